"""Plain, slow, obviously-correct CPU FP64 oracle for exact diagonalization of the
tight-binding / Hubbard model (Siro & Harju, arXiv:1511.00863).

TEST INFRASTRUCTURE ONLY. Only the test suite, the smoke check and the benchmark's CPU
baseline leg may import this package. The CUDA library never calls it and shares no code
with it; the two meet only through the seeded input generators in `ed_inputs`.

Each function cites the passage of the paper it follows (section, equation, algorithm).
Where the paper is silent the reading used is stated in the docstring.

Module map:
  basis        single-species occupation basis and its ranking (Sec. 2.1, Eq. 2)
  hamiltonian  explicit sparse H and matrix-free rows (Sec. 1 Eq. 1 plus the on-site term)
  tridiag      lowest eigenvalue of the Lanczos tridiagonal T (Sec. 2.2, Eq. for T)
  lanczos      Algorithm 1 in FP64, optional full reorthogonalisation (Sec. 2.2)
  dense        dense diagonalisation for small dimensions
  observables  double occupancy of a state vector (the on-site term; dE0/dU)
  complex_hopping  H with a complex amplitude per bond (Sec. 2.1: the checkerboard lattice's
               complex hoppings) and its real view
  mlp          the learned start-vector network, its loss and gradient (no counterpart in
               the paper; test oracle of the library's MLP kernels)
  bethe        ground-state energy of the periodic Hubbard ring from the Lieb-Wu
               Bethe-ansatz equations (an exact method of its own, used to pin the
               full-size ring workloads beyond the explicit matrix's reach)
"""
from . import basis, hamiltonian, tridiag, lanczos, dense, mlp, observables, complex_hopping, bethe  # noqa: F401
