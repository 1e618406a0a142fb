"""Pins of the CPU oracle against what the paper and the mathematics fix.

None of these compare the oracle with itself: every expected value comes from a number
printed in the paper (tests/golden), a closed form, a symmetry of the model, or a
library routine (LAPACK eigensolvers, math.comb) on a special case.
"""
import math
import os

import numpy as np
import pytest
import scipy.linalg as sla
import scipy.sparse as sp

import ed_inputs
from oracle import basis, dense, hamiltonian, lanczos, tridiag

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _hopping_matrix(n_sites, bonds, t=1.0):
    h = np.zeros((n_sites, n_sites))
    for i, j in bonds:
        h[i, j] -= t
        h[j, i] -= t
    return h


def _free_fermion_E0(n_sites, bonds, n_up, n_dn, t=1.0):
    eps = np.linalg.eigvalsh(_hopping_matrix(n_sites, bonds, t))
    return eps[:n_up].sum() + eps[:n_dn].sum()


def _lanczos_E0(n_sites, bonds, n_up, n_dn, t, U, seed=11, tol=1e-14, steps=300):
    H = hamiltonian.hamiltonian_csr(n_sites, bonds, n_up, n_dn, t, U)
    f1 = lanczos.normalized_start(ed_inputs.start_vector_raw(seed, H.shape[0]))
    return lanczos.lanczos(lambda v: H @ v, f1, max_steps=steps, tol=tol).E0


# ----------------------------------------------------------------------------- basis
def test_dimensions_printed_in_paper():
    for line in open(os.path.join(GOLDEN, "paper_dims.txt")):
        line = line.split("#")[0].split()
        if not line:
            continue
        if line[0] == "V":
            L, nu, nd, p, gb, rel = int(line[1]), int(line[2]), int(line[3]), int(line[4]), float(line[5]), float(line[6])
            dim = math.comb(L, nu) * math.comb(L, nd)
            assert abs(dim * p / 1e9 - gb) <= rel * gb
        else:
            L, nu, nd, val, rel = int(line[0]), int(line[1]), int(line[2]), float(line[3]), float(line[4])
            if L <= 14:   # enumeration is cheap up to 14 sites
                dim = basis.dimension(L, nu, nd)
            else:
                dim = len(basis.species_states(L, nu)) ** 2
            assert abs(dim - val) <= rel * val


@pytest.mark.parametrize("L,N", [(1, 0), (1, 1), (5, 2), (8, 4), (12, 3), (10, 10)])
def test_species_states_ascending_and_counted(L, N):
    s = basis.species_states(L, N)
    assert len(s) == math.comb(L, N)
    assert np.all(np.diff(s) > 0)
    assert np.all(basis.popcount(s) == N)
    assert np.all(basis.rank_of(s, s) == np.arange(len(s)))


@pytest.mark.parametrize("L,nu,nd", [(6, 1, 4), (7, 3, 2), (8, 0, 5), (5, 5, 2)])
def test_dimension_unequal_fillings(L, nu, nd):
    """Eq. 2 with N_up != N_dn (every dimension the paper prints is at N_up = N_dn), for the
    enumerated count and for the size of the explicit H."""
    expect = math.comb(L, nu) * math.comb(L, nd)
    assert basis.dimension(L, nu, nd) == expect
    H = hamiltonian.hamiltonian_csr(L, ed_inputs.ring_bonds(L), nu, nd, 1.0, 2.0)
    assert H.shape == (expect, expect)


def test_popcount_against_python():
    rng = np.random.default_rng(0)
    a = rng.integers(0, 2**62, size=1000)
    assert np.array_equal(basis.popcount(a), [bin(int(v)).count("1") for v in a])


# ------------------------------------------------------------------------ hamiltonian
CASES = [
    (5, ed_inputs.ring_bonds(5), 2, 2, 1.0, 3.0),
    (6, ed_inputs.ring_bonds(6), 3, 2, 1.0, 2.5),
    (6, ed_inputs.ring_bonds(6), 2, 4, 0.7, 1.0),
    (8, ed_inputs.torus_bonds(2, 4), 2, 3, 1.0, 4.0),
    (6, ed_inputs.torus_bonds(3, 2), 3, 3, 1.3, -2.0),
]


@pytest.mark.parametrize("case", CASES)
def test_hamiltonian_symmetric(case):
    H = hamiltonian.hamiltonian_csr(*case)
    assert abs(H - H.T).max() == 0.0


@pytest.mark.parametrize("case", CASES)
def test_trace_closed_form(case):
    L, bonds, nu, nd, t, U = case
    H = hamiltonian.hamiltonian_csr(*case)
    # each site is doubly occupied in C(L-1,nu-1)*C(L-1,nd-1) basis states
    expect = U * L * math.comb(L - 1, nu - 1) * math.comb(L - 1, nd - 1)
    assert abs(H.diagonal().sum() - expect) <= 1e-12 * max(1.0, abs(expect))


@pytest.mark.parametrize("L,N", [(6, 2), (8, 3), (12, 3), (7, 4)])
def test_hop_count_closed_form(L, N):
    bonds = ed_inputs.ring_bonds(L)
    _, lists = hamiltonian.species_hop_table(L, N, bonds)
    # a bond moves a particle iff exactly one end is occupied: 2*C(L-2, N-1) states
    assert sum(len(x) for x in lists) == 2 * len(bonds) * math.comb(L - 2, N - 1)


def test_tensor_product_split_eq3():
    """H(U=0) = H_up (x) I + I (x) H_dn (Sec. 2.1, Eq. 3) as a property of the state-by-
    state construction; the single-species H_sigma is the N_other = 0 case."""
    L, bonds = 6, ed_inputs.ring_bonds(6)
    nu, nd = 3, 2
    H = hamiltonian.hamiltonian_csr(L, bonds, nu, nd, 1.0, 0.0)
    Hu = hamiltonian.hamiltonian_csr(L, bonds, nu, 0, 1.0, 0.0)
    Hd = hamiltonian.hamiltonian_csr(L, bonds, nd, 0, 1.0, 0.0)
    K = sp.kron(Hu, sp.identity(Hd.shape[0])) + sp.kron(sp.identity(Hu.shape[0]), Hd)
    assert abs(H - K).max() == 0.0


@pytest.mark.parametrize("case", CASES)
def test_rows_match_columns(case):
    """Rows from the hops out of each state equal H built column by column."""
    H = hamiltonian.hamiltonian_csr(*case)
    x = ed_inputs.uniform_pm1(7, H.shape[0])
    rows = np.arange(H.shape[0])
    assert np.allclose(hamiltonian.hv_rows(*case, x, rows), H @ x, rtol=0, atol=1e-13)


@pytest.mark.parametrize("L,bonds,N", [
    (8, ed_inputs.ring_bonds(8), 3),
    (9, np.array([[0, 5], [3, 8], [1, 2], [7, 0], [6, 4], [2, 8], [5, 1], [8, 3]]), 4),
])
def test_hop_table_rebuilds_the_single_species_hamiltonian(L, bonds, N):
    """The per-state hop lists (the reference of the device hop tables) hold, for state r,
    the hopped states' ranks and signs in bond order: summing -sign |target><r| over them
    gives the one-species Hamiltonian at U = 0 (pinned above by the free-fermion energies
    and the symmetries), and entry k of state r comes from the k-th bond that moves one of
    its particles."""
    states, lists = hamiltonian.species_hop_table(L, N, bonds)
    n = len(states)
    M = np.zeros((n, n))
    for r, lst in enumerate(lists):
        for tgt, sg in lst:
            M[tgt, r] += -1.0 * sg
    H = hamiltonian.hamiltonian_csr(L, bonds, N, 0, 1.0, 0.0).toarray()
    assert np.array_equal(M, H)
    for r, lst in enumerate(lists):
        movers = [b for b, (i, j) in enumerate(bonds) if ((states[r] >> i) & 1) != ((states[r] >> j) & 1)]
        assert len(movers) == len(lst)
        for (tgt, _), b in zip(lst, movers):
            i, j = bonds[b]
            assert states[tgt] == states[r] ^ ((1 << int(i)) | (1 << int(j)))


def test_wrap_sign_is_fermionic():
    """Ring wrap-around hop with N particles crosses the other N-1: sign (-1)^(N-1)."""
    for N in (2, 3, 4):
        states, lists = hamiltonian.species_hop_table(6, N, np.array([[5, 0]]))
        for r, lst in enumerate(lists):
            for tgt, sgn in lst:
                assert sgn == (-1) ** (N - 1)


# ------------------------------------------------------------------ closed-form energies
@pytest.mark.parametrize("L,nu,nd", [(6, 2, 2), (6, 3, 1), (8, 2, 3), (5, 2, 2), (4, 2, 2)])
def test_U0_free_fermions_ring(L, nu, nd):
    """U = 0: E0 = sum of the lowest N_up and N_dn single-particle levels (even N included,
    which fails if the fermion signs are wrong)."""
    bonds = ed_inputs.ring_bonds(L)
    E = dense.spectrum(L, bonds, nu, nd, 1.0, 0.0)[0]
    assert abs(E - _free_fermion_E0(L, bonds, nu, nd)) <= 1e-12


def test_U0_free_fermions_torus():
    bonds = ed_inputs.torus_bonds(4, 4)
    E = _lanczos_E0(16, bonds, 2, 2, 1.0, 0.0)
    assert abs(E - (-12.0)) <= 1e-10


def test_U0_ring12_closed_form():
    """L = 12 ring, 3/3: odd N gives E0_sigma = -2 sin(pi N / L) / sin(pi / L)."""
    E = _lanczos_E0(12, ed_inputs.ring_bonds(12), 3, 3, 1.0, 0.0)
    expect = 2 * (-2 * math.sin(math.pi * 3 / 12) / math.sin(math.pi / 12))
    assert abs(expect - (-4 * (1 + math.sqrt(3)))) < 1e-13
    assert abs(E - expect) <= 1e-12 * abs(expect)


@pytest.mark.parametrize("U", [0.0, 1.0, 4.0, 8.0, -3.0])
@pytest.mark.parametrize("t", [1.0, 0.5])
def test_two_site_hubbard(U, t):
    """One bond, one up and one down electron: E0 = (U - sqrt(U^2 + 16 t^2)) / 2."""
    bonds = np.array([[0, 1]])
    E = dense.spectrum(2, bonds, 1, 1, t, U)[0]
    assert abs(E - (U - math.sqrt(U * U + 16 * t * t)) / 2) <= 1e-13


def test_two_site_doubled_bond():
    """The L = 2 'ring' lists the pair twice: amplitude 2t, E0 = (U - sqrt(U^2 + 64 t^2))/2."""
    E = dense.spectrum(2, ed_inputs.ring_bonds(2), 1, 1, 1.0, 4.0)[0]
    assert abs(E - (4 - math.sqrt(16 + 64)) / 2) <= 1e-13


@pytest.mark.parametrize("L,bonds,nu,nd,U", [
    (6, ed_inputs.ring_bonds(6), 3, 1, 2.0),
    (8, ed_inputs.torus_bonds(2, 4), 2, 3, 4.0),
    (6, ed_inputs.torus_bonds(3, 2), 1, 2, 1.5),
])
def test_spin_swap_symmetry(L, bonds, nu, nd, U):
    a = dense.spectrum(L, bonds, nu, nd, 1.0, U)[0]
    b = dense.spectrum(L, bonds, nd, nu, 1.0, U)[0]
    assert abs(a - b) <= 1e-12 * max(1, abs(a))


@pytest.mark.parametrize("L,bonds,nu,nd,U", [
    (6, ed_inputs.ring_bonds(6), 2, 1, 3.0),
    (8, ed_inputs.torus_bonds(2, 4), 2, 3, 4.0),
    (4, ed_inputs.ring_bonds(4), 1, 1, 2.0),
])
def test_particle_hole_symmetry_bipartite(L, bonds, nu, nd, U):
    """On a bipartite lattice E0(L-Nu, L-Nd) = E0(Nu, Nd) + U (L - Nu - Nd)."""
    a = dense.spectrum(L, bonds, nu, nd, 1.0, U)[0]
    b = dense.spectrum(L, bonds, L - nu, L - nd, 1.0, U)[0]
    assert abs(b - (a + U * (L - nu - nd))) <= 1e-11 * max(1, abs(b))


def test_energy_monotone_in_U():
    L, bonds = 6, ed_inputs.ring_bonds(6)
    Es = [dense.spectrum(L, bonds, 3, 3, 1.0, U)[0] for U in (0.0, 1.0, 2.0, 4.0, 8.0)]
    assert all(np.diff(Es) > 0)


@pytest.mark.parametrize("L,bonds,nu,nd", [
    (6, ed_inputs.ring_bonds(6), 3, 3),
    (5, ed_inputs.ring_bonds(5), 2, 1),
    (8, ed_inputs.torus_bonds(2, 4), 1, 3),
])
def test_variational_bound_and_concavity_in_U(L, bonds, nu, nd):
    """E0(U) = min over unit psi of <psi|H_0|psi> + U <psi|D|psi> (D = number of doubly
    occupied sites) is a minimum of functions linear in U, hence concave, and lies below the
    line through the U = 0 ground state: E0(U) <= E0(0) + U <D>_0, evaluated here with the
    U = 0 ground state's own energy functional (<psi0|H(U)|psi0>, no closed form of D)."""
    Us = np.linspace(0.0, 8.0, 9)
    E = np.array([dense.spectrum(L, bonds, nu, nd, 1.0, U)[0] for U in Us])
    assert np.all(E[:-2] - 2 * E[1:-1] + E[2:] <= 1e-12)
    _, psi0 = dense.ground_state(L, bonds, nu, nd, 1.0, 0.0)
    for U, e in zip(Us, E):
        H = hamiltonian.hamiltonian_csr(L, bonds, nu, nd, 1.0, U)
        assert e <= float(psi0 @ (H @ psi0)) + 1e-12


# ----------------------------------------------------------------------- tridiagonal
def test_sturm_against_lapack():
    rng = np.random.default_rng(3)
    for m in (1, 2, 5, 40, 200):
        a = rng.normal(size=m) * 3
        b = np.abs(rng.normal(size=m - 1)) + 0.01
        ref = sla.eigh_tridiagonal(a, b, eigvals_only=True)[0]
        assert abs(tridiag.lowest_eigenvalue(a, b) - ref) <= 4e-15 * max(1, np.abs(ref))


def test_sturm_closed_form():
    """a = 0, b = 1: eigenvalues 2 cos(k pi / (m + 1)); the lowest is -2 cos(pi/(m+1))."""
    for m in (3, 17, 100):
        E = tridiag.lowest_eigenvalue(np.zeros(m), np.ones(m - 1))
        assert abs(E + 2 * math.cos(math.pi / (m + 1))) <= 1e-14


def test_sturm_count_brackets():
    rng = np.random.default_rng(4)
    a = rng.normal(size=30)
    b = rng.uniform(0.1, 1, size=29)
    w = sla.eigh_tridiagonal(a, b, eigvals_only=True)
    for k, x in enumerate((w[:-1] + w[1:]) / 2):
        assert tridiag.sturm_count(a, b, x) == k + 1


# --------------------------------------------------------------------------- lanczos
@pytest.mark.parametrize("case", CASES)
def test_lanczos_matches_dense(case):
    E_dense = dense.spectrum(*case)[0]
    E = _lanczos_E0(*case)
    assert abs(E - E_dense) <= 1e-11 * max(1, abs(E_dense))


@pytest.mark.parametrize("reorth", [False, True])
def test_lanczos_on_tridiagonal_returns_its_entries(reorth):
    """Algorithm 1 applied to an unreduced symmetric tridiagonal matrix T (positive off-
    diagonal) from f_1 = e_1 produces f_j = e_j, a_j = T_jj and b_{j+1} = T_{j,j+1}: the
    Krylov basis of e_1 under T is the unit-vector basis. In FP64 every step is exact
    (each subtraction cancels equal numbers, sqrt(b^2) rounds back to b), so the
    coefficients must match bit for bit. The start is given with norm 3, which Algorithm 1
    normalises. fixed_steps must run all m steps although E0(j) settles earlier; at step m
    the residual is exactly zero (breakdown). Small off-diagonals (down to 0.01 against a
    spread of diagonal entries) must not be taken for a breakdown."""
    rng = np.random.default_rng(12)
    m = 40
    a = rng.normal(size=m) * 2.0
    b = rng.uniform(0.01, 1.0, size=m - 1)
    b[7] = 0.01
    T = sp.diags([b, a, b], [-1, 0, 1], format="csr")
    e1 = np.zeros(m)
    e1[0] = 3.0
    r = lanczos.lanczos(lambda v: T @ v, e1, max_steps=m, tol=1e-12, reorth=reorth,
                        fixed_steps=True)
    assert r.steps == m and r.breakdown
    assert np.array_equal(np.array(r.alpha), a)
    assert np.array_equal(np.array(r.beta[:-1]), b) and r.beta[-1] == 0.0
    ref = sla.eigh_tridiagonal(a, b, eigvals_only=True)[0]
    assert abs(r.E0 - ref) <= 4e-15 * max(1.0, abs(ref))
    # the same run with the convergence test on stops as soon as E0(j) settles, before m
    r2 = lanczos.lanczos(lambda v: T @ v, e1, max_steps=m, tol=1e-12, reorth=reorth)
    assert r2.converged and not r2.breakdown and r2.steps < m
    assert r2.alpha == r.alpha[:r2.steps]


def test_normalized_start_is_unit_and_parallel():
    raw = ed_inputs.start_vector_raw(5, 1000) * 7.5
    f = lanczos.normalized_start(raw)
    assert abs(np.linalg.norm(f) - 1.0) <= 1e-15
    k = int(np.argmax(np.abs(raw)))
    assert np.allclose(f * (raw[k] / f[k]), raw, rtol=1e-14, atol=0)
    assert np.sign(f[k]) == np.sign(raw[k])


@pytest.mark.parametrize("case", CASES[:3])
def test_dense_ground_state_is_a_gauged_eigenvector(case):
    """ground_state returns a unit eigenvector for the lowest eigenvalue, gauged so that its
    largest-magnitude entry (lowest index on ties) is positive."""
    E0, psi = dense.ground_state(*case)
    H = hamiltonian.hamiltonian_csr(*case)
    assert abs(np.linalg.norm(psi) - 1.0) <= 1e-13
    assert np.max(np.abs(H @ psi - E0 * psi)) <= 1e-11
    k = int(np.argmax(np.abs(psi)))
    assert psi[k] > 0


def test_lanczos_breakdown_on_eigenvector():
    case = (2, np.array([[0, 1]]), 1, 1, 1.0, 0.0)
    E0, psi = dense.ground_state(*case)
    H = hamiltonian.hamiltonian_csr(*case)
    r = lanczos.lanczos(lambda v: H @ v, psi)
    assert r.breakdown and r.steps == 1
    assert abs(r.E0 - (-2.0)) <= 1e-14


def test_lanczos_full_reorth_keeps_orthogonality():
    case = (6, ed_inputs.ring_bonds(6), 3, 3, 1.0, 4.0)
    H = hamiltonian.hamiltonian_csr(*case)
    f1 = lanczos.normalized_start(ed_inputs.start_vector_raw(2, H.shape[0]))
    r = lanczos.lanczos(lambda v: H @ v, f1, max_steps=60, fixed_steps=True)
    a, b = np.array(r.alpha), np.array(r.beta[:-1])
    # with full reorthogonalisation T's spectrum lies inside H's (no ghost copies)
    w_T = sla.eigh_tridiagonal(a, b, eigvals_only=True)
    w_H = np.linalg.eigvalsh(H.toarray())
    assert w_T[0] >= w_H[0] - 1e-10 and w_T[-1] <= w_H[-1] + 1e-10
    assert abs(w_T[0] - w_H[0]) <= 1e-10


# ------------------------------------------------- error-bound scale |H| |x| of the H.v tests
RANDOM_BONDS = (9, np.array([[0, 5], [3, 8], [1, 2], [7, 0], [6, 4], [2, 8], [5, 1], [8, 3]]),
                4, 3, 1.3, -1.5)


@pytest.mark.parametrize("case", CASES + [RANDOM_BONDS])
def test_abs_rows_match_abs_matrix(case):
    """(|H| |x|)_g from the hops out of each state equals |H| @ |x| with H built column by
    column (Eq. 1 plus the on-site term): every row, a U of either sign, a doubled bond
    (the 2x4 lattice) and a bond listed in both orders (the random list)."""
    H = hamiltonian.hamiltonian_csr(*case)
    x = ed_inputs.uniform_pm1(17, H.shape[0])
    rows = np.arange(H.shape[0])
    ref = abs(H) @ np.abs(x)
    got = hamiltonian.hv_abs_rows(*case, x, rows)
    assert np.all(got >= 0)
    assert np.allclose(got, ref, rtol=1e-14, atol=0)
    # and it bounds the signed rows term by term
    assert np.all(np.abs(hamiltonian.hv_rows(*case, x, rows)) <= got * (1 + 1e-14))


# ------------------------------------------------------------------ Bethe-ansatz ring pin
from oracle import bethe  # noqa: E402


@pytest.mark.parametrize("L,nu,nd", [(4, 2, 2), (6, 3, 3), (8, 4, 4), (6, 2, 2), (5, 2, 2),
                                     (7, 3, 2), (6, 1, 1), (9, 3, 3)])
@pytest.mark.parametrize("U", [0.5, 4.0, 8.0])
def test_bethe_ansatz_matches_diagonalisation(L, nu, nd, U):
    """The Lieb-Wu ring energy equals the oracle's E0 (dense eigh, or Algorithm 1 with full
    reorthogonalisation above the dense limit) on small periodic rings: half filling with
    odd and even particle numbers per spin (the 16-site ring workload is even), and open-
    shell fillings whose ground state has higher spin."""
    E_bethe = bethe.ring_ground_energy(L, nu, nd, U)
    bonds = ed_inputs.ring_bonds(L)
    if math.comb(L, nu) * math.comb(L, nd) <= 2000:
        ref = dense.spectrum(L, bonds, nu, nd, 1.0, U)[0]
    else:
        ref = _lanczos_E0(L, bonds, nu, nd, 1.0, U, tol=1e-15, steps=400)
    assert abs(E_bethe - ref) <= 1e-12 * abs(ref), (E_bethe, ref)


def test_bethe_quantum_number_parity():
    """I_j integers for even M, half-odd for odd M; J_a integers for odd N - M, half-odd for
    even N - M; both sets consecutive."""
    for N, M in [(16, 8), (12, 6), (5, 2), (4, 1), (7, 3)]:
        I, J = bethe.ground_state_numbers(16, N, M)
        assert len(I) == N and len(J) == M
        assert np.all(np.diff(I) == 1) and np.all(np.diff(J) == 1)
        assert np.all((I - (0.0 if M % 2 == 0 else 0.5)) % 1.0 == 0.0)
        assert np.all((J - (0.0 if (N - M) % 2 == 1 else 0.5)) % 1.0 == 0.0)
