"""Reorthogonalisation on the GPU (ed_opts.reorth = 1 full, 2 partial) against the oracle's
Algorithm 1 with full reorthogonalisation (two Gram-Schmidt passes, Sec. 2.2 plus the
reading that the oracle reorthogonalises), and its effect: no spurious copies ("ghosts") of
converged eigenvalues in T_m."""
import os

import numpy as np
import pytest
import scipy.linalg as sla

import ed_inputs
from oracle import hamiltonian, lanczos as olz

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")

# 6-site ring, 3/3, U = 4 (dim 400): without reorthogonalisation T_120 holds two copies of
# the lowest and of the highest eigenvalue of H; with it, one.
CASE = (6, ed_inputs.ring_bonds(6), 3, 3, 1.0, 4.0)


@pytest.fixture(scope="module")
def ed():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1511_00863_gb300 as m
    return m


@pytest.fixture(scope="module")
def ref():
    H = hamiltonian.hamiltonian_csr(*CASE)
    w = np.linalg.eigvalsh(H.toarray())
    f1 = olz.normalized_start(ed_inputs.start_vector_raw(21, H.shape[0]))
    full = olz.lanczos(lambda v: H @ v, f1, max_steps=60, reorth=True, fixed_steps=True)
    plain = olz.lanczos(lambda v: H @ v, f1, max_steps=120, reorth=False, fixed_steps=True)
    return w, f1, full, plain


def _run(ed, f1, steps, dtype, reorth):
    L, bonds, nu, nd, t, U = CASE
    b = ed.ed_build_basis(L, bonds, nu, nd)
    try:
        tdt = torch.float32 if dtype == "f32" else torch.float64
        return ed.ed_lanczos_solve(b, t, U, ed.make_opts(max_steps=steps, tol=0.0, seed=1, dtype=dtype,
                                                         reorth=reorth),
                                   f1=torch.tensor(f1, dtype=tdt, device="cuda"),
                                   raise_not_converged=False)
    finally:
        ed.ed_basis_destroy(b)


def _copies(res, e, tol):
    n = res["steps"]
    T = sla.eigvalsh_tridiagonal(np.asarray(res["alpha"][:n]), np.asarray(res["beta"][:n - 1]))
    return int(np.sum(np.abs(T - e) <= tol * max(1.0, abs(e))))


@pytest.mark.parametrize("dtype", ["f64", "f64n"])
def test_full_reorth_follows_oracle(ed, ref, dtype):
    """60 steps with full reorthogonalisation: a_j and b_{j+1} equal the oracle's fully
    reorthogonalised run to 1e-10 (without it the two runs would part once the extreme Ritz
    values converge)."""
    w, f1, full, _ = ref
    res = _run(ed, f1, 60, dtype, 1)
    assert res["steps"] == 60
    assert np.allclose(res["alpha"], full.alpha, rtol=1e-10, atol=1e-10), \
        np.max(np.abs(np.asarray(res["alpha"]) - full.alpha))
    assert np.allclose(res["beta"], full.beta, rtol=1e-10, atol=1e-10)


@pytest.mark.parametrize("dtype", ["f64", "f64n", "f32"])
@pytest.mark.parametrize("reorth", [1, 2])
def test_no_ghost_eigenvalues(ed, ref, dtype, reorth):
    """120 steps: the plain recurrence (oracle, and the GPU without reorthogonalisation)
    duplicates the extreme eigenvalues of H in T_120; with full or partial
    reorthogonalisation each appears once, and every Ritz value lies in [E_min, E_max]."""
    w, f1, _, plain = ref
    tol = 1e-8 if dtype != "f32" else 1e-5
    assert _copies({"steps": 120, "alpha": plain.alpha, "beta": plain.beta}, w[0], 1e-8) >= 2
    if reorth == 1 and dtype == "f64":
        assert _copies(_run(ed, f1, 120, dtype, 0), w[0], tol) >= 2
    res = _run(ed, f1, 120, dtype, reorth)
    assert res["steps"] == 120
    assert _copies(res, w[0], tol) == 1
    assert _copies(res, w[-1], tol) == 1
    n = res["steps"]
    T = sla.eigvalsh_tridiagonal(np.asarray(res["alpha"]), np.asarray(res["beta"][:n - 1]))
    assert T[0] >= w[0] - tol * abs(w[0]) and T[-1] <= w[-1] + tol * abs(w[-1])


def _golden(name):
    out = {}
    for line in open(os.path.join(GOLDEN, name)):
        f = line.split()
        if f and not f[0].startswith("#") and len(f) == 2:
            out[f[0]] = float(f[1])
    return out


@pytest.mark.parametrize("dtype,reorth,tol", [("f32", 1, 1e-6), ("f32", 2, 1e-6), ("f64", 2, 1e-10),
                                              ("f64n", 1, 1e-10)])
def test_reorth_E0_ring12(ed, dtype, reorth, tol):
    """E0 of the 12-site ring, 3/3, U = 4 with reorthogonalisation against the stored oracle
    value (FP32 within 1e-6, the FP64 forms within 1e-10)."""
    E_ref = _golden("lanczos_ring12_3_3_U4.txt")["E0"]
    w = ed_inputs.workload("ring12_3_3")
    b = ed.ed_build_basis(w["n_sites"], w["bonds"], w["n_up"], w["n_dn"])
    try:
        res = ed.ed_lanczos_solve(b, w["t"], 4.0, ed.make_opts(max_steps=200, tol=1e-9 if dtype == "f32" else 1e-12,
                                                               seed=w["seed"], dtype=dtype, reorth=reorth),
                                  raise_not_converged=False)
    finally:
        ed.ed_basis_destroy(b)
    assert abs(res["E0"] - E_ref) <= tol * abs(E_ref), (res["E0"], E_ref)


def test_reorth_rejected_for_complex_and_out_of_range(ed):
    b = ed.ed_build_basis(4, ed_inputs.ring_bonds(4), 2, 2)
    try:
        with pytest.raises(ed.EdError):
            ed.ed_lanczos_solve(b, 1.0, 1.0, ed.make_opts(max_steps=10, dtype="c32", reorth=1))
        with pytest.raises(ed.EdError):
            ed.ed_lanczos_solve(b, 1.0, 1.0, ed.make_opts(max_steps=10, reorth=3))
    finally:
        ed.ed_basis_destroy(b)
