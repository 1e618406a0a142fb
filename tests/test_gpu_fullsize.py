"""E0 of the full-size workloads at U != 0 against values independent of the GPU code: the
oracle's Algorithm 1 with full reorthogonalisation on the 4x4 torus (stored by
tests/golden/make_lanczos_goldens.py) and the Lieb-Wu Bethe-ansatz energies of the periodic
rings (stored by tests/golden/make_small_goldens.py from oracle/bethe.py). FP64 forms within
1e-10 relative, FP32 within 1e-6 relative."""
import os

import numpy as np
import pytest

import ed_inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


@pytest.fixture(scope="module")
def ed():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1511_00863_gb300 as m
    return m


def lanczos_golden(name):
    E0, ab = None, []
    for line in open(os.path.join(GOLDEN, name)):
        f = line.split()
        if not f or f[0].startswith("#"):
            continue
        if f[0] == "E0":
            E0 = float(f[1])
        elif f[0] == "ab":
            ab.append((float(f[2]), float(f[3])))
    return E0, np.array(ab)


def bethe_golden(workload, U):
    for line in open(os.path.join(GOLDEN, "bethe_rings.txt")):
        f = line.split()
        if f and not f[0].startswith("#") and f[0] == workload and abs(float(f[4]) - U) < 1e-15:
            return float(f[5])
    raise KeyError((workload, U))


def _solve(ed, name, dtype, U=None, tol=1e-12, max_steps=400, f1=None):
    w = ed_inputs.workload(name)
    b = ed.ed_build_basis(w["n_sites"], w["bonds"], w["n_up"], w["n_dn"])
    try:
        return ed.ed_lanczos_solve(b, w["t"], w["U"] if U is None else U,
                                   ed.make_opts(max_steps=max_steps, tol=tol, seed=w["seed"], dtype=dtype),
                                   f1=f1, raise_not_converged=False)
    finally:
        ed.ed_basis_destroy(b)


@pytest.mark.parametrize("dtype,tol", [("f64", 1e-10), ("f64n", 1e-10), ("f32", 1e-6)])
def test_torus4x4_U4_E0_vs_oracle(ed, dtype, tol):
    E_ref, _ = lanczos_golden("lanczos_torus4x4_5_5_U4.txt")
    res = _solve(ed, "torus4x4_5_5", dtype, tol=1e-12 if dtype != "f32" else 1e-9)
    assert abs(res["E0"] - E_ref) <= tol * abs(E_ref), (res["E0"], E_ref, res["steps"])


@pytest.mark.parametrize("dtype,tol", [("f64", 1e-11), ("f64n", 1e-11), ("f32", 2e-5)])
def test_torus4x4_U4_first_steps_vs_oracle(ed, dtype, tol):
    """a_1..a_20, b_2..b_21 of the benchmark workload (the fused H.v variant the benchmark
    times for the FP64-accurate and FP32 forms) against the oracle's first 20 steps from the
    same seeded start vector."""
    _, ab = lanczos_golden("lanczos_torus4x4_5_5_U4.txt")
    res = _solve(ed, "torus4x4_5_5", dtype, tol=0.0, max_steps=20)
    assert res["steps"] == 20
    assert np.allclose(res["alpha"], ab[:, 0], rtol=tol, atol=tol), np.max(np.abs(res["alpha"] - ab[:, 0]))
    assert np.allclose(res["beta"], ab[:, 1], rtol=tol, atol=tol), np.max(np.abs(res["beta"] - ab[:, 1]))


@pytest.mark.parametrize("dtype,tol", [("f64", 1e-10), ("f32", 1e-6), ("f64n", 1e-10)])
def test_ring16_U4_E0_vs_bethe_ansatz(ed, dtype, tol):
    E_ref = bethe_golden("ring16_8_8", 4.0)
    res = _solve(ed, "ring16_8_8", dtype, U=4.0, tol=1e-12 if dtype != "f32" else 1e-9)
    assert abs(res["E0"] - E_ref) <= tol * abs(E_ref), (res["E0"], E_ref, res["steps"])


@pytest.mark.slow
def test_ring18_U4_fp32_E0_vs_bethe_ansatz(ed):
    """The 18-site 9/9 basis (2,363,904,400 states) in FP32 at U = 4: E0 within 1e-6 of the
    Bethe-ansatz energy."""
    E_ref = bethe_golden("ring18_9_9", 4.0)
    res = _solve(ed, "ring18_9_9", "f32", U=4.0, tol=1e-9, max_steps=300)
    assert abs(res["E0"] - E_ref) <= 1e-6 * abs(E_ref), (res["E0"], E_ref, res["steps"])


@pytest.mark.slow
def test_ring18_U4_fp64_accurate_split_rows_vs_bethe_ansatz(ed):
    """The FP64-accurate form of the 18-site 9/9 basis: its 389 KB int64 rows exceed shared
    memory, so the split-row fused kernel (schedule 30, two slices of the down states) runs
    by itself; E0 at U = 4 within 1e-10 of the Bethe-ansatz energy."""
    E_ref = bethe_golden("ring18_9_9", 4.0)
    w = ed_inputs.workload("ring18_9_9")
    b = ed.ed_build_basis(w["n_sites"], w["bonds"], w["n_up"], w["n_dn"])
    try:
        opts = ed.make_opts(max_steps=400, tol=1e-12, seed=w["seed"], dtype="f64")
        st = ed.ed_lanczos_init(b, opts)
        try:
            assert ed.ed_lanczos_schedule(st) == 30
        finally:
            ed.ed_lanczos_destroy(st)
        res = ed.ed_lanczos_solve(b, w["t"], 4.0, opts, raise_not_converged=False)
    finally:
        ed.ed_basis_destroy(b)
    assert abs(res["E0"] - E_ref) <= 1e-10 * abs(E_ref), (res["E0"], E_ref, res["steps"])
