"""The mixed-precision solve (FP32 Lanczos, its Ritz vector, FP64-accurate Lanczos from it)
against stored oracle energies: E0 within 1e-10 relative on the 12-site ring, the full-size
4x4 torus and 16-site ring at U = 4 and every instance of the 256-instance batch; the
Rayleigh quotient of the FP32 Ritz vector obeys the Kato-Temple bound; a poor FP32 phase
only costs refinement steps."""
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


def _golden_E0(name):
    for line in open(os.path.join(GOLDEN, name)):
        f = line.split()
        if f and f[0] == "E0":
            return float(f[1])


def _bethe(workload, U):
    for line in open(os.path.join(GOLDEN, "bethe_rings.txt")):
        f = line.split()
        if f and f[0] == workload and abs(float(f[4]) - U) < 1e-15:
            return float(f[5])


@pytest.mark.parametrize("name,E_ref_fn,tol", [
    ("ring12_3_3", lambda: _golden_E0("lanczos_ring12_3_3_U4.txt"), 1e-10),
    ("torus4x4_5_5", lambda: _golden_E0("lanczos_torus4x4_5_5_U4.txt"), 1e-10),
    ("ring16_8_8", lambda: _bethe("ring16_8_8", 4.0), 1e-10),
])
def test_mixed_solve_reaches_fp64_accuracy(ed, name, E_ref_fn, tol):
    w = ed_inputs.workload(name)
    E_ref = E_ref_fn()
    b = ed.ed_build_basis(w["n_sites"], w["bonds"], w["n_up"], w["n_dn"])
    try:
        res = ed.ed_lanczos_solve_mixed(b, w["t"], 4.0, ed.make_opts(max_steps=300, tol=1e-9, seed=w["seed"],
                                                                     dtype="f32"), refine_steps=64,
                                        refine_tol=1e-12)
    finally:
        ed.ed_basis_destroy(b)
    assert abs(res["E0"] - E_ref) <= tol * abs(E_ref), res
    assert res["steps32"] >= 2 and res["residual"] > 0.0
    assert res["steps64"] <= 32   # the FP32 Ritz vector leaves few steps to the FP64 form
    # the FP32 phase alone is less accurate than the refined energy (or as accurate)
    assert abs(res["E0"] - E_ref) <= abs(res["E0_fp32"] - E_ref) + 1e-12 * abs(E_ref)


def test_rayleigh_quotient_kato_temple(ed):
    """One refinement step: E0 = a_1 = the Rayleigh quotient rho of the FP32 Ritz vector; its
    distance to the exact E0 is at most residual^2 / (E1 - rho) (Kato-Temple), with E0, E1
    from the dense spectrum of a small ring."""
    from oracle import dense
    L, bonds, nu, nd, U = 7, ed_inputs.ring_bonds(7), 3, 3, 2.0   # non-degenerate ground state
    w = dense.spectrum(L, bonds, nu, nd, 1.0, U)
    assert w[1] - w[0] > 1.0
    b = ed.ed_build_basis(L, bonds, nu, nd)
    try:
        res = ed.ed_lanczos_solve_mixed(b, 1.0, U, ed.make_opts(max_steps=200, tol=1e-7, seed=3, dtype="f32"),
                                        refine_steps=1, refine_tol=0.0)
    finally:
        ed.ed_basis_destroy(b)
    assert res["E0"] >= w[0] - 1e-12 * abs(w[0])   # a Rayleigh quotient bounds E0 from above
    # rho - E0 <= r^2 / (E1 - rho) for rho below (E0 + E1) / 2
    assert res["E0"] < 0.5 * (w[0] + w[1])
    assert res["E0"] - w[0] <= res["residual"] ** 2 / (w[1] - res["E0"]) * (1 + 1e-6) + 1e-13 * abs(w[0])


def test_poor_fp32_phase_costs_only_refinement_steps(ed):
    """Two FP32 steps give a poor psi; the FP64-accurate run from it still reaches the
    oracle's E0, with more steps."""
    E_ref = _golden_E0("lanczos_ring12_3_3_U4.txt")
    w = ed_inputs.workload("ring12_3_3")
    b = ed.ed_build_basis(w["n_sites"], w["bonds"], w["n_up"], w["n_dn"])
    try:
        res = ed.ed_lanczos_solve_mixed(b, 1.0, 4.0, ed.make_opts(max_steps=2, tol=0.0, seed=1, dtype="f32"),
                                        refine_steps=300, refine_tol=1e-13)
    finally:
        ed.ed_basis_destroy(b)
    assert res["steps32"] == 2 and res["steps64"] > 16
    assert abs(res["E0"] - E_ref) <= 1e-10 * abs(E_ref), res


def test_mixed_solve_every_batch_instance(ed):
    """Every instance of the 256-instance batch (lattices, fillings, U of the batched
    workload) through the mixed solve: E0 within 1e-10 of the oracle's."""
    ref = {}
    for line in open(os.path.join(GOLDEN, "batched_E0.txt")):
        f = line.split()
        if f and not f[0].startswith("#"):
            ref[int(f[0])] = float(f[6])
    errs = []
    for i, w in enumerate(ed_inputs.batched_instances()):
        b = ed.ed_build_basis(w["n_sites"], w["bonds"], w["n_up"], w["n_dn"])
        try:
            res = ed.ed_lanczos_solve_mixed(b, w["t"], w["U"], ed.make_opts(max_steps=300, tol=1e-9, seed=4,
                                                                           dtype="f32"),
                                            refine_steps=300, refine_tol=1e-13)
        finally:
            ed.ed_basis_destroy(b)
        errs.append(abs(res["E0"] - ref[i]) / max(1.0, abs(ref[i])))
    assert max(errs) <= 1e-10, (int(np.argmax(errs)), max(errs))


def test_mixed_solve_rejects_other_dtypes(ed):
    b = ed.ed_build_basis(4, ed_inputs.ring_bonds(4), 2, 2)
    try:
        with pytest.raises(ed.EdError):
            ed.ed_lanczos_solve_mixed(b, 1.0, 1.0, ed.make_opts(max_steps=10, dtype="f64"))
        with pytest.raises(ed.EdError):
            ed.ed_lanczos_solve_mixed(b, 1.0, 1.0, ed.make_opts(max_steps=10, dtype="f32"), refine_steps=0)
    finally:
        ed.ed_basis_destroy(b)
