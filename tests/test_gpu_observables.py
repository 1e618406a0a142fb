"""Double occupancy of the ground-state vector (ed_double_occupancy) against the oracle on
the same vector, against dense ground states, against Hellmann-Feynman (dE0/dU from
Lanczos energies at U +- h) and against closed forms."""
import math

import numpy as np
import pytest

import ed_inputs
from oracle import dense, observables

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ed():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1511_00863_gb300 as m
    return m


def _ground_state(ed, b, U, tol=1e-13):
    dim = ed.ed_basis_dims(b)[2]
    psi = torch.empty(dim, dtype=torch.float64, device="cuda")
    res = ed.ed_lanczos_ground_state(b, 1.0, U, ed.make_opts(max_steps=600, tol=tol, seed=3), psi)
    return psi, res["E0"]


@pytest.mark.parametrize("case", [
    (8, ed_inputs.ring_bonds(8), 3, 3, 4.0),
    (8, ed_inputs.torus_bonds(2, 4), 1, 3, 5.0),
    (6, ed_inputs.ring_bonds(6), 3, 3, 3.0),
])
def test_vs_oracle_and_dense(ed, case):
    L, bonds, nu, nd, U = case
    b = ed.ed_build_basis(L, bonds, nu, nd)
    try:
        psi, E0 = _ground_state(ed, b, U)
        D, site = ed.ed_double_occupancy(b, psi)
    finally:
        ed.ed_basis_destroy(b)
    p = psi.cpu().numpy()
    # the kernel on this vector vs the oracle on the same vector
    Dr, site_r = observables.double_occupancy(L, nu, nd, p)
    assert abs(D - Dr) <= 1e-13 * max(1.0, Dr)
    assert np.allclose(site, site_r, rtol=1e-13, atol=1e-15)
    # the whole pipeline vs the dense ground state
    Ed, pd = dense.ground_state(L, bonds, nu, nd, 1.0, U)
    Dd, _ = observables.double_occupancy(L, nu, nd, pd)
    assert abs(D - Dd) <= 1e-8 * max(1.0, Dd), (D, Dd)


@pytest.mark.parametrize("U", [0.0, 2.0, 8.0])
def test_two_site_closed_form(ed, U):
    b = ed.ed_build_basis(2, np.array([[0, 1]]), 1, 1)
    try:
        psi, _ = _ground_state(ed, b, U)
        D, site = ed.ed_double_occupancy(b, psi)
    finally:
        ed.ed_basis_destroy(b)
    assert abs(D - 0.5 * (1.0 - U / math.sqrt(U * U + 16.0))) <= 1e-12
    assert abs(site[0] - site[1]) <= 1e-12


@pytest.mark.parametrize("name,U,h,tol", [
    ("ring12_3_3", 4.0, 1e-3, 2e-6),
    ("torus4x4_5_5", 4.0, 1e-3, 2e-6),
])
def test_hellmann_feynman_full_size(ed, name, U, h, tol):
    w = ed_inputs.workload(name)
    b = ed.ed_build_basis(w["n_sites"], w["bonds"], w["n_up"], w["n_dn"])
    try:
        psi, _ = _ground_state(ed, b, U)
        D, site = ed.ed_double_occupancy(b, psi)
        o = ed.make_opts(max_steps=600, tol=1e-13, seed=3)
        Ep = ed.ed_lanczos_solve(b, 1.0, U + h, o)["E0"]
        Em = ed.ed_lanczos_solve(b, 1.0, U - h, o)["E0"]
    finally:
        ed.ed_basis_destroy(b)
    dE = (Ep - Em) / (2 * h)
    assert abs(dE - D) <= tol * max(1.0, abs(D)), (dE, D)
    # translation-invariant lattice, non-degenerate ground state: the same D_i on every site
    # (to first order in the eigenvector error, ~1e-7 here)
    assert np.allclose(site, D / w["n_sites"], rtol=2e-6)


def test_U0_closed_shell_ring(ed):
    # free fermions, closed shells: D_i = (N/L)^2 on every site (to first order in the
    # eigenvector error: E0 converged to 1e-13 leaves psi accurate to ~1e-8)
    L, n = 12, 3
    b = ed.ed_build_basis(L, ed_inputs.ring_bonds(L), n, n)
    try:
        psi, _ = _ground_state(ed, b, 0.0)
        D, site = ed.ed_double_occupancy(b, psi)
    finally:
        ed.ed_basis_destroy(b)
    assert np.allclose(site, (n / L) ** 2, rtol=1e-7, atol=0.0)
    assert abs(D - n * n / L) <= 1e-7 * (n * n / L)


def test_zero_vector_is_an_argument_error(ed):
    b = ed.ed_build_basis(4, ed_inputs.ring_bonds(4), 2, 2)
    try:
        psi = torch.zeros(ed.ed_basis_dims(b)[2], dtype=torch.float64, device="cuda")
        with pytest.raises(ed.EdError) as ei:
            ed.ed_double_occupancy(b, psi)
        assert ei.value.status == ed.ED_ERR_ARG
    finally:
        ed.ed_basis_destroy(b)
