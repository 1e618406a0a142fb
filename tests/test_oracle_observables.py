"""Pins of the oracle's double occupancy (oracle/observables.py) against the mathematics:
the two-site closed form, Hellmann-Feynman (dE0/dU from dense energies), the U = 0 product
state on closed-shell rings, and E0 = <H(U=0)> + U D."""
import math

import numpy as np
import pytest

import ed_inputs
from oracle import dense, hamiltonian, observables


@pytest.mark.parametrize("U", [0.0, 1.0, 4.0, 8.0])
def test_two_site_closed_form(U):
    # single bond, N_up = N_dn = 1: E0 = (U - sqrt(U^2 + 16 t^2)) / 2, so
    # D = dE0/dU = (1 - U / sqrt(U^2 + 16 t^2)) / 2
    E0, psi = dense.ground_state(2, np.array([[0, 1]]), 1, 1, 1.0, U)
    D, per_site = observables.double_occupancy(2, 1, 1, psi)
    assert abs(D - 0.5 * (1.0 - U / math.sqrt(U * U + 16.0))) <= 1e-13
    assert abs(per_site[0] - per_site[1]) <= 1e-13


HF_CASES = [
    (6, ed_inputs.ring_bonds(6), 3, 3, 1.0, 3.0),
    (8, ed_inputs.torus_bonds(2, 4), 1, 3, 1.0, 5.0),
    (7, np.array([[0, 1], [1, 2], [2, 3], [3, 4], [4, 5], [5, 6], [6, 0], [0, 3], [2, 5]]), 3, 2, 1.0, 2.0),
]


@pytest.mark.parametrize("case", HF_CASES)
def test_hellmann_feynman(case):
    L, bonds, nu, nd, t, U = case
    w = dense.spectrum(L, bonds, nu, nd, t, U)
    assert w[1] - w[0] > 1e-6   # non-degenerate ground state
    E0, psi = dense.ground_state(L, bonds, nu, nd, t, U)
    D, per_site = observables.double_occupancy(L, nu, nd, psi)
    h = 1e-4
    dE = (dense.spectrum(L, bonds, nu, nd, t, U + h)[0] - dense.spectrum(L, bonds, nu, nd, t, U - h)[0]) / (2 * h)
    assert abs(dE - D) <= 1e-7, (dE, D)
    assert abs(per_site.sum() - D) <= 1e-14
    assert 0.0 <= D <= min(nu, nd)


@pytest.mark.parametrize("case", HF_CASES)
def test_energy_splits_into_kinetic_and_on_site(case):
    L, bonds, nu, nd, t, U = case
    E0, psi = dense.ground_state(L, bonds, nu, nd, t, U)
    D, _ = observables.double_occupancy(L, nu, nd, psi)
    H0 = hamiltonian.hamiltonian_csr(L, bonds, nu, nd, t, 0.0)
    assert abs(float(psi @ (H0 @ psi)) + U * D - E0) <= 1e-12 * max(1.0, abs(E0))


@pytest.mark.parametrize("L,n", [(6, 1), (7, 3), (5, 1)])
def test_U0_closed_shell_ring_is_uniform_product(L, n):
    # at U = 0 the closed-shell ground state is a product of up and down Slater determinants:
    # D_i = <n_i,up><n_i,dn> = (n / L)^2 on every site of the ring
    _, psi = dense.ground_state(L, ed_inputs.ring_bonds(L), n, n, 1.0, 0.0)
    D, per_site = observables.double_occupancy(L, n, n, psi)
    assert np.allclose(per_site, (n / L) ** 2, atol=1e-12)
    assert abs(D - n * n / L) <= 1e-12


def test_normalisation_is_irrelevant():
    _, psi = dense.ground_state(6, ed_inputs.ring_bonds(6), 2, 3, 1.0, 2.0)
    a = observables.double_occupancy(6, 2, 3, psi)
    b = observables.double_occupancy(6, 2, 3, -3.5 * psi)
    assert abs(a[0] - b[0]) <= 1e-14 and np.allclose(a[1], b[1], atol=1e-14)
