"""Pins of the oracle's complex-hopping Hamiltonian (oracle/complex_hopping.py): Hermiticity,
the real limit, free fermions through the single-particle matrix, the flux-threaded ring's
closed form, gauge invariance, complex conjugation, and the real-view Lanczos against dense
diagonalisation."""
import math

import numpy as np
import pytest

import ed_inputs
from oracle import complex_hopping as ch
from oracle import hamiltonian, lanczos as olz


def _rand_tb(nb, seed):
    r = np.random.default_rng(seed)
    return r.uniform(0.5, 1.5, nb) * np.exp(1j * r.uniform(-math.pi, math.pi, nb))


CASES = [
    (6, ed_inputs.ring_bonds(6), 3, 2),
    (8, ed_inputs.torus_bonds(2, 4), 2, 3),
    (7, np.array([[0, 1], [1, 2], [2, 3], [3, 4], [4, 5], [5, 6], [6, 0], [0, 3], [2, 5], [1, 4]]), 3, 3),
]


@pytest.mark.parametrize("case", CASES)
def test_hermitian(case):
    L, bonds, nu, nd = case
    H = ch.hamiltonian_csr_complex(L, bonds, _rand_tb(len(bonds), 1), nu, nd, 1.0, 2.5)
    assert abs(H - H.getH()).max() <= 1e-15


@pytest.mark.parametrize("case", CASES)
def test_real_limit_is_the_real_hamiltonian(case):
    L, bonds, nu, nd = case
    Hc = ch.hamiltonian_csr_complex(L, bonds, np.ones(len(bonds)), nu, nd, 0.7, 3.0)
    Hr = hamiltonian.hamiltonian_csr(L, bonds, nu, nd, 0.7, 3.0)
    assert abs(Hc - Hr).max() == 0.0


@pytest.mark.parametrize("case", CASES)
def test_free_fermions_from_single_particle_matrix(case):
    L, bonds, nu, nd = case
    tb = _rand_tb(len(bonds), 2)
    H = ch.hamiltonian_csr_complex(L, bonds, tb, nu, nd, 1.0, 0.0).toarray()
    assert abs(np.linalg.eigvalsh(H)[0] - ch.u0_energy(L, bonds, tb, nu, nd, 1.0)) <= 1e-12


@pytest.mark.parametrize("L,n,phi", [(7, 3, 0.3), (8, 3, 1.1), (6, 2, -0.7)])
def test_flux_ring_closed_form(L, n, phi):
    # tau = t e^{i phi} on every bond (i, i+1): single-particle levels -2t cos(2 pi m / L + phi)
    e = np.sort(-2.0 * np.cos(2 * np.pi * np.arange(L) / L + phi))
    tb = np.full(L, np.exp(1j * phi))
    h = ch.single_particle_matrix(L, ed_inputs.ring_bonds(L), tb, 1.0)
    assert np.allclose(np.linalg.eigvalsh(h), e, atol=1e-13)
    H = ch.hamiltonian_csr_complex(L, ed_inputs.ring_bonds(L), tb, n, n, 1.0, 0.0).toarray()
    assert abs(np.linalg.eigvalsh(H)[0] - 2 * e[:n].sum()) <= 1e-12


@pytest.mark.parametrize("case", CASES)
def test_gauge_and_conjugation_invariance(case):
    L, bonds, nu, nd = case
    tb = _rand_tb(len(bonds), 3)
    theta = np.random.default_rng(4).uniform(-math.pi, math.pi, L)
    b = np.asarray(bonds)
    tg = tb * np.exp(1j * (theta[b[:, 0]] - theta[b[:, 1]]))
    w = np.linalg.eigvalsh(ch.hamiltonian_csr_complex(L, bonds, tb, nu, nd, 1.0, 2.0).toarray())
    wg = np.linalg.eigvalsh(ch.hamiltonian_csr_complex(L, bonds, tg, nu, nd, 1.0, 2.0).toarray())
    wc = np.linalg.eigvalsh(ch.hamiltonian_csr_complex(L, bonds, np.conj(tb), nu, nd, 1.0, 2.0).toarray())
    assert np.allclose(w, wg, atol=1e-11) and np.allclose(w, wc, atol=1e-11)


def test_real_view_lanczos_reaches_dense_ground_state():
    L, bonds, nu, nd = CASES[2]
    tb = _rand_tb(len(bonds), 5)
    H = ch.hamiltonian_csr_complex(L, bonds, tb, nu, nd, 1.0, 3.0)
    E = np.linalg.eigvalsh(H.toarray())[0]
    f1 = olz.normalized_start(ed_inputs.start_vector_raw(9, 2 * H.shape[0]))
    res = olz.lanczos(ch.real_view_matvec(H), f1, max_steps=300, tol=1e-14)
    assert abs(res.E0 - E) <= 1e-10 * abs(E)


@pytest.mark.parametrize("case", CASES)
def test_matrix_free_rows_match_the_matrix(case):
    L, bonds, nu, nd = case
    tb = _rand_tb(len(bonds), 6)
    H = ch.hamiltonian_csr_complex(L, bonds, tb, nu, nd, 0.9, 1.7)
    r = np.random.default_rng(7)
    x = r.normal(size=H.shape[0]) + 1j * r.normal(size=H.shape[0])
    rows = np.arange(H.shape[0])
    assert np.allclose(ch.hv_rows_complex(L, bonds, tb, nu, nd, 0.9, 1.7, x, rows), H @ x, atol=1e-13)


@pytest.mark.parametrize("species", ["up", "down"])
def test_one_particle_sector_is_the_hopping_matrix(species):
    """With one particle in the lattice the many-body basis is the site basis (state 1 << s
    has rank s) and no fermion sign arises, so H is the first-quantised matrix of the model:
    bond b = (i, j) moves the particle from j to i with amplitude -t tau_b (row i, column j)
    and back with -t conj(tau_b). This fixes which end of a bond gets tau and which its
    conjugate, a convention every spectrum is blind to (conjugating all tau leaves the
    spectrum unchanged)."""
    L, bonds = 7, CASES[2][1]
    tb = _rand_tb(len(bonds), 8)
    t = 0.8
    nu, nd = (1, 0) if species == "up" else (0, 1)
    H = ch.hamiltonian_csr_complex(L, bonds, tb, nu, nd, t, 5.0).toarray()
    h = np.zeros((L, L), dtype=complex)
    for (i, j), tau in zip(bonds, tb):
        h[i, j] += -t * tau
        h[j, i] += -t * np.conj(tau)
    assert np.array_equal(H, h)
    assert np.array_equal(ch.single_particle_matrix(L, bonds, tb, t), h)
    x = np.random.default_rng(9).normal(size=L) + 1j
    assert np.allclose(ch.hv_rows_complex(L, bonds, tb, nu, nd, t, 5.0, x, np.arange(L)), h @ x,
                       rtol=0, atol=1e-14)
