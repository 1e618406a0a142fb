"""Dense diagonalisation for small dimensions: the full spectrum of H via LAPACK
(numpy.linalg.eigh). This is the plain definition of the ground-state energy (Sec. 1:
"the lowest eigenvalue, i.e. the ground state energy")."""
from __future__ import annotations

import numpy as np

from .hamiltonian import hamiltonian_csr

MAX_DENSE_DIM = 4000


def spectrum(n_sites, bonds, n_up, n_dn, t, U) -> np.ndarray:
    H = hamiltonian_csr(n_sites, bonds, n_up, n_dn, t, U)
    if H.shape[0] > MAX_DENSE_DIM:
        raise ValueError("dimension too large for dense diagonalisation")
    return np.linalg.eigvalsh(H.toarray())


def ground_state(n_sites, bonds, n_up, n_dn, t, U):
    """(E0, psi0) with the sign gauge: the largest |psi| entry positive (lowest index on
    ties)."""
    H = hamiltonian_csr(n_sites, bonds, n_up, n_dn, t, U)
    if H.shape[0] > MAX_DENSE_DIM:
        raise ValueError("dimension too large for dense diagonalisation")
    w, v = np.linalg.eigh(H.toarray())
    psi = v[:, 0].copy()
    k = int(np.argmax(np.abs(psi)))
    if psi[k] < 0:
        psi = -psi
    return float(w[0]), psi
