"""Ground-state observables from a state vector: double occupancy.

The on-site term of the model (Sec. 1, Eq. 1 extended by the interaction the paper adds,
reading R6: U sum_i n_i,up n_i,dn) counts doubly occupied sites, so

    D_i = <psi| n_i,up n_i,dn |psi> / <psi|psi>,      D = sum_i D_i = dE0/dU

(the last equality by Hellmann-Feynman, since dH/dU = sum_i n_i,up n_i,dn for a
normalised, non-degenerate ground state). psi is indexed as in Sec. 4, Eqs. 5-6: global
index = rank_up * dim_dn + rank_dn.

TEST INFRASTRUCTURE ONLY (see the package header).
"""
from __future__ import annotations

import numpy as np

from .basis import species_states


def double_occupancy(n_sites: int, n_up: int, n_dn: int, psi: np.ndarray):
    """(D, [D_0 .. D_{L-1}]) in FP64 for the state psi (any normalisation)."""
    up = species_states(n_sites, n_up)
    dn = species_states(n_sites, n_dn)
    p2 = np.asarray(psi, dtype=np.float64).reshape(len(up), len(dn)) ** 2
    norm2 = float(p2.sum())
    per_site = np.zeros(n_sites)
    for i in range(n_sites):
        occ_up = ((up >> np.uint32(i)) & np.uint32(1)).astype(np.float64)
        occ_dn = ((dn >> np.uint32(i)) & np.uint32(1)).astype(np.float64)
        per_site[i] = float(occ_up @ p2 @ occ_dn) / norm2
    return float(per_site.sum()), per_site
