"""The Hamiltonian in the fixed-(N_up, N_dn) basis, from its second-quantised definition.

H = -t * sum_<ij> sum_sigma (c+_{i sigma} c_{j sigma} + h.c.)      (Sec. 1, Eq. 1)
    + U * sum_i n_{i up} n_{i dn}                                    (Sec. 1, on-site term)

Readings where the paper is silent (it defers the construction to its Ref. [Siro 2012]):
  * <ij> runs over an explicit bond list; a pair listed twice gets both hoppings (they add).
  * Global index of the pair (up state, down state) = rank_up * dim_dn + rank_dn: the vector
    is dim_up sub-vectors of length dim_dn with the up configuration fixed inside each
    (Sec. 4, Eqs. 5-6 and the indexing of Algorithm 2).
  * Fermion sign: creation operators ordered by ascending site within a species, all up
    operators before all down operators. Then c+_i c_j (one of i, j occupied, the other
    empty) gives (-1)^(number of same-species particles strictly between i and j); the
    other species contributes no sign because the hopping bilinear is parity-even.
  * Matrix element: <s'| H |s> = -t * sign for the hopped state s' (real t).
  * The interaction is U * (number of doubly occupied sites): diagonal in this basis
    (Sec. 1: "such interaction terms are diagonal").

Everything here is built state by state from these rules in FP64; nothing uses the
tensor-product split of Eq. 3 (tests check that split as a property of the result).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from .basis import popcount, rank_of, species_states


def _between_mask(i: int, j: int) -> int:
    lo, hi = min(i, j), max(i, j)
    return ((1 << hi) - 1) & ~((1 << (lo + 1)) - 1)


def hops_of(bits: np.ndarray, bonds: np.ndarray):
    """All single-particle hops out of each state in `bits` (one species).

    For every bond (i, j), in bond-list order, and every state with exactly one of the
    sites i, j occupied, the particle moves to the empty end. Yields, per bond,
    (source positions, hopped bit strings, fermion sign +-1).
    """
    bits = np.asarray(bits, dtype=np.int64)
    for (i, j) in np.asarray(bonds).reshape(-1, 2):
        i, j = int(i), int(j)
        if i == j:
            raise ValueError("bond with i == j")
        bi = (bits >> i) & 1
        bj = (bits >> j) & 1
        src = np.nonzero(bi != bj)[0]
        s = bits[src]
        s2 = s ^ ((1 << i) | (1 << j))
        npass = popcount(s & _between_mask(i, j))
        sign = np.where(npass % 2 == 0, 1.0, -1.0)
        yield src, s2, sign


def species_hop_table(n_sites: int, n_particles: int, bonds: np.ndarray):
    """Per-state hop list of one species, in bond-list order.

    Returns (states, lists) where lists[r] is the list of (target rank, sign) pairs of the
    hops out of state r, ordered by bond index. Used to check the device tables entry by
    entry.
    """
    states = species_states(n_sites, n_particles)
    lists = [[] for _ in range(len(states))]
    for src, s2, sign in hops_of(states, bonds):
        tgt = rank_of(states, s2)
        for r, t_, sg in zip(src.tolist(), tgt.tolist(), sign.tolist()):
            lists[r].append((t_, int(sg)))
    return states, lists


def hamiltonian_csr(n_sites, bonds, n_up, n_dn, t, U) -> sp.csr_matrix:
    """Explicit sparse H (FP64, CSR), built by applying Eq. 1 and the on-site term to
    every basis state. Column = source state, row = hopped state; duplicates add."""
    up = species_states(n_sites, n_up)
    dn = species_states(n_sites, n_dn)
    dim_dn = len(dn)
    dim = len(up) * dim_dn
    g = np.arange(dim, dtype=np.int64)
    ub = up[g // dim_dn]
    db = dn[g % dim_dn]
    rows, cols, vals = [], [], []
    # hopping of up particles: the down configuration is untouched
    for src, s2, sign in hops_of(ub, bonds):
        tgt = rank_of(up, s2) * dim_dn + (src % dim_dn)
        rows.append(tgt); cols.append(src); vals.append(-t * sign)
    # hopping of down particles: the up configuration is untouched
    for src, s2, sign in hops_of(db, bonds):
        tgt = (src // dim_dn) * dim_dn + rank_of(dn, s2)
        rows.append(tgt); cols.append(src); vals.append(-t * sign)
    # on-site interaction: U times the number of doubly occupied sites
    diag = U * popcount(ub & db).astype(np.float64)
    rows.append(g); cols.append(g); vals.append(diag)
    H = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                      shape=(dim, dim)).tocsr()
    H.sum_duplicates()
    return H


def hv_rows(n_sites, bonds, n_up, n_dn, t, U, x: np.ndarray, rows: np.ndarray) -> np.ndarray:
    """(H x)[g] for the global indices `rows` only, without forming H.

    Row g of H is found from the hops out of state g: the states that hop into g are
    exactly those reached from g by one hop, with the same sign and amplitude (the hop
    is reversible and the sites between its ends do not change). Each output is summed
    in plain FP64, diagonal first, then up hops and down hops in bond order.
    """
    up = species_states(n_sites, n_up)
    dn = species_states(n_sites, n_dn)
    dim_dn = len(dn)
    rows = np.asarray(rows, dtype=np.int64)
    ub = up[rows // dim_dn]
    db = dn[rows % dim_dn]
    y = U * popcount(ub & db).astype(np.float64) * x[rows]
    for src, s2, sign in hops_of(ub, bonds):
        col = rank_of(up, s2) * dim_dn + (rows[src] % dim_dn)
        np.add.at(y, src, -t * sign * x[col])
    for src, s2, sign in hops_of(db, bonds):
        col = (rows[src] // dim_dn) * dim_dn + rank_of(dn, s2)
        np.add.at(y, src, -t * sign * x[col])
    return y


def hv_abs_rows(n_sites, bonds, n_up, n_dn, t, U, x: np.ndarray, rows: np.ndarray) -> np.ndarray:
    """(|H| |x|)[g] for the rows `rows`: the scale of a floating-point error bound."""
    up = species_states(n_sites, n_up)
    dn = species_states(n_sites, n_dn)
    dim_dn = len(dn)
    rows = np.asarray(rows, dtype=np.int64)
    ub = up[rows // dim_dn]
    db = dn[rows % dim_dn]
    ax = np.abs(x)
    y = abs(U) * popcount(ub & db).astype(np.float64) * ax[rows]
    for src, s2, _ in hops_of(ub, bonds):
        col = rank_of(up, s2) * dim_dn + (rows[src] % dim_dn)
        np.add.at(y, src, abs(t) * ax[col])
    for src, s2, _ in hops_of(db, bonds):
        col = (rows[src] // dim_dn) * dim_dn + rank_of(dn, s2)
        np.add.at(y, src, abs(t) * ax[col])
    return y
