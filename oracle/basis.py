"""Single-species occupation-number basis (Sec. 2.1).

A single-species basis state is an integer whose set bits are the occupied sites
(Sec. 2.1, after Eq. 3); bit i is site i. The paper leaves the order of the basis to
its Ref. [Siro 2012]; the reading used here is ascending integer value, and the rank of
a state is its position in that ascending list (found by binary search, deliberately not
by any closed formula). The two-species dimension is C(Ns, N_up) * C(Ns, N_dn) (Eq. 2).
"""
from __future__ import annotations

import itertools

import numpy as np

_POP8 = np.array([bin(i).count("1") for i in range(256)], dtype=np.int64)


def popcount(a: np.ndarray) -> np.ndarray:
    """Number of set bits of each element of an integer array (byte table, no tricks)."""
    a = np.asarray(a, dtype=np.uint64)
    out = np.zeros(a.shape, dtype=np.int64)
    for k in range(8):
        out += _POP8[((a >> np.uint64(8 * k)) & np.uint64(0xFF)).astype(np.int64)]
    return out


def species_states(n_sites: int, n_particles: int) -> np.ndarray:
    """All n_sites-bit integers with exactly n_particles set bits, ascending (int64)."""
    if not (0 <= n_particles <= n_sites):
        raise ValueError("need 0 <= n_particles <= n_sites")
    vals = [sum(1 << p for p in c) for c in itertools.combinations(range(n_sites), n_particles)]
    return np.array(sorted(vals), dtype=np.int64)


def rank_of(states: np.ndarray, s: np.ndarray) -> np.ndarray:
    """Position of each s in the ascending list `states` (binary search); raises if absent."""
    s = np.asarray(s, dtype=np.int64)
    r = np.searchsorted(states, s)
    if np.any(r >= len(states)) or np.any(states[np.minimum(r, len(states) - 1)] != s):
        raise ValueError("state not in basis")
    return r


def dimension(n_sites: int, n_up: int, n_dn: int) -> int:
    """dim H = C(Ns, N_up) * C(Ns, N_dn) (Sec. 2.1, Eq. 2), counted by enumeration."""
    return len(species_states(n_sites, n_up)) * len(species_states(n_sites, n_dn))
