"""Seeded synthetic inputs shared by the oracle tests, the GPU tests and the benchmark.

This module holds no arithmetic of the method (no Hamiltonian, no Lanczos): only the
problem descriptions (bond lists of the lattices the paper studies, Sec. 2.1) and the
random numbers the method draws (the random unit start vector of Algorithm 1, Sec. 2.2).

Random numbers come from SplitMix64 (Steele, Lea & Flood, "Fast splittable pseudorandom
number generators", OOPSLA 2014), used counter-style: element i is the (i+1)-th output of
the generator seeded with `seed`. The CUDA library implements the same published
generator independently for its device-side start vector.
"""
from __future__ import annotations

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_MIX1 = np.uint64(0xBF58476D1CE4E5B9)
_MIX2 = np.uint64(0x94D049BB133111EB)


# --------------------------------------------------------------------------- lattices
def ring_bonds(L: int) -> np.ndarray:
    """Periodic 1D ring (Sec. 2.1, Fig. 1 top): bonds (i, i+1 mod L).

    Periodic boundaries are always used (Sec. 2.1). For L == 2 both bonds join the same
    pair, so the pair appears twice and its hoppings add; L == 1 has no bond.
    """
    if L < 2:
        return np.zeros((0, 2), dtype=np.int32)
    return np.array([(i, (i + 1) % L) for i in range(L)], dtype=np.int32)


def torus_bonds(Lx: int, Ly: int) -> np.ndarray:
    """Periodic Lx x Ly square lattice, site index x + Lx*y, nearest-neighbour bonds.

    Every site emits a bond to its +x neighbour when Lx >= 2 and to its +y neighbour
    when Ly >= 2, with periodic wrap (Sec. 2.1). An extent-2 direction therefore lists
    each pair twice (the hoppings add), an extent-1 direction lists nothing.
    """
    out = []
    for y in range(Ly):
        for x in range(Lx):
            s = x + Lx * y
            if Lx >= 2:
                out.append((s, (x + 1) % Lx + Lx * y))
            if Ly >= 2:
                out.append((s, x + Lx * ((y + 1) % Ly)))
    return np.array(out, dtype=np.int32).reshape(-1, 2)


# --------------------------------------------------------------------------- SplitMix64
def splitmix64(seed: int, n: int, offset: int = 0) -> np.ndarray:
    """Outputs offset+1 .. offset+n of SplitMix64 seeded with `seed`, as uint64."""
    with np.errstate(over="ignore"):
        k = np.arange(offset + 1, offset + n + 1, dtype=np.uint64)
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + k * _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _MIX1
        z = (z ^ (z >> np.uint64(27))) * _MIX2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform_pm1(seed: int, n: int, offset: int = 0) -> np.ndarray:
    """uniform[-1, 1) doubles: 2 * (top 53 bits * 2^-53) - 1, exact in FP64."""
    z = splitmix64(seed, n, offset)
    u = (z >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)
    return 2.0 * u - 1.0


def checkerboard_lattice(Lx: int, Ly: int, phi: float = np.pi / 4, t2: float = 0.3,
                         t3: float = -0.2):
    """A checkerboard-type periodic Lx x Ly lattice with complex nearest-neighbour hoppings
    (the paper's second geometry, Sec. 2.1 Fig. 1, whose amplitudes it does not print; these
    are synthetic stand-ins): site x + Lx y, sublattice A where x + y is even.
      * nearest neighbours (+x, +y): relative amplitude exp(+-i phi), the sign of the phase
        set by the sublattice of the first site and flipped between x and y bonds;
      * next-nearest (the two diagonals): real +-t2, alternating with the sublattice;
      * third neighbours (+2x, +2y): real t3 (on a 4-wide axis the two neighbours at +-2
        coincide; that pair is listed once).
    Returns (bonds [n_bonds][2], complex amplitudes [n_bonds])."""
    bonds, amp = [], []
    def site(x, y):
        return (x % Lx) + Lx * (y % Ly)
    for y in range(Ly):
        for x in range(Lx):
            s, a = site(x, y), (x + y) % 2 == 0
            bonds.append((s, site(x + 1, y))); amp.append(np.exp(1j * phi * (1 if a else -1)))
            bonds.append((s, site(x, y + 1))); amp.append(np.exp(1j * phi * (-1 if a else 1)))
            bonds.append((s, site(x + 1, y + 1))); amp.append(t2 if a else -t2)
            bonds.append((s, site(x + 1, y - 1))); amp.append(-t2 if a else t2)
            if Lx != 4 or x < 2:
                bonds.append((s, site(x + 2, y))); amp.append(t3)
            if Ly != 4 or y < 2:
                bonds.append((s, site(x, y + 2))); amp.append(t3)
    return np.array(bonds, dtype=np.int32), np.array(amp, dtype=np.complex128)


def start_vector_raw(seed: int, dim: int) -> np.ndarray:
    """The un-normalised random start vector (Algorithm 1 requires norm 1; each side
    normalises it itself)."""
    return uniform_pm1(seed, dim)


# --------------------------------------------------------------------------- workloads
def workload(name: str) -> dict:
    """The synthetic workloads: lattice, fillings, t, U, dtype, seed."""
    if name == "ring12_3_3":      # L=12 ring, 3/3, dim 220^2, FP64, U in {0, 4}
        return dict(n_sites=12, bonds=ring_bonds(12), n_up=3, n_dn=3, t=1.0, U=4.0,
                    dtype="f64", seed=1)
    if name == "torus4x4_5_5":    # 4x4 periodic, 5/5, dim 4368^2, FP64, U=4
        return dict(n_sites=16, bonds=torus_bonds(4, 4), n_up=5, n_dn=5, t=1.0, U=4.0,
                    dtype="f64", seed=2)
    if name == "ring16_8_8":      # L=16 ring, half filling, dim 12870^2, U=4
        return dict(n_sites=16, bonds=ring_bonds(16), n_up=8, n_dn=8, t=1.0, U=4.0,
                    dtype="f32", seed=3)
    if name == "ring14_7_7":      # L=14 ring, 7/7, dim 3432^2 (learned start)
        return dict(n_sites=14, bonds=ring_bonds(14), n_up=7, n_dn=7, t=1.0, U=4.0,
                    dtype="f32", seed=5)
    if name == "ring26_13_0":     # L=26 ring, 13 particles of one spin, dim 10,400,600
        return dict(n_sites=26, bonds=ring_bonds(26), n_up=13, n_dn=0, t=1.0, U=4.0,
                    dtype="f64", seed=7)
    if name == "checker4x4_5_5":  # checkerboard-type 4x4, complex NN hoppings, dim 4368^2
        bonds, amp = checkerboard_lattice(4, 4)
        return dict(n_sites=16, bonds=bonds, t_bond=amp, n_up=5, n_dn=5, t=1.0, U=4.0,
                    dtype="c64", seed=8)
    if name == "ring18_3_9":      # L=18 ring, 3 up, 9 down: the 18-site rows at 39.7 M states
        return dict(n_sites=18, bonds=ring_bonds(18), n_up=3, n_dn=9, t=1.0, U=4.0,
                    dtype="f32", seed=6)
    if name == "ring18_9_9":      # L=18 ring, half filling, dim 48620^2 = 2.36e9, FP32
        return dict(n_sites=18, bonds=ring_bonds(18), n_up=9, n_dn=9, t=1.0, U=4.0,
                    dtype="f32", seed=6)
    raise KeyError(name)


def batched_instances(seed: int = 4, count: int = 256) -> list[dict]:
    """Draws `count` (lattice, filling, U) instances: lattices uniform over rings
    L = 8..12 and periodic 2x4 / 3x4 rectangles, N_up, N_dn uniform in [1, L/2],
    U uniform[0, 8), t = 1. Deterministic in `seed` (SplitMix64 stream)."""
    kinds = [("ring", L) for L in range(8, 13)] + [("rect", (2, 4)), ("rect", (3, 4))]
    r = splitmix64(seed, 4 * count)
    out = []
    for m in range(count):
        z0, z1, z2, z3 = (int(v) for v in r[4 * m:4 * m + 4])
        kind, geo = kinds[z0 % len(kinds)]
        if kind == "ring":
            L = geo
            bonds = ring_bonds(L)
            name = f"ring{L}"
        else:
            L = geo[0] * geo[1]
            bonds = torus_bonds(*geo)
            name = f"rect{geo[0]}x{geo[1]}"
        half = L // 2
        n_up = 1 + z1 % half
        n_dn = 1 + z2 % half
        U = 8.0 * ((z3 >> 11) * 2.0 ** -53)
        out.append(dict(name=name, n_sites=L, bonds=bonds, n_up=n_up, n_dn=n_dn,
                        t=1.0, U=U))
    return out


def random_lattices(seed: int = 7, count: int = 6) -> list[dict]:
    """Irregular bond lists for robustness tests of the row-staged H.v: L uniform in 10..12
    sites, L..2L random pairs (i != j; pairs may repeat, in either order) plus the first pair
    listed once more and the second reversed; N_up uniform in [3, L - 3] (at least 120 up
    states), N_dn uniform over the fillings in [1, L - 1] with C(L, N_up) C(L, N_dn) <=
    400,000; U uniform in [-2, 8), t = 1. Lattice m draws from the SplitMix64 stream seeded
    seed * 1000 + m."""
    from math import comb
    out = []
    for m in range(count):
        r = iter(int(v) for v in splitmix64(seed * 1000 + m, 256))
        L = 10 + next(r) % 3
        nb = L + next(r) % (L + 1)
        bonds = []
        while len(bonds) < nb:
            i, j = next(r) % L, next(r) % L
            if i != j:
                bonds.append((i, j))
        bonds += [bonds[0], bonds[1][::-1]]
        n_up = 3 + next(r) % (L - 5)
        fits = [n for n in range(1, L) if comb(L, n_up) * comb(L, n) <= 400_000]
        n_dn = fits[next(r) % len(fits)]
        U = -2.0 + 10.0 * ((next(r) >> 11) * 2.0 ** -53)
        out.append(dict(name=f"random{m}_L{L}_{n_up}_{n_dn}", n_sites=L,
                        bonds=np.array(bonds, dtype=np.int64), n_up=n_up, n_dn=n_dn,
                        t=1.0, U=U))
    return out


def heldout_U(seed: int = 5, count: int = 16) -> np.ndarray:
    """Held-out interaction strengths uniform[0, 8) for the learned-start evaluation."""
    return 8.0 * (splitmix64(seed ^ 0x5555, count) >> np.uint64(11)).astype(np.float64) * 2.0 ** -53
