"""Ground-state energy of the periodic Hubbard ring from the Lieb-Wu Bethe-ansatz equations.

TEST INFRASTRUCTURE ONLY (an independent pin of the full-size ring workloads, whose basis is
too large for the oracle's explicit matrix). The paper itself computes E0 numerically with
Algorithm 1 (Sec. 2.2); this module gives the same quantity for the 1D ring (Sec. 2.1,
Fig. 1 top: periodic chain, nearest-neighbour hopping, plus the on-site U term of Sec. 1)
by an exact method of its own (E. H. Lieb and F. Y. Wu, Phys. Rev. Lett. 20, 1445 (1968);
the finite-ring form with periodic boundary conditions for fermions as in Essler et al.,
"The One-Dimensional Hubbard Model", Cambridge 2005, Ch. 3).

For N electrons of which M have spin down on an L-site ring, H = -t sum (c+c + h.c.) +
U sum n_up n_dn, the eigenstates of the regular Bethe ansatz carry charge momenta k_j
(j = 1..N) and spin rapidities lambda_a (a = 1..M) obeying, with u = U / (4t) > 0,

    L k_j = 2 pi I_j - sum_a theta((sin k_j - lambda_a) / u)
    sum_j theta((lambda_a - sin k_j) / u) = 2 pi J_a + sum_b theta((lambda_a - lambda_b) / (2u))

where theta(x) = 2 arctan(x), and E = -2t sum_j cos k_j. Taking logarithms of the product
form fixes the parity of the quantum numbers: I_j is an integer when M is even and a
half-odd integer when M is odd; J_a is an integer when N - M is odd and a half-odd integer
when N - M is even. The lowest state with M rapidities takes both sets consecutive and as
centred as their parity allows (where the centred set has the other parity, the two
choices one half to either side are mirror images, k -> -k, with the same energy; at half
filling they differ by L, the same momenta modulo 2 pi).

Reading (the paper is silent; it uses periodic boundaries, Sec. 2.1): the fermion sign of
the oracle's Hamiltonian (creation operators in ascending site order) makes the hop across
the ring's closing bond carry (-1)^(N_sigma - 1) relative to an open chain, i.e. the
Hamiltonian is exactly the periodic fermion ring these equations describe.

Solved by Newton's method on the N + M logarithmic equations (analytic Jacobian, dense
numpy linear solves), continued in u from a large value, where the charge momenta are close
to 2 pi I_j / L, down to the requested one.
"""
from __future__ import annotations

import numpy as np


def _theta(x):
    return 2.0 * np.arctan(x)


def _dtheta(x):
    return 2.0 / (1.0 + x * x)


def ground_state_numbers(L: int, N: int, M: int):
    """Quantum numbers (I_j, J_a) of the repulsive ground state."""
    if not (0 <= M <= N <= 2 * L and N - M <= L and M <= L):
        raise ValueError("need 0 <= M <= N, N - M <= L, M <= L")
    shift_I = 0.0 if M % 2 == 0 else 0.5
    shift_J = 0.0 if (N - M) % 2 == 1 else 0.5
    # n consecutive numbers of the given parity, as centred as possible (the lower of the
    # two centred choices when the centred set has the other parity)
    def centred(n, shift):
        q = np.arange(n, dtype=np.float64) - (n - 1) / 2.0
        if n and (q[0] - shift) % 1.0 != 0.0:
            q = q - 0.5
        return q
    return centred(N, shift_I), centred(M, shift_J)


def _residual(v, L, N, M, u, I, J):
    k, lam = v[:N], v[N:]
    sk = np.sin(k)
    r1 = L * k - 2 * np.pi * I + _theta((sk[:, None] - lam[None, :]) / u).sum(axis=1)
    r2 = (_theta((lam[:, None] - sk[None, :]) / u).sum(axis=1) - 2 * np.pi * J
          - _theta((lam[:, None] - lam[None, :]) / (2 * u)).sum(axis=1))
    return np.concatenate([r1, r2])


def _jacobian(v, L, N, M, u):
    k, lam = v[:N], v[N:]
    sk, ck = np.sin(k), np.cos(k)
    a = _dtheta((sk[:, None] - lam[None, :]) / u) / u           # N x M
    b = _dtheta((lam[:, None] - sk[None, :]) / u) / u           # M x N
    c = _dtheta((lam[:, None] - lam[None, :]) / (2 * u)) / (2 * u)  # M x M
    Jm = np.zeros((N + M, N + M))
    Jm[np.arange(N), np.arange(N)] = L + ck * a.sum(axis=1)
    Jm[:N, N:] = -a
    Jm[N:, :N] = -b * ck[None, :]
    Jm[N + np.arange(M), N + np.arange(M)] = b.sum(axis=1) - c.sum(axis=1) + np.diag(c)
    Jm[N:, N:] += c - np.diag(np.diag(c))
    return Jm


def _newton(v, L, N, M, u, I, J, iters=200):
    for _ in range(iters):
        r = _residual(v, L, N, M, u, I, J)
        dv = np.linalg.solve(_jacobian(v, L, N, M, u), -r)
        step = 1.0
        rn = np.linalg.norm(r)
        while step > 1e-6:   # damped step: accept the first that does not increase |r|
            v2 = v + step * dv
            if np.linalg.norm(_residual(v2, L, N, M, u, I, J)) <= rn * (1 - 1e-4 * step) or rn < 1e-13:
                break
            step *= 0.5
        v = v2
        if np.max(np.abs(step * dv)) < 1e-15 and np.linalg.norm(_residual(v, L, N, M, u, I, J)) < 1e-11:
            break
    return v


def solve(L: int, N: int, M: int, U: float, t: float = 1.0):
    """(E0, k, lambda, max residual) of the repulsive ground state (U > 0)."""
    if U <= 0:
        raise ValueError("the regular ground-state solution used here needs U > 0")
    I, J = ground_state_numbers(L, N, M)
    u_target = U / (4.0 * t)
    # start where the spin rapidities decouple from a free-fermion-like charge sector:
    # large u, k_j = 2 pi I_j / L, lambda from the u -> infinity limit (Heisenberg-like
    # equations with sin k -> 0 replaced by iterating the second equation)
    u = max(8.0, 2.0 * u_target)
    k = 2 * np.pi * I / L
    lam = np.zeros(M)
    for _ in range(200 if M else 0):   # fixed point of the second equation at fixed k
        rhs = 2 * np.pi * J + _theta((lam[:, None] - lam[None, :]) / (2 * u)).sum(axis=1)
        # invert sum_j theta((lam - sin k_j)/u) = rhs for each lam by bisection
        lo, hi = np.full(M, -1e6), np.full(M, 1e6)
        for _ in range(200):
            mid = 0.5 * (lo + hi)
            f = _theta((mid[:, None] - np.sin(k)[None, :]) / u).sum(axis=1) - rhs
            lo = np.where(f < 0, mid, lo)
            hi = np.where(f >= 0, mid, hi)
        lam_new = 0.5 * (lo + hi)
        if np.max(np.abs(lam_new - lam)) < 1e-14:
            lam = lam_new
            break
        lam = lam_new
    v = np.concatenate([k, lam])
    us = np.geomspace(u, u_target, 40) if u != u_target else [u_target]
    for uu in us:
        v = _newton(v, L, N, M, uu, I, J)
    res = np.max(np.abs(_residual(v, L, N, M, u_target, I, J)))
    k, lam = v[:N], v[N:]
    return float(-2.0 * t * np.sum(np.cos(k))), k, lam, float(res)


def ring_ground_energy(L: int, n_up: int, n_dn: int, U: float, t: float = 1.0,
                       spins=None) -> float:
    """E0 of the periodic L-site Hubbard ring with n_up, n_dn electrons (U > 0).

    A Bethe state with M spin rapidities is the highest-weight member of a spin multiplet
    with S = N/2 - M; the sector (n_up, n_dn) holds every multiplet with S >= |n_up - n_dn|/2,
    i.e. every M' <= min(n_up, n_dn). E0 is the lowest of those ground energies (away from
    half filling an open-shell ring can have a ground state of higher spin). `spins`
    restricts the M' searched (None = all)."""
    N = n_up + n_dn
    cands = range(min(n_up, n_dn) + 1) if spins is None else spins
    best = None
    for M in cands:
        E, _, _, res = solve(L, N, M, U, t)
        if res > 1e-9:
            raise RuntimeError(f"Bethe equations not solved (M = {M}, residual {res:g})")
        best = E if best is None else min(best, E)
    return best
