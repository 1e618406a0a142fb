"""Algorithm 1 (Sec. 2.2): the Lanczos iteration in FP64, written in the paper's order.

    b_1 = 0, f_0 = 0, f_1 a random vector of norm 1
    for j = 1..m:
        q_j = H f_j - b_j f_{j-1}
        a_j = q_j . f_j
        q_j = q_j - a_j f_j
        b_{j+1} = ||q_j||;  stop if b_{j+1} = 0
        f_{j+1} = q_j / b_{j+1}

Readings where the paper is silent:
  * Full reorthogonalisation (optional, default on): after q_j - a_j f_j, two classical
    Gram-Schmidt passes against every stored f_1..f_j.
  * Convergence: after step j the estimate E0(j) = lambda_min(T_j); stop when
    |E0(j) - E0(j-1)| <= tol * max(|E0(j)|, 1), or after max_steps steps.
  * Breakdown ("if b_{j+1} = 0"): b_{j+1} <= 1e-13 * max(1, max_i(|a_i| + b_i)) over the
    steps so far; then E0 = lambda_min(T_j) is exact for the invariant subspace reached.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from .tridiag import lowest_eigenvalue

BREAKDOWN_REL = 1e-13


@dataclass
class LanczosResult:
    E0: float
    steps: int
    alpha: list = field(default_factory=list)
    beta: list = field(default_factory=list)    # beta[j-1] = b_{j+1}
    E0_history: list = field(default_factory=list)
    breakdown: bool = False
    converged: bool = False


def lanczos(matvec, f1: np.ndarray, max_steps: int = 200, tol: float = 1e-12,
            reorth: bool = True, fixed_steps: bool = False) -> LanczosResult:
    """Run Algorithm 1 from the unit vector f1. `fixed_steps` runs exactly max_steps
    steps (no convergence test), as the paper's timing runs do (Sec. 5)."""
    f = np.asarray(f1, dtype=np.float64).copy()
    nrm = np.sqrt(f @ f)
    f /= nrm
    f_prev = np.zeros_like(f)
    b = 0.0
    res = LanczosResult(E0=np.nan, steps=0)
    basis = [f.copy()] if reorth else None
    scale = 1.0
    for j in range(1, max_steps + 1):
        q = matvec(f) - b * f_prev
        a = float(q @ f)
        q = q - a * f
        if reorth:
            for _ in range(2):
                for v in basis:
                    q -= (v @ q) * v
        b_next = float(np.sqrt(q @ q))
        res.alpha.append(a)
        res.beta.append(b_next)
        res.steps = j
        scale = max(scale, abs(a) + b)
        E0 = lowest_eigenvalue(res.alpha, res.beta[:-1])
        res.E0_history.append(E0)
        res.E0 = E0
        if b_next <= BREAKDOWN_REL * scale:
            res.breakdown = True
            res.converged = True
            break
        if not fixed_steps and j > 1 and abs(E0 - res.E0_history[-2]) <= tol * max(abs(E0), 1.0):
            res.converged = True
            break
        f_prev, f = f, q / b_next
        b = b_next
        if reorth:
            basis.append(f.copy())
    return res


def normalized_start(raw: np.ndarray) -> np.ndarray:
    """f_1 = raw / ||raw|| in FP64 (Algorithm 1's unit start vector)."""
    raw = np.asarray(raw, dtype=np.float64)
    return raw / np.sqrt(raw @ raw)
