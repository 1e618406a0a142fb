"""Writes the stored oracle results of the full-size workloads (expected values of the GPU
parity tests and the reference energies of the benchmark's time-to-E0 studies).

Only the CPU oracle (`oracle/`) and the seeded input generators (`ed_inputs`) are used:
Algorithm 1 (Sec. 2.2) in FP64 from the workload's seeded start vector, with the oracle's
matrix-free rows of H (Sec. 1 Eq. 1 plus the on-site term) as the product. The rows are
split into chunks that worker processes evaluate in parallel; every row is still the
oracle's plain FP64 sum, and the Lanczos recurrence runs unchanged in this process.

Usage (from the repository root):
    python tests/golden/make_lanczos_goldens.py torus4x4_5_5 [--workers 6]
    python tests/golden/make_lanczos_goldens.py ring16_8_8 --no-reorth

The 4x4 torus (dim 19,079,424) runs with full reorthogonalisation to |dE0| <= 1e-14 |E0|
(about 25 GB of host memory, tens of minutes on 6 cores). The 16-site ring (dim
165,636,900, 1.3 GB per vector) cannot hold its Krylov basis in host memory and runs the
plain three-term recurrence of Algorithm 1; ghost copies do not move the converged lowest
Ritz value (Paige).
"""
from __future__ import annotations

import argparse
import multiprocessing as mp
import os
import sys
import time
from multiprocessing import shared_memory

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import ed_inputs  # noqa: E402
from oracle import lanczos as olz  # noqa: E402
from oracle import basis as obasis  # noqa: E402

CHUNK = 1 << 20
_W = {}


def _init(name, dim, shx, shy, U):
    sys.path.insert(0, ROOT)
    from oracle import hamiltonian
    w = ed_inputs.workload(name)
    _W["args"] = (w["n_sites"], w["bonds"], w["n_up"], w["n_dn"], w["t"], U)
    _W["hv"] = hamiltonian.hv_rows
    _W["shx"] = shared_memory.SharedMemory(name=shx)
    _W["shy"] = shared_memory.SharedMemory(name=shy)
    _W["x"] = np.ndarray((dim,), dtype=np.float64, buffer=_W["shx"].buf)
    _W["y"] = np.ndarray((dim,), dtype=np.float64, buffer=_W["shy"].buf)


def _rows(lo_hi):
    lo, hi = lo_hi
    rows = np.arange(lo, hi, dtype=np.int64)
    _W["y"][lo:hi] = _W["hv"](*_W["args"], _W["x"], rows)
    return hi - lo


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("workload")
    ap.add_argument("--U", type=float, default=None)
    ap.add_argument("--workers", type=int, default=6)
    ap.add_argument("--no-reorth", action="store_true")
    ap.add_argument("--tol", type=float, default=1e-14)
    ap.add_argument("--max-steps", type=int, default=300)
    ap.add_argument("--record", type=int, default=20, help="a_j, b_j+1 stored for j <= this")
    ap.add_argument("--out", default=None)
    args = ap.parse_args()
    w = ed_inputs.workload(args.workload)
    U = w["U"] if args.U is None else args.U
    dim = obasis.dimension(w["n_sites"], w["n_up"], w["n_dn"])
    shx = shared_memory.SharedMemory(create=True, size=dim * 8)
    shy = shared_memory.SharedMemory(create=True, size=dim * 8)
    x = np.ndarray((dim,), dtype=np.float64, buffer=shx.buf)
    y = np.ndarray((dim,), dtype=np.float64, buffer=shy.buf)
    spans = [(lo, min(lo + CHUNK, dim)) for lo in range(0, dim, CHUNK)]
    ctx = mp.get_context("spawn")
    t_start = time.time()
    nmv = [0]
    with ctx.Pool(args.workers, initializer=_init,
                  initargs=(args.workload, dim, shx.name, shy.name, U)) as pool:
        def matvec(v):
            x[:] = v
            done = sum(pool.imap_unordered(_rows, spans))
            assert done == dim
            nmv[0] += 1
            print(f"  H.v {nmv[0]}: {time.time() - t_start:.0f} s", flush=True)
            return y.copy()

        f1 = olz.normalized_start(ed_inputs.start_vector_raw(w["seed"], dim))
        res = olz.lanczos(matvec, f1, max_steps=args.max_steps, tol=args.tol,
                          reorth=not args.no_reorth)
    shx.close(); shx.unlink(); shy.close(); shy.unlink()
    out = args.out or os.path.join(os.path.dirname(os.path.abspath(__file__)),
                                   f"lanczos_{args.workload}_U{U:g}.txt")
    m = min(args.record, res.steps)
    with open(out, "w") as fh:
        fh.write(f"# Oracle Algorithm 1 (Sec. 2.2) in FP64 on workload {args.workload}: "
                 f"{w['n_sites']} sites, {len(w['bonds'])} bonds, N_up={w['n_up']}, "
                 f"N_dn={w['n_dn']}, t={w['t']}, U={U}, dim={dim}\n")
        fh.write(f"# start vector: SplitMix64 seed {w['seed']}, normalised in FP64; "
                 f"reorthogonalisation: {'none' if args.no_reorth else 'full (two passes)'}; "
                 f"stop: |E0(j)-E0(j-1)| <= {args.tol:g} max(|E0|,1) or {args.max_steps} steps\n")
        fh.write(f"# written by tests/golden/make_lanczos_goldens.py "
                 f"({time.time() - t_start:.0f} s, {args.workers} workers)\n")
        fh.write(f"E0 {res.E0!r}\n")
        fh.write(f"steps {res.steps}\n")
        fh.write(f"converged {int(res.converged)}\n")
        fh.write(f"breakdown {int(res.breakdown)}\n")
        fh.write(f"dE0_last {abs(res.E0_history[-1] - res.E0_history[-2]) if res.steps > 1 else 0.0!r}\n")
        for j in range(m):
            fh.write(f"ab {j + 1} {res.alpha[j]!r} {res.beta[j]!r}\n")
        for j in range(res.steps):
            fh.write(f"E0_hist {j + 1} {res.E0_history[j]!r}\n")
    print(f"E0 = {res.E0!r} after {res.steps} steps -> {out}", flush=True)


if __name__ == "__main__":
    main()
