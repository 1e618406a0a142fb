"""Writes stored oracle energies used as references by the GPU tests and the benchmark:

  bethe_rings.txt     ground-state energies of periodic Hubbard rings from the Lieb-Wu
                      Bethe-ansatz equations (oracle/bethe.py): the 16-site ring at half
                      filling (U = 4), the 14-site ring at half filling for the learned-start
                      training grid and held-out U values, the 18-site ring at half filling.
  batched_E0.txt      E0 of every instance of the 256-instance batch (ed_inputs.
                      batched_instances), by the oracle's Algorithm 1 with full
                      reorthogonalisation on the explicit sparse H (dense eigh below
                      dimension 2000).
  lanczos_ring12_3_3_U4.txt  Algorithm 1 on the 12-site ring, 3/3, U = 4, seed 1.

Only oracle/ and ed_inputs are used. Usage (repository root):
    python tests/golden/make_small_goldens.py [bethe|batched|ring12]...
"""
from __future__ import annotations

import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import ed_inputs  # noqa: E402
from oracle import bethe, dense, hamiltonian, lanczos as olz  # noqa: E402


def write_bethe():
    rows = []
    rows.append(("ring16_8_8", 16, 8, 8, 4.0))
    rows.append(("ring18_9_9", 18, 9, 9, 4.0))
    for U in [0.5 * k for k in range(1, 17)]:
        rows.append(("ring14_7_7", 14, 7, 7, U))
    for U in ed_inputs.heldout_U():
        rows.append(("ring14_7_7", 14, 7, 7, float(U)))
    with open(os.path.join(HERE, "bethe_rings.txt"), "w") as fh:
        fh.write("# Lieb-Wu Bethe-ansatz ground-state energies of periodic Hubbard rings, t = 1\n")
        fh.write("# (oracle/bethe.py; written by tests/golden/make_small_goldens.py bethe)\n")
        fh.write("# columns: workload n_sites n_up n_dn U E0\n")
        for name, L, nu, nd, U in rows:
            E = bethe.ring_ground_energy(L, nu, nd, U)
            fh.write(f"{name} {L} {nu} {nd} {U!r} {E!r}\n")
            print(name, U, E, flush=True)


def _oracle_E0(w, seed=4):
    L, bonds, nu, nd, t, U = w["n_sites"], w["bonds"], w["n_up"], w["n_dn"], w["t"], w["U"]
    H = hamiltonian.hamiltonian_csr(L, bonds, nu, nd, t, U)
    if H.shape[0] <= 2000:
        return float(np.linalg.eigvalsh(H.toarray())[0]), "dense"
    f1 = olz.normalized_start(ed_inputs.start_vector_raw(seed, H.shape[0]))
    r = olz.lanczos(lambda v: H @ v, f1, max_steps=600, tol=1e-15)
    return float(r.E0), f"lanczos {r.steps} steps"


def write_batched():
    insts = ed_inputs.batched_instances()
    t0 = time.time()
    with open(os.path.join(HERE, "batched_E0.txt"), "w") as fh:
        fh.write("# Oracle E0 of the 256 instances of ed_inputs.batched_instances(seed=4)\n")
        fh.write("# (written by tests/golden/make_small_goldens.py batched)\n")
        fh.write("# columns: index lattice n_sites n_up n_dn U E0 method\n")
        for i, w in enumerate(insts):
            E, how = _oracle_E0(w)
            fh.write(f"{i} {w['name']} {w['n_sites']} {w['n_up']} {w['n_dn']} {w['U']!r} {E!r} {how}\n")
            fh.flush()
            print(i, w["name"], E, how, f"{time.time() - t0:.0f}s", flush=True)


def write_ring12():
    w = ed_inputs.workload("ring12_3_3")
    H = hamiltonian.hamiltonian_csr(w["n_sites"], w["bonds"], w["n_up"], w["n_dn"], w["t"], w["U"])
    f1 = olz.normalized_start(ed_inputs.start_vector_raw(w["seed"], H.shape[0]))
    r = olz.lanczos(lambda v: H @ v, f1, max_steps=300, tol=1e-14)
    with open(os.path.join(HERE, "lanczos_ring12_3_3_U4.txt"), "w") as fh:
        fh.write("# Oracle Algorithm 1 (Sec. 2.2) in FP64, explicit sparse H, ring12_3_3: 12 sites, "
                 f"N_up=N_dn=3, t=1, U={w['U']}, dim={H.shape[0]}, seed {w['seed']}, full reorth.\n")
        fh.write("# (written by tests/golden/make_small_goldens.py ring12)\n")
        fh.write(f"E0 {r.E0!r}\nsteps {r.steps}\n")
        for j in range(min(20, r.steps)):
            fh.write(f"ab {j + 1} {r.alpha[j]!r} {r.beta[j]!r}\n")


if __name__ == "__main__":
    what = sys.argv[1:] or ["bethe", "ring12", "batched"]
    for w in what:
        {"bethe": write_bethe, "batched": write_batched, "ring12": write_ring12}[w]()
