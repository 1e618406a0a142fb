"""The seeded input generators (`ed_inputs.py`) against what fixes them independently: the
published SplitMix64 output stream, the exactness of the uniform mapping, the lattices'
bond counts, and the workload recipe (sizes the paper prints, Sec. 2.1; the batch recipe's
stated ranges).
"""
import math

import numpy as np

import ed_inputs
from oracle.basis import species_states


def test_splitmix64_published_stream():
    # the first outputs of SplitMix64 started from state 0 (the generator's reference
    # implementation by S. Vigna)
    got = [int(x) for x in ed_inputs.splitmix64(0, 3)]
    assert got == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]
    # an offset continues the same stream
    assert int(ed_inputs.splitmix64(0, 1, offset=2)[0]) == 0x06C45D188009454F


def test_uniform_pm1_exact_and_in_range():
    z = ed_inputs.splitmix64(11, 4096)
    u = ed_inputs.uniform_pm1(11, 4096)
    assert ((u >= -1.0) & (u < 1.0)).all()
    # 2 (k 2^-53) - 1 with k the top 53 bits: exact in FP64, so it inverts exactly
    k = ((u + 1.0) * 2.0 ** 52).astype(np.uint64)
    assert (k == (z >> np.uint64(11))).all()
    assert abs(u.mean()) < 0.05 and abs((u * u).mean() - 1.0 / 3.0) < 0.02


def test_lattice_bond_counts():
    assert len(ed_inputs.ring_bonds(12)) == 12 and len(ed_inputs.ring_bonds(1)) == 0
    assert len(ed_inputs.ring_bonds(2)) == 2  # the pair twice: the two hoppings add
    assert len(ed_inputs.torus_bonds(4, 4)) == 32
    assert len(ed_inputs.torus_bonds(2, 4)) == 16  # extent-2 direction lists pairs twice
    assert len(ed_inputs.torus_bonds(1, 4)) == 4


def test_workload_sizes():
    dims = {"ring12_3_3": 220 ** 2, "torus4x4_5_5": 4368 ** 2, "ring16_8_8": 12870 ** 2,
            "ring14_7_7": 3432 ** 2, "ring26_13_0": 10_400_600, "checker4x4_5_5": 4368 ** 2,
            "ring18_9_9": 48620 ** 2}
    for name, dim in dims.items():
        w = ed_inputs.workload(name)
        L = w["n_sites"]
        assert math.comb(L, w["n_up"]) * math.comb(L, w["n_dn"]) == dim, name
    assert len(species_states(16, 5)) == 4368


def test_batch_recipe():
    inst = ed_inputs.batched_instances()
    assert len(inst) == 256
    kinds = {f"ring{L}" for L in range(8, 13)} | {"rect2x4", "rect3x4"}
    dims = []
    for i in inst:
        assert i["name"] in kinds
        L = i["n_sites"]
        assert 1 <= i["n_up"] <= L // 2 and 1 <= i["n_dn"] <= L // 2
        assert 0.0 <= i["U"] < 8.0 and i["t"] == 1.0
        dims.append(math.comb(L, i["n_up"]) * math.comb(L, i["n_dn"]))
    assert min(dims) >= 64 and max(dims) <= 853_776
    assert sum(dims) == 14_934_709  # the batch's total dimension
    assert len({i["name"] for i in inst}) == len(kinds)  # every lattice kind is drawn
    again = ed_inputs.batched_instances()  # deterministic in the seed
    assert all(a["name"] == b["name"] and a["n_up"] == b["n_up"] and a["n_dn"] == b["n_dn"]
               and a["U"] == b["U"] for a, b in zip(inst, again))


def test_heldout_U():
    U = ed_inputs.heldout_U()
    assert U.shape == (16,) and ((U >= 0) & (U < 8)).all()
    assert not np.isin(U, np.arange(17) * 0.5).any()  # none on the training grid


def test_random_lattices_as_described():
    from math import comb
    cases = ed_inputs.random_lattices()
    again = ed_inputs.random_lattices()
    assert all(a["name"] == b["name"] and np.array_equal(a["bonds"], b["bonds"]) and a["U"] == b["U"]
               for a, b in zip(cases, again))
    for c in cases:
        L, b = c["n_sites"], c["bonds"]
        assert 10 <= L <= 12 and L + 2 <= len(b) <= 2 * L + 2
        assert np.all(b[:, 0] != b[:, 1]) and b.min() >= 0 and b.max() < L
        assert tuple(b[-2]) == tuple(b[0]) and tuple(b[-1]) == tuple(b[1][::-1])
        assert 3 <= c["n_up"] <= L - 3 and 1 <= c["n_dn"] <= L - 1
        assert comb(L, c["n_up"]) * comb(L, c["n_dn"]) <= 400_000
        assert -2.0 <= c["U"] < 8.0 and c["t"] == 1.0
