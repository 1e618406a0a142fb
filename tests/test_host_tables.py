"""Host logic of the fused H.v plan (no GPU): the down-hop tables built by
ed_hv_down_tables, the same code the library runs for every plan.

The kernel's down part (Sec. 4, Eq. 6) gathers, for every column of a staged row, the
row's elements at the column's hop targets. The tables must keep each column's hops
exactly (as a multiset, split by fermion sign for real tables, with their amplitude
indices for complex ones), put padding on zero slots, keep the slot map a permutation
inside aligned groups of G columns, and order the columns by hop count. The bank-conflict
schedule is checked against a modelled wavefront count.
"""
import numpy as np
import pytest

import ed_inputs
from oracle.basis import rank_of, species_states
from oracle.hamiltonian import hops_of

pytestmark = pytest.mark.filterwarnings("ignore::DeprecationWarning")

ed = pytest.importorskip("paper_1511_00863_gb300")

SIGN = np.int64(1) << 31


def hop_table(n_sites, n_particles, bonds):
    """Library-format hop table [maxhops][dim] of one species, hops of a state in bond
    order (target rank | sign << 31, padding = dim), amplitude numbers 2 b + (particle at
    the bond's second site), and the bit strings."""
    states = species_states(n_sites, n_particles)
    n = len(states)
    lists = [[] for _ in range(n)]
    bonds = np.asarray(bonds).reshape(-1, 2)
    for b, (src, s2, sign) in enumerate(hops_of(states, bonds)):
        tg = rank_of(states, s2)
        at_j = (states[src] >> int(bonds[b, 1])) & 1
        for r, t, sg, aj in zip(src, tg, sign, at_j):
            lists[r].append((int(t) | (int(SIGN) if sg < 0 else 0), 2 * b + int(aj)))
    mh = max((len(l) for l in lists), default=0)
    hop = np.full((mh, n), n, dtype=np.int64)
    amp = np.zeros((mh, n), dtype=np.int32)
    for r, l in enumerate(lists):
        for k, (e, a) in enumerate(l):
            hop[k, r] = e
            amp[k, r] = a
    return hop.astype(np.uint32).view(np.int32), amp, states.astype(np.uint32)


def check_tables(hop, amp, bits, V, G, cplx):
    n = bits.size
    mh = hop.shape[0]
    out = ed.ed_hv_down_tables(hop, bits, V, G, hop_amp=amp if cplx else None,
                               complex_entries=cplx)
    T, kpn, lo, pos, ld = out["table"], out["kpn"], out["slot_lo"], out["colpos"], out["ld"]
    assert ld == (n + 31) // 32 * 32
    h = hop.view(np.uint32).astype(np.int64)
    tgt = h & 0x3FFFFFFF
    neg = (h >> 31) & 1
    valid = tgt < n
    npos = (valid & (neg == 0)).sum(0)
    nneg = (valid & (neg == 1)).sum(0)
    # column order: hop count desc, +1 count desc, rank asc
    assert sorted(pos.tolist()) == list(range(n))
    perm = np.empty(n, dtype=np.int64)
    perm[pos] = np.arange(n)
    key = list(zip(-(npos + nneg)[perm], -npos[perm], perm))
    assert key == sorted(key)
    # slot map: a permutation inside each aligned group of G columns
    assert (np.sort(lo.reshape(-1, G), axis=1) == np.arange(G)).all()
    slot_of = (np.arange(ld) & ~(G - 1)) | lo
    col_of_slot = np.empty(ld, dtype=np.int64)
    col_of_slot[slot_of] = np.arange(ld)
    chunk = 32 * V
    entry_slot = T & 0xFFFF if cplx else T
    entry_amp = T >> 16
    for c in range(kpn.shape[0]):
        cols = np.arange(c * chunk, min((c + 1) * chunk, ld))
        real = cols[cols < n]
        if cplx:
            assert kpn[c, 0] == ((npos + nneg)[perm[real]].max() if real.size else 0)
            assert kpn[c, 1] == 0
        else:
            assert kpn[c, 0] == (npos[perm[real]].max() if real.size else 0)
            assert kpn[c, 1] == (nneg[perm[real]].max() if real.size else 0)
        groups = [(0, int(kpn[c, 0]), None)] if cplx else [
            (0, int(kpn[c, 0]), 0), (int(kpn[c, 0]), int(kpn[c, 0] + kpn[c, 1]), 1)]
        for p in cols:
            for k0, k1, sgn in groups:
                s = entry_slot[k0:k1, p].astype(np.int64)
                zero = s >= ld
                assert (s[zero] < ld + G).all(), "padding outside the zero slots"
                got = sorted(zip(col_of_slot[s[~zero]].tolist(),
                                 entry_amp[k0:k1, p][~zero].tolist() if cplx else [0] * int((~zero).sum())))
                want = []
                if p < n:
                    d = perm[p]
                    for k in range(mh):
                        if valid[k, d] and (sgn is None or neg[k, d] == sgn):
                            want.append((int(pos[tgt[k, d]]),
                                         int(2 * amp[k, d] + neg[k, d]) if cplx else 0))
                assert got == sorted(want), f"column {p} rows {k0}..{k1}"
    return out


def modelled_wavefronts(out, V, G, cplx):
    """Shared-memory wavefronts per phase and step: the largest number of distinct slots in
    one bank group (slot mod G) among the G lanes of a phase."""
    T, kpn, ld = out["table"], out["kpn"], out["ld"]
    S = (T & 0xFFFF if cplx else T).astype(np.int64)
    chunk = 32 * V
    total = steps = 0
    for c in range(kpn.shape[0]):
        for k in range(int(kpn[c, 0] + kpn[c, 1])):
            for v in range(V):
                for ph in range(0, 32, G):
                    cols = c * chunk + (ph + np.arange(G)) * V + v
                    cols = cols[cols < ld]
                    if cols.size == 0:
                        continue
                    sl = np.unique(S[k, cols])
                    total += np.bincount(sl % G, minlength=G).max()
                    steps += 1
    return total / steps


def test_torus_int64_geometry():
    """4x4 periodic lattice, 5 particles (dim 4368): the int64 R=1 geometry (V=2, G=16)."""
    hop, amp, bits = hop_table(16, 5, ed_inputs.torus_bonds(4, 4))
    out = check_tables(hop, amp, bits, 2, 16, False)
    # with slots and hop order both chosen: ~1.56 (2.2 with the slot map alone)
    assert modelled_wavefronts(out, 2, 16, False) < 1.7


@pytest.mark.parametrize("V,G", [(4, 32), (4, 16), (4, 8), (2, 8)])
def test_ring_geometries(V, G):
    hop, amp, bits = hop_table(12, 6, ed_inputs.ring_bonds(12))
    out = check_tables(hop, amp, bits, V, G, False)
    assert modelled_wavefronts(out, V, G, False) < 2.0


@pytest.mark.parametrize("V,G", [(2, 16), (2, 8)])
def test_complex_entries(V, G):
    """Complex tables: one group of all hops, amplitude indices travel with their hops."""
    bonds, _ = ed_inputs.checkerboard_lattice(4, 3)
    hop, amp, bits = hop_table(12, 4, bonds)
    check_tables(hop, amp, bits, V, G, True)


def test_tiny_and_empty():
    # fewer states than one chunk; a species without hops (all sites filled)
    hop, amp, bits = hop_table(6, 2, ed_inputs.ring_bonds(6))
    check_tables(hop, amp, bits, 2, 16, False)
    hop, amp, bits = hop_table(5, 5, ed_inputs.ring_bonds(5))
    assert hop.shape[0] == 0
    out = ed.ed_hv_down_tables(hop, bits, 2, 16)
    assert out["table"].shape[0] == 1 and (out["table"][0, :bits.size] >= out["ld"]).all()


def test_bad_geometry():
    hop, amp, bits = hop_table(6, 2, ed_inputs.ring_bonds(6))
    with pytest.raises(ed.EdError) as e:
        ed.ed_hv_down_tables(hop, bits, 2, 12)
    assert e.value.status == ed.ED_ERR_ARG
    bad = amp.copy()
    bad[0, 0] = 40000  # 2 a + 1 does not fit the 16-bit index field
    with pytest.raises(ed.EdError) as e:
        ed.ed_hv_down_tables(hop, bits, 2, 16, hop_amp=bad, complex_entries=True)
    assert e.value.status == ed.ED_ERR_ARG


SPLIT_CASES = [
    (12, ed_inputs.ring_bonds(12), 6, 2, 16),     # half filling: equal slices
    (10, ed_inputs.ring_bonds(10), 3, 4, 32),     # unequal slices (site 0 occupied in 36 of 120)
    (8, ed_inputs.torus_bonds(2, 4), 4, 1, 16),   # doubled bonds
    (9, np.array([[0, 5], [3, 8], [1, 2], [7, 0], [6, 4], [2, 8], [5, 1]]), 4, 2, 8),
    (14, ed_inputs.ring_bonds(14), 7, 4, 32),     # the FP32 geometry on a longer row
]


@pytest.mark.parametrize("L,bonds,N,V,G", SPLIT_CASES)
def test_split_tables_keep_every_hop(L, bonds, N, V, G):
    """Split-row tables (rows longer than shared memory, staged as two slices cut by the
    occupation of site 0): each slice holds exactly the states with site 0 occupied / empty
    and at least one padding column; its slot map is a permutation inside aligned groups of
    G; each column decodes to exactly its state's hops, by sign, the in-slice ones as slots
    (padding on the slice's zero slots) and the cross-slice ones as columns of the other
    slice (padding on one of its padding columns); the in-slice gathers keep the modelled
    bank conflicts of the plain tables."""
    check_split(L, bonds, N, V, G, 0, wavefront_bound=2.0)


def check_split(L, bonds, N, V, G, site, wavefront_bound=None):
    hop, _, bits = hop_table(L, N, bonds)
    n = bits.size
    out = ed.ed_hv_split_tables(hop, bits, V, G, site=site)
    T, X, kpn, lo, cs, pos, ld = (out[k] for k in ("table", "xtable", "kpn", "slot_lo", "cstart",
                                                   "colpos", "ld"))
    CW = 32 * V
    occ = ((bits >> site) & 1) == 1
    nsl = [int(occ.sum()), int(n - occ.sum())]
    assert cs[0] == 0 and cs[2] == ld
    for s_ in range(2):
        assert cs[s_ + 1] - cs[s_] == (nsl[s_] + 1 + CW - 1) // CW * CW
    # every rank has a distinct column inside its slice
    assert len(set(pos.tolist())) == n
    assert np.all((pos < cs[1]) == occ)
    col2rank = {int(p): d for d, p in enumerate(pos)}
    assert (np.sort(lo.reshape(-1, G), axis=1) == np.arange(G)).all()
    h = hop.view(np.uint32).astype(np.int64)
    tgt, neg = h & 0x3FFFFFFF, (h >> 31) & 1
    for s_ in range(2):
        c0, c1, o = int(cs[s_]), int(cs[s_ + 1]), 1 - s_
        lds, ldo = c1 - c0, int(cs[o + 1] - cs[o])
        slot_of = (np.arange(lds) & ~(G - 1)) | lo[c0:c1]
        col_of_slot = np.empty(lds, dtype=np.int64)
        col_of_slot[slot_of] = np.arange(c0, c1)
        assert (c1 - 1) not in col2rank and (int(cs[o + 1]) - 1) not in col2rank
        for p in range(c0, c1):
            c = p // CW
            ip, im, xp, xm = (int(v) for v in kpn[c])
            assert T.shape[0] >= ip + im and X.shape[0] >= xp + xm
            got = {(+1, 0): [], (-1, 0): [], (+1, 1): [], (-1, 1): []}
            for k in range(ip + im):
                e = int(T[k, p])
                assert e < lds + G
                if e >= lds:
                    continue
                got[(+1 if k < ip else -1, 0)].append(int(col_of_slot[e]))
            for k in range(xp + xm):
                e = int(X[k, p])
                assert e < ldo
                if cs[o] + e in col2rank:
                    got[(+1 if k < xp else -1, 1)].append(int(cs[o] + e))
                else:
                    assert e == ldo - 1
            d = col2rank.get(p)
            want = {key: [] for key in got}
            if d is not None:
                for k in range(h.shape[0]):
                    if tgt[k, d] < n:
                        t = int(tgt[k, d])
                        want[(-1 if neg[k, d] else +1, int(occ[t] != occ[d]))].append(int(pos[t]))
            for key in got:
                assert sorted(got[key]) == sorted(want[key]), (p, key)
        # per chunk: the rows are the largest counts of the chunk's columns
        for c in range(c0 // CW, c1 // CW):
            cols = [col2rank[p] for p in range(c * CW, (c + 1) * CW) if p in col2rank]
            cnt = np.zeros((4, max(len(cols), 1)), dtype=np.int64)
            for j, d in enumerate(cols):
                for k in range(h.shape[0]):
                    if tgt[k, d] < n:
                        cnt[2 * int(occ[tgt[k, d]] != occ[d]) + int(neg[k, d]), j] += 1
            assert list(kpn[c]) == list(cnt.max(axis=1)), c
        if wavefront_bound is not None:
            sub = {"table": T[:, c0:c1], "kpn": kpn[c0 // CW:c1 // CW, :2], "ld": lds}
            assert modelled_wavefronts(sub, V, G, False) < wavefront_bound


def test_split_tables_bad_geometry():
    hop, _, bits = hop_table(8, 4, ed_inputs.ring_bonds(8))
    with pytest.raises(ed.EdError) as e:
        ed.ed_hv_split_tables(hop, bits, 2, 12)
    assert e.value.status == ed.ED_ERR_ARG


def _random_lattice(rng):
    """A bond list on 5-11 sites with random pairs, one of them listed twice and one in both
    orders (duplicates add), and a random filling with at least one state per slice."""
    L = int(rng.integers(5, 12))
    nb = int(rng.integers(L, 2 * L + 1))
    bonds = []
    while len(bonds) < nb:
        i, j = (int(v) for v in rng.integers(0, L, size=2))
        if i != j:
            bonds.append((i, j))
    bonds += [bonds[0], bonds[1][::-1]]
    N = int(rng.integers(1, L))
    return L, np.array(bonds), N


@pytest.mark.parametrize("seed", range(40))
def test_random_lattices_all_geometries(seed):
    """Seeded random bond lists (irregular degrees, doubled and reversed bonds) through both
    table builders at every geometry the ABI allows (V from 1 to 8, odd V included, and G of
    8, 16 and 32), real and complex entries, and the split tables cut at a random site."""
    rng = np.random.default_rng(1000 + seed)
    L, bonds, N = _random_lattice(rng)
    hop, amp, bits = hop_table(L, N, bonds)
    V = int(rng.choice([1, 2, 3, 4, 8]))
    G = int(rng.choice([8, 16, 32]))
    check_tables(hop, amp, bits, V, G, False)
    check_tables(hop, amp, bits, V, G, True)
    check_split(L, bonds, N, V, G, int(rng.integers(0, L)))


@pytest.mark.parametrize("case", ed_inputs.random_lattices(), ids=lambda c: c["name"])
def test_random_lattice_workloads_at_kernel_geometries(case):
    """The random lattices the GPU parity tests run: both species' tables at the geometries
    of the fused H.v's variants (int64: V = 2 with G = 16 or 8; FP32: V = 4 with G = 32, 16
    or 8), every hop decoded back and every slot inside the staged row or its zero slots."""
    for n in (case["n_up"], case["n_dn"]):
        hop, amp, bits = hop_table(case["n_sites"], n, case["bonds"])
        for V, G in ((2, 16), (2, 8), (4, 32), (4, 16), (4, 8)):
            check_tables(hop, amp, bits, V, G, False)
