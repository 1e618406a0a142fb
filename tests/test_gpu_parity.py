"""GPU parity: the CUDA path through the C ABI against the CPU oracle on the same seeded
inputs. Integer work (basis, hop targets, signs) must match bit for bit; floating point
within the stated error bounds."""
import math

import numpy as np
import pytest

import ed_inputs
from oracle import basis as obasis
from oracle import dense, hamiltonian, lanczos as olz

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

EPS64 = 2.0 ** -53
EPS32 = 2.0 ** -24


@pytest.fixture(scope="module")
def ed():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1511_00863_gb300 as m
    return m


class _DevView:
    def __init__(self, ptr, n, typestr):
        self.__cuda_array_interface__ = {"shape": (n,), "typestr": typestr, "data": (ptr, False),
                                         "version": 3, "strides": None}


def dev_to_numpy(ptr, n, typestr):
    return torch.as_tensor(_DevView(ptr, n, typestr), device="cuda").cpu().numpy()


def _oracle_tables(L, N, bonds):
    states, lists = hamiltonian.species_hop_table(L, N, bonds)
    return states, lists


TABLE_CASES = [
    ("ring6_3_2", 6, ed_inputs.ring_bonds(6), 3, 2),
    ("rect2x4_2_3", 8, ed_inputs.torus_bonds(2, 4), 2, 3),
    ("ring12_3_3", 12, ed_inputs.ring_bonds(12), 3, 3),
    ("torus4x4_5_5", 16, ed_inputs.torus_bonds(4, 4), 5, 5),
    ("ring16_8_7", 16, ed_inputs.ring_bonds(16), 8, 7),
    ("empty_full", 5, ed_inputs.ring_bonds(5), 0, 5),
    ("single_site", 1, np.zeros((0, 2), np.int32), 1, 0),
    ("doubled_pair", 2, ed_inputs.ring_bonds(2), 1, 1),
    ("random_bonds", 9, np.array([[0, 5], [3, 8], [1, 2], [7, 0], [6, 4], [2, 8], [5, 1]]), 4, 3),
    ("single_species_up", 10, ed_inputs.ring_bonds(10), 4, 0),
    ("single_species_dn", 10, ed_inputs.ring_bonds(10), 0, 4),
]


@pytest.mark.parametrize("name,L,bonds,nu,nd", TABLE_CASES, ids=[c[0] for c in TABLE_CASES])
def test_basis_tables_bit_exact(ed, name, L, bonds, nu, nd):
    b = ed.ed_build_basis(L, bonds, nu, nd)
    try:
        du, dd, d = ed.ed_basis_dims(b)
        assert (du, dd, d) == (math.comb(L, nu), math.comb(L, nd), math.comb(L, nu) * math.comb(L, nd))
        tb = ed.ed_basis_tables(b)
        for N, dim, bits_ptr, hop_ptr, mh in ((nu, du, tb["up_bits"], tb["hop_up"], tb["maxhops_up"]),
                                              (nd, dd, tb["dn_bits"], tb["hop_dn"], tb["maxhops_dn"])):
            states, lists = _oracle_tables(L, N, bonds)
            bits = dev_to_numpy(bits_ptr, dim, "<u4")
            assert np.array_equal(bits.astype(np.int64), states)
            assert mh == max(len(x) for x in lists)
            if mh == 0:
                continue
            hop = dev_to_numpy(hop_ptr, mh * dim, "<u4").reshape(mh, dim)
            for r in range(dim):
                for k in range(mh):
                    e = int(hop[k, r])
                    if k < len(lists[r]):
                        tgt, sgn = lists[r][k]
                        assert (e & 0x3FFFFFFF) == tgt and (e >> 31) == (1 if sgn < 0 else 0), (r, k)
                        assert (e >> 30) & 1 == 0
                    else:
                        assert e == dim, (r, k)
    finally:
        ed.ed_basis_destroy(b)


HV_CASES = [
    (5, ed_inputs.ring_bonds(5), 2, 2, 1.0, 3.0),
    (6, ed_inputs.ring_bonds(6), 3, 2, 0.7, 2.5),
    (8, ed_inputs.torus_bonds(2, 4), 2, 3, 1.0, 4.0),
    (12, ed_inputs.ring_bonds(12), 3, 3, 1.0, 4.0),
    (9, np.array([[0, 5], [3, 8], [1, 2], [7, 0], [6, 4], [2, 8], [5, 1]]), 4, 3, 1.3, -1.5),
    (8, ed_inputs.ring_bonds(8), 0, 3, 1.0, 2.0),
    (10, ed_inputs.ring_bonds(10), 4, 0, 1.0, 2.0),
    (4, ed_inputs.ring_bonds(4), 4, 4, 1.0, 2.0),
]


def _hv_bound(case, x, rows, eps, extra=4.0):
    L, bonds, nu, nd, t, U = case
    absy = hamiltonian.hv_abs_rows(L, bonds, nu, nd, t, U, x, rows)
    nh = 2 * len(bonds) + 2
    return extra * nh * eps * absy + 1e-300


@pytest.mark.parametrize("case", HV_CASES)
@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_hv_small_elementwise(ed, case, dtype):
    L, bonds, nu, nd, t, U = case
    b = ed.ed_build_basis(L, bonds, nu, nd)
    try:
        dim = ed.ed_basis_dims(b)[2]
        x = ed_inputs.uniform_pm1(21, dim)
        tdt = torch.float64 if dtype == "f64" else torch.float32
        xd = torch.tensor(x, device="cuda", dtype=tdt)
        yd = torch.empty_like(xd)
        ed.ed_hv(b, t, U, xd, yd)
        xr = xd.double().cpu().numpy()
        rows = np.arange(dim)
        ref = hamiltonian.hv_rows(L, bonds, nu, nd, t, U, xr, rows)
        eps = EPS64 if dtype == "f64" else EPS32
        bound = _hv_bound(case, xr, rows, eps)
        err = np.abs(yd.double().cpu().numpy() - ref)
        assert np.all(err <= bound), float((err / bound).max())
    finally:
        ed.ed_basis_destroy(b)


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_hv_rejects_overlap_and_misalignment(ed, dtype):
    """ed_hv refuses, with ED_ERR_ARG and before any launch, an output that overlaps the
    input (the same buffer, or one shifted by 16 bytes) and vectors that are not 16-byte
    aligned (shifted by one element). The output keeps its contents, and a valid call on the
    same basis afterwards matches the oracle."""
    case = HV_CASES[0]
    L, bonds, nu, nd, t, U = case
    b = ed.ed_build_basis(L, bonds, nu, nd)
    try:
        dim = ed.ed_basis_dims(b)[2]
        tdt = torch.float64 if dtype == "f64" else torch.float32
        es = 8 if dtype == "f64" else 4
        buf = torch.zeros(dim + 16 // es, device="cuda", dtype=tdt)
        other = torch.full((dim + 1,), 7.0, device="cuda", dtype=tdt)
        assert buf.data_ptr() % 16 == 0 and other.data_ptr() % 16 == 0
        a = buf[:dim]
        cases = [(a, a, "overlap"), (a, buf[16 // es:], "overlap"),
                 (other[1:], buf[:dim], "aligned"), (buf[:dim], other[1:], "aligned")]
        for x, y, word in cases:
            before = y.clone()
            with pytest.raises(ed.EdError) as ei:
                ed.ed_hv(b, t, U, x, y)
            assert ei.value.status == ed.ED_ERR_ARG and word in str(ei.value), str(ei.value)
            torch.cuda.synchronize()
            assert torch.equal(y, before)
        x = ed_inputs.uniform_pm1(21, dim)
        xd = torch.tensor(x, device="cuda", dtype=tdt)
        yd = torch.empty_like(xd)
        ed.ed_hv(b, t, U, xd, yd)
        xr = xd.double().cpu().numpy()
        rows = np.arange(dim)
        ref = hamiltonian.hv_rows(L, bonds, nu, nd, t, U, xr, rows)
        bound = _hv_bound(case, xr, rows, EPS64 if dtype == "f64" else EPS32)
        assert np.all(np.abs(yd.double().cpu().numpy() - ref) <= bound)
    finally:
        ed.ed_basis_destroy(b)


FULL = [("torus4x4_5_5", "f64"), ("ring16_8_8", "f32"), ("ring16_8_8", "f64")]


@pytest.mark.parametrize("name,dtype", FULL)
def test_hv_full_size_sampled(ed, name, dtype):
    """Full-size workloads: sampled rows (both ends, sub-vector borders, random) against
    the oracle's matrix-free rows."""
    w = ed_inputs.workload(name)
    L, bonds, nu, nd, t, U = w["n_sites"], w["bonds"], w["n_up"], w["n_dn"], w["t"], w["U"]
    b = ed.ed_build_basis(L, bonds, nu, nd)
    try:
        du, dd, dim = ed.ed_basis_dims(b)
        tdt = torch.float64 if dtype == "f64" else torch.float32
        x = ed_inputs.uniform_pm1(w["seed"], dim)
        xd = torch.from_numpy(x).to(device="cuda", dtype=tdt)
        del x
        yd = torch.empty_like(xd)
        ed.ed_hv(b, t, U, xd, yd)
        torch.cuda.synchronize()
        rng = np.random.default_rng(5)
        rows = np.unique(np.concatenate([
            [0, 1, dim - 1, dim - 2], np.arange(0, dim, dd)[:50], np.arange(dd - 1, dim, dd)[-50:],
            rng.integers(0, dim, 3000)]))
        xr = xd.double().cpu().numpy()
        ref = hamiltonian.hv_rows(L, bonds, nu, nd, t, U, xr, rows)
        got = yd[torch.from_numpy(rows).cuda()].double().cpu().numpy()
        bound = _hv_bound((L, bonds, nu, nd, t, U), xr, rows, EPS64 if dtype == "f64" else EPS32)
        err = np.abs(got - ref)
        assert np.all(err <= bound), float((err / bound).max())
    finally:
        ed.ed_basis_destroy(b)


def test_start_vector_matches_generator(ed):
    n = 100003
    ref = olz.normalized_start(ed_inputs.start_vector_raw(77, n))
    out = torch.empty(n, dtype=torch.float64, device="cuda")
    ed.ed_start_vector(n, 77, out)
    got = out.cpu().numpy()
    assert np.all(np.abs(got - ref) <= 2 * EPS64 * np.abs(ref))
    o32 = torch.empty(n, dtype=torch.float32, device="cuda")
    ed.ed_start_vector(n, 77, o32)
    g32 = o32.cpu().numpy().astype(np.float64)
    assert np.all(np.abs(g32 - ref) <= 1.0000001 * EPS32 * np.abs(ref) * 2)


# --------------------------------------------------------------------------- Lanczos
def _solve(ed, L, bonds, nu, nd, t, U, dtype="f64", seed=1, max_steps=300, tol=1e-13, f1=None):
    b = ed.ed_build_basis(L, bonds, nu, nd)
    try:
        return ed.ed_lanczos_solve(b, t, U, ed.make_opts(max_steps=max_steps, tol=tol, seed=seed,
                                                         dtype=dtype), f1=f1,
                                   raise_not_converged=False)
    finally:
        ed.ed_basis_destroy(b)


F64_KINDS = ["f64", "f64n"]   # fixed-point FP64-accurate path, native FP64 path


@pytest.mark.parametrize("dtype", F64_KINDS)
@pytest.mark.parametrize("U", [0.0, 4.0])
def test_lanczos_ring12_fp64(ed, U, dtype):
    L, bonds = 12, ed_inputs.ring_bonds(12)
    res = _solve(ed, L, bonds, 3, 3, 1.0, U, seed=1, max_steps=200, tol=1e-12, dtype=dtype)
    if U == 0.0:
        ref = -4 * (1 + math.sqrt(3))
    else:
        H = hamiltonian.hamiltonian_csr(L, bonds, 3, 3, 1.0, U)
        f1 = olz.normalized_start(ed_inputs.start_vector_raw(1, H.shape[0]))
        ref = olz.lanczos(lambda v: H @ v, f1, max_steps=300, tol=1e-14).E0
    assert res["status"] in (0, 1)
    assert abs(res["E0"] - ref) <= 1e-10 * abs(ref), (res["E0"], ref)


def test_lanczos_ring12_fp32(ed):
    L, bonds = 12, ed_inputs.ring_bonds(12)
    H = hamiltonian.hamiltonian_csr(L, bonds, 3, 3, 1.0, 4.0)
    f1 = olz.normalized_start(ed_inputs.start_vector_raw(1, H.shape[0]))
    ref = olz.lanczos(lambda v: H @ v, f1, max_steps=300, tol=1e-14).E0
    res = _solve(ed, L, bonds, 3, 3, 1.0, 4.0, dtype="f32", max_steps=300, tol=1e-9)
    assert abs(res["E0"] - ref) <= 1e-6 * abs(ref), (res["E0"], ref)


RANDOM_CASES = []
_rng = np.random.default_rng(123)
for _k in range(8):
    _L = int(_rng.integers(4, 9))
    _nb = int(_rng.integers(_L - 1, 2 * _L))
    _pairs = set()
    while len(_pairs) < _nb:
        i, j = (int(v) for v in _rng.integers(0, _L, 2))
        if i != j:
            _pairs.add((i, j))
    _nu = int(_rng.integers(0, _L + 1))
    _nd = int(_rng.integers(0, _L + 1))
    RANDOM_CASES.append((_L, np.array(sorted(_pairs)), _nu, _nd, 1.0, float(_rng.uniform(-2, 8))))


@pytest.mark.parametrize("dtype", F64_KINDS)
@pytest.mark.parametrize("case", RANDOM_CASES)
def test_lanczos_random_lattices_vs_dense(ed, case, dtype):
    L, bonds, nu, nd, t, U = case
    if math.comb(L, nu) * math.comb(L, nd) > 2000:
        pytest.skip("dense reference limited to dim <= 2000")
    ref = dense.spectrum(L, bonds, nu, nd, t, U)[0]
    res = _solve(ed, L, bonds, nu, nd, t, U, seed=3, dtype=dtype)
    assert abs(res["E0"] - ref) <= 1e-10 * max(1.0, abs(ref)), (res, ref)


@pytest.mark.parametrize("dtype", F64_KINDS + ["f32"])
@pytest.mark.parametrize("U", [0.0, 4.0, 8.0])
def test_two_site_closed_form(ed, U, dtype):
    res = _solve(ed, 2, np.array([[0, 1]]), 1, 1, 1.0, U, seed=4, dtype=dtype)
    if dtype == "f32":
        assert abs(res["E0"] - (U - math.sqrt(U * U + 16)) / 2) <= 1e-6
        return
    assert abs(res["E0"] - (U - math.sqrt(U * U + 16)) / 2) <= 1e-12


@pytest.mark.parametrize("dtype", F64_KINDS)
def test_breakdown_on_eigenvector(ed, dtype):
    case = (2, np.array([[0, 1]]), 1, 1, 1.0, 0.0)
    E0, psi = dense.ground_state(*case)
    f1 = torch.tensor(psi, device="cuda")
    res = _solve(ed, *case, f1=f1, dtype=dtype)
    assert res["status"] == ed.ED_BREAKDOWN and res["steps"] == 1
    assert abs(res["E0"] - (-2.0)) <= 1e-14


@pytest.mark.parametrize("dtype", F64_KINDS)
def test_alpha_beta_follow_oracle(ed, dtype):
    """First steps of Algorithm 1 from the same start vector (no reorthogonalisation on
    either side): a_j and b_{j+1} agree to rounding level."""
    L, bonds, nu, nd, t, U = 8, ed_inputs.torus_bonds(2, 4), 3, 3, 1.0, 4.0
    H = hamiltonian.hamiltonian_csr(L, bonds, nu, nd, t, U)
    f1 = olz.normalized_start(ed_inputs.start_vector_raw(6, H.shape[0]))
    ref = olz.lanczos(lambda v: H @ v, f1, max_steps=12, reorth=False, fixed_steps=True)
    res = _solve(ed, L, bonds, nu, nd, t, U, max_steps=12, tol=0.0,
                 f1=torch.tensor(f1, device="cuda"), dtype=dtype)
    assert res["steps"] == 12
    assert np.allclose(res["alpha"], ref.alpha, rtol=1e-11, atol=1e-11)
    assert np.allclose(res["beta"], ref.beta, rtol=1e-11, atol=1e-11)


@pytest.mark.parametrize("dtype", F64_KINDS + ["f32"])
def test_step_api_matches_solve(ed, dtype):
    L, bonds, nu, nd, t, U = 6, ed_inputs.ring_bonds(6), 3, 3, 1.0, 2.0
    b = ed.ed_build_basis(L, bonds, nu, nd)
    try:
        opts = ed.make_opts(max_steps=10, tol=0.0, seed=8, dtype=dtype)
        full = ed.ed_lanczos_solve(b, t, U, opts)
        st = ed.ed_lanczos_init(b, opts)
        try:
            a, bb = [], []
            for _ in range(10):
                s, aj, bj = ed.ed_lanczos_step(st, t, U)
                a.append(aj)
                bb.append(bj)
            E, j = ed.ed_lanczos_energy(st)
        finally:
            ed.ed_lanczos_destroy(st)
        assert j == 10
        assert np.array_equal(np.array(a), full["alpha"]) and np.array_equal(np.array(bb), full["beta"])
        assert E == full["E0"]
    finally:
        ed.ed_basis_destroy(b)


@pytest.mark.parametrize("name,dtype,expect,tol", [
    ("torus4x4_5_5", "f64", -24.0, 1e-10),
    ("torus4x4_5_5", "f64n", -24.0, 1e-10),
    ("ring16_8_8", "f32", -20.109357968503396, 1e-6),
    ("ring16_8_8", "f64", -20.109357968503396, 1e-10),
])
def test_full_size_U0_closed_form(ed, name, dtype, expect, tol):
    """U = 0 at full size: E0 = sum of the lowest single-particle levels."""
    w = ed_inputs.workload(name)
    eps = np.linalg.eigvalsh(_hop_matrix(w["n_sites"], w["bonds"]))
    assert abs(eps[:w["n_up"]].sum() + eps[:w["n_dn"]].sum() - expect) < 1e-12
    res = _solve(ed, w["n_sites"], w["bonds"], w["n_up"], w["n_dn"], 1.0, 0.0, dtype=dtype,
                 seed=w["seed"], max_steps=300, tol=1e-12 if dtype == "f64" else 1e-9)
    assert abs(res["E0"] - expect) <= tol * abs(expect), res["E0"]


def _hop_matrix(L, bonds):
    h = np.zeros((L, L))
    for i, j in bonds:
        h[i, j] -= 1
        h[j, i] -= 1
    return h


def test_fixed_point_matches_native_fp64_from_seeded_start(ed):
    """The FP64-accurate fixed-point run and the native FP64 run from the same seeded device
    start vector produce the same a_j, b_j to rounding level."""
    L, bonds, nu, nd, t, U = 12, ed_inputs.ring_bonds(12), 3, 3, 1.0, 4.0
    b = ed.ed_build_basis(L, bonds, nu, nd)
    try:
        out = {}
        for dt in F64_KINDS:
            out[dt] = ed.ed_lanczos_solve(b, t, U, ed.make_opts(max_steps=15, tol=0.0, seed=1,
                                                                dtype=dt))
        assert np.allclose(out["f64"]["alpha"], out["f64n"]["alpha"], rtol=1e-11, atol=1e-12)
        assert np.allclose(out["f64"]["beta"], out["f64n"]["beta"], rtol=1e-11, atol=1e-12)
    finally:
        ed.ed_basis_destroy(b)


@pytest.mark.parametrize("dtype", ["f64", "f32", "f64n"])
def test_cached_solves_repeat_exactly(ed, dtype):
    """Solves on one basis reuse its cached workspace and graph; changing U or the start
    vector between them must not leak state: a repeated solve returns the same bits."""
    L, bonds, nu, nd = 8, ed_inputs.ring_bonds(8), 3, 3
    b = ed.ed_build_basis(L, bonds, nu, nd)
    try:
        opts = ed.make_opts(max_steps=80, tol=0.0, seed=3, dtype=dtype)
        first = ed.ed_lanczos_solve(b, 1.0, 4.0, opts)
        other = ed.ed_lanczos_solve(b, 1.0, 2.0, opts)
        dim = ed.ed_basis_dims(b)[2]
        tdt = torch.float32 if dtype == "f32" else torch.float64
        f1 = torch.tensor(ed_inputs.uniform_pm1(5, dim), device="cuda", dtype=tdt)
        ed.ed_lanczos_solve(b, 1.0, 4.0, opts, f1=f1)
        again = ed.ed_lanczos_solve(b, 1.0, 4.0, opts)
        assert other["E0"] != first["E0"]
        assert again["E0"] == first["E0"]
        assert np.array_equal(again["alpha"], first["alpha"])
        assert np.array_equal(again["beta"], first["beta"])
    finally:
        ed.ed_basis_destroy(b)


# Every fused H.v variant (schedule id) on a lattice whose down rows span several warp chunks
# with a ragged tail (dim_dn = 462, rows padded to 480), long-range bonds for mixed fermion
# signs and uneven hop counts: a_j, b_{j+1} of the first steps follow the oracle.
VARIANT_LATTICE = (11, np.array([[i, (i + 1) % 11] for i in range(11)] +
                                [[0, 5], [2, 9], [3, 7], [1, 8], [4, 10], [6, 0]]), 3, 5, 1.0, 3.5)
F32_VARIANTS = [1, 2, 3, 4, 5, 6, 7, 14, 31]   # 31: split-row kernel, forced
F64_VARIANTS = [8, 9, 10, 11, 12, 13, 30]      # 30: split-row kernel, forced


@pytest.fixture(scope="module")
def variant_reference():
    L, bonds, nu, nd, t, U = VARIANT_LATTICE
    H = hamiltonian.hamiltonian_csr(L, bonds, nu, nd, t, U)
    f1 = olz.normalized_start(ed_inputs.start_vector_raw(21, H.shape[0]))
    return f1, olz.lanczos(lambda v: H @ v, f1, max_steps=16, reorth=False, fixed_steps=True)


@pytest.mark.parametrize("variant", F32_VARIANTS + F64_VARIANTS)
def test_every_variant_follows_oracle(ed, variant, variant_reference):
    L, bonds, nu, nd, t, U = VARIANT_LATTICE
    f1, ref = variant_reference
    dtype = "f32" if variant in F32_VARIANTS else "f64"
    b = ed.ed_build_basis(L, bonds, nu, nd)
    try:
        opts = ed.make_opts(max_steps=16, tol=0.0, seed=1, dtype=dtype, schedule=variant)
        st = ed.ed_lanczos_init(b, opts)
        try:
            assert ed.ed_lanczos_schedule(st) == variant
        finally:
            ed.ed_lanczos_destroy(st)
        fdev = torch.tensor(f1, dtype=torch.float32 if dtype == "f32" else torch.float64,
                            device="cuda")
        res = ed.ed_lanczos_solve(b, t, U, opts, f1=fdev, raise_not_converged=False)
    finally:
        ed.ed_basis_destroy(b)
    assert res["steps"] == 16
    tol = 2e-5 if dtype == "f32" else 1e-11
    assert np.allclose(res["alpha"], ref.alpha, rtol=tol, atol=tol), (res["alpha"], ref.alpha)
    assert np.allclose(res["beta"], ref.beta, rtol=tol, atol=tol), (res["beta"], ref.beta)


@pytest.mark.parametrize("dtype", ["f32", "f64"])
def test_down_dimension_above_2_15(ed, dtype):
    """L=18 ring with N_dn=9: 48,620 down states, so the FP32 fused H.v addresses shared-memory
    slots above 2^15 (16-bit table entries) and the int64 rows exceed shared memory (general
    kernels). First steps follow the oracle from the same start vector."""
    L, bonds, nu, nd, t, U = 18, ed_inputs.ring_bonds(18), 1, 9, 1.0, 2.0
    H = hamiltonian.hamiltonian_csr(L, bonds, nu, nd, t, U)
    f1 = olz.normalized_start(ed_inputs.start_vector_raw(5, H.shape[0]))
    ref = olz.lanczos(lambda v: H @ v, f1, max_steps=6, reorth=False, fixed_steps=True)
    b = ed.ed_build_basis(L, bonds, nu, nd)
    try:
        # 18 up rows: automatic selection would take the element-parallel kernels, so the
        # FP32 fused variant (R = 1) is requested explicitly
        opts = ed.make_opts(max_steps=6, tol=0.0, seed=1, dtype=dtype,
                            schedule=2 if dtype == "f32" else -1)
        st = ed.ed_lanczos_init(b, opts)
        try:
            variant = ed.ed_lanczos_schedule(st)
        finally:
            ed.ed_lanczos_destroy(st)
        assert variant == (2 if dtype == "f32" else 0)
        fdev = torch.tensor(f1, dtype=torch.float32 if dtype == "f32" else torch.float64,
                            device="cuda")
        res = ed.ed_lanczos_solve(b, t, U, opts, f1=fdev, raise_not_converged=False)
    finally:
        ed.ed_basis_destroy(b)
    tol = 2e-5 if dtype == "f32" else 1e-11
    assert np.allclose(res["alpha"], ref.alpha, rtol=tol, atol=tol), (res["alpha"], ref.alpha)
    assert np.allclose(res["beta"], ref.beta, rtol=tol, atol=tol), (res["beta"], ref.beta)


@pytest.mark.parametrize("tol", [1e-14, 0.0])
@pytest.mark.parametrize("dtype", ["f64", "f32"])
@pytest.mark.parametrize("lattice", ["torus2x4", "ring10"])
def test_per_step_lowest_ritz_value_matches_lapack(ed, dtype, lattice, tol):
    """E0(j) reported for every step equals lambda_min of T_j assembled from the returned a_j,
    b_j, by LAPACK, to a few ulps of ||T_j||: with a convergence test (tol > 0) each step's
    device Sturm multisection, warm-started from E0(j-1); without one (tol = 0) the history
    computed after the run, one multisection per step side by side."""
    import scipy.linalg
    if lattice == "torus2x4":
        L, bonds, nu, nd, U = 8, ed_inputs.torus_bonds(2, 4), 3, 4, 6.0
    else:
        L, bonds, nu, nd, U = 10, ed_inputs.ring_bonds(10), 5, 4, 2.5
    b = ed.ed_build_basis(L, bonds, nu, nd)
    try:
        res = ed.ed_lanczos_solve(b, 1.0, U, ed.make_opts(max_steps=120, tol=tol, seed=3,
                                                          dtype=dtype), raise_not_converged=False)
    finally:
        ed.ed_basis_destroy(b)
    a, bt, hist = res["alpha"], res["beta"], res["E0_hist"]
    n = res["steps"]
    assert n >= 10
    for j in range(1, n + 1):
        w = scipy.linalg.eigvalsh_tridiagonal(a[:j], bt[:j - 1], select="i", select_range=(0, 0))
        scale = np.max(np.abs(a[:j])) + (np.max(np.abs(bt[:j - 1])) if j > 1 else 0.0)
        assert abs(hist[j - 1] - w[0]) <= 8 * EPS64 * max(scale, 1.0), (j, hist[j - 1], w[0])
    assert res["E0"] == hist[n - 1]


@pytest.mark.slow
def test_ring18_half_filling_U0_closed_form(ed):
    """The 18-site 9/9 basis (2,363,904,400 states; 9.5 GB per FP32 vector; int64 indices
    throughout) on one GPU: at U = 0 the closed-shell E0 is 2 x (-2t sin(pi N/L)/sin(pi/L))
    for N = 9 per species."""
    w = ed_inputs.workload("ring18_9_9")
    L, N = w["n_sites"], w["n_up"]
    ref = 2 * (-2.0 * math.sin(math.pi * N / L) / math.sin(math.pi / L))
    b = ed.ed_build_basis(L, w["bonds"], N, N)
    try:
        assert ed.ed_basis_dims(b)[2] == math.comb(18, 9) ** 2
        opts = ed.make_opts(max_steps=400, tol=1e-9, seed=w["seed"], dtype="f32")
        st = ed.ed_lanczos_init(b, opts)
        try:
            assert ed.ed_lanczos_schedule(st) == 31   # the split-row fused kernel (two 97 KB slices)
        finally:
            ed.ed_lanczos_destroy(st)
        res = ed.ed_lanczos_solve(b, 1.0, 0.0, opts, raise_not_converged=False)
    finally:
        ed.ed_basis_destroy(b)
    assert abs(res["E0"] - ref) <= 1e-6 * abs(ref), (res["E0"], ref, res["steps"])



# ----------------------------------------------------------------- single spin species
@pytest.mark.parametrize("dtype", ["f64", "f32"])
@pytest.mark.parametrize("fill", [(8, 0), (0, 8)])
def test_single_species_alpha_beta_follow_oracle(ed, dtype, fill):
    """All particles of one spin (the paper's one-species workloads): the occupied species
    forms one long row internally whichever slot it is given in; a_j, b_{j+1} follow the
    oracle from the same start vector."""
    nu, nd = fill
    L, bonds, t, U = 16, ed_inputs.ring_bonds(16), 1.0, 3.0
    H = hamiltonian.hamiltonian_csr(L, bonds, nu, nd, t, U)
    f1 = olz.normalized_start(ed_inputs.start_vector_raw(31, H.shape[0]))
    ref = olz.lanczos(lambda v: H @ v, f1, max_steps=16, reorth=False, fixed_steps=True)
    b = ed.ed_build_basis(L, bonds, nu, nd)
    try:
        du, dd, dim = ed.ed_basis_dims(b)
        assert (du, dd) == (math.comb(16, nu), math.comb(16, nd)) and dim == math.comb(16, 8)
        fdev = torch.tensor(f1, dtype=torch.float32 if dtype == "f32" else torch.float64,
                            device="cuda")
        res = ed.ed_lanczos_solve(b, t, U, ed.make_opts(max_steps=16, tol=0.0, dtype=dtype),
                                  f1=fdev, raise_not_converged=False)
    finally:
        ed.ed_basis_destroy(b)
    tol = 2e-5 if dtype == "f32" else 1e-11
    assert np.allclose(res["alpha"], ref.alpha, rtol=tol, atol=tol)
    assert np.allclose(res["beta"], ref.beta, rtol=tol, atol=tol)


@pytest.mark.parametrize("fill", [(13, 0), (0, 13)])
def test_single_species_ring26_closed_form(ed, fill):
    """26-site ring with 13 particles of one spin (dim 10,400,600, one row of the layout):
    free fermions, closed shell, E0 = -2t sin(pi N/L) / sin(pi/L)."""
    w = ed_inputs.workload("ring26_13_0")
    L, N = w["n_sites"], 13
    ref = -2.0 * math.sin(math.pi * N / L) / math.sin(math.pi / L)
    b = ed.ed_build_basis(L, w["bonds"], *fill)
    try:
        res = ed.ed_lanczos_solve(b, 1.0, w["U"], ed.make_opts(max_steps=600, tol=1e-13, seed=w["seed"]))
    finally:
        ed.ed_basis_destroy(b)
    assert abs(res["E0"] - ref) <= 1e-11 * abs(ref), (res["E0"], ref, res["steps"])


@pytest.mark.parametrize("name", ["variant_lattice", "ring14_7_7"])
def test_fp32_norm_accumulation_matches_fp64_norm(ed, name):
    """The FP32 path accumulates dot products per thread as compensated FP32 pairs (Dot2),
    summed in FP64: b_{j+1} returned by a step equals the FP64 norm of the very FP32 vector
    q the step wrote (read back through ed_lanczos_buffers) to 1e-12 relative over several
    steps (the lattice with padded rows of the variant tests, and the 11.8 M-state 14-site
    ring). FP32 products summed in FP64 would be off by ~1e-11 relative at this size, a
    plain FP32 running sum by ~1e-7; Dot2 measures ~2e-14 here (its bound, gamma_n^2 for n
    terms per thread, is far looser)."""
    if name == "ring14_7_7":
        w = ed_inputs.workload(name)
        L, bonds, nu, nd, t, U = w["n_sites"], w["bonds"], w["n_up"], w["n_dn"], w["t"], w["U"]
    else:
        L, bonds, nu, nd, t, U = VARIANT_LATTICE
    b = ed.ed_build_basis(L, bonds, nu, nd)
    try:
        du, dd, dim = ed.ed_basis_dims(b)
        st = ed.ed_lanczos_init(b, ed.make_opts(max_steps=20, tol=0.0, seed=3, dtype="f32"))
        try:
            for _ in range(5):
                s, a_j, b_j1 = ed.ed_lanczos_step(st, t, U)
                bufs = ed.ed_lanczos_buffers(st)
                n = du * bufs["ld"]
                q = dev_to_numpy(bufs["f_next"], n, "<f4").astype(np.float64)
                norm = float(np.sqrt(q @ q))          # FP64 norm of the FP32 values
                assert abs(b_j1 - norm) <= 1e-12 * norm, (b_j1, norm)
                assert bufs["scale_next"] == pytest.approx(1.0 / b_j1, rel=1e-15)
        finally:
            ed.ed_lanczos_destroy(st)
    finally:
        ed.ed_basis_destroy(b)


@pytest.mark.parametrize("t,U", [(1e-3, 1e6), (1e4, 0.5), (1.0, 1e-9)])
@pytest.mark.parametrize("tol", [1e-14, 0.0])
def test_per_step_lowest_ritz_value_at_extreme_scales(ed, t, U, tol):
    """E0(j) at every step against LAPACK on the returned a_j, b_j when the entries of T span
    many orders of magnitude (U / t up to 1e9) or sit far from 1 in size: the bisection's
    float-float rounds (FP32 exponents, rescaled) and its FP64 finish must still give E0 to a
    few units in the last place of ||T_j||."""
    import scipy.linalg
    L, nu, nd = 8, 3, 3
    b = ed.ed_build_basis(L, ed_inputs.ring_bonds(L), nu, nd)
    try:
        res = ed.ed_lanczos_solve(b, t, U, ed.make_opts(max_steps=60, tol=tol, seed=5, dtype="f64"),
                                  raise_not_converged=False)
    finally:
        ed.ed_basis_destroy(b)
    a, bt, hist = res["alpha"], res["beta"], res["E0_hist"]
    n = res["steps"]
    assert n >= 3
    for j in range(1, n + 1):
        w = scipy.linalg.eigvalsh_tridiagonal(a[:j], bt[:j - 1], select="i", select_range=(0, 0))
        scale = np.max(np.abs(a[:j])) + (np.max(np.abs(bt[:j - 1])) if j > 1 else 0.0)
        assert abs(hist[j - 1] - w[0]) <= 8 * EPS64 * max(scale, 1e-300), (j, hist[j - 1], w[0])


# ------------------------------------------------- irregular lattices on the row-staged path
RANDOM_LARGE = ed_inputs.random_lattices()


def _tuple(case):
    return (case["n_sites"], case["bonds"], case["n_up"], case["n_dn"], case["t"], case["U"])


@pytest.fixture(scope="module")
def random_large_reference():
    """Oracle a_j, b_{j+1} of 12 steps of plain Algorithm 1 (no reorthogonalisation) from
    the seeded start, one explicit H per lattice."""
    out = {}
    for case in RANDOM_LARGE:
        H = hamiltonian.hamiltonian_csr(*_tuple(case))
        f1 = olz.normalized_start(ed_inputs.start_vector_raw(41, H.shape[0]))
        out[case["name"]] = (f1, olz.lanczos(lambda v: H @ v, f1, max_steps=12, reorth=False,
                                             fixed_steps=True))
    return out


@pytest.mark.parametrize("dtype", ["f64", "f32"])
@pytest.mark.parametrize("case", RANDOM_LARGE, ids=lambda c: c["name"])
def test_random_lattices_hv_elementwise(ed, case, dtype):
    """ed_hv on irregular bond lists (uneven degrees, a doubled and a reversed bond, U of
    either sign) with 210 to 792 up rows, every element against the oracle's rows within
    the rounding bound."""
    L, bonds, nu, nd, t, U = _tuple(case)
    b = ed.ed_build_basis(L, bonds, nu, nd)
    try:
        dim = ed.ed_basis_dims(b)[2]
        tdt = torch.float64 if dtype == "f64" else torch.float32
        xd = torch.tensor(ed_inputs.uniform_pm1(43, dim), device="cuda", dtype=tdt)
        yd = torch.empty_like(xd)
        ed.ed_hv(b, t, U, xd, yd)
        xr = xd.double().cpu().numpy()
        rows = np.arange(dim)
        ref = hamiltonian.hv_rows(L, bonds, nu, nd, t, U, xr, rows)
        bound = _hv_bound(_tuple(case), xr, rows, EPS64 if dtype == "f64" else EPS32)
        err = np.abs(yd.double().cpu().numpy() - ref)
        assert np.all(err <= bound), float((err / bound).max())
    finally:
        ed.ed_basis_destroy(b)


@pytest.mark.parametrize("dtype", F64_KINDS + ["f32"])
@pytest.mark.parametrize("case", RANDOM_LARGE, ids=lambda c: c["name"])
def test_random_lattices_alpha_beta_follow_oracle(ed, case, dtype, random_large_reference):
    """The fused Lanczos step (autotuned variant) on the same irregular lattices: 12 steps
    of a_j, b_{j+1} from the oracle's start vector against the oracle's plain Algorithm 1."""
    L, bonds, nu, nd, t, U = _tuple(case)
    f1, ref = random_large_reference[case["name"]]
    fdev = torch.tensor(f1, dtype=torch.float32 if dtype == "f32" else torch.float64,
                        device="cuda")
    res = _solve(ed, L, bonds, nu, nd, t, U, max_steps=12, tol=0.0, f1=fdev, dtype=dtype)
    assert res["steps"] == 12
    tol = 2e-5 if dtype == "f32" else 1e-11
    assert np.allclose(res["alpha"], ref.alpha, rtol=tol, atol=tol), (res["alpha"], ref.alpha)
    assert np.allclose(res["beta"], ref.beta, rtol=tol, atol=tol), (res["beta"], ref.beta)
