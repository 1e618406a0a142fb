"""Python binding of libed, the GB300 CUDA library for exact diagonalization of the
tight-binding / Hubbard model by the Lanczos method (Siro & Harju, arXiv:1511.00863).

Argument marshalling only: every function forwards to the C entry point of the same name
declared in include/ed.h. Vectors are torch CUDA tensors (device memory owned by the
caller); the CUDA stream defaults to torch's current stream. There is no fallback: if the
compiled library is missing, importing this package raises.
"""
from __future__ import annotations

import ctypes
import os
from ctypes import POINTER, byref, c_double, c_int, c_int32, c_int64, c_uint32, c_uint64, c_void_p

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
# ED_LIB_PATH selects another build of the same library (e.g. a debug or instrumented one)
LIB_PATH = os.environ.get("ED_LIB_PATH") or os.path.join(_HERE, "libed.so")

ED_OK, ED_BREAKDOWN = 0, 1
ED_ERR_ARG, ED_ERR_OOM, ED_ERR_CUDA, ED_ERR_TIMEOUT, ED_ERR_NOT_CONVERGED = -1, -2, -3, -4, -5
ED_F64, ED_F32, ED_F64_NATIVE, ED_C32, ED_C64 = 0, 1, 2, 3, 4
ED_MAX_STEPS = 1000


class EdError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"libed status {status}: {message}")
        self.status = status


class ed_lattice(ctypes.Structure):
    _fields_ = [("n_sites", c_int32), ("n_bonds", c_int32), ("bonds", POINTER(c_int32)),
                ("t_bond", POINTER(c_double))]


class ed_params(ctypes.Structure):
    _fields_ = [("t", c_double), ("U", c_double)]


class ed_opts(ctypes.Structure):
    _fields_ = [("max_steps", c_int32), ("tol", c_double), ("reorth", c_int32),
                ("seed", c_uint64), ("dtype", c_int), ("schedule", c_int32)]


if not os.path.exists(LIB_PATH):
    raise ImportError(f"libed.so not built ({LIB_PATH}); run __graft_entry__.build() or "
                      "python -m paper_1511_00863_gb300.build")
_lib = ctypes.CDLL(LIB_PATH)

_SIGS = {
    "ed_build_basis": (c_int, [POINTER(ed_lattice), c_int32, c_int32, c_void_p, POINTER(c_void_p)]),
    "ed_basis_dims": (c_int, [c_void_p, POINTER(c_int64), POINTER(c_int64), POINTER(c_int64)]),
    "ed_basis_filling": (c_int, [c_void_p, POINTER(c_int32), POINTER(c_int32), POINTER(c_int32)]),
    "ed_basis_tables": (c_int, [c_void_p, POINTER(c_void_p), POINTER(c_void_p), POINTER(c_void_p),
                                POINTER(c_void_p), POINTER(c_int32), POINTER(c_int32)]),
    "ed_basis_destroy": (None, [c_void_p]),
    "ed_hv": (c_int, [c_void_p, POINTER(ed_params), c_int, c_void_p, c_void_p, c_void_p]),
    "ed_start_vector": (c_int, [c_int64, c_uint64, c_int, c_void_p, c_void_p]),
    "ed_start_vector_noalloc": (c_int, [c_int64, c_uint64, c_int, c_void_p, c_void_p]),
    "ed_lanczos_init": (c_int, [c_void_p, POINTER(ed_opts), c_void_p, c_void_p, POINTER(c_void_p)]),
    "ed_lanczos_step": (c_int, [c_void_p, POINTER(ed_params), POINTER(c_double), POINTER(c_double)]),
    "ed_lanczos_run": (c_int, [c_void_p, POINTER(ed_params), c_int32, POINTER(ctypes.c_float)]),
    "ed_lanczos_energy": (c_int, [c_void_p, POINTER(c_double), POINTER(c_int32)]),
    "ed_lanczos_schedule": (c_int, [c_void_p, POINTER(c_int32)]),
    "ed_lanczos_buffers": (c_int, [c_void_p, POINTER(c_void_p), POINTER(c_void_p), POINTER(c_double),
                                   POINTER(c_double), POINTER(c_int64), POINTER(c_void_p)]),
    "ed_lanczos_destroy": (None, [c_void_p]),
    "ed_lanczos_solve": (c_int, [c_void_p, POINTER(ed_params), POINTER(ed_opts), c_void_p, c_void_p,
                                 POINTER(c_double), POINTER(c_int32), POINTER(c_double),
                                 POINTER(c_double), POINTER(c_double)]),
    "ed_lanczos_solve_mixed": (c_int, [c_void_p, POINTER(ed_params), POINTER(ed_opts), c_void_p, c_int32,
                                       c_double, c_void_p, POINTER(c_double), POINTER(c_int32),
                                       POINTER(c_double), POINTER(c_int32), POINTER(c_double)]),
    "ed_lanczos_solve_batched": (c_int, [c_int32, POINTER(c_void_p), POINTER(ed_params),
                                         POINTER(ed_opts), c_void_p, POINTER(c_double),
                                         POINTER(c_int32), POINTER(c_int32), POINTER(c_int32)]),
    "ed_lanczos_solve_batched_mixed": (c_int, [c_int32, POINTER(c_void_p), POINTER(ed_params),
                                               POINTER(ed_opts), c_int32, c_double, c_void_p,
                                               POINTER(c_double), POINTER(c_int32), POINTER(c_int32),
                                               POINTER(c_int32), POINTER(c_int32)]),
    "ed_selftest_barrier_timeout": (c_int, [c_int32, c_int32, c_void_p]),
    "ed_lanczos_ground_state": (c_int, [c_void_p, POINTER(ed_params), POINTER(ed_opts), c_void_p,
                                        c_void_p, c_void_p, POINTER(c_double), POINTER(c_int32)]),
    "ed_double_occupancy": (c_int, [c_void_p, c_void_p, c_void_p, POINTER(c_double), POINTER(c_double)]),
    "ed_mlp_create": (c_int, [c_int32, c_uint64, c_void_p, POINTER(c_void_p)]),
    "ed_mlp_params": (c_int, [c_void_p, POINTER(c_void_p), POINTER(c_int64)]),
    "ed_mlp_loss_grad": (c_int, [c_void_p, c_void_p, c_double, c_void_p, c_void_p, c_int64,
                                 c_double, POINTER(c_double), POINTER(c_void_p)]),
    "ed_mlp_train_step": (c_int, [c_void_p, c_void_p, c_double, c_void_p, c_int64, c_double,
                                  c_uint64, POINTER(c_double)]),
    "ed_mlp_infer": (c_int, [c_void_p, c_void_p, c_double, c_int, c_void_p]),
    "ed_mlp_destroy": (None, [c_void_p]),
    "ed_hv_down_tables": (c_int, [c_void_p, c_void_p, c_void_p, c_int64, c_int32, c_int32, c_int32,
                                  c_int32, c_int32, c_void_p, c_int32, POINTER(c_int32), c_void_p,
                                  c_void_p, c_void_p]),
    "ed_hv_split_tables": (c_int, [c_void_p, c_void_p, c_int64, c_int32, c_int32, c_int32, c_int32,
                                   c_void_p, c_void_p, c_int32, c_int32, POINTER(c_int32),
                                   POINTER(c_int32), POINTER(c_int32), c_void_p, c_void_p, c_void_p,
                                   c_void_p]),
    "ed_last_error": (ctypes.c_char_p, []),
}
for _name, (_res, _args) in _SIGS.items():
    _fn = getattr(_lib, _name)
    _fn.restype = _res
    _fn.argtypes = _args


def _check(status: int) -> int:
    if status < 0:
        raise EdError(status, _lib.ed_last_error().decode(errors="replace"))
    return status


def _stream(stream):
    if stream is None:
        import torch
        return c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return c_void_p(stream)
    return c_void_p(stream.cuda_stream)


def _ptr(t, dtype_code=None, numel=None):
    """Device pointer of a contiguous CUDA tensor (checked), or NULL for None."""
    if t is None:
        return c_void_p(None)
    import torch
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.is_contiguous()):
        raise ValueError("expected a contiguous CUDA tensor")
    if dtype_code is not None:
        want = {ED_F32: torch.float32, ED_C32: torch.complex64,
                ED_C64: torch.complex128}.get(dtype_code, torch.float64)
        if t.dtype != want:
            raise ValueError(f"expected {want}, got {t.dtype}")
    if numel is not None and t.numel() != numel:
        raise ValueError(f"expected {numel} elements, got {t.numel()}")
    return c_void_p(t.data_ptr())


def dtype_code(dtype) -> int:
    if dtype in (ED_F64_NATIVE, "f64n", "f64_native"):
        return ED_F64_NATIVE
    if dtype in (ED_F64, "f64", "float64", "fp64"):
        return ED_F64
    if dtype in (ED_F32, "f32", "float32", "fp32"):
        return ED_F32
    if dtype in (ED_C32, "c32", "complex64"):
        return ED_C32
    if dtype in (ED_C64, "c64", "complex128"):
        return ED_C64
    import torch
    if dtype == torch.float64:
        return ED_F64
    if dtype == torch.float32:
        return ED_F32
    if dtype == torch.complex64:
        return ED_C32
    if dtype == torch.complex128:
        return ED_C64
    raise ValueError(f"unknown dtype {dtype!r}")


# ------------------------------------------------------------------------ basis
def ed_build_basis(n_sites: int, bonds, n_up: int, n_dn: int, stream=None, t_bond=None) -> c_void_p:
    """t_bond: None, or one complex relative amplitude per bond (then only the complex
    dtypes apply)."""
    b = np.ascontiguousarray(np.asarray(bonds, dtype=np.int32).reshape(-1, 2))
    tb = None
    if t_bond is not None:
        tc = np.asarray(t_bond, dtype=np.complex128).reshape(-1)
        if tc.shape[0] != b.shape[0]:
            raise ValueError("t_bond needs one amplitude per bond")
        tb = np.ascontiguousarray(np.stack([tc.real, tc.imag], axis=1).reshape(-1))
    lat = ed_lattice(n_sites, b.shape[0], b.ctypes.data_as(POINTER(c_int32)),
                     tb.ctypes.data_as(POINTER(c_double)) if tb is not None else None)
    out = c_void_p()
    _check(_lib.ed_build_basis(byref(lat), n_up, n_dn, _stream(stream), byref(out)))
    return out


def ed_basis_dims(basis) -> tuple[int, int, int]:
    du, dd, d = c_int64(), c_int64(), c_int64()
    _check(_lib.ed_basis_dims(basis, byref(du), byref(dd), byref(d)))
    return du.value, dd.value, d.value


def ed_hv_down_tables(hop, bits, V: int, G: int, hop_amp=None, complex_entries: bool = False):
    """Host-only: the fused H.v's down tables of one species (no GPU needed).

    hop: int32 [maxhops][dim] (target | sign << 31), bits: uint32 [dim], hop_amp: optional
    int32 [maxhops][dim]. Returns dict(table [rows][ld] uint32, kpn [chunks][2] uint8,
    slot_lo [ld] uint8, colpos [dim] int32, ld).
    """
    hop = np.ascontiguousarray(hop, dtype=np.int32)
    bits = np.ascontiguousarray(bits, dtype=np.uint32)
    mh, dim = (hop.shape if hop.ndim == 2 else (0, bits.size))
    ld = (dim + 31) // 32 * 32
    amp = None if hop_amp is None else np.ascontiguousarray(hop_amp, dtype=np.int32)
    cap = max(1, 2 * mh)
    table = np.zeros((cap, ld), dtype=np.uint32)
    kpn = np.zeros(2 * ((ld + 32 * V - 1) // (32 * V)), dtype=np.uint8)
    lo = np.zeros(ld, dtype=np.uint8)
    colpos = np.zeros(dim, dtype=np.int32)
    rows = c_int32(0)
    _check(_lib.ed_hv_down_tables(hop.ctypes.data if mh else None,
                                  None if amp is None else amp.ctypes.data, bits.ctypes.data,
                                  dim, mh, ld, V, G, int(complex_entries), table.ctypes.data, cap,
                                  byref(rows), kpn.ctypes.data, lo.ctypes.data, colpos.ctypes.data))
    return {"table": table[:rows.value].copy(), "kpn": kpn.reshape(-1, 2), "slot_lo": lo,
            "colpos": colpos, "ld": ld}


def ed_hv_split_tables(hop, bits, V: int, G: int, site: int = 0):
    """Host-only: the split-row fused H.v's down tables of one species (no GPU needed).

    Returns dict(table [rows][ld] uint16 in-slice slots, xtable [xrows][ld] uint16 columns in
    the other slice, kpn [chunks][4] uint8, slot_lo [ld] uint8, cstart [3], colpos [dim]
    int32, ld)."""
    hop = np.ascontiguousarray(hop, dtype=np.int32)
    bits = np.ascontiguousarray(bits, dtype=np.uint32)
    mh, dim = (hop.shape if hop.ndim == 2 else (0, bits.size))
    cols = 2 * ((dim + 32 * V) // (32 * V) + 1) * 32 * V
    cap = max(1, 2 * mh)
    table = np.zeros(cap * cols, dtype=np.uint16)
    xtable = np.zeros(cap * cols, dtype=np.uint16)
    kpn = np.zeros(4 * (cols // (32 * V)), dtype=np.uint8)
    lo = np.zeros(cols, dtype=np.uint8)
    cstart = np.zeros(3, dtype=np.int32)
    colpos = np.zeros(dim, dtype=np.int32)
    rows, xrows, ld = c_int32(0), c_int32(0), c_int32(0)
    _check(_lib.ed_hv_split_tables(hop.ctypes.data if mh else None, bits.ctypes.data, dim, mh, V, G,
                                   site, table.ctypes.data, xtable.ctypes.data, cap, cols,
                                   byref(rows), byref(xrows), byref(ld), cstart.ctypes.data,
                                   kpn.ctypes.data, lo.ctypes.data, colpos.ctypes.data))
    n, nx, w = rows.value * ld.value, xrows.value * ld.value, ld.value
    return {"table": table[:n].reshape(rows.value, w).copy(),
            "xtable": xtable[:nx].reshape(xrows.value, w).copy(),
            "kpn": kpn[:4 * (w // (32 * V))].reshape(-1, 4).copy(), "slot_lo": lo[:w].copy(),
            "cstart": cstart.copy(), "colpos": colpos, "ld": w}


def ed_basis_filling(basis):
    """(n_sites, n_up, n_dn)."""
    L, nu, nd = c_int32(), c_int32(), c_int32()
    _check(_lib.ed_basis_filling(basis, byref(L), byref(nu), byref(nd)))
    return L.value, nu.value, nd.value


def ed_basis_tables(basis) -> dict:
    ub, db, hu, hd = c_void_p(), c_void_p(), c_void_p(), c_void_p()
    mu, md = c_int32(), c_int32()
    _check(_lib.ed_basis_tables(basis, byref(ub), byref(db), byref(hu), byref(hd), byref(mu),
                                byref(md)))
    return dict(up_bits=ub.value, dn_bits=db.value, hop_up=hu.value, hop_dn=hd.value,
                maxhops_up=mu.value, maxhops_dn=md.value)


def ed_basis_destroy(basis) -> None:
    _lib.ed_basis_destroy(basis)


# ------------------------------------------------------------------------ H.v
def ed_hv(basis, t: float, U: float, x, y, stream=None) -> None:
    code = dtype_code(x.dtype)
    dim = ed_basis_dims(basis)[2]
    p = ed_params(t, U)
    _check(_lib.ed_hv(basis, byref(p), code, _ptr(x, code, dim), _ptr(y, code, dim),
                      _stream(stream)))


def ed_start_vector(dim: int, seed: int, out, stream=None) -> None:
    code = dtype_code(out.dtype)
    _check(_lib.ed_start_vector(dim, seed, code, _ptr(out, code, dim), _stream(stream)))


def ed_start_vector_noalloc(dim: int, seed: int, out, stream=None) -> None:
    """ed_start_vector without any device allocation (scratch in static device memory);
    for callers that must not allocate device memory while they run."""
    code = dtype_code(out.dtype)
    _check(_lib.ed_start_vector_noalloc(dim, seed, code, _ptr(out, code, dim), _stream(stream)))


# ------------------------------------------------------------------------ Lanczos
def make_opts(max_steps=200, tol=1e-12, reorth=0, seed=1, dtype=ED_F64, schedule=-1) -> ed_opts:
    return ed_opts(max_steps, tol, reorth, seed, dtype_code(dtype), schedule)


def ed_lanczos_init(basis, opts: ed_opts, f1=None, stream=None) -> c_void_p:
    dim = ed_basis_dims(basis)[2]
    out = c_void_p()
    _check(_lib.ed_lanczos_init(basis, byref(opts), _ptr(f1, opts.dtype, dim), _stream(stream),
                                byref(out)))
    return out


def ed_lanczos_step(st, t: float, U: float) -> tuple[int, float, float]:
    a, b = c_double(), c_double()
    p = ed_params(t, U)
    s = _check(_lib.ed_lanczos_step(st, byref(p), byref(a), byref(b)))
    return s, a.value, b.value


def ed_lanczos_run(st, t: float, U: float, nsteps: int, time_hv: bool = False):
    """Enqueue nsteps iterations; with time_hv, returns the summed fused H.v time (ms)."""
    p = ed_params(t, U)
    if time_hv:
        ms = ctypes.c_float()
        _check(_lib.ed_lanczos_run(st, byref(p), nsteps, byref(ms)))
        return ms.value
    _check(_lib.ed_lanczos_run(st, byref(p), nsteps, None))
    return None


def ed_lanczos_schedule(st) -> int:
    v = c_int32()
    _check(_lib.ed_lanczos_schedule(st, byref(v)))
    return v.value


def ed_lanczos_energy(st) -> tuple[float, int]:
    e, j = c_double(), c_int32()
    _check(_lib.ed_lanczos_energy(st, byref(e), byref(j)))
    return e.value, j.value


def ed_lanczos_destroy(st) -> None:
    _lib.ed_lanczos_destroy(st)


def ed_lanczos_solve(basis, t: float, U: float, opts: ed_opts, f1=None, stream=None,
                     raise_not_converged: bool = True, history: bool = True) -> dict:
    """history=False skips the per-step E0(j) (computed then only at the last step)."""
    dim = ed_basis_dims(basis)[2]
    p = ed_params(t, U)
    E0, steps = c_double(), c_int32()
    alpha = (c_double * opts.max_steps)()
    beta = (c_double * opts.max_steps)()
    hist = (c_double * opts.max_steps)() if history else None
    s = _lib.ed_lanczos_solve(basis, byref(p), byref(opts), _ptr(f1, opts.dtype, dim),
                              _stream(stream), byref(E0), byref(steps), alpha, beta, hist)
    if s < 0 and not (s == ED_ERR_NOT_CONVERGED and not raise_not_converged):
        _check(s)
    n = steps.value
    return dict(status=s, E0=E0.value, steps=n, alpha=np.array(alpha[:n]), beta=np.array(beta[:n]),
                E0_hist=np.array(hist[:n]) if history else None)


def ed_lanczos_buffers(st) -> dict:
    """Device pointers and scales of the state's two work vectors (see include/ed.h)."""
    fn, fc, cp = c_void_p(), c_void_p(), c_void_p()
    sn, sc = c_double(), c_double()
    ld = c_int64()
    _check(_lib.ed_lanczos_buffers(st, byref(fn), byref(fc), byref(sn), byref(sc), byref(ld), byref(cp)))
    return dict(f_next=fn.value, f_cur=fc.value, scale_next=sn.value, scale_cur=sc.value, ld=ld.value,
                colpos=cp.value)


def ed_lanczos_solve_mixed(basis, t: float, U: float, opts: ed_opts, f1=None, refine_steps: int = 64,
                           refine_tol: float = 1e-12, stream=None, raise_not_converged: bool = True) -> dict:
    """FP32 Lanczos, its Ritz vector, then FP64-accurate Lanczos from it (at most
    refine_steps steps, convergence test refine_tol)."""
    dim = ed_basis_dims(basis)[2]
    p = ed_params(t, U)
    E0, e32, res = c_double(), c_double(), c_double()
    s32, s64 = c_int32(), c_int32()
    s = _lib.ed_lanczos_solve_mixed(basis, byref(p), byref(opts), _ptr(f1, opts.dtype, dim), refine_steps,
                                    refine_tol, _stream(stream), byref(E0), byref(s32), byref(e32),
                                    byref(s64), byref(res))
    if s < 0 and not (s == ED_ERR_NOT_CONVERGED and not raise_not_converged):
        _check(s)
    return dict(status=s, E0=E0.value, steps32=s32.value, E0_fp32=e32.value, steps64=s64.value,
                residual=res.value)


def ed_lanczos_solve_batched(bases, ts, Us, opts: ed_opts, stream=None,
                             raise_not_converged: bool = True) -> dict:
    """All instances in one persistent launch; ts, Us: per-instance parameters."""
    n = len(bases)
    arr = (c_void_p * n)(*[b.value if isinstance(b, c_void_p) else b for b in bases])
    params = (ed_params * n)(*[ed_params(float(t), float(u)) for t, u in zip(ts, Us)])
    E0 = (c_double * n)()
    steps = (c_int32 * n)()
    status = (c_int32 * n)()
    used = c_int32()
    s = _lib.ed_lanczos_solve_batched(n, arr, params, byref(opts), _stream(stream), E0, steps,
                                      status, byref(used))
    if s < 0 and not (s == ED_ERR_NOT_CONVERGED and not raise_not_converged):
        _check(s)
    return dict(status=s, E0=np.array(E0[:]), steps=np.array(steps[:]),
                inst_status=np.array(status[:]), schedule=used.value)


def ed_lanczos_solve_batched_mixed(bases, ts, Us, opts: ed_opts, refine_steps: int = 32,
                                   refine_tol: float = 1e-12, stream=None,
                                   raise_not_converged: bool = True) -> dict:
    """All instances in one persistent launch: FP32 Lanczos (opts), Ritz vector, FP64
    refinement (see include/ed.h)."""
    n = len(bases)
    arr = (c_void_p * n)(*[b.value if isinstance(b, c_void_p) else b for b in bases])
    params = (ed_params * n)(*[ed_params(float(t), float(u)) for t, u in zip(ts, Us)])
    E0 = (c_double * n)()
    s32 = (c_int32 * n)()
    s64 = (c_int32 * n)()
    status = (c_int32 * n)()
    used = c_int32()
    s = _lib.ed_lanczos_solve_batched_mixed(n, arr, params, byref(opts), refine_steps, refine_tol,
                                            _stream(stream), E0, s32, s64, status, byref(used))
    if s < 0 and not (s == ED_ERR_NOT_CONVERGED and not raise_not_converged):
        _check(s)
    return dict(status=s, E0=np.array(E0[:]), steps32=np.array(s32[:]), steps64=np.array(s64[:]),
                inst_status=np.array(status[:]), schedule=used.value)


def ed_selftest_barrier_timeout(ctas: int = 4, timeout_ms: int = 50, stream=None) -> int:
    """Returns the raw status: ED_ERR_TIMEOUT means the bounded wait ran out as intended."""
    return _lib.ed_selftest_barrier_timeout(ctas, timeout_ms, _stream(stream))


def ed_lanczos_ground_state(basis, t: float, U: float, opts: ed_opts, psi, f1=None,
                            stream=None, raise_not_converged: bool = True) -> dict:
    dim = ed_basis_dims(basis)[2]
    p = ed_params(t, U)
    E0, steps = c_double(), c_int32()
    s = _lib.ed_lanczos_ground_state(basis, byref(p), byref(opts), _ptr(f1, ED_F64, dim),
                                     _stream(stream), _ptr(psi, ED_F64, dim), byref(E0), byref(steps))
    if s < 0 and not (s == ED_ERR_NOT_CONVERGED and not raise_not_converged):
        _check(s)
    return dict(status=s, E0=E0.value, steps=steps.value)


def ed_double_occupancy(basis, psi, stream=None):
    """(D, D_site): double occupancy of the FP64 state psi (device, basis order)."""
    import numpy as np
    dim = ed_basis_dims(basis)[2]
    n_sites = ed_basis_filling(basis)[0]
    D = c_double()
    site = (c_double * max(n_sites, 1))()
    _check(_lib.ed_double_occupancy(basis, _ptr(psi, ED_F64, dim), _stream(stream), byref(D), site))
    return D.value, np.array(site[:n_sites])


def ed_mlp_create(n_sites: int, seed: int, stream=None) -> c_void_p:
    out = c_void_p()
    _check(_lib.ed_mlp_create(n_sites, seed, _stream(stream), byref(out)))
    return out


def ed_mlp_params(mlp):
    """(device pointer, count) of the FP32 master parameters."""
    p, n = c_void_p(), c_int64()
    _check(_lib.ed_mlp_params(mlp, byref(p), byref(n)))
    return p.value, n.value


def ed_mlp_loss_grad(mlp, basis, U: float, idx, target, weight_scale: float):
    """Returns (loss, device pointer of the gradient)."""
    n = idx.numel()
    loss, g = c_double(), c_void_p()
    if target.numel() != n or idx.dtype.itemsize != 8:
        raise ValueError("idx (int64) and target (float64) must have the same length")
    _check(_lib.ed_mlp_loss_grad(mlp, basis, U, _ptr(idx), _ptr(target, ED_F64, n), n,
                                 weight_scale, byref(loss), byref(g)))
    return loss.value, g.value


def ed_mlp_train_step(mlp, basis, U: float, psi, batch: int, lr: float, seed: int) -> float:
    loss = c_double()
    _check(_lib.ed_mlp_train_step(mlp, basis, U, _ptr(psi, ED_F64), batch, lr, seed, byref(loss)))
    return loss.value


def ed_mlp_infer(mlp, basis, U: float, out) -> None:
    code = dtype_code(out.dtype)
    dim = ed_basis_dims(basis)[2]
    _check(_lib.ed_mlp_infer(mlp, basis, U, code, _ptr(out, code, dim)))


def ed_mlp_destroy(mlp) -> None:
    _lib.ed_mlp_destroy(mlp)


def ed_last_error() -> str:
    return _lib.ed_last_error().decode(errors="replace")
