"""The C-ABI library loads and exports every function include/ed.h declares (no GPU)."""
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = []
    for h in os.listdir(os.path.join(ROOT, "include")):
        if h.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", h)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names += re.findall(r"\b(ed_[a-z0-9_]+)\s*\(", txt)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib_path():
    import __graft_entry__
    b = __graft_entry__._build_module()
    if not os.path.exists(b.LIB):
        b.build()
    return b.LIB


def test_header_declares_the_boundary():
    names = _declared()
    for n in ("ed_build_basis", "ed_hv", "ed_lanczos_step", "ed_lanczos_solve"):
        assert n in names


def test_library_exports_every_declared_symbol(lib_path):
    out = subprocess.run(["nm", "-D", "--defined-only", lib_path], capture_output=True,
                         text=True, check=True).stdout
    exported = set(line.split()[-1] for line in out.splitlines() if line.strip())
    missing = [n for n in _declared() if n not in exported]
    assert not missing, missing


def test_binding_loads_and_covers_header(lib_path):
    import paper_1511_00863_gb300 as ed
    for n in _declared():
        assert callable(getattr(ed, n)), n


def test_argument_errors_without_gpu(lib_path):
    """Invalid arguments are rejected on the host before any CUDA call."""
    import paper_1511_00863_gb300 as ed
    with pytest.raises(ed.EdError) as e:
        ed.ed_build_basis(40, [[0, 1]], 1, 1, stream=0)
    assert e.value.status == ed.ED_ERR_ARG and "n_sites" in str(e.value)
    with pytest.raises(ed.EdError):
        ed.ed_build_basis(4, [[0, 0]], 1, 1, stream=0)
    with pytest.raises(ed.EdError):
        ed.ed_build_basis(4, [[0, 1]], 5, 1, stream=0)
    bad = [((4, [[0, 4]], 1, 1), "bond 0"), ((4, [[-1, 2]], 1, 1), "bond 0"),
           ((4, [[0, 1]], -1, 1), "particle numbers"), ((0, [], 0, 0), "n_sites"),
           ((33, [[0, 1]], 1, 1), "n_sites"), ((32, [[0, 31]], 33, 0), "particle numbers")]
    for args, word in bad:
        with pytest.raises(ed.EdError) as e:
            ed.ed_build_basis(*args, stream=0)
        assert e.value.status == ed.ED_ERR_ARG and word in str(e.value), str(e.value)


def test_batched_argument_errors_without_gpu(lib_path):
    """The batched entry points reject bad options on the host before any CUDA call: the mixed
    solve's FP32 phase must be ED_F32, its refinement length must be in range, neither takes
    reorthogonalisation, and the plain batch takes only ED_F32 or ED_F64_NATIVE."""
    import paper_1511_00863_gb300 as ed
    bases = [None]   # not reached: the options are checked first
    cases = [
        (lambda: ed.ed_lanczos_solve_batched_mixed(bases, [1.0], [4.0], ed.make_opts(dtype="f64"), stream=0),
         "ED_F32"),
        (lambda: ed.ed_lanczos_solve_batched_mixed(bases, [1.0], [4.0], ed.make_opts(dtype="f32"),
                                                   refine_steps=0, stream=0), "refine_steps"),
        (lambda: ed.ed_lanczos_solve_batched_mixed(bases, [1.0], [4.0], ed.make_opts(dtype="f32", reorth=1),
                                                   stream=0), "reorth"),
        (lambda: ed.ed_lanczos_solve_batched(bases, [1.0], [4.0], ed.make_opts(dtype="c32"), stream=0),
         "dtype"),
        (lambda: ed.ed_lanczos_solve_batched(bases, [1.0], [4.0], ed.make_opts(dtype="f32", max_steps=0),
                                             stream=0), "max_steps"),
    ]
    for call, word in cases:
        with pytest.raises(ed.EdError) as e:
            call()
        assert e.value.status == ed.ED_ERR_ARG and word in str(e.value), str(e.value)


def test_null_arguments_rejected_without_gpu(lib_path):
    """Every entry point called with NULL pointers and zero sizes returns ED_ERR_ARG with a
    message, on the host and before any CUDA call; the destroy functions accept NULL."""
    import ctypes

    import paper_1511_00863_gb300 as ed
    scalars = (ctypes.c_int, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64, ctypes.c_double)
    for name, (res, args) in ed._SIGS.items():
        if name == "ed_last_error":
            continue
        vals = [0 if a in scalars else None for a in args]
        r = getattr(ed._lib, name)(*vals)
        if res is None:
            assert name.endswith("_destroy")
            continue
        assert r == ed.ED_ERR_ARG, (name, r)
        msg = ed._lib.ed_last_error().decode()
        assert msg.startswith(name + ":"), (name, msg)
