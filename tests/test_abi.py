"""The C-ABI library builds for sm_103a, loads, and exports every function
include/sv.h declares (no compute call: this runs without a GPU)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared(header: str) -> list[str]:
    text = open(os.path.join(ROOT, "include", header)).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:int|void|const char\*)\s+(sv_\w+)\s*\(", text, flags=re.M)))


@pytest.fixture(scope="module")
def libsv():
    from paper_1805_03442_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = _declared("sv.h")
    for required in ("sv_init", "sv_step", "sv_run_to", "sv_dt_cfl", "sv_read_state",
                     "sv_write_state", "sv_free"):
        assert required in names


def test_every_declared_symbol_is_exported(libsv):
    headers = [f for f in os.listdir(os.path.join(ROOT, "include")) if f.endswith(".h")]
    for h in headers:
        for name in _declared(h):
            assert hasattr(libsv, name), f"{name} declared in {h} but not exported"


def test_binding_names_match_header():
    from paper_1805_03442_gb300 import sv
    assert set(sv.EXPORTS) <= set(_declared("sv.h"))


def test_argument_errors_without_gpu(libsv):
    """sv_required_bytes validates its input on the host only."""
    from paper_1805_03442_gb300 import sv
    sv._lib = None
    L = sv.lib()
    p = sv.Params().c()
    g = sv.grid((16,), (1.0,))
    n = ctypes.c_size_t()
    assert L.sv_required_bytes(ctypes.byref(p), ctypes.byref(g), ctypes.byref(n)) == 0
    assert n.value >= 2 * 4 * 16 * 4 + 4 * 16 * 8
    bad = sv.grid((16, 8), (1.0, 1.0))            # unequal cell sizes
    assert L.sv_required_bytes(ctypes.byref(p), ctypes.byref(bad), ctypes.byref(n)) == sv.SV_EINVAL
    p.limiter = 7
    assert L.sv_required_bytes(ctypes.byref(p), ctypes.byref(g), ctypes.byref(n)) == sv.SV_EINVAL
    assert L.sv_strerror(sv.SV_ENONPHYS).startswith(b"non-physical")


def _rb(L, p, g):
    n = ctypes.c_size_t()
    return L.sv_required_bytes(ctypes.byref(p), ctypes.byref(g), ctypes.byref(n)), n.value


def test_host_validation_edge_cases(libsv):
    """Degenerate and out-of-range inputs are rejected on the host, before any
    CUDA call; the smallest valid grids are accepted."""
    from paper_1805_03442_gb300 import sv
    sv._lib = None
    L = sv.lib()
    ok = sv.Params().c()
    assert _rb(L, ok, sv.grid((1,), (1.0,)))[0] == 0                 # one periodic cell
    assert _rb(L, ok, sv.grid((2, 2, 2), (1.0, 1.0, 1.0)))[0] == 0
    empty = sv.grid((16,), (1.0,))
    empty.n[0] = 0                                                   # no cells
    assert _rb(L, ok, empty)[0] == sv.SV_EINVAL
    for dim in (0, 4):
        g = sv.grid((16,), (1.0,))
        g.dim = dim
        assert _rb(L, ok, g)[0] == sv.SV_EINVAL
    neg = sv.grid((16,), (1.0,))
    neg.L[0] = -1.0
    assert _rb(L, ok, neg)[0] == sv.SV_EINVAL
    for field, value in [("gamma", 1.0), ("cfl", 0.0), ("c_tau", -1.0), ("tau0", 0.0),
                         ("precision", 5), ("precision", -1), ("method", 2)]:
        p = sv.Params().c()
        setattr(p, field, value)
        assert _rb(L, p, sv.grid((16,), (1.0,)))[0] == sv.SV_EINVAL, field
    # the perturbation layout: every dimension, not with Heun
    ps = sv.Params(precision=sv.FP32_PS).c()
    for n in [(8,), (8, 8), (8, 8, 8)]:
        assert _rb(L, ps, sv.grid(n))[0] == 0
    assert _rb(L, sv.Params(precision=sv.FP32_PS, method=sv.HEUN).c(), sv.grid((8,)))[0] == sv.SV_EINVAL
    # walls need at least two cells; 3D is periodic; the driven boundary is 1D x = 0 only
    assert _rb(L, ok, sv.grid((1,), (1.0,), bc=(sv.BC_REFLECT, sv.BC_REFLECT)))[0] == sv.SV_EINVAL
    assert _rb(L, ok, sv.grid((4, 4, 4), (1, 1, 1), bc=(sv.BC_REFLECT,)))[0] == sv.SV_EINVAL
    assert _rb(L, ok, sv.grid((8,), (1.0,), bc=(sv.BC_PERIODIC, sv.BC_DRIVEN)))[0] == sv.SV_EINVAL
    assert _rb(L, ok, sv.grid((8, 8), (1, 1), bc=(sv.BC_DRIVEN, sv.BC_OUTFLOW)))[0] == sv.SV_EINVAL
    # the bytes of a float 1D solver: two state buffers, a double staging buffer
    rc, nbytes = _rb(L, ok, sv.grid((1000,), (1.0,)))
    assert rc == 0 and nbytes >= 2 * 4 * 1000 * 4 + 4 * 1000 * 8


def test_batch_and_noalloc_validation(libsv):
    from paper_1805_03442_gb300 import sv
    sv._lib = None
    L = sv.lib()
    p = sv.Params().c()
    runs = (sv._Run * 2)()
    for r in runs:
        r.n, r.L, r.t_end, r.S, r.tau0, r.mode = 64, 1.0, 0.1, 1.0, 0.1, 1
    n = ctypes.c_size_t()
    assert L.sv_batch_required_bytes(ctypes.byref(p), runs, 2, 8, ctypes.byref(n)) == 0
    assert n.value > 0
    assert L.sv_batch_required_bytes(ctypes.byref(p), runs, 0, 8, ctypes.byref(n)) == sv.SV_EINVAL
    runs[1].n = 0
    assert L.sv_batch_required_bytes(ctypes.byref(p), runs, 2, 8, ctypes.byref(n)) == sv.SV_EINVAL
    runs[1].n, runs[1].t_end = 64, -1.0
    assert L.sv_batch_required_bytes(ctypes.byref(p), runs, 2, 8, ctypes.byref(n)) == sv.SV_EINVAL
    # the allocation-free step checks its arguments before touching the device
    dt, fl = ctypes.c_double(), ctypes.c_uint32()
    a, b = ctypes.c_void_p(1 << 20), ctypes.c_void_p(2 << 20)
    f = L.sv_step1d_noalloc
    assert f(ctypes.byref(p), 0, 1.0, a, b, ctypes.byref(dt), ctypes.byref(fl), None) == sv.SV_EINVAL
    assert f(ctypes.byref(p), 16, 1.0, a, a, ctypes.byref(dt), ctypes.byref(fl), None) == sv.SV_EINVAL
    assert f(ctypes.byref(p), sv.NOALLOC_MAX_CELLS + 1, 1.0, a, b, ctypes.byref(dt),
             ctypes.byref(fl), None) == sv.SV_ESIZE
    ps = sv.Params(precision=sv.FP32_PS).c()
    assert f(ctypes.byref(ps), 16, 1.0, a, b, ctypes.byref(dt), ctypes.byref(fl), None) == sv.SV_EINVAL
    # buffers that share any byte: U_out starting inside U_in, or U_in inside U_out
    # (16 float cells: 4 * 16 * 4 = 256 bytes per buffer)
    for off in (16, 255, -255):
        c = ctypes.c_void_p((1 << 20) + off)
        assert f(ctypes.byref(p), 16, 1.0, a, c, ctypes.byref(dt), ctypes.byref(fl),
                 None) == sv.SV_EINVAL, off
    pd = sv.Params(precision=sv.FP64).c()       # double: 512 bytes per buffer
    c = ctypes.c_void_p((1 << 20) + 300)
    assert f(ctypes.byref(pd), 16, 1.0, a, c, ctypes.byref(dt), ctypes.byref(fl), None) == sv.SV_EINVAL


def test_wait_limit_and_probe_validation(libsv):
    """The failure-path hook and the FP64 probe check their arguments before
    touching the device."""
    from paper_1805_03442_gb300 import sv
    sv._lib = None
    L = sv.lib()
    assert L.sv_set_wait_limit(None, 1) == sv.SV_EINVAL
    assert L.sv_measure_fp64_peak(None, None) == sv.SV_EINVAL
