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
