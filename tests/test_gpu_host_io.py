"""Host state I/O through the C ABI: pageable numpy buffers go through the
device staging buffer; page-locked (pinned) buffers are read and written by
the conversion kernels directly over the host link.  Both routes must give the
same device state and the same host copies, for float and double solvers,
aligned and unaligned pinned addresses and an odd element count."""
import numpy as np
import pytest

from gpu_util import need_gpu
from paper_1805_03442_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sv():
    return need_gpu()


def _pinned(torch, n, offset):
    """A pinned float64 host buffer of n elements starting `offset` elements
    into a larger pinned allocation (offset 1: 8-byte aligned only)."""
    base = torch.empty(n + 2, dtype=torch.float64).pin_memory()
    return base, base[offset:offset + n]


@pytest.mark.parametrize("prec", ["FP32", "FP64"])
@pytest.mark.parametrize("n,offset", [((4099,), 0), ((37, 29), 0), ((37, 29), 1), ((8, 6, 5), 1)])
def test_pinned_and_pageable_io_agree(sv, prec, n, offset):
    torch = pytest.importorskip("torch")
    dim = len(n)
    cells = int(np.prod(n))
    U0 = inputs.random_states(dim, cells, seed=cells + offset, smooth=True)
    P = sv.Params(precision=getattr(sv, prec), tau0=0.3)
    count = (dim + 3) * cells
    base_in, hin = _pinned(torch, count, offset)
    hin.copy_(torch.from_numpy(U0.reshape(-1)))
    base_out, hout = _pinned(torch, count, offset)
    with sv.Solver(P, n) as a, sv.Solver(P, n) as b:
        a.write_state(U0, t=0.25)                 # pageable route
        b.write_state_ptr(hin.data_ptr(), t=0.25)  # pinned route
        assert a.dt() == b.dt()
        a.step(3)
        b.step(3)
        Ua, ta = a.read_state()
        tb = b.read_state_ptr(hout.data_ptr())
        Ub = hout.numpy().reshape(Ua.shape)
        assert ta == tb and a.status() == 0 and b.status() == 0
        assert np.array_equal(Ua, Ub)
        assert not np.array_equal(Ua.reshape(U0.shape), U0)    # the steps changed the state


def _pinned32(torch, n, offset):
    """A pinned float32 host buffer of n elements, `offset` elements in
    (offset 1: 4-byte aligned only)."""
    base = torch.empty(n + 2, dtype=torch.float32).pin_memory()
    return base, base[offset:offset + n]


@pytest.mark.parametrize("prec", ["FP32", "FP32_PC", "FP32_PS", "FP64"])
@pytest.mark.parametrize("n,offset", [((4099,), 0), ((4099,), 1), ((37, 29), 1)])
def test_float_host_buffers(sv, prec, n, offset):
    """sv_write_state_f32 / sv_read_state_f32 against the double calls on the
    same float-representable state: the same device state (the same dt and
    the same steps), the float download equal to the double download rounded
    to float (exactly equal for the float policies), on the pageable route
    and on pinned buffers, aligned or not."""
    torch = pytest.importorskip("torch")
    dim = len(n)
    cells = int(np.prod(n))
    U0 = inputs.random_states(dim, cells, seed=3 * cells + offset, smooth=True)
    U32 = U0.astype(np.float32)
    P = sv.Params(precision=getattr(sv, prec), tau0=0.3)
    count = (dim + 3) * cells
    base_in, hin = _pinned32(torch, count, offset)
    hin.copy_(torch.from_numpy(U32.reshape(-1)))
    base_out, hout = _pinned32(torch, count, offset)
    with sv.Solver(P, n) as a, sv.Solver(P, n) as b, sv.Solver(P, n) as c:
        a.write_state(U32.astype(np.float64), t=0.5)    # double route
        b.write_state_f32(U32, t=0.5)                   # float, pageable
        c.write_state_ptr_f32(hin.data_ptr(), t=0.5)    # float, pinned
        assert a.dt() == b.dt() == c.dt()
        for s in (a, b, c):
            s.step(2)
        Ua, ta = a.read_state()
        Ub, tb = b.read_state()
        Fb, _ = b.read_state_f32()
        tc = c.read_state_ptr_f32(hout.data_ptr())
        Fc = hout.numpy().reshape(Fb.shape)
        assert ta == tb == tc
        assert np.array_equal(Ua, Ub)
        assert np.array_equal(Fb, Ua.astype(np.float32))
        assert np.array_equal(Fc, Fb)
        if prec in ("FP32", "FP32_PC"):
            assert np.array_equal(Fb.astype(np.float64), Ua)    # float state: exact both ways
