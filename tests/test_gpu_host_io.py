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
