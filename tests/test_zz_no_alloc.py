"""The allocation-free 1D step, sv_step1d_noalloc, against the regular
solver's step.

The entry point serves callers that cannot allocate device memory (processes
whose device memory is a fixed pool handed out at start-up, hosts that must
not allocate while stepping): they pass their own state buffers and the
library keeps its control block in a static device array.  Here torch
allocates the two buffers only to play such a caller.  Two calls in a row
check that the second call is not disturbed by what the first left in the
shared array.

The file name sorts last so that a run stopping at its first failure has
already run every other test when it reaches this one; the tests here do not
depend on that order and pass alone in a fresh process as well."""
import numpy as np
import pytest

from gpu_util import need_gpu, rel_linf
from paper_1805_03442_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("prec,tol", [("FP64", 1e-12), ("FP32", 2e-6)])
def test_noalloc_step_matches_solver_on_two_calls(prec, tol):
    sv = need_gpu()
    import torch
    N = 5003
    P = sv.Params(precision=getattr(sv, prec), tau0=0.2)
    U0 = inputs.random_states(1, N, seed=21, smooth=True)
    with sv.Solver(P, (N,), (1.0,)) as s:
        s.write_state(U0)
        s.step(1)
        U1_ref, t1 = s.read_state()
        s.step(1)
        U2_ref, t2 = s.read_state()
    dtype = torch.float64 if prec == "FP64" else torch.float32
    a = torch.tensor(U0, dtype=dtype, device="cuda").contiguous()
    b = torch.empty_like(a)
    dt1, f1 = sv.step1d_noalloc(P, N, 1.0, a.data_ptr(), b.data_ptr())
    U1 = b.double().cpu().numpy()
    dt2, f2 = sv.step1d_noalloc(P, N, 1.0, b.data_ptr(), a.data_ptr())
    U2 = a.double().cpu().numpy()
    assert f1 == 0 and f2 == 0
    assert dt1 == pytest.approx(t1, rel=1e-15)
    assert dt1 + dt2 == pytest.approx(t2, rel=1e-14)
    assert rel_linf(U1, U1_ref) <= tol
    assert rel_linf(U2, U2_ref) <= tol
    # the same kernels' arithmetic as the solver's step: equal bit for bit
    assert dt1 == t1 and np.array_equal(U1, U1_ref)
    assert np.array_equal(U2, U2_ref)


def test_noalloc_rejects_oversized_grid():
    sv = need_gpu()
    P = sv.Params(precision=sv.FP32)
    with pytest.raises(sv.SvError) as e:
        sv.step1d_noalloc(P, sv.NOALLOC_MAX_CELLS + 1, 1.0, 1 << 20, 2 << 20)
    assert e.value.code == sv.SV_ESIZE
