"""Checkpoint and restart: a run stopped after K steps, read to the host
(sv_read_state: the state and its time) and uploaded into a fresh solver
(sv_write_state) continues bit for bit as the run that was never stopped, in
every precision policy, in 1D (sliding warps and block tiles), 2D and 3D.
The full-state float policies also go through float host buffers
(sv_read_state_f32 / sv_write_state_f32), which carry their device state
exactly (the perturbation layout's float buffers hold U rounded to float, not
its device perturbations, so they are not a checkpoint of it)."""
import numpy as np
import pytest

from gpu_util import need_gpu
from paper_1805_03442_gb300 import inputs

pytestmark = pytest.mark.gpu

K, M = 7, 5


@pytest.fixture(scope="module")
def sv():
    return need_gpu()


def _state(n, seed):
    return inputs.random_states(len(n), int(np.prod(n)), seed=seed, smooth=True)


@pytest.mark.parametrize("prec", ["FP64", "FP32", "FP32_PC", "FP32_PS"])
@pytest.mark.parametrize("n", [(5000,), (1 << 16,), (130, 64), (36, 30, 8)])
def test_restart_continues_bitwise(sv, n, prec):
    P = sv.Params(precision=getattr(sv, prec), tau0=0.1)
    h = 1.0 / n[0]
    L = tuple(x * h for x in n)
    U0 = _state(n, 11 + len(n))
    with sv.Solver(P, n, L) as s:
        s.write_state(U0)
        s.step(K)
        Uk, tk = s.read_state()
        Uk32 = s.read_state_f32()[0] if prec in ("FP32", "FP32_PC") else None
        s.step(M)
        Ua, ta = s.read_state()
        assert s.status() == 0
    with sv.Solver(P, n, L) as r:
        r.write_state(Uk, t=tk)
        r.step(M)
        Ub, tb = r.read_state()
        assert r.status() == 0
    assert tb == ta
    assert np.array_equal(Ub, Ua)
    if Uk32 is not None:
        with sv.Solver(P, n, L) as r:
            r.write_state_f32(Uk32, t=tk)
            r.step(M)
            Uc, tc = r.read_state()
        assert tc == ta and np.array_equal(Uc, Ua)
