"""Parity in the stiff-source regime, where the source time-step cap
dt <= c_tau min_j tau_j (a reading of the paper: eq. 16 bounds only the
advection) sets every step rather than eq. 16: tau0 = 1e-3, the lower end of
the stability sweep's range, with general closure exponents of eq. 6.

Both sides take the cap on their own state: the FP64 kernels as
c_tau tau0 rho^tau_rho T^tau_T folded as a maximum of -tau, the float kernels
as c_tau tau0 2^-a with a = -(tau_rho log2 rho + tau_T log2 T) folded as a
maximum in float.  dt is compared to 1e-13 (FP64) and 1e-5 (float: the SFU
log2 / exp2 carry ~2^-22 each), the states as in the other parity tests."""

import numpy as np
import pytest

from gpu_util import assert_fp64_parity, field_rel_linf, need_gpu, oracle_params, rel_linf
from oracle import orc as O
from paper_1805_03442_gb300 import inputs

pytestmark = pytest.mark.gpu

STIFF = dict(tau0=1e-3, S=1.3, tau_rho=-0.7, tau_T=-1.9, Q_rho=0.4, Q_T=-0.6, I_rho=-0.3, I_T=0.8)


@pytest.fixture(scope="module")
def sv():
    return need_gpu()


def _cap_is_active(Po, U, N, h):
    """The oracle's dt equals the tau cap, well below eq. 16's advective bound."""
    dt = O.dt_cfl(Po, U, N, h)
    P_adv = oracle_params_like(Po, c_tau=1e30)
    dt_adv = O.dt_cfl(P_adv, U, N, h)
    assert dt < 0.5 * dt_adv
    return dt


def _spacing(N):
    """h = 1/256 from 256 cells up (the cap binds at coarse spacing only), 1/N below."""
    return 1.0 / min(N, 256)


def oracle_params_like(Po, **over):
    d = dict(Po.__dict__)
    d.update(over)
    return O.Params(**d)


@pytest.mark.parametrize("limiter", [0, 1])
@pytest.mark.parametrize("N", [5, 33, 1000, 4099, 8192])
def test_fp64_tau_cap_steps(sv, N, limiter):
    P = sv.Params(precision=sv.FP64, limiter=limiter, **STIFF)
    Po = oracle_params(P)
    h = _spacing(N)
    U0 = inputs.random_states(1, N, seed=100 + N, smooth=True)
    _cap_is_active(Po, U0, N, h)
    with sv.Solver(P, (N,), (N * h,)) as s:
        s.write_state(U0)
        dts = []
        for _ in range(4):
            dts.append(s.dt())
            s.step(1)
        U, t = s.read_state()
        assert s.status() == 0
    ref, rdts = U0.copy(), []
    for _ in range(4):
        rdts.append(O.dt_cfl(Po, ref, N, h))
        ref, rc = O.step(Po, ref, N, h, rdts[-1])
        assert rc == 0
    assert np.allclose(dts, rdts, rtol=1e-13, atol=0)
    assert t == pytest.approx(sum(rdts), rel=1e-14)
    assert_fp64_parity(U, ref)


@pytest.mark.parametrize("precision", ["FP32", "FP32_PC"])
@pytest.mark.parametrize("N", [5, 33, 1000, 4099, 8192])
def test_fp32_tau_cap_steps(sv, precision, N):
    P = sv.Params(precision=getattr(sv, precision), **STIFF)
    Po = oracle_params(P)
    h = _spacing(N)
    U0 = inputs.random_states(1, N, seed=200 + N, smooth=True)
    U0 = U0.astype(np.float32).astype(np.float64)
    _cap_is_active(Po, U0, N, h)
    with sv.Solver(P, (N,), (N * h,)) as s:
        s.write_state(U0)
        dt0 = s.dt()
        s.step(1)
        U1, _ = s.read_state()
        dts = [dt0]
        for _ in range(3):                   # the float finalize's cap on later states
            dts.append(s.dt())
            Uk, _ = s.read_state()
            assert dts[-1] == pytest.approx(O.dt_cfl(Po, Uk, N, h), rel=1e-5)
            s.step(1)
        assert s.status() == 0
    assert dt0 == pytest.approx(O.dt_cfl(Po, U0, N, h), rel=1e-5)
    ref, rc = O.step(Po, U0, N, h, dt0)         # same dt: compare the step's arithmetic
    assert rc == 0
    assert rel_linf(U1, ref) <= 2e-6
    assert max(field_rel_linf(U1, ref).values()) <= 2e-6


def test_tau_cap_run_to_matches_oracle(sv):
    """sv_run_to over 62 capped steps (the last one clamped to t_end): same
    step count and time as the oracle, states within 1e-12.  (Much longer and
    the medium's unstable short waves, Im omega ~ 250 here, amplify rounding
    in the oracle itself: a one-ulp change of the initial state moves its own
    result by 3e-12 by t = 0.0137, 1073 steps.)"""
    N = 700
    P = sv.Params(precision=sv.FP64, limiter=1, **STIFF)
    Po = oracle_params(P)
    U0 = inputs.random_states(1, N, seed=17, smooth=True)
    t_end = 0.008
    with sv.Solver(P, (N,), (1.0,)) as s:
        s.write_state(U0)
        rc, k = s.run_to(t_end)
        U, t = s.read_state()
    ref, tr, kr, rcr = O.run(Po, U0, N, 1.0 / N, t_end)
    assert rc == 0 and rcr == 0
    assert k == kr and k > 50 and t == tr == t_end
    assert_fp64_parity(U, ref)
