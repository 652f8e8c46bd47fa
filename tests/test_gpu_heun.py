"""The Heun (SSP-RK2) method option on the GPU (SV_HEUN, two launches per
step) against the oracle's Heun integration; same error measure and
tolerances as the MUSCL-Hancock parity tests."""
import math

import numpy as np
import pytest

from gpu_util import assert_fp64_parity, need_gpu, oracle_params, rel_linf
from oracle import dispersion as D
from oracle import orc as O
from paper_1805_03442_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sv():
    return need_gpu()


@pytest.mark.parametrize("N", [5, 33, 1000, 4099])
@pytest.mark.parametrize("params", [dict(tau0=0.3),
                                    dict(tau0=0.05, S=0.7, Q_rho=0.4, Q_T=-0.3, I_rho=0.2, I_T=0.5),
                                    dict(tau0=math.inf, S=0.0)])
def test_fp64_heun_matches_oracle(sv, N, params):
    P = sv.Params(precision=sv.FP64, method=sv.HEUN, **params)
    Po = oracle_params(P)
    h = 1.0 / N
    U0 = inputs.random_states(1, N, seed=N + 7, smooth=True)
    with sv.Solver(P, (N,), (1.0,)) as s:
        s.write_state(U0)
        s.step(3)
        U, t = s.read_state()
        assert s.status() == 0
    ref = U0
    for _ in range(3):
        ref, rc = O.step_heun(Po, ref, N, h, O.dt_cfl(Po, ref, N, h))
        assert rc == 0
    assert_fp64_parity(U, ref)


def test_fp32_heun_one_step(sv):
    N = 4099
    P = sv.Params(precision=sv.FP32, method=sv.HEUN, tau0=0.3)
    Po = oracle_params(P)
    U0 = inputs.random_states(1, N, seed=2, smooth=True).astype(np.float32).astype(np.float64)
    with sv.Solver(P, (N,), (1.0,)) as s:
        s.write_state(U0)
        dt = s.dt()
        s.step(1)
        U, _ = s.read_state()
    ref, _ = O.step_heun(Po, U0, N, 1.0 / N, dt)
    assert rel_linf(U, ref) <= 2e-6


@pytest.mark.parametrize("prec", ["FP32", "FP64"])
def test_heun_growth_rate(sv, prec):
    N, k = 1024, 2 * math.pi
    P = sv.Params(precision=getattr(sv, prec), method=sv.HEUN, tau0=0.08)
    Po = oracle_params(P)
    w = D.growing_acoustic_root(Po, k)
    md = D.eigenmode(Po, k, w)
    U0 = inputs.waves_1d(P.gamma, N, 1.0, inputs.equilibrium_primitive(P.Ck, P.S),
                         [inputs.Mode(m=1, shape=md["prim"], scale=1e-4)])
    x = inputs.cell_centres(N, 1.0)
    ts, amps = [], []
    with sv.Solver(P, (N,), (1.0,)) as s:
        s.write_state(U0)
        t = 0.0
        while t < math.log(100.0) / w.imag:
            s.run_to(t + 0.05)
            U, t = s.read_state()
            ts.append(t)
            amps.append(np.sum(U[1] / U[0] * np.exp(-1j * k * x)) / N)
    growth = np.polyfit(ts, np.log(np.abs(amps)), 1)[0]
    assert abs(growth - w.imag) <= 0.02 * w.imag


def test_heun_rejected_where_not_built(sv):
    with pytest.raises(sv.SvError):
        sv.Solver(sv.Params(method=sv.HEUN), (16, 16), (1.0, 1.0))
    with pytest.raises(sv.SvError):
        sv.Solver(sv.Params(method=sv.HEUN), (64,), (1.0,), bc=(sv.BC_REFLECT, sv.BC_REFLECT))
