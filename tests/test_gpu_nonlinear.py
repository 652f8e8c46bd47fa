"""The one-wavelength eigenmode run into its nonlinear stage (Sec. 3: the
linear growth of eq. 8 gives way to a train of shocks) on the GPU, against the
oracle's statistics stored in tests/golden/nonlinear_stage.json (written by
oracle/nonlinear_stage.py --golden).

The run ends, in the oracle and on the GPU alike, when the pumped shocks have
steepened the density spikes until the pressure goes negative: every setting
of N = 1024 / 2048, CFL 0.4 / 0.2 and minmod / van Leer collapses between
t = 13.3 and 14.5, so the collapse is a property of the model's solution that
the GPU must reproduce.  With van Leer its time is reproducible: one-ulp
perturbations of the initial state move the oracle's collapse by 1e-4
(14.0228-14.0229).  With minmod it is not: the limiter's grid-scale noise
amplification (tests/test_oracle_noise.py) moves it across 13.3-14.5 under the
same perturbations, so for minmod only that band is a prediction.

Bounds.  FP64: the same shock count and spacing at t = 10, mean velocity jump
and max density within 3% (after ~30000 steps two correct FP64 codes that
round differently differ at the percent level in the shock amplitudes with
minmod, at 1e-4 with van Leer); collapse within 0.05 of the oracle with van
Leer, inside 13.0-15.0 with minmod.
Float: the perturbation layout (FP32_PS) follows the same shock train within
5%; the full-state float policy is seeded by its own rounding noise (a float
state rounds the O(1) background at 6e-8 each step, which the medium's
short-wave instability amplifies) and collapses earlier, which the last test
records."""
import json
import math
import os

import pytest

from gpu_util import need_gpu
from oracle import dispersion as D
from oracle import orc as O
from oracle.nonlinear_stage import snapshot
from paper_1805_03442_gb300 import inputs

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "nonlinear_stage.json")


@pytest.fixture(scope="module")
def sv():
    return need_gpu()


def _golden(limiter):
    return next(r for r in json.load(open(GOLDEN))["runs"] if r["limiter"] == limiter)


def _run(sv, prec, limiter, marks):
    N = 1024
    P = sv.Params(precision=prec, tau0=0.08, S=1.0, limiter=limiter)
    Po = O.Params(tau0=0.08, S=1.0, limiter=limiter)
    k = 2 * math.pi
    w = D.growing_acoustic_root(Po, k)
    md = D.eigenmode(Po, k, w)
    U0 = inputs.waves_1d(1.4, N, 1.0, inputs.equilibrium_primitive(0.1, 1.0),
                         [inputs.Mode(m=1, shape=md["prim"], scale=1e-4)])
    out = {}
    with sv.Solver(P, (N,), (1.0,)) as s:
        s.write_state(U0)
        for mark in marks:
            rc, _ = s.run_to(mark, check=False)
            U, t = s.read_state()
            if rc != 0:
                out["collapse_t"], out["rc"] = t, rc
                break
            out[mark] = snapshot(U)
    return out


@pytest.mark.parametrize("limiter", [0, 1])
def test_fp64_shock_train_and_collapse(sv, limiter):
    g = _golden(limiter)
    r = _run(sv, sv.FP64, limiter, (5.0, 10.0, g["t_end"]))
    assert r[5.0]["count"] == g["t5"]["count"] == 0
    assert r[10.0]["count"] == g["t10"]["count"]
    assert r[10.0]["spacing"] == pytest.approx(g["t10"]["spacing"])
    assert r[10.0]["jump"] == pytest.approx(g["t10"]["jump"], rel=0.03)
    assert r[10.0]["max_rho"] == pytest.approx(g["t10"]["max_rho"], rel=0.03)
    assert r["rc"] in (sv.SV_ENONPHYS, sv.SV_EDT)
    if limiter == 1:
        assert abs(r["collapse_t"] - g["collapse_t"]) <= 0.05
    else:
        assert 13.0 <= r["collapse_t"] <= 15.0


def test_fp32_perturbation_layout_shock_train(sv):
    g = _golden(0)
    r = _run(sv, sv.FP32_PS, 0, (5.0, 10.0))
    assert r[5.0]["count"] == 0
    assert r[10.0]["count"] == g["t10"]["count"]
    assert r[10.0]["spacing"] == pytest.approx(g["t10"]["spacing"])
    assert r[10.0]["jump"] == pytest.approx(g["t10"]["jump"], rel=0.05)
    assert r[10.0]["max_rho"] == pytest.approx(g["t10"]["max_rho"], rel=0.05)


def test_fp32_full_state_is_noise_seeded(sv):
    """The full-state float run already carries many small noise-seeded shocks
    at t = 5, where the oracle has none, and collapses before t = 10."""
    g = _golden(0)
    r = _run(sv, sv.FP32, 0, (5.0, 10.0, g["t_end"]))
    assert r[5.0]["count"] > 5
    assert r["collapse_t"] < 10.0 < g["collapse_t"]
