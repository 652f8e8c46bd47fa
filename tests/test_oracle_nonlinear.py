"""The nonlinear stage of the one-wavelength eigenmode run (Sec. 3, the
shock-train stage after the linear growth): the shock detector of
oracle/nonlinear_stage.py pinned on hand-built states, and the stored oracle
statistics (tests/golden/nonlinear_stage.json, written by that script) checked
for what they must show."""
import json
import os

import numpy as np
import pytest

from oracle.nonlinear_stage import shocks, snapshot
from paper_1805_03442_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "nonlinear_stage.json")


def _state(u, p=None):
    N = len(u)
    p = np.ones(N) if p is None else p
    return inputs.prim_to_cons(1.4, np.ones(N), [u], p, np.full(N, 1.1))


def test_sawtooth_has_its_jumps():
    """A periodic sawtooth of three teeth: velocity rising linearly by 0.6 over
    each third and dropping back in one cell -- three shocks, spacing 1/3,
    jump 0.6 (up to the one-cell rise the drop takes back)."""
    N = 300
    x = (np.arange(N) % 100) / 100.0
    s = shocks(_state(0.6 * x - 0.3))
    assert s["count"] == 3
    assert s["spacing"] == pytest.approx(1.0 / 3.0)
    assert s["jump"] == pytest.approx(0.6 * 99 / 100, rel=1e-12)


def test_smooth_wave_and_rest_have_none():
    N = 256
    x = (np.arange(N) + 0.5) / N
    assert shocks(_state(1e-3 * np.sin(2 * np.pi * x)))["count"] == 0
    assert shocks(_state(np.zeros(N)))["count"] == 0


def test_pressure_ratio_across_a_jump():
    N = 200
    u = np.where(np.arange(N) < 100, 0.5, -0.5)     # two jumps: one compressive
    p = np.where(np.arange(N) < 100, 1.0, 3.0)
    s = snapshot(_state(u, p))
    assert s["count"] == 1 and s["jump"] == pytest.approx(1.0)
    assert s["p_ratio"] == pytest.approx(3.0)
    assert s["max_rho"] == 1.0 and s["min_p"] == pytest.approx(1.0)


def test_golden_oracle_statistics():
    """The stored oracle runs: no shock at t = 5 (still linear), a train of
    three by t = 10, and the loss of positivity between t = 13 and 15, before
    the 20 periods (t = 14.58) run out."""
    g = json.load(open(GOLDEN))
    assert {r["limiter"] for r in g["runs"]} == {0, 1}
    for r in g["runs"]:
        assert r["N"] == 1024 and r["cfl"] == 0.4
        assert r["t5"]["count"] == 0
        assert r["t10"]["count"] == 3 and r["t10"]["spacing"] == pytest.approx(1 / 3)
        assert 13.0 < r["collapse_t"] < 15.0 and r["collapse_t"] < r["t_end"]
        assert not r["at_collapse"]["min_p"] > 0 and r["t10"]["min_p"] > 0   # p < 0 or NaN
