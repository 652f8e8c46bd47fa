"""Pins of the oracle's Heun (SSP-RK2) integration of the MUSCL spatial
operator (the predictor-corrector form of eqs. 10-11): second order on smooth
flow, conservation, stationarity, exact-Riemann and eq.-8 growth checks."""
import math

import numpy as np
import pytest

from oracle import dispersion as D
from oracle import orc as O
from oracle.riemann import Riemann
from paper_1805_03442_gb300 import inputs


def test_second_order_on_smooth_advection(orc):
    P = O.Params(limiter=O.MC).frozen()
    errs = []
    for N in (64, 128, 256):
        h = 1.0 / N
        x = inputs.cell_centres(N, 1.0)

        def avg(t):
            return 1 + 0.2 * (np.cos(2 * np.pi * (x - h / 2 - t)) - np.cos(2 * np.pi * (x + h / 2 - t))) \
                / (2 * np.pi * h)

        U = inputs.prim_to_cons(P.gamma, avg(0), [np.ones(N)], np.ones(N), np.full(N, 0.5))
        Ue, _, _, rc = O.run_heun(P, U, N, h, 1.0)
        assert rc == 0
        errs.append(np.mean(np.abs(Ue[0] - avg(1.0))))
    rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(rates > 1.8), rates


def test_conservation_and_stationarity(orc):
    P = O.Params(tau0=0.2, Q_rho=0.3, I_T=-0.2)
    N = 64
    U = inputs.random_states(1, N, seed=6, smooth=True)
    U1 = U.copy()
    for _ in range(5):
        U1, rc = O.step_heun(P, U1, N, 1.0 / N, O.dt_cfl(P, U1, N, 1.0 / N))
        assert rc == 0
    for f in (0, 1):
        assert abs(math.fsum(U1[f]) - math.fsum(U[f])) <= 1e-13 * math.fsum(np.abs(U[f]))
    E = np.repeat(D.equilibrium(P)[:, None], N, axis=1)
    E1, _ = O.step_heun(P, E, N, 1.0 / N, O.dt_cfl(P, E, N, 1.0 / N))
    assert np.array_equal(E1[:2], E[:2]) and np.max(np.abs(E1 - E)) < 1e-14


def test_frozen_double_tube_matches_exact_riemann(orc):
    P = O.Params().frozen()
    N, L, t_end = 800, 1.0, 0.1
    h = L / N
    outer, inner = (1.0, 0.0, 1.0, 0.3), (0.125, 0.0, 0.1, 0.9)
    U, t, _, rc = O.run_heun(P, inputs.double_tube_1d(P.gamma, N, L, outer, inner), N, h, t_end)
    assert rc == 0 and t == t_end
    x = inputs.cell_centres(N, L)
    R = Riemann(P.gamma, *outer[:3], *inner[:3])
    ex = R.sample_array((x - 0.25) / t_end)
    _, _, c, _, s = R.wave_speeds()
    xc, xs = 0.25 + c * t_end, 0.25 + s * t_end
    plateau = (x > xc + 10 * h) & (x < xs - 3 * h)
    assert np.mean(np.abs(U[0][plateau] - ex[0][plateau])) <= 1e-3
    half = 0.5 * (R.star_densities()[1] + inner[0])
    i = np.where((x > xc) & (x < 0.5) & (U[0] < half))[0][0]
    xsh = x[i - 1] + (half - U[0][i - 1]) / (U[0][i] - U[0][i - 1]) * h
    assert abs(xsh - xs) <= h


def test_linear_growth_rate_matches_eq8(orc):
    P = O.Params(tau0=0.08)
    N, k = 256, 2 * math.pi
    w = D.growing_acoustic_root(P, k)
    md = D.eigenmode(P, k, w)
    U = inputs.waves_1d(P.gamma, N, 1.0, inputs.equilibrium_primitive(P.Ck, P.S),
                        [inputs.Mode(m=1, shape=md["prim"], scale=1e-4)])
    x = inputs.cell_centres(N, 1.0)
    ts, amps, t = [], [], 0.0
    while t < math.log(100.0) / w.imag:
        U, t, _, rc = O.run_heun(P, U, N, 1.0 / N, t + 0.05, t0=t)
        assert rc == 0
        ts.append(t)
        amps.append(np.sum(U[1] / U[0] * np.exp(-1j * k * x)) / N)
    growth = np.polyfit(ts, np.log(np.abs(amps)), 1)[0]
    assert abs(growth - w.imag) <= 0.02 * w.imag
