"""Pins of the forced-source (spatial) problem of the paper's Sec. 3: a wave
driven at x = 0 into the active medium, free outflow at x = 1.  Behind the
front the solution oscillates at the driving frequency with an amplitude that
grows as exp(-Im k x), k the spatial root of eq. 8 for real omega."""
import math

import numpy as np
import pytest

from oracle import dispersion as D
from oracle import orc as O
from paper_1805_03442_gb300 import inputs


def test_spatial_root_solves_eq8():
    """The spatial root, put back into the quartic of eq. 8, gives zero: the
    spatial and temporal problems are one dispersion relation."""
    for params in (dict(S=0.5, tau0=0.0135), dict(S=0.8, tau0=0.05, Q_rho=0.4, I_T=0.3)):
        P = O.Params(**params)
        w = 74.0
        k = D.spatial_root(P, w)
        coef = D.quartic(P, k)          # quartic in omega at this (complex) k
        val = np.polyval(coef, w)
        assert abs(val) <= 1e-10 * np.sum(np.abs(coef) * np.abs(w) ** np.arange(4, -1, -1))
        assert k.real > 0


def driven_amplitude(P, N, t_end, w, k, amp=1e-4, samples=32):
    md = D.eigenmode(P, k, w)
    base = D.equilibrium(P)
    drv = O.drive(w, k, base, amp * md["cons"])
    U = np.repeat(base[:, None], N, axis=1)
    U, t, _, rc = O.run_driven(P, U, N, 1.0 / N, t_end, drv)
    assert rc == 0
    Tp = 2 * math.pi / w
    acc = np.zeros(N, dtype=complex)
    for i in range(samples):
        U, t, _, rc = O.run_driven(P, U, N, 1.0 / N, t_end + (i + 1) * Tp / samples, drv, t0=t)
        acc += (U[1] / U[0]) * np.exp(1j * w * t)
    return 2 * acc / samples


def test_spatial_growth_matches_eq8():
    """S = 0.5, tau_rho = -1, tau_T = -1.5 (the paper's set), wavelength ~0.1,
    omega tau0 ~ 1: the measured spatial growth of the driven wave agrees with
    -Im k of eq. 8 within 2% and its wavenumber within 0.5%."""
    P = O.Params(S=0.5, tau0=0.0135)
    w = 2 * math.pi / 0.1 * 1.18
    k = D.spatial_root(P, w)
    N = 2000
    a = driven_amplitude(P, N, 1.0, w, k)
    x = inputs.cell_centres(N, 1.0)
    sel = (x > 0.1) & (x < 0.5)
    growth = np.polyfit(x[sel], np.log(np.abs(a[sel])), 1)[0]
    kr = np.polyfit(x[sel], np.unwrap(np.angle(a[sel])), 1)[0]
    assert k.imag < 0
    assert abs(growth + k.imag) <= 0.02 * abs(k.imag)
    assert abs(kr - k.real) <= 0.005 * k.real
