"""Conservation budget of one step (the pin list's budget check): on a periodic
grid the flux differences of eq. 15 telescope, so the sums of rho and rho v
do not change and the sums of E and E_nu change by dt times the summed source
Y at the half-step states (the Y vector of Sec. 2.3 with the closures of
eq. 6).

The half-step states are known in closed form on a checkerboard: cells that
alternate between two states A and B along every axis have one-sided
differences of opposite sign on every axis, so every limited slope is zero
(minmod, van Leer and MC alike), the predictor's flux difference
F(U + 0) - F(U - 0) vanishes, and U^{n+1/2} = U + dt/2 Y(U) cell by cell.  The
expected budget is then dt sum_j Y(U_j + dt/2 Y(U_j)), written here from the
source's definition (reading 1: Y_E = rho (Q - I), Y_Enu = (rho C_k T - E_nu)
/ tau + rho Q, with tau, Q, I the power laws of eq. 6 and I0 = Q0 = S / tau0).
A source taken at U^n instead of U^{n+1/2}, a half step of dt instead of
dt/2, or a flux that does not telescope fails these tests."""
import math

import numpy as np
import pytest

from oracle import orc as O

GENERAL = dict(tau0=0.05, S=0.7, tau_rho=-1.0, tau_T=-1.5, Q_rho=0.4, Q_T=-0.3, I_rho=0.2,
               I_T=0.5)


def source(P, U):
    """(Y_E, Y_Enu) of conserved states U (nf, ncell): eq. 6 closures and the
    Y vector of Sec. 2.3 under reading 1 (R = 1, T = p / rho)."""
    dim = U.shape[0] - 3
    rho, E, Ev = U[0], U[dim + 1], U[dim + 2]
    kin = sum(U[1 + a] ** 2 for a in range(dim)) / (2.0 * rho)
    p = (P.gamma - 1.0) * (E - kin - Ev)
    T = p / rho
    Q0 = P.S / P.tau0
    tau = P.tau0 * rho ** P.tau_rho * T ** P.tau_T
    Q = Q0 * rho ** P.Q_rho * T ** P.Q_T
    I = Q0 * rho ** P.I_rho * T ** P.I_T
    return rho * (Q - I), (rho * P.Ck * T - Ev) / tau + rho * Q


def state(gamma, rho, vel, p, ev):
    """Conserved state of one cell (eq. 5)."""
    m = [rho * v for v in vel]
    E = p / (gamma - 1.0) + 0.5 * rho * sum(v * v for v in vel) + ev
    return np.array([rho, *m, E, ev])


def checkerboard(gamma, n):
    """Two states, out of equilibrium and moving, alternating along every axis
    (x fastest in the flat layout)."""
    dim = len(n)
    A = state(gamma, 1.0, [0.3, -0.2, 0.1][:dim], 1.0, 0.45)
    B = state(gamma, 1.2, [-0.1, 0.25, -0.15][:dim], 0.8, 0.2)
    idx = np.indices(tuple(reversed(n))).sum(axis=0).reshape(-1) % 2
    return np.where(idx[None, :] == 0, A[:, None], B[:, None])


def budget(P, U, dt):
    yE, yEv = source(P, U)
    Uh = U.copy()
    dim = U.shape[0] - 3
    Uh[dim + 1] += 0.5 * dt * yE
    Uh[dim + 2] += 0.5 * dt * yEv
    hE, hEv = source(P, Uh)
    return dt * np.sum(hE), dt * np.sum(hEv), dt * np.sum(yE), dt * np.sum(yEv)


@pytest.mark.parametrize("limiter", [0, 1, 2])
@pytest.mark.parametrize("n", [(16,), (8, 6), (4, 6, 8)])
def test_step_changes_sums_by_the_half_step_source(orc, n, limiter):
    P = O.Params(limiter=limiter, **GENERAL)
    U = checkerboard(P.gamma, n)
    dim = len(n)
    h = 1.0 / n[0]
    dt = O.dt_cfl(P, U, n, h)
    Un, rc = O.step(P, U, n, h, dt)
    assert rc == 0
    dS = Un.sum(axis=1) - U.sum(axis=1)
    scale = np.abs(U).sum(axis=1)
    # mass and momentum: conserved to rounding
    for f in range(dim + 1):
        assert abs(dS[f]) <= 1e-14 * scale[f] + 1e-15, (f, dS[f])
    bE, bEv, bE0, bEv0 = budget(P, U, dt)
    assert abs(bE) > 1e-6 and abs(bEv) > 1e-6
    assert dS[dim + 1] == pytest.approx(bE, rel=1e-12, abs=1e-14 * scale[dim + 1])
    assert dS[dim + 2] == pytest.approx(bEv, rel=1e-12, abs=1e-14 * scale[dim + 2])
    # the source at U^n instead of the half step is visibly different
    assert abs(bEv0 - bEv) > 1e3 * max(1e-12 * abs(bEv), 1e-14 * scale[dim + 2])


def test_checkerboard_slopes_vanish(orc):
    """The premise: every cell's one-sided differences have opposite signs on
    every axis, and the step keeps the two-state checkerboard (all A cells and
    all B cells update alike)."""
    n = (6, 4, 4)
    P = O.Params(**GENERAL)
    U = checkerboard(P.gamma, n)
    shape = (U.shape[0],) + tuple(reversed(n))
    G = U.reshape(shape)
    for ax in range(1, 4):
        a = G - np.roll(G, 1, axis=ax)
        b = np.roll(G, -1, axis=ax) - G
        assert np.all(a * b <= 0)
    h = 1.0 / n[0]
    Un, _ = O.step(P, U, n, h, O.dt_cfl(P, U, n, h))
    par = np.indices(tuple(reversed(n))).sum(axis=0).reshape(-1) % 2
    for k in (0, 1):
        cells = Un[:, par == k]
        assert np.allclose(cells, cells[:, :1], rtol=1e-14, atol=1e-15)


def test_frozen_limit_conserves_every_field(orc):
    """tau0 = inf (no source): all four sums, E and E_nu included, are
    conserved."""
    P = O.Params(tau0=math.inf, S=0.0)
    n = (32,)
    U = checkerboard(P.gamma, n)
    h = 1.0 / n[0]
    Un, rc = O.step(P, U, n, h, O.dt_cfl(P, U, n, h))
    assert rc == 0
    assert np.allclose(Un.sum(axis=1), U.sum(axis=1), rtol=1e-14, atol=1e-14)
