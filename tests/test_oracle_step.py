"""Pins of the oracle's MUSCL-Hancock step (eqs. 13-16) against what the paper
and the mathematics fix: stationarity of the equilibrium, exact conservation on
periodic grids, symmetries, reduction of 2D/3D to 1D, the exact Riemann
solution in the frozen limit, second-order convergence on smooth flow, and the
linear growth rate of eq. 8."""
import math

import numpy as np
import pytest

from oracle import dispersion as D
from oracle import orc as O
from oracle.riemann import Riemann
from paper_1805_03442_gb300 import inputs


def _grid_state(dim, n, seed, smooth=True):
    ncell = int(np.prod(n))
    return inputs.random_states(dim, ncell, seed, smooth=smooth)


@pytest.mark.parametrize("dim,n", [(1, (16,)), (2, (8, 6)), (3, (5, 4, 6))])
def test_equilibrium_is_stationary(orc, dim, n):
    P = O.Params(S=0.7, tau0=0.2, Q_rho=0.3, I_T=-0.2)
    U0 = D.equilibrium(P, dim)
    U = np.repeat(U0[:, None], int(np.prod(n)), axis=1)
    h = 1.0 / n[0]
    Un, rc = O.step(P, U, n, h, O.dt_cfl(P, U, n, h))
    assert rc == 0
    assert np.array_equal(Un[: dim + 1], U[: dim + 1])        # rho, momenta: fluxes cancel
    assert np.max(np.abs(Un - U)) < 1e-14


@pytest.mark.parametrize("dim,n", [(1, (37,)), (2, (9, 7)), (3, (5, 6, 4))])
def test_step_cell_matches_step_bitwise(orc, dim, n):
    P = O.Params(tau0=0.3)
    U = _grid_state(dim, n, 3)
    h = 0.1
    dt = O.dt_cfl(P, U, n, h)
    Un, _ = O.step(P, U, n, h, dt)
    for idx in [0, 1, int(np.prod(n)) // 2, int(np.prod(n)) - 1]:
        assert np.array_equal(O.step_cell(P, U, n, h, dt, idx), Un[:, idx])


@pytest.mark.parametrize("dim,n", [(1, (64,)), (2, (12, 10)), (3, (6, 5, 7))])
def test_conservation(orc, dim, n):
    """Periodic grid: sum rho and sum rho v are invariant (no momentum source,
    f = 0); in the frozen limit sum E and sum E_nu are invariant as well."""
    h = 1.0 / n[0]
    for P, fields in ((O.Params(tau0=0.2), range(dim + 1)), (O.Params().frozen(), range(dim + 3))):
        U = _grid_state(dim, n, 5)
        U1, steps = U.copy(), 0
        for _ in range(5):
            U1, rc = O.step(P, U1, n, h, O.dt_cfl(P, U1, n, h))
            assert rc == 0
        for f in fields:
            s0, s1 = math.fsum(U[f]), math.fsum(U1[f])
            assert abs(s1 - s0) <= 1e-13 * math.fsum(np.abs(U[f])), f


def test_mirror_symmetry_1d(orc):
    P = O.Params(tau0=0.3, Q_T=0.4)
    n = (40,)
    U = _grid_state(1, n, 11)
    h = 0.05
    dt = O.dt_cfl(P, U, n, h)
    mir = np.array([1, -1, 1, 1])[:, None]
    Um = (U * mir)[:, ::-1].copy()
    A, _ = O.step(P, U, n, h, dt)
    B, _ = O.step(P, Um, n, h, dt)
    assert np.allclose((B * mir)[:, ::-1], A, rtol=1e-13, atol=1e-13)


@pytest.mark.parametrize("dim,axis", [(2, 0), (2, 1), (3, 0), (3, 1), (3, 2)])
def test_multid_reduces_to_1d(orc, dim, axis):
    """A state varying along one axis only, with zero transverse velocity, must
    evolve exactly as the 1D problem along that axis (the transverse fluxes
    cancel)."""
    P = O.Params(tau0=0.3)
    N = 24
    U1 = _grid_state(1, (N,), 17)
    h = 1.0 / N
    dt = O.dt_cfl(P, U1, (N,), h)
    ref, _ = O.step(P, U1, (N,), h, dt)
    shape = [3] * dim
    shape[dim - 1 - axis] = N                                 # arrays are (z, y, x)
    n = tuple(reversed(shape))
    nf = dim + 3
    U = np.zeros((nf,) + tuple(shape))
    line = [slice(None) if d == dim - 1 - axis else None for d in range(dim)]
    src = {0: 0, 1 + axis: 1, 1 + dim: 2, 2 + dim: 3}
    for f in range(nf):
        if f in src:
            U[f] = np.broadcast_to(U1[src[f]][tuple(line)], shape)
    Un, _ = O.step(P, U.reshape(nf, -1), n, h, dt)
    Un = Un.reshape((nf,) + tuple(shape))
    for f, g in src.items():
        assert np.allclose(Un[f], np.broadcast_to(ref[g][tuple(line)], shape), rtol=1e-13, atol=1e-13)
    for f in range(1, dim + 1):
        if f != 1 + axis:
            assert np.max(np.abs(Un[f])) < 1e-14


def test_2d_transpose_symmetry(orc):
    P = O.Params(tau0=0.3)
    nx, ny = 7, 9
    U = _grid_state(2, (nx, ny), 23).reshape(5, ny, nx)
    h = 0.1
    dt = 0.5 * O.dt_cfl(P, U.reshape(5, -1), (nx, ny), h)
    A, _ = O.step(P, U.reshape(5, -1), (nx, ny), h, dt)
    Ut = U.transpose(0, 2, 1)[[0, 2, 1, 3, 4]].copy()
    B, _ = O.step(P, Ut.reshape(5, -1), (ny, nx), h, dt)
    Bt = B.reshape(5, nx, ny).transpose(0, 2, 1)[[0, 2, 1, 3, 4]]
    assert np.allclose(Bt, A.reshape(5, ny, nx), rtol=1e-13, atol=1e-13)


def test_dt_eq16_by_hand(orc):
    """Uniform u = 0.5, c = sqrt(1.4): dt = cfl h / max(2|u|, |u| + c); a short
    tau caps it at c_tau tau with tau = tau0 rho^tau_rho T^tau_T."""
    P = O.Params(tau0=10.0)
    N, h = 8, 0.01
    U = inputs.prim_to_cons(1.4, np.full(N, 1.0), [np.full(N, 0.5)], np.full(N, 1.0), np.full(N, 0.2))
    assert O.dt_cfl(P, U, (N,), h) == pytest.approx(0.4 * h / (0.5 + math.sqrt(1.4)), rel=1e-15)
    U = inputs.prim_to_cons(1.4, np.full(N, 2.0), [np.full(N, 0.5)], np.full(N, 1.0), np.full(N, 0.2))
    P = O.Params(tau0=1e-4)
    tau = 1e-4 * 2.0 ** -1.0 * 0.5 ** -1.5
    assert O.dt_cfl(P, U, (N,), h) == pytest.approx(0.5 * tau, rel=1e-14)


def test_frozen_double_tube_matches_exact_riemann(orc):
    """Frozen limit (Q = I = 0, 1/tau = 0): two Sod tubes at L/4 and 3L/4 on a
    periodic domain, compared with the exact solution before the waves meet.
    Gates: post-shock plateau density L1 <= 1e-3 and shock position (half-jump
    crossing) within one cell."""
    P = O.Params().frozen()
    N, L, t_end = 800, 1.0, 0.1
    h = L / N
    outer, inner = (1.0, 0.0, 1.0, 0.3), (0.125, 0.0, 0.1, 0.9)
    U = inputs.double_tube_1d(P.gamma, N, L, outer, inner)
    Ue, t, _, rc = O.run(P, U, N, h, t_end)
    assert rc == 0 and t == t_end
    x = inputs.cell_centres(N, L)
    R = Riemann(P.gamma, *outer[:3], *inner[:3], evL=outer[3], evR=inner[3])
    ex = R.sample_array((x - 0.25) / t_end)
    _, _, c, _, s = R.wave_speeds()
    xc, xs = 0.25 + c * t_end, 0.25 + s * t_end
    plateau = (x > xc + 10 * h) & (x < xs - 3 * h)
    assert plateau.sum() > 30
    assert np.mean(np.abs(Ue[0][plateau] - ex[0][plateau])) <= 1e-3
    rs = R.star_densities()[1]
    half = 0.5 * (rs + inner[0])
    i = np.where((x > xc) & (x < 0.5) & (Ue[0] < half))[0][0]
    xsh = x[i - 1] + (half - Ue[0][i - 1]) / (Ue[0][i] - Ue[0][i - 1]) * h
    assert abs(xsh - xs) <= h
    # mirror tube at 3L/4 gives the mirrored solution
    assert np.allclose(Ue[0][:N // 2], Ue[0][N // 2:][::-1], rtol=1e-12)


@pytest.mark.parametrize("limiter,order", [(O.MINMOD, 1.7), (O.MC, 1.9)])
def test_second_order_on_smooth_advection(orc, limiter, order):
    """Entropy wave rho = 1 + 0.2 sin(2 pi (x - t)), u = p = 1 in the frozen
    limit is translated exactly; L1 error must fall at second order."""
    P = O.Params(limiter=limiter).frozen()
    errs = []
    for N in (64, 128, 256):
        h = 1.0 / N
        x = inputs.cell_centres(N, 1.0)

        def avg(t):
            a, b = x - h / 2 - t, x + h / 2 - t
            return 1 + 0.2 * (np.cos(2 * np.pi * a) - np.cos(2 * np.pi * b)) / (2 * np.pi * h)

        U = inputs.prim_to_cons(P.gamma, avg(0), [np.ones(N)], np.ones(N), np.full(N, 0.5))
        Ue, _, _, _ = O.run(P, U, N, h, 1.0)
        errs.append(np.mean(np.abs(Ue[0] - avg(1.0))))
    rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(rates > order), rates


@pytest.mark.parametrize("params", [dict(tau0=0.08),
                                    dict(tau0=0.1, S=0.6, Q_rho=0.5, Q_T=0.5)])
def test_linear_growth_rate_matches_eq8(orc, params):
    """A growing eigenmode of amplitude 1e-4 on one wavelength (N = 256) grows
    at Im omega of eq. 8 within 2% and oscillates at Re omega within 1%."""
    P = O.Params(**params)
    N, L = 256, 1.0
    h = L / N
    k = 2 * math.pi / L
    w = D.growing_acoustic_root(P, k)
    assert w.imag > 0
    md = D.eigenmode(P, k, w)
    base = inputs.equilibrium_primitive(P.Ck, P.S)
    U = inputs.waves_1d(P.gamma, N, L, base, [inputs.Mode(m=1, shape=md["prim"], scale=1e-4)])
    x = inputs.cell_centres(N, L)
    ts, amps, t = [], [], 0.0
    t_stop = math.log(100.0) / w.imag
    while t < t_stop:
        U, t, _, rc = O.run(P, U, N, h, t + 0.05, t0=t)
        assert rc == 0
        ts.append(t)
        amps.append(np.sum(U[1] / U[0] * np.exp(-1j * k * x)) / N)
    ts, amps = np.array(ts), np.array(amps)
    growth = np.polyfit(ts, np.log(np.abs(amps)), 1)[0]
    freq = -np.polyfit(ts, np.unwrap(np.angle(amps)), 1)[0]
    assert abs(growth - w.imag) <= 0.02 * w.imag
    assert abs(freq - w.real) <= 0.01 * w.real
