"""Pins of the oracle's 2D step with boundaries, medium map and driven cells
(orc_step2m; the paper's two-dimensional active-sector problem, Sec. 3).

Each pin is fixed by something other than the function itself: the periodic
step, the 1D boundary step, symmetry, exact conservation at solid walls, the
steady states of both media, the definition of the driven cells."""
import math

import numpy as np
import pytest

from oracle import orc as O
from paper_1805_03442_gb300 import inputs

PER, WALL, OUT = O.PERIODIC, O.REFLECT, O.OUTFLOW


def rnd(nx, ny, seed):
    return inputs.random_states(2, nx * ny, seed=seed, smooth=True)


def dt_of(P, U, nx, ny, h):
    return O.dt_cfl(P, U, (nx, ny), h)


@pytest.mark.parametrize("nx,ny", [(12, 10), (7, 9), (1, 6), (5, 1)])
def test_periodic_equals_periodic_step(nx, ny):
    P = O.Params(tau0=0.3)
    U = rnd(nx, ny, nx * 31 + ny)
    h = 1.0 / max(nx, ny)
    dt = dt_of(P, U, nx, ny, h)
    a, rc = O.step2m(P, U, nx, ny, h, dt, (PER, PER, PER, PER))
    b, rc2 = O.step(P, U, (nx, ny), h, dt)
    assert rc == rc2 == 0
    assert np.array_equal(a, b)


@pytest.mark.parametrize("bcx", [(WALL, WALL), (OUT, OUT), (WALL, OUT), (OUT, WALL), (PER, WALL)])
def test_rows_of_y_uniform_data_equal_the_1d_boundary_step(bcx):
    """Data uniform in y with v = 0: every row is the 1D step with the same x
    boundaries (the y fluxes cancel exactly)."""
    nx, ny = 23, 4
    P = O.Params(tau0=0.2)
    U1 = inputs.random_states(1, nx, seed=8, smooth=True)
    U2 = np.zeros((5, ny, nx))
    for f, g in ((0, 0), (1, 1), (3, 2), (4, 3)):
        U2[f] = U1[g][None, :]
    U2 = U2.reshape(5, -1)
    h = 1.0 / nx
    dt = 0.8 * O.dt_cfl(P, U1, (nx,), h)
    for bcy in ((PER, PER), (WALL, WALL), (OUT, OUT)):
        out2, rc2 = O.step2m(P, U2, nx, ny, h, dt, bcx + bcy)
        out1, rc1 = O.step_bc1(P, U1, nx, h, dt, *bcx)
        assert rc1 == rc2 == 0
        o2 = out2.reshape(5, ny, nx)
        for j in range(ny):
            for f, g in ((0, 0), (1, 1), (3, 2), (4, 3)):
                assert np.array_equal(o2[f, j], out1[g])
            assert np.all(o2[2, j] == 0.0)


@pytest.mark.parametrize("bc", [(WALL, OUT, OUT, WALL), (OUT, OUT, WALL, WALL), (PER, WALL, OUT, PER)])
def test_transposed_problem_gives_transposed_result(bc):
    nx, ny = 9, 13
    P = O.Params(tau0=0.25)
    U = rnd(nx, ny, 5).reshape(5, ny, nx)
    h = 0.1
    dt = 0.7 * dt_of(P, U.reshape(5, -1), nx, ny, h)
    a, rc = O.step2m(P, U.reshape(5, -1), nx, ny, h, dt, bc)
    Ut = U.transpose(0, 2, 1)[[0, 2, 1, 3, 4]]          # swap axes and momenta
    bt = (bc[2], bc[3], bc[0], bc[1])
    b, rc2 = O.step2m(P, np.ascontiguousarray(Ut).reshape(5, -1), ny, nx, h, dt, bt)
    assert rc == rc2 == 0
    bb = b.reshape(5, nx, ny).transpose(0, 2, 1)[[0, 2, 1, 3, 4]]
    assert np.array_equal(a.reshape(5, ny, nx), bb)


def test_walls_conserve_mass_and_energy():
    """Solid walls on all sides: the mirrored face states give zero mass and
    energy flux through the walls, and with zero Q/I exponents E has no source,
    so the totals of rho and E change only by rounding."""
    nx, ny = 20, 17
    P = O.Params(tau0=0.3)
    U = rnd(nx, ny, 3)
    h = 0.05
    m0, e0 = U[0].sum(), U[3].sum()
    U2, t, k, rc = O.run2m(P, U, nx, ny, h, 0.2, (WALL, WALL, WALL, WALL))
    assert rc == 0 and k > 10
    assert abs(U2[0].sum() - m0) <= 1e-13 * m0
    assert abs(U2[3].sum() - e0) <= 1e-13 * abs(e0)
    # an open boundary lets mass through
    U3, _, _, _ = O.run2m(P, U, nx, ny, h, 0.2, (WALL, OUT, WALL, WALL))
    assert abs(U3[0].sum() - m0) > 1e-8 * m0


def test_wall_mirror_symmetry():
    """A state mirror-symmetric about x = Lx/2 (u odd) between two walls stays
    mirror-symmetric."""
    nx, ny = 16, 6
    P = O.Params(tau0=0.3)
    U = rnd(nx, ny, 9).reshape(5, ny, nx)
    U[:, :, nx // 2:] = U[:, :, : nx // 2][:, :, ::-1]
    U[1, :, nx // 2:] *= -1.0
    out, t, k, rc = O.run2m(P, U.reshape(5, -1), nx, ny, 0.1, 0.15, (WALL, WALL, OUT, PER))
    assert rc == 0
    o = out.reshape(5, ny, nx)
    mir = o[:, :, ::-1].copy()
    mir[1] *= -1.0
    assert np.allclose(o, mir, rtol=0, atol=1e-13)


def test_medium_map_everywhere_and_nowhere():
    nx, ny = 11, 8
    P = O.Params(S=1.0, tau0=0.2)
    U = rnd(nx, ny, 4)
    h = 0.1
    dt = dt_of(P, U, nx, ny, h)
    bc = (OUT, WALL, OUT, OUT)
    plain, _ = O.step2m(P, U, nx, ny, h, dt, bc)
    every = O.Medium2(np.zeros(ny), np.full(ny, nx))
    a, _ = O.step2m(P, U, nx, ny, h, dt, bc, every)
    assert np.array_equal(a, plain)
    none = O.Medium2(np.zeros(ny), np.zeros(ny))
    b, _ = O.step2m(P, U, nx, ny, h, dt, bc, none)
    frozen, _ = O.step2m(P.frozen(), U, nx, ny, h, dt, bc)
    assert np.array_equal(b, frozen)
    assert not np.array_equal(a, b)


def test_medium_map_is_local():
    """One step reaches two cells: a cell whose 5x5 neighbourhood lies in one
    medium takes that medium's uniform-map value, bit for bit."""
    pb = inputs.sector_problem(40)
    P = O.Params(S=1.0, tau0=0.05)
    lo, hi = pb.maps[0], pb.maps[1]
    U = rnd(pb.nx, pb.ny, 6)
    dt = 0.5 * dt_of(P, U, pb.nx, pb.ny, pb.h)
    bc = (OUT, OUT, OUT, OUT)
    mixed, _ = O.step2m(P, U, pb.nx, pb.ny, pb.h, dt, bc, O.Medium2(lo, hi))
    active, _ = O.step2m(P, U, pb.nx, pb.ny, pb.h, dt, bc)
    frozen, _ = O.step2m(P.frozen(), U, pb.nx, pb.ny, pb.h, dt, bc)
    i = np.arange(pb.nx)[None, :]
    inside = (i >= lo[:, None]) & (i < hi[:, None])
    pad = np.pad(inside, 2, mode="edge")
    win = np.stack([pad[2 + a: 2 + a + pb.ny, 2 + b: 2 + b + pb.nx]
                    for a in range(-2, 3) for b in range(-2, 3)])
    all_in, all_out = win.all(axis=0), (~win).all(axis=0)
    m, ac, fr = (x.reshape(5, pb.ny, pb.nx) for x in (mixed, active, frozen))
    assert all_in.sum() > 50 and all_out.sum() > 50
    assert np.array_equal(m[:, all_in], ac[:, all_in])
    assert np.array_equal(m[:, all_out], fr[:, all_out])
    assert not np.array_equal(m, ac) and not np.array_equal(m, fr)


def test_rest_state_stays_at_rest():
    """rho = p = 1, v = 0, e_nu = C_k + S is steady in the active medium (pump
    balances relaxation) and in the frozen one; with the sector map, walls and
    outflow and no driving it stays put up to rounding."""
    pb = inputs.sector_problem(48)
    P = O.Params(S=1.0, tau0=0.05)
    U = inputs.sector_rest_state(1.4, P.Ck, P.S, pb.nx, pb.ny)
    M = O.Medium2(pb.maps[0], pb.maps[1])
    out, t, k, rc = O.run2m(P, U, pb.nx, pb.ny, pb.h, 0.05, pb.bc, M)
    assert rc == 0 and k > 5
    assert np.max(np.abs(out - U)) <= 1e-13


def test_driven_cells_hold_the_pulse():
    pb = inputs.sector_problem(120)
    P = O.Params(S=1.0, tau0=0.05)
    lo, hi, dlo, dhi = pb.maps
    U = inputs.sector_rest_state(1.4, P.Ck, P.S, pb.nx, pb.ny)
    M = O.Medium2(lo, hi, dlo, dhi, pb.omega, pb.amp)
    t, dt = 0.013, 0.7 * O.dt_cfl(P, U, (pb.nx, pb.ny), pb.h)
    out, rc = O.step2m(P, U, pb.nx, pb.ny, pb.h, dt, pb.bc, M, t)
    assert rc == 0
    o = out.reshape(5, pb.ny, pb.nx)
    s = pb.amp * math.sin(pb.omega * (t + dt))
    n_driven = 0
    for j in range(pb.ny):
        for i in range(dlo[j], dhi[j]):
            rho, p = 1.0 + s, 1.0 + 1.4 * s
            ev = rho * (P.Ck + P.S)
            want = [rho, 0.0, 0.0, p / 0.4 + ev, ev]
            assert np.allclose(o[:, j, i], want, rtol=1e-15, atol=1e-15)
            n_driven += 1
    assert n_driven >= 8
    # everything else started at rest and moves only next to the source
    far = o[:, :, pb.nx - 3:]
    assert np.max(np.abs(far - U.reshape(5, pb.ny, pb.nx)[:, :, pb.nx - 3:])) <= 1e-14


def test_sector_amplifies_and_outside_does_not():
    """Linear stage of the active-sector problem at low resolution: the wave
    leaving the source is stronger inside the sector than at the same radius
    outside it."""
    pb = inputs.sector_problem(96)
    P = O.Params(S=1.0, tau0=0.0135)
    lo, hi, dlo, dhi = pb.maps
    U = inputs.sector_rest_state(1.4, P.Ck, P.S, pb.nx, pb.ny)
    M = O.Medium2(lo, hi, dlo, dhi, pb.omega, pb.amp)
    out, t, k, rc = O.run2m(P, U, pb.nx, pb.ny, pb.h, 0.4, pb.bc, M)
    assert rc == 0
    rho = out[0].reshape(pb.ny, pb.nx) - 1.0
    x = (np.arange(pb.nx) + 0.5) * pb.h - pb.apex[0]
    y = (np.arange(pb.ny) + 0.5) * pb.h - pb.apex[1]
    X, Y = np.meshgrid(x, y)
    r = np.hypot(X, Y)
    ang = np.degrees(np.arctan2(Y, X))
    ring = (r > 0.25) & (r < 0.4)           # 2.5-4 wavelengths out, 7 cells per wavelength
    inside = np.abs(rho[ring & (np.abs(ang) < 10)]).max()
    outside = np.abs(rho[ring & (np.abs(ang) > 40) & (np.abs(ang) < 140)]).max()
    assert inside > 2.0 * outside


def test_bad_arguments():
    U = rnd(4, 4, 1)
    P = O.Params()
    assert O.step2m(P, U, 4, 4, 0.1, 1e-3, (WALL, WALL, 7, PER))[1] == -3
    assert O.step2m(P, rnd(1, 4, 1), 1, 4, 0.1, 1e-3, (WALL, WALL, PER, PER))[1] == -3
