"""Pins of the oracle's 1D boundary conditions (solid walls, free outflow) and
of the colliding-shock test the paper uses to verify its schemes."""
import json
import math
import os

import numpy as np
import pytest

from oracle import orc as O
from paper_1805_03442_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "woodward_colella.json")
MIR = np.array([1.0, -1.0, 1.0, 1.0])[:, None]


def wc_state(N):
    g = json.load(open(GOLDEN))["initial"]
    x = inputs.cell_centres(N, 1.0)
    p = np.where(x < g["x_left"], g["p_left"], np.where(x <= g["x_right"], g["p_middle"], g["p_right"]))
    return inputs.prim_to_cons(g["gamma"], np.full(N, g["rho"]), [np.full(N, g["u"])], p,
                               np.full(N, 0.3))


def test_periodic_ghosts_equal_the_periodic_step(orc):
    P = O.Params(tau0=0.3)
    N = 50
    U = inputs.random_states(1, N, seed=4, smooth=True)
    dt = O.dt_cfl(P, U, N, 1.0 / N)
    a, _ = O.step(P, U, N, 1.0 / N, dt)
    b, _ = O.step_bc1(P, U, N, 1.0 / N, dt, O.PERIODIC, O.PERIODIC)
    assert np.array_equal(a, b)


@pytest.mark.parametrize("params", [dict(tau0=0.3), dict(tau0=math.inf, S=0.0)])
def test_wall_equals_mirrored_periodic_domain(orc, params):
    """A domain with walls at both ends evolves exactly like the periodic domain
    of twice the length holding the mirror image (x -> 2L - x, v -> -v)."""
    P = O.Params(**params)
    N, h = 40, 1.0 / 40
    U = inputs.random_states(1, N, seed=8, smooth=True)
    D = np.concatenate([U, (U * MIR)[:, ::-1]], axis=1)
    for _ in range(6):
        dt = O.dt_cfl(P, U, N, h)
        U, rc = O.step_bc1(P, U, N, h, dt, O.REFLECT, O.REFLECT)
        D, _ = O.step(P, D, 2 * N, h, dt)
        assert rc == 0
        assert np.array_equal(U, D[:, :N])


def test_outflow_keeps_a_uniform_flow(orc):
    P = O.Params(tau0=0.2)
    N = 30
    U = inputs.prim_to_cons(1.4, np.full(N, 1.0), [np.full(N, 0.3)], np.full(N, 1.0),
                            np.full(N, P.Ck + P.S))
    U1, _, _, rc = O.run_bc1(P, U, N, 1.0 / N, 0.05, O.OUTFLOW, O.OUTFLOW)
    assert rc == 0
    assert np.allclose(U1, U, rtol=1e-13, atol=1e-14)


def test_walls_conserve_mass(orc):
    P = O.Params().frozen()
    N = 400
    U = wc_state(N)
    U1, t, k, rc = O.run_bc1(P, U, N, 1.0 / N, 0.01, O.REFLECT, O.REFLECT)
    assert rc == 0 and k > 100
    assert abs(math.fsum(U1[0]) - math.fsum(U[0])) <= 1e-13 * math.fsum(U[0])


def test_colliding_shocks_as_printed():
    """The two strong shocks collide at t1 = 0.028 with a peak at x = 0.7 (N = 1000,
    solid walls, frozen ideal gas gamma 1.4)."""
    g = json.load(open(GOLDEN))
    P = O.Params().frozen()
    N = g["grid_cells_fig1"]
    x = inputs.cell_centres(N, 1.0)
    U, t, _, rc = O.run_bc1(P, wc_state(N), N, 1.0 / N, g["collision_time"], O.REFLECT, O.REFLECT)
    assert rc == 0 and t == g["collision_time"]
    p = 0.4 * (U[2] - 0.5 * U[1] ** 2 / U[0] - U[3])
    assert abs(x[np.argmax(p)] - g["collision_position"]) <= 0.02
    # shortly before, the two shocks are still apart: two separate pressure maxima
    U0, _, _, _ = O.run_bc1(P, wc_state(N), N, 1.0 / N, 0.02, O.REFLECT, O.REFLECT)
    p0 = 0.4 * (U0[2] - 0.5 * U0[1] ** 2 / U0[0] - U0[3])
    left, right = p0[x < 0.69].max(), p0[x > 0.71].max()
    assert min(left, right) > 10 * p0[np.abs(x - 0.7) < 0.005].min()


def test_colliding_shocks_converge():
    """At the comparison time t = 0.038, coarse solutions approach a fine-grid
    solution as the grid is refined (the paper's N = 200 ... 1600 vs a very fine
    run)."""
    g = json.load(open(GOLDEN))
    P = O.Params().frozen()
    T = g["comparison_time"]
    Nf = 3200
    Uf, _, _, _ = O.run_bc1(P, wc_state(Nf), Nf, 1.0 / Nf, T, O.REFLECT, O.REFLECT)
    errs = []
    for N in (200, 400, 800, 1600):
        U, _, _, rc = O.run_bc1(P, wc_state(N), N, 1.0 / N, T, O.REFLECT, O.REFLECT)
        assert rc == 0
        errs.append(np.mean(np.abs(U[0] - Uf[0].reshape(N, -1).mean(axis=1))))
    assert all(b < a for a, b in zip(errs, errs[1:])), errs
    assert errs[-1] < 0.35 * errs[0]
