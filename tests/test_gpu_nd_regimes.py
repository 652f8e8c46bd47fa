"""The 2D / 3D kernels in the regimes that so far only the 1D tests reached.

* The positivity guard: the hand-built periodic states of test_oracle_guard.py
  (case a: an extrapolated state with p < 0; case b: half-step face states
  with p < 0) laid along the x, y or z axis of a 2D / 3D grid, uniform across
  it with no transverse velocity.  One step against the ND oracle at the GPU's
  dt, in every launch configuration; the guarded cells must take the
  first-order upwind value that the oracle pins in exact arithmetic.
* The stiff-source regime, where the cap dt <= c_tau min tau (a reading of the
  paper: eq. 16 bounds only the advection) sets every step: tau0 = 1e-3 with
  general closure exponents of eq. 6, four steps against the oracle.

Tolerances as in the 1D tests: FP64 to 1e-12 (assert_fp64_parity), float to
2e-6 after one step on float-representable inputs; dt to 1e-13 / 1e-5."""
import numpy as np
import pytest

from gpu_util import assert_fp64_parity, need_gpu, oracle_params, rel_linf
from oracle import orc as O
from paper_1805_03442_gb300 import inputs
from test_oracle_guard import CASE_A, CASE_B, FROZEN, embed_nd
from test_gpu_taucap import STIFF, oracle_params_like

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sv():
    return need_gpu()


GUARD_GRIDS = [(2, 0, 7, (5,)), (2, 1, 7, (37,)), (2, 0, 70, (3,)), (2, 1, 70, (9,)),
               (3, 0, 7, (5, 4)), (3, 1, 7, (4, 3)), (3, 2, 7, (3, 5)), (3, 2, 20, (17, 4))]


@pytest.mark.parametrize("prec", ["FP64", "FP32"])
@pytest.mark.parametrize("grid", GUARD_GRIDS, ids=lambda g: f"{g[0]}d-axis{g[1]}-x{g[2]}-{g[3]}")
@pytest.mark.parametrize("name", ["a", "b"])
def test_guard_states_nd(sv, prec, grid, name):
    dim, axis, reps, other = grid
    case = CASE_A if name == "a" else CASE_B
    U0, n = embed_nd(case, reps, dim, axis, other)
    if prec == "FP32":
        U0 = U0.astype(np.float32).astype(np.float64)
    P = sv.Params(precision=getattr(sv, prec), cfl=10.0 if name == "b" else 0.4, **FROZEN)
    Po = oracle_params(P)
    h = 1.0 / n[0]
    L = tuple(x * h for x in n)
    with sv.Solver(P, n, L) as s:
        results = []
        for c in range(len(s.configs())):
            s.set_config(c)
            s.write_state(U0)
            dt = s.dt()
            s.step(1)
            U, _ = s.read_state()
            results.append((U, dt, s.status()))
    dt = results[0][1]
    if name == "b":
        assert dt == pytest.approx(float(case["r"]) * h, rel=1e-6)
    ref, rc = O.step(Po, U0, n, h, dt)
    tol = 1e-12 if prec == "FP64" else 2e-6
    shape = (U0.shape[0],) + tuple(reversed(n))
    j = case["j"]
    for c, (U, dtc, flags) in enumerate(results):
        assert dtc == dt
        assert bool(flags & sv.FLAG_NONPHYS) == (rc != 0), (c, flags, rc)
        assert rel_linf(U, ref) <= tol, (c, rel_linf(U, ref))
        # the guarded cells: every sixth cell along the axis from j, every
        # transverse position
        sel = [slice(None)] * (dim + 1)
        sel[dim - axis] = slice(j, None, 6)
        got, want = U.reshape(shape)[tuple(sel)], ref.reshape(shape)[tuple(sel)]
        assert np.max(np.abs(got - want)) <= (1e-12 if prec == "FP64" else 1e-4), c


TAU_SHAPES = [(7, 5), (37, 29), (300, 70), (5, 4, 6), (33, 17, 9), (65, 40, 20)]


def _tau_run(sv, P, Po, U0, n, h, nsteps):
    with sv.Solver(P, n, tuple(x * h for x in n)) as s:
        s.write_state(U0)
        dts = []
        for _ in range(nsteps):
            dts.append(s.dt())
            s.step(1)
        U, t = s.read_state()
        assert s.status() == 0
    ref, rdts = U0.copy(), []
    for _ in range(nsteps):
        rdts.append(O.dt_cfl(Po, ref, n, h))
        ref, rc = O.step(Po, ref, n, h, rdts[-1])
        assert rc == 0
    return U, t, dts, ref, rdts


def _spacing(n):
    """h = 1/64 from 64 cells up (the cap binds at coarse spacing), 1/n_x below."""
    return 1.0 / min(n[0], 64)


@pytest.mark.parametrize("limiter", [0, 1])
@pytest.mark.parametrize("n", TAU_SHAPES)
def test_fp64_tau_cap_nd(sv, n, limiter):
    P = sv.Params(precision=sv.FP64, limiter=limiter, **STIFF)
    Po = oracle_params(P)
    h = _spacing(n)
    U0 = inputs.random_states(len(n), int(np.prod(n)), seed=200 + sum(n), smooth=True)
    assert O.dt_cfl(Po, U0, n, h) < 0.5 * O.dt_cfl(oracle_params_like(Po, c_tau=1e30), U0, n, h)
    U, t, dts, ref, rdts = _tau_run(sv, P, Po, U0, n, h, 4)
    assert np.allclose(dts, rdts, rtol=1e-13, atol=0)
    assert t == pytest.approx(sum(rdts), rel=1e-14)
    assert_fp64_parity(U, ref)


@pytest.mark.parametrize("precision", ["FP32", "FP32_PC"])
@pytest.mark.parametrize("n", TAU_SHAPES)
def test_fp32_tau_cap_nd(sv, precision, n):
    P = sv.Params(precision=getattr(sv, precision), **STIFF)
    Po = oracle_params(P)
    h = _spacing(n)
    U0 = inputs.random_states(len(n), int(np.prod(n)), seed=300 + sum(n), smooth=True)
    U0 = U0.astype(np.float32).astype(np.float64)
    assert O.dt_cfl(Po, U0, n, h) < 0.5 * O.dt_cfl(oracle_params_like(Po, c_tau=1e30), U0, n, h)
    U, t, dts, ref, rdts = _tau_run(sv, P, Po, U0, n, h, 1)
    assert dts[0] == pytest.approx(rdts[0], rel=1e-5)
    ref, _ = O.step(Po, U0, n, h, dts[0])
    assert rel_linf(U, ref) <= 2e-6
