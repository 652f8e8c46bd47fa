"""GPU parity of the positivity guard: the hand-built states of
test_oracle_guard.py (a cell whose extrapolated state has p < 0, and a cell
whose half-step face states have p < 0), tiled periodically over small grids
(sliding-warp kernels) and over grids of >= 4096 cells (the block-tile kernel
of the float benchmark line), one step against the oracle at the GPU's dt, in
every launch configuration of the solver."""
import numpy as np
import pytest

from gpu_util import field_rel_linf, need_gpu, oracle_params, rel_linf
from oracle import orc as O
from test_oracle_guard import CASE_A, CASE_B, FROZEN, _array

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sv():
    return need_gpu()


def _tiled(case, reps):
    return np.tile(_array(case["cells"]), (1, reps))


@pytest.mark.parametrize("prec", ["FP64", "FP32"])
@pytest.mark.parametrize("reps", [1, 7, 700])
@pytest.mark.parametrize("name", ["a", "b"])
def test_guard_states_match_oracle(sv, prec, reps, name):
    case = CASE_A if name == "a" else CASE_B
    # case (b) needs a half step long enough to drive the face states below
    # zero pressure: dt = h/2 at |v| = 10 is cfl = 10 (eq. 16 with 2|v| = 20)
    P = sv.Params(precision=getattr(sv, prec), cfl=10.0 if name == "b" else 0.4, **FROZEN)
    Po = oracle_params(P)
    U0 = _tiled(case, reps)
    if prec == "FP32":
        U0 = U0.astype(np.float32).astype(np.float64)
    N = U0.shape[1]
    h = 1.0 / N
    with sv.Solver(P, (N,), (1.0,)) as s:
        ncfg = len(s.configs())
        results = []
        for c in range(ncfg):
            s.set_config(c)
            s.write_state(U0)
            dt = s.dt()
            s.step(1)
            U, _ = s.read_state()
            results.append((U, dt, s.status()))
    ref, rc = O.step(Po, U0, (N,), h, results[0][1])
    if name == "b":
        expect_r = float(case["r"])
        assert results[0][1] == pytest.approx(expect_r * h, rel=1e-6)
    for c, (U, dt, flags) in enumerate(results):
        assert dt == results[0][1]
        assert bool(flags & sv.FLAG_NONPHYS) == (rc != 0), (c, flags, rc)
        tol = 1e-12 if prec == "FP64" else 2e-6
        assert rel_linf(U, ref) <= tol, (c, rel_linf(U, ref))
        assert max(field_rel_linf(U, ref).values()) <= tol, (c, field_rel_linf(U, ref))
    # the guarded cells take the first-order upwind value of the oracle pins
    j = case["j"]
    for U, _, _ in results:
        assert np.max(np.abs(U[:, j::6] - ref[:, j::6])) <= (1e-12 if prec == "FP64" else 1e-4)
