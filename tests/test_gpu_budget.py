"""The conservation budget of one step on the GPU (see test_oracle_budget.py):
on checkerboards of two states, where every limited slope is zero and the
half-step states have a closed form, one step changes the device's field sums
(sv_conservation, compensated double sums) by zero for rho and rho v and by
dt times the summed half-step source for E and E_nu.  The expectation is
written from the source's definition, not taken from the oracle or the GPU.

FP64: to 1e-12 of the budget.  Float policies: the update rounds every cell's
E once (and alike in all cells of one colour, so the roundings add up rather
than cancel), which bounds |d sum - budget| by about N eps_f max|E|; the SFU
approximations of the source add ~1e-6 of it."""
import numpy as np
import pytest

from gpu_util import need_gpu
from test_oracle_budget import GENERAL, budget, checkerboard

pytestmark = pytest.mark.gpu

EPS_F = 2.0 ** -24


@pytest.fixture(scope="module")
def sv():
    return need_gpu()


@pytest.mark.parametrize("prec", ["FP64", "FP32", "FP32_PC", "FP32_PS"])
@pytest.mark.parametrize("n", [(16,), (4096,), (130, 64), (36, 30, 8)])
def test_budget_every_configuration(sv, n, prec):
    P = sv.Params(precision=getattr(sv, prec), **GENERAL)
    U0 = checkerboard(P.gamma, n)
    if prec != "FP64":
        U0 = U0.astype(np.float32).astype(np.float64)
    dim = len(n)
    ncell = int(np.prod(n))
    h = 1.0 / n[0]
    with sv.Solver(P, n, tuple(x * h for x in n)) as s:
        ncfg = len(s.configs())
        for c in range(ncfg):
            s.set_config(c)
            s.write_state(U0)
            c0 = s.conservation()
            dt = s.dt()
            s.step(1)
            c1 = s.conservation()
            assert s.status() == 0
            d = c1 - c0
            bE, bEv, _, _ = budget(P, U0, dt)
            mx = np.max(np.abs(U0), axis=1)
            if prec == "FP64":
                tol_cons = 1e-14 * np.abs(U0).sum(axis=1)
                tol = [1e-12 * abs(bE) + 1e-14 * np.abs(U0[dim + 1]).sum(),
                       1e-12 * abs(bEv) + 1e-14 * np.abs(U0[dim + 2]).sum()]
            else:
                tol_cons = 2 * ncell * EPS_F * mx
                tol = [2 * ncell * EPS_F * mx[dim + 1] + 1e-5 * abs(bE),
                       2 * ncell * EPS_F * mx[dim + 2] + 1e-5 * abs(bEv)]
            for f in range(dim + 1):
                assert abs(d[f]) <= tol_cons[f], (c, f, d[f], tol_cons[f])
            assert abs(d[dim + 1] - bE) <= tol[0], (c, d[dim + 1], bE, tol[0])
            assert abs(d[dim + 2] - bEv) <= tol[1], (c, d[dim + 2], bEv, tol[1])
