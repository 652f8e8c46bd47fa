"""Parity of the fused 2D / 3D unsplit CUDA steps (through the C ABI) with the
FP64 oracle.  Error measure and tolerances as for 1D: <= 1e-12 for the FP64
kernels, <= 2e-6 after one step for the FP32 kernels (max |gpu - oracle| over
max(|field|, 1), per field)."""
import math

import numpy as np
import pytest

from gpu_util import assert_fp64_parity, need_gpu, oracle_params, rel_linf
from oracle import orc as O
from paper_1805_03442_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sv():
    return need_gpu()


def _gpu_steps(sv, P, U0, n, L, nsteps):
    with sv.Solver(P, n, L) as s:
        s.write_state(U0)
        dts = []
        for _ in range(nsteps):
            dts.append(s.dt())
            s.step(1)
        U, t = s.read_state()
        assert s.status() == 0
    return U, t, dts


def _oracle_steps(Po, U0, n, h, dts):
    U = U0.copy()
    for dt in dts:
        U, rc = O.step(Po, U, n, h, dt)
        assert rc == 0
    return U


SHAPES_2D = [(7, 5), (37, 29), (300, 70), (513, 260)]
SHAPES_3D = [(5, 4, 6), (33, 17, 9), (65, 40, 20)]
PARAMS = [dict(tau0=0.3), dict(tau0=0.05, S=0.7, Q_rho=0.4, Q_T=-0.3, I_rho=0.2, I_T=0.5),
          dict(tau0=math.inf, S=0.0)]


@pytest.mark.parametrize("n", SHAPES_2D + SHAPES_3D)
@pytest.mark.parametrize("params", PARAMS)
def test_fp64_matches_oracle(sv, n, params):
    P = sv.Params(precision=sv.FP64, **params)
    Po = oracle_params(P)
    dim = len(n)
    h = 1.0 / n[0]
    L = tuple(x * h for x in n)
    U0 = inputs.random_states(dim, int(np.prod(n)), seed=sum(n), smooth=True)
    U, t, dts = _gpu_steps(sv, P, U0, n, L, 3)
    ref_dt = O.dt_cfl(Po, U0, n, h)
    assert dts[0] == pytest.approx(ref_dt, rel=1e-13)
    ref = _oracle_steps(Po, U0, n, h, dts)
    assert_fp64_parity(U, ref)


@pytest.mark.parametrize("limiter", [1, 2])
@pytest.mark.parametrize("n", [(37, 29), (33, 17, 9)])
def test_fp64_other_limiters(sv, n, limiter):
    P = sv.Params(precision=sv.FP64, tau0=0.2, limiter=limiter)
    Po = oracle_params(P)
    h = 1.0 / n[0]
    U0 = inputs.random_states(len(n), int(np.prod(n)), seed=4, smooth=True)
    U, _, dts = _gpu_steps(sv, P, U0, n, tuple(x * h for x in n), 2)
    assert_fp64_parity(U, _oracle_steps(Po, U0, n, h, dts))


@pytest.mark.parametrize("precision", ["FP32", "FP32_P64", "FP32_PC"])
@pytest.mark.parametrize("n", [(37, 29), (513, 260), (33, 17, 9), (65, 40, 20)])
def test_fp32_one_step(sv, precision, n):
    P = sv.Params(precision=getattr(sv, precision), tau0=0.3)
    Po = oracle_params(P)
    h = 1.0 / n[0]
    U0 = inputs.random_states(len(n), int(np.prod(n)), seed=7, smooth=True)
    U0 = U0.astype(np.float32).astype(np.float64)
    U, _, dts = _gpu_steps(sv, P, U0, n, tuple(x * h for x in n), 1)
    assert dts[0] == pytest.approx(O.dt_cfl(Po, U0, n, h), rel=1e-5)
    assert rel_linf(U, _oracle_steps(Po, U0, n, h, dts)) <= 2e-6


@pytest.mark.parametrize("prec", ["FP64", "FP32"])
@pytest.mark.parametrize("n", [(64, 48), (24, 20, 16)])
def test_conservation_and_stationarity(sv, prec, n):
    dim = len(n)
    P = sv.Params(precision=getattr(sv, prec), tau0=0.1)
    h = 1.0 / n[0]
    L = tuple(x * h for x in n)
    U0 = inputs.random_states(dim, int(np.prod(n)), seed=1, smooth=True)
    with sv.Solver(P, n, L) as s:
        s.write_state(U0)
        c0 = s.conservation()
        s.step(12)          # these random states go non-physical near step 35 (oracle too)
        c1 = s.conservation()
        assert s.status() == 0
    tol = 1e-13 if prec == "FP64" else 1e-6
    for f in range(dim + 1):
        assert abs(c1[f] - c0[f]) <= tol * np.sum(np.abs(U0[f]))
    with sv.Solver(P, n, L) as s:             # uniform equilibrium stays put
        E0, _ = s.read_state()
        s.step(20)
        E1, _ = s.read_state()
    assert np.array_equal(E1[: dim + 1], E0[: dim + 1])
    assert rel_linf(E1, E0) <= (1e-14 if prec == "FP64" else 2e-6)


def test_2d_full_size_sampled(sv):
    """8192 x 8192 FP32 (the 2D benchmark workload and launch configuration):
    one step checked on sampled cells against the oracle cell by cell."""
    nx = ny = 8192
    P = sv.Params(precision=sv.FP32, tau0=0.1)
    Po = oracle_params(P)
    h = 1.0 / nx
    U0 = inputs.plane_wave_2d(P.gamma, nx, ny, 1.0, inputs.equilibrium_primitive(P.Ck, P.S),
                              7, 4, 1e-3, 1e-5, seed=3)
    U0 = U0.astype(np.float32).astype(np.float64)
    with sv.Solver(P, (nx, ny), (1.0, 1.0)) as s:
        s.write_state(U0)
        dt = s.dt()
        s.step(1)
        U, _ = s.read_state()
    rng = np.random.default_rng(8)
    edge = [0, 1, nx - 1, nx, nx * ny - 1, 253, 254, 255, 256, 257, nx * 255 + 17, nx * 256 + 17]
    idx = np.unique(np.concatenate([edge, rng.integers(0, nx * ny, 100)]))
    scale = np.maximum(np.max(np.abs(U0), axis=1), 1.0)
    errs = [np.max(np.abs(U[:, i] - O.step_cell(Po, U0, (nx, ny), h, dt, int(i))) / scale) for i in idx]
    assert max(errs) <= 2e-6, (idx[int(np.argmax(errs))], max(errs))


def test_3d_full_size_sampled(sv):
    """512^3 FP32 (the 3D benchmark workload and launch configuration): one step
    checked on sampled cells against the oracle cell by cell."""
    n = 512
    P = sv.Params(precision=sv.FP32, tau0=0.08, cfl=0.3)
    Po = oracle_params(P)
    h = 1.0 / n
    U0 = inputs.random_field_3d(P.gamma, n, 1.0, inputs.equilibrium_primitive(P.Ck, P.S), 1e-3,
                                seed=5)
    U0 = U0.astype(np.float32).astype(np.float64)
    with sv.Solver(P, (n, n, n), (1.0, 1.0, 1.0)) as s:
        s.write_state(U0)
        dt = s.dt()
        s.step(1)
        U, _ = s.read_state()
    rng = np.random.default_rng(9)
    edge = [0, n - 1, n * n - 1, n ** 3 - 1, 29, 30, 31, 32, n * 13 + 5, n * 14 + 5, n * n * 128 + 7]
    idx = np.unique(np.concatenate([edge, rng.integers(0, n ** 3, 60)]))
    scale = np.maximum(np.max(np.abs(U0), axis=1), 1.0)
    errs = [np.max(np.abs(U[:, i] - O.step_cell(Po, U0, (n, n, n), h, dt, int(i))) / scale)
            for i in idx]
    assert max(errs) <= 2e-6, (idx[int(np.argmax(errs))], max(errs))
