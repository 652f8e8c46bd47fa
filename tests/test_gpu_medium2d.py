"""2D boundaries, the active-medium map and driven cells on the GPU (through
the C ABI) against the FP64 oracle (orc_step2m / orc_run2m): the paper's
two-dimensional active-sector problem, Sec. 3.  Error measure as for the other
parity tests (max |gpu - oracle| over max(|field|, 1), per field): <= 1e-12
for FP64, <= 2e-6 after one step for FP32."""
import math

import numpy as np
import pytest

from gpu_util import assert_fp64_parity, need_gpu, oracle_params, rel_linf
from oracle import orc as O
from paper_1805_03442_gb300 import inputs

pytestmark = pytest.mark.gpu

PER, WALL, OUT = 0, 1, 2
BCS = [(WALL, WALL, WALL, WALL), (OUT, WALL, OUT, OUT), (PER, WALL, OUT, PER), (WALL, OUT, PER, PER)]
SHAPES = [(7, 5), (130, 77), (300, 40), (513, 260)]


@pytest.fixture(scope="module")
def sv():
    return need_gpu()


def gpu_steps(sv, P, U0, n, h, bc, nsteps, medium=None):
    with sv.Solver(P, n, tuple(x * h for x in n), bc=bc) as s:
        if medium is not None:
            s.set_medium2d(*medium)
        s.write_state(U0)
        dts = []
        for _ in range(nsteps):
            dts.append(s.dt())
            s.step(1)
        U, t = s.read_state()
        assert s.status() == 0
    return U, t, dts


def oracle_steps(Po, U0, n, h, bc, dts, M=None):
    U, t = U0.copy(), 0.0
    for dt in dts:
        U, rc = O.step2m(Po, U, n[0], n[1], h, dt, bc, M, t)
        assert rc == 0
        t += dt
    return U


@pytest.mark.parametrize("bc", BCS)
@pytest.mark.parametrize("n", SHAPES)
def test_fp64_boundaries_match_oracle(sv, bc, n):
    P = sv.Params(precision=sv.FP64, tau0=0.3)
    Po = oracle_params(P)
    h = 1.0 / n[0]
    U0 = inputs.random_states(2, n[0] * n[1], seed=sum(n) + sum(bc), smooth=True)
    U, t, dts = gpu_steps(sv, P, U0, n, h, bc, 3)
    assert dts[0] == pytest.approx(O.dt_cfl(Po, U0, n, h), rel=1e-13)
    ref = oracle_steps(Po, U0, n, h, bc, dts)
    assert_fp64_parity(U, ref)


@pytest.mark.parametrize("bc", BCS[:2])
def test_fp32_boundaries_one_step(sv, bc):
    n = (300, 70)
    P = sv.Params(precision=sv.FP32, tau0=0.3)
    Po = oracle_params(P)
    h = 1.0 / n[0]
    U0 = inputs.random_states(2, n[0] * n[1], seed=3, smooth=True).astype(np.float32).astype(np.float64)
    U, t, dts = gpu_steps(sv, P, U0, n, h, bc, 1)
    ref = oracle_steps(Po, U0, n, h, bc, dts)
    assert rel_linf(U, ref) <= 2e-6


def sector(sv, nx, prec, S=1.0, tau0=0.0135):
    pb = inputs.sector_problem(nx)
    P = sv.Params(precision=prec, S=S, tau0=tau0)
    lo, hi, dlo, dhi = pb.maps
    U0 = inputs.sector_rest_state(1.4, P.Ck, P.S, pb.nx, pb.ny)
    return pb, P, U0, (lo, hi, dlo, dhi, pb.omega, pb.amp), O.Medium2(lo, hi, dlo, dhi, pb.omega, pb.amp)


@pytest.mark.parametrize("nx", [96, 200])
def test_fp64_sector_problem_matches_oracle(sv, nx):
    pb, P, U0, med, M = sector(sv, nx, sv.FP64)
    Po = oracle_params(P)
    n = (pb.nx, pb.ny)
    with sv.Solver(P, n, (pb.nx * pb.h, pb.ny * pb.h), bc=pb.bc) as s:
        s.set_medium2d(*med)
        s.write_state(U0)
        rc, k = s.run_to(0.1)
        U, t = s.read_state()
    ref, tr, kr, rcr = O.run2m(Po, U0, pb.nx, pb.ny, pb.h, 0.1, pb.bc, M)
    assert rc == 0 and rcr == 0 and k == kr and t == tr == 0.1
    assert_fp64_parity(U, ref)
    # the source has been pulsing: the state is no longer at rest
    assert np.max(np.abs(U[0] - 1.0)) > 1e-4


def test_fp32_sector_problem_close_to_oracle(sv):
    """FP32 over 60 steps of the sector problem: the waves the source launched
    agree with the FP64 oracle to within float rounding of O(1) fields."""
    pb, P, U0, med, M = sector(sv, 160, sv.FP32)
    Po = oracle_params(P)
    n = (pb.nx, pb.ny)
    with sv.Solver(P, n, (pb.nx * pb.h, pb.ny * pb.h), bc=pb.bc) as s:
        s.set_medium2d(*med)
        s.write_state(U0)
        s.step(60)
        U, t = s.read_state()
        k = s.time()[1]
        assert s.status() == 0 and k == 60
    ref, tr, kr, rcr = O.run2m(Po, U0, pb.nx, pb.ny, pb.h, t, pb.bc, M)
    assert rcr == 0 and abs(kr - k) <= 1
    amp = np.max(np.abs(ref[0] - 1.0))
    assert amp > 1e-4
    assert np.max(np.abs(U[0] - ref[0])) <= 2e-3 * amp + 1e-6


@pytest.mark.parametrize("prec", ["FP32", "FP64"])
def test_subnormal_speeds_do_not_stop_the_run(sv, prec):
    """Gas at rest with velocities whose squares are subnormal in float (the
    far tail of a wave spreading into still gas): the eq. 16 bound is that of
    the gas at rest, and stepping goes on."""
    n = (64, 48)
    P = sv.Params(precision=getattr(sv, prec))
    rest = inputs.sector_rest_state(1.4, P.Ck, P.S, *n)
    tiny = rest.copy()
    tiny[1, ::7] = 3e-22                  # (3e-22)^2 = 9e-44 < FLT_MIN
    tiny[2, ::5] = -2e-21
    dts = []
    for U in (rest, tiny):
        with sv.Solver(P, n, None, bc=(OUT, WALL, OUT, OUT)) as s:
            s.write_state(U)
            dts.append(s.dt())
            s.step(30)
            assert s.status() == 0 and s.time()[1] == 30
    assert dts[1] == dts[0]


def test_medium_map_everywhere_and_nowhere(sv):
    n = (130, 77)
    h = 1.0 / n[0]
    P = sv.Params(precision=sv.FP64, S=1.0, tau0=0.2)
    U0 = inputs.random_states(2, n[0] * n[1], seed=12, smooth=True)
    bc = (OUT, WALL, OUT, OUT)
    plain, _, _ = gpu_steps(sv, P, U0, n, h, bc, 2)
    every, _, _ = gpu_steps(sv, P, U0, n, h, bc, 2,
                            (np.zeros(n[1]), np.full(n[1], n[0])))
    none, _, _ = gpu_steps(sv, P, U0, n, h, bc, 2, (np.zeros(n[1]), np.zeros(n[1])))
    frozen, _, _ = gpu_steps(sv, sv.Params(precision=sv.FP64, S=1.0, tau0=math.inf), U0, n, h, bc, 2)
    assert np.array_equal(plain, every)
    assert np.array_equal(none, frozen)


def test_walls_conserve_mass_and_energy(sv):
    n = (257, 130)
    h = 1.0 / n[0]
    P = sv.Params(precision=sv.FP64, tau0=0.3)
    U0 = inputs.random_states(2, n[0] * n[1], seed=21, smooth=True)
    with sv.Solver(P, n, tuple(x * h for x in n), bc=(WALL, WALL, WALL, WALL)) as s:
        s.write_state(U0)
        s0 = s.conservation()
        s.step(40)
        s1 = s.conservation()
        assert s.status() == 0
    assert abs(s1[0] - s0[0]) <= 1e-13 * s0[0]
    assert abs(s1[3] - s0[3]) <= 1e-13 * abs(s0[3])


def test_configs_bitwise_with_boundaries_and_medium(sv):
    pb, P, U0, med, M = sector(sv, 200, sv.FP32)
    n = (pb.nx, pb.ny)
    L = (pb.nx * pb.h, pb.ny * pb.h)
    out = []
    with sv.Solver(P, n, L, bc=pb.bc) as s:
        ncfg = len(s.configs())
    for c in range(ncfg):
        with sv.Solver(P, n, L, bc=pb.bc) as s:
            s.set_config(c)
            s.set_medium2d(*med)
            s.write_state(U0)
            s.step(25)
            out.append(s.read_state()[0])
    for o in out[1:]:
        assert np.array_equal(o, out[0])


def test_bad_medium_and_boundaries(sv):
    P = sv.Params(precision=sv.FP32)
    with sv.Solver(P, (40, 30), None, bc=(WALL, OUT, OUT, OUT)) as s:
        with pytest.raises(sv.SvError):
            s.set_medium2d(np.zeros(30), np.full(30, 41))          # beyond nx
        with pytest.raises(sv.SvError):
            s.set_medium2d(np.full(30, 5), np.full(30, 4))         # lo > hi
        with pytest.raises(sv.SvError):
            s.set_medium2d(np.zeros(30), None)                     # half a pair
    with sv.Solver(P, (64,), None) as s:
        with pytest.raises(sv.SvError):
            s.set_medium2d(np.zeros(1), np.ones(1))
    for bad in [dict(n=(40, 30, 20), bc=(WALL, 0, 0, 0)), dict(n=(1, 30), bc=(WALL, WALL, 0, 0)),
                dict(n=(40, 30), bc=(3, OUT, 0, 0))]:
        with pytest.raises(sv.SvError):
            sv.Solver(P, bad["n"], None, bc=bad["bc"])
