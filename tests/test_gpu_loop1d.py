"""The persistent 1D step loop (one cooperative launch for many steps) against
per-step launches and against the oracle, through the C ABI.

Both launch modes run the same per-cell arithmetic, and the dt reduction is a
maximum (exact in any order), so the two must agree bit for bit: states,
times and step counts."""
import numpy as np
import pytest

from gpu_util import assert_fp64_parity, need_gpu, oracle_params, rel_linf
from oracle import orc as O
from paper_1805_03442_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sv():
    return need_gpu()


def wave_state(N, amp=1e-3, seed=0):
    modes = inputs.random_phase_modes(seed, inputs.acoustic_shape(1.4), 6, 1, amp)
    return inputs.waves_1d(1.4, N, 1.0, inputs.equilibrium_primitive(0.1, 1.0), modes)


def run_modes(sv, P, N, U0, nsteps=None, t_end=None, bc=(0, 0), drive=None):
    out = {}
    for mode in (sv.LAUNCH_PER_STEP, sv.LAUNCH_PERSISTENT):
        with sv.Solver(P, (N,), (1.0,), bc=bc) as s:
            s.set_launch(mode)
            assert s.launch == mode
            if drive is not None:
                s.set_drive(*drive)
            s.write_state(U0)
            if t_end is None:
                s.step(nsteps)
                rc = 0
            else:
                rc, _ = s.run_to(t_end, check=False)
            U, t = s.read_state()
            out[mode] = (U, t, s.time()[1], s.status(), rc)
    return out[sv.LAUNCH_PER_STEP], out[sv.LAUNCH_PERSISTENT]


def assert_same(a, b):
    assert np.array_equal(a[0], b[0], equal_nan=True)
    assert a[1:] == b[1:]


@pytest.mark.parametrize("prec", ["FP32", "FP64", "FP32_P64", "FP32_PC", "FP32_PS"])
@pytest.mark.parametrize("N", [1, 63, 200, 1601, 4099, 100000])
def test_bitwise_equal_to_per_step(sv, prec, N):
    P = sv.Params(precision=getattr(sv, prec))
    U0 = wave_state(N, seed=N)
    a, b = run_modes(sv, P, N, U0, nsteps=57)
    assert_same(a, b)


@pytest.mark.parametrize("limiter", ["MINMOD", "VANLEER", "MC"])
@pytest.mark.parametrize("src", ["frozen", "qi_zero", "general"])
def test_bitwise_limiters_sources(sv, limiter, src):
    over = {"frozen": dict(tau0=float("inf")), "qi_zero": dict(),
            "general": dict(Q_rho=0.5, Q_T=-0.7, I_rho=1.0, I_T=0.6)}[src]
    P = sv.Params(precision=sv.FP32, limiter=getattr(sv, limiter), **over)
    N = 3000
    U0 = wave_state(N, amp=1e-2, seed=3)
    a, b = run_modes(sv, P, N, U0, nsteps=40)
    assert_same(a, b)


@pytest.mark.parametrize("bc", [(1, 1), (2, 2), (1, 2), (0, 1)])
def test_bitwise_walls_outflow(sv, bc):
    N = 1000
    P = sv.Params(precision=sv.FP64, tau0=0.3)
    U0 = inputs.random_states(1, N, seed=11, smooth=True)
    a, b = run_modes(sv, P, N, U0, nsteps=25, bc=bc)
    assert_same(a, b)


def test_bitwise_driven(sv):
    N = 2000
    P = sv.Params(precision=sv.FP32)
    U0 = wave_state(N, amp=0.0)
    ev0 = P.Ck + P.S
    base = [1.0, 0.0, 1.0 / 0.4 + ev0, ev0]
    amp = [1e-3, 1e-3, 1e-3 / 0.4 * 1.4, 1e-4]
    a, b = run_modes(sv, P, N, U0, nsteps=300, bc=(3, 2), drive=(20.0, 17.0 - 0.3j, base, amp))
    assert_same(a, b)


def test_run_to_lands_on_t_end(sv):
    N = 1600
    P = sv.Params(precision=sv.FP32)
    U0 = wave_state(N, amp=1e-2, seed=5)
    a, b = run_modes(sv, P, N, U0, t_end=0.37)
    assert_same(a, b)
    assert b[1] == 0.37 and b[4] == 0


def test_more_steps_than_one_launch(sv):
    """70000 steps span two persistent launches (65536 steps each at most).
    Frozen medium: the waves neither grow nor steepen into failure."""
    N = 200
    P = sv.Params(precision=sv.FP32, tau0=float("inf"))
    U0 = wave_state(N, amp=1e-3, seed=9)
    a, b = run_modes(sv, P, N, U0, nsteps=70000)
    assert_same(a, b)
    assert b[2] == 70000 and b[3] == 0


def test_matches_oracle(sv):
    N = 1000
    P = sv.Params(precision=sv.FP64, limiter=sv.VANLEER)
    U0 = wave_state(N, amp=1e-2, seed=1)
    with sv.Solver(P, (N,), (1.0,)) as s:
        assert s.launch == sv.LAUNCH_PERSISTENT
        s.write_state(U0)
        rc, k = s.run_to(0.25)
        U, t = s.read_state()
    ref, t_ref, k_ref, rc_ref = O.run(oracle_params(P), U0, (N,), 1.0 / N, 0.25)
    assert rc == 0 and rc_ref == 0
    assert k == k_ref and t == t_ref == 0.25
    assert_fp64_parity(U, ref)


def test_nonphysical_stops_the_loop(sv):
    """Two streams flying apart open a near-vacuum that goes non-physical after
    a few dozen steps (the oracle fails there too): every block of the loop
    stops at the same step, and the result is the per-step launches' one."""
    N = 500
    x = inputs.cell_centres(N, 1.0)
    v = np.where(x < 0.5, -3.0, 3.0)
    U0 = inputs.prim_to_cons(1.4, np.ones(N), [v], np.full(N, 1e-2), np.full(N, 0.5))
    P = sv.Params(precision=sv.FP64, tau0=0.2)
    _, _, k_ref, rc_ref = O.run(oracle_params(P), U0, (N,), 1.0 / N, 0.05, max_steps=5000)
    assert rc_ref == -1 and k_ref > 5
    a, b = run_modes(sv, P, N, U0, t_end=0.05)
    assert_same(a, b)
    assert b[4] in (sv.SV_ENONPHYS, sv.SV_EDT) and b[3] != 0


def test_auto_mode(sv):
    P = sv.Params(precision=sv.FP32)
    with sv.Solver(P, (1000,), (1.0,)) as s:
        assert s.launch == sv.LAUNCH_PERSISTENT
    with sv.Solver(P, (8000,), (1.0,)) as s:
        assert s.launch == sv.LAUNCH_PER_STEP
    with sv.Solver(P, (20000,), (1.0,)) as s:
        assert s.launch == sv.LAUNCH_PER_STEP
    with sv.Solver(P, (1 << 22,), (1.0,)) as s:
        assert s.launch == sv.LAUNCH_PER_STEP
        s.set_launch(sv.LAUNCH_PERSISTENT)
        assert s.launch == sv.LAUNCH_PERSISTENT
    with sv.Solver(sv.Params(precision=sv.FP32, method=sv.HEUN), (1000,), (1.0,)) as s:
        assert s.launch == sv.LAUNCH_PER_STEP
        with pytest.raises(sv.SvError):
            s.set_launch(sv.LAUNCH_PERSISTENT)
    with sv.Solver(P, (64, 64), (1.0, 1.0)) as s:
        assert s.launch == sv.LAUNCH_PER_STEP
        with pytest.raises(sv.SvError):
            s.set_launch(sv.LAUNCH_PERSISTENT)


def test_persistent_full_grid_matches(sv):
    """Forced persistent mode on a grid larger than one chunk per warp (every
    warp then owns several chunks): still bitwise the per-step result."""
    N = 1 << 21
    P = sv.Params(precision=sv.FP32)
    U0 = wave_state(N, seed=4)
    a, b = run_modes(sv, P, N, U0, nsteps=12)
    assert_same(a, b)


@pytest.mark.parametrize("prec", ["FP32", "FP64"])
def test_barrier_wait_limit_ends_with_estall(sv, prec):
    """The failure path of the persistent loop's bounded grid-barrier wait:
    with the wait limited to one poll, the blocks that arrive before the last
    one give up, raise the stall flag and leave the launch, which ends with
    SV_ESTALL instead of hanging.  Nothing faults and nothing spins: the wait
    simply runs out.  After a new upload (and the default limit) the solver
    steps exactly as a fresh per-step solver does."""
    N = 4000                                     # 63 chunks: 63 co-resident blocks
    P = sv.Params(precision=getattr(sv, prec))
    U0 = wave_state(N, seed=5)
    with sv.Solver(P, (N,), (1.0,)) as s:
        s.set_launch(sv.LAUNCH_PERSISTENT)
        s.write_state(U0)
        s.set_wait_limit(1)
        rc, _ = s.run_to(0.05, check=False)
        assert rc == sv.SV_ESTALL
        assert s.status() & sv.FLAG_STALL
        s.set_wait_limit(0)
        s.write_state(U0)
        assert s.status() == 0
        rc, k = s.run_to(0.05, check=False)
        assert rc == 0 and s.status() == 0
        U, t = s.read_state()
    with sv.Solver(P, (N,), (1.0,)) as r:
        r.set_launch(sv.LAUNCH_PER_STEP)
        r.write_state(U0)
        rc2, k2 = r.run_to(0.05, check=False)
        U2, t2 = r.read_state()
    assert rc2 == 0 and k == k2 and t == t2
    assert np.array_equal(U, U2)
    with pytest.raises(Exception):
        s2 = sv.Solver(P, (N,), (1.0,))
        try:
            s2.set_wait_limit(-1)
        finally:
            s2.close()
