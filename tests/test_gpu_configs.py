"""Launch configurations and the autotuner on the GPU, through the C ABI.

Every configuration of a solver runs the same per-cell arithmetic (only the
work decomposition changes), and the dt reduction is a maximum, so all of them
must give bitwise the same states, times and step counts.  The autotuner must
leave the state exactly as it found it."""
import numpy as np
import pytest

from gpu_util import need_gpu
from paper_1805_03442_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sv():
    return need_gpu()


def wave_1d(N, amp=1e-2, seed=0):
    modes = inputs.random_phase_modes(seed, inputs.acoustic_shape(1.4), 6, 1, amp)
    return inputs.waves_1d(1.4, N, 1.0, inputs.equilibrium_primitive(0.1, 1.0), modes)


def run_each_config(sv, P, n, U0, steps, bc=(0, 0)):
    out = []
    with sv.Solver(P, n, None, bc=bc) as s:
        descs = s.configs()
    for i in range(len(descs)):
        with sv.Solver(P, n, None, bc=bc) as s:
            s.set_config(i)
            assert s.config == i
            s.write_state(U0)
            s.step(steps)
            U, t = s.read_state()
            out.append((U, t, s.time()[1], s.status()))
    return descs, out


def assert_all_equal(out):
    for o in out[1:]:
        assert np.array_equal(o[0], out[0][0], equal_nan=True)
        assert o[1:] == out[0][1:]


@pytest.mark.parametrize("prec", ["FP32", "FP32_PC", "FP32_PS"])
@pytest.mark.parametrize("N", [4096, 5001, 65536 + 3])
def test_1d_float_configs_bitwise(sv, N, prec):
    P = sv.Params(precision=getattr(sv, prec))
    descs, out = run_each_config(sv, P, (N,), wave_1d(N, seed=N), 30)
    assert len(descs) == 5 and "block tiles" in descs[0] and "4 cells per thread" in descs[2]
    assert "4 blocks/SM" in descs[3] and "sliding" in descs[4]
    assert_all_equal(out)


@pytest.mark.parametrize("bc", [(1, 1), (2, 1)])
def test_1d_float_configs_walls(sv, bc):
    N = 6000
    P = sv.Params(precision=sv.FP32, tau0=0.3)
    U0 = inputs.random_states(1, N, seed=7, smooth=True)
    _, out = run_each_config(sv, P, (N,), U0, 20, bc=bc)
    assert_all_equal(out)


def test_1d_other_solvers_have_one_config(sv):
    for P, N in [(sv.Params(precision=sv.FP64), 8192), (sv.Params(precision=sv.FP32), 1000),
                 (sv.Params(precision=sv.FP32, method=sv.HEUN), 8192)]:
        with sv.Solver(P, (N,)) as s:
            assert len(s.configs()) == 1
            with pytest.raises(sv.SvError):
                s.set_config(1)


@pytest.mark.parametrize("prec", ["FP32", "FP64", "FP32_PS"])
def test_2d_configs_bitwise(sv, prec):
    nx, ny = 130, 300                 # several x tiles and a ragged x tile; 300 planes
    P = sv.Params(precision=getattr(sv, prec))
    U0 = inputs.random_states(2, nx * ny, seed=3, smooth=True)
    descs, out = run_each_config(sv, P, (nx, ny), U0, 6)
    assert len(descs) == 4 and all("planes per block" in d for d in descs)
    assert_all_equal(out)


def test_3d_configs_bitwise(sv):
    n = (40, 20, 150)
    P = sv.Params(precision=sv.FP32)
    U0 = inputs.random_states(3, n[0] * n[1] * n[2], seed=4, smooth=True)
    _, out = run_each_config(sv, P, n, U0, 5)
    assert_all_equal(out)


@pytest.mark.parametrize("n", [(1 << 18,), (256, 256)])
def test_autotune_restores_state(sv, n):
    P = sv.Params(precision=sv.FP32)
    cells = int(np.prod(n))
    U0 = wave_1d(cells, seed=2).reshape(4, -1) if len(n) == 1 else \
        inputs.random_states(2, cells, seed=2, smooth=True)
    with sv.Solver(P, n, None) as s:
        s.write_state(U0, t=0.125)
        s.step(3)
        before, tb = s.read_state()
        kb = s.time()[1]
        best, us = s.autotune(steps=5)
        after, ta = s.read_state()
        assert np.array_equal(before, after) and ta == tb and s.time()[1] == kb
        assert s.status() == 0
        assert 0 <= best < len(s.configs()) and s.config == best
        assert len(us) == len(s.configs()) and all(np.isfinite(us))
        assert us[best] == min(us)
        # stepping on after tuning matches an untuned solver
        s.step(4)
        U1, t1 = s.read_state()
    with sv.Solver(P, n, None) as r:
        r.write_state(U0, t=0.125)
        r.step(7)
        U2, t2 = r.read_state()
    assert np.array_equal(U1, U2) and t1 == t2


def test_cold_autotune_restores_state(sv):
    """Trials with an L2-evicting write before every timed step leave the
    state, time and step count exactly as they were, and time every
    configuration."""
    N = 1 << 20
    P = sv.Params(precision=sv.FP32)
    with sv.Solver(P, (N,), None) as s:
        s.write_state(wave_1d(N, seed=5), t=0.25)
        s.step(2)
        before, tb = s.read_state()
        kb = s.time()[1]
        best, us = s.autotune(steps=3, cold=True)
        after, ta = s.read_state()
        assert np.array_equal(before, after) and ta == tb and s.time()[1] == kb
        assert s.status() == 0 and s.config == best
        assert len(us) == len(s.configs()) and all(np.isfinite(us)) and us[best] == min(us)


def test_autotune_stopped_trials(sv):
    """A solver whose next dt is 0 (run ended) times nothing: every entry is
    +inf and the configuration stays."""
    N = 8192
    P = sv.Params(precision=sv.FP32)
    with sv.Solver(P, (N,)) as s:
        s.write_state(wave_1d(N), t=0.0)
        bad = wave_1d(N)
        bad[0, 5] = -1.0                  # non-physical: the first dt collapses
        s.write_state(bad)
        best, us = s.autotune(steps=3)
        assert best == 0 and all(np.isinf(us))


def test_batch_configs_bitwise(sv):
    from test_gpu_batch import _mini_sweep
    runs, states = _mini_sweep(13, 16)
    P = sv.Params(precision=sv.FP32)
    res = []
    with sv.Batch(P, runs, states) as b:
        descs = b.configs()
        assert len(descs) == 2 and b.config == 0
        for i in range(len(descs)):
            b.set_config(i)
            b.reset_initial()
            b.run()
            b.sync()
            res.append([b.read(j) for j in range(len(runs))])
    for a, c in zip(res[0], res[1]):
        assert np.array_equal(a[0], c[0], equal_nan=True)
        assert a[1:] == c[1:]


def test_tune_solver_cache(sv, tmp_path):
    from paper_1805_03442_gb300 import tune
    cache = tune.Cache(str(tmp_path / "cache.json"))
    P = sv.Params(precision=sv.FP32)
    N = 1 << 16
    dev = tune.device_name()
    key = tune.solver_key(P, (N,))
    with sv.Solver(P, (N,)) as s:
        s.write_state(wave_1d(N))
        r = tune.tune_solver(s, key, dev, cache, steps=3)
        assert not r["cached"] and s.configs()[s.config] == r["config"]
    with sv.Solver(P, (N,)) as s:
        r2 = tune.tune_solver(s, key, dev, tune.Cache(cache.path))
        assert r2["cached"] and r2["config"] == r["config"]
