"""The batched sweep kernel (sv_batch_*): each run must be identical, bit for
bit, to the same run advanced alone by a 1D solver (same precision, same
per-cell arithmetic), FP64 runs must match the oracle, and the logged mode
amplitude must grow at the rate of eq. 8."""
import math
from dataclasses import dataclass, replace

import numpy as np
import pytest

from gpu_util import assert_fp64_parity, need_gpu, oracle_params, rel_linf
from oracle import dispersion as D
from oracle import orc as O
from paper_1805_03442_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sv():
    return need_gpu()


@dataclass
class Run:
    n: int
    t_end: float
    S: float
    tau0: float
    tau_rho: float = -1.0
    tau_T: float = -1.5
    Q_rho: float = 0.0
    Q_T: float = 0.0
    I_rho: float = 0.0
    I_T: float = 0.0
    m: int = 1
    L: float = 1.0


def _mini_sweep(seed: int, nruns: int):
    rng = np.random.default_rng(seed)
    runs, states = [], []
    for i in range(nruns):
        r = inputs.sweep_runs(seed * 1000 + i, 1, n_lo=33, n_hi=700)[0]
        run = Run(n=r.N, t_end=0.25 * r.t_end, S=r.S, tau0=max(r.tau0, 2e-3), tau_rho=r.tau_rho,
                  tau_T=r.tau_T, Q_rho=r.Q_rho, Q_T=r.Q_T, I_rho=r.I_rho, I_T=r.I_T, m=r.m)
        if i % 7 == 3:                       # zero exponents (the qi_zero kernel when alone)
            run = replace(run, Q_rho=0.0, Q_T=0.0, I_rho=0.0, I_T=0.0)
        if i % 11 == 5:                      # frozen limit (no source when alone)
            run = replace(run, tau0=math.inf, S=0.0)
        base = inputs.equilibrium_primitive(0.1, run.S)
        shape = inputs.acoustic_shape(1.4)
        U = inputs.waves_1d(1.4, run.n, run.L, base,
                            [inputs.Mode(m=run.m, shape=shape, scale=1e-3 * float(rng.uniform(0.5, 2)))])
        runs.append(run)
        states.append(U)
    return runs, states


def _single(sv, prec, run, U0):
    P = sv.Params(precision=prec, S=run.S, tau0=run.tau0, tau_rho=run.tau_rho, tau_T=run.tau_T,
                  Q_rho=run.Q_rho, Q_T=run.Q_T, I_rho=run.I_rho, I_T=run.I_T)
    with sv.Solver(P, (run.n,), (run.L,)) as s:
        s.write_state(U0)
        rc, k = s.run_to(run.t_end, check=False)
        U, t = s.read_state()
        flags = s.status()
    return U, t, k, flags


@pytest.mark.parametrize("prec", ["FP32", "FP64", "FP32_PC", "FP32_PS"])
def test_batch_equals_looped_single_runs(sv, prec):
    runs, states = _mini_sweep(3, 40)
    P = sv.Params(precision=getattr(sv, prec))
    with sv.Batch(P, runs, states, log_cap=16) as b:
        b.run()
        b.sync()
        ok = 0
        for i, (run, U0) in enumerate(zip(runs, states)):
            Ub, tb, kb, fb = b.read(i)
            Us, ts, ks, fs = _single(sv, P.precision, run, U0)
            # runs that blow up (strongly unstable draws) must fail identically too
            assert fb == fs, (i, fb, fs)
            assert tb == ts and kb == ks, (i, tb, ts, kb, ks)
            assert np.array_equal(Ub, Us, equal_nan=True), (i, np.nanmax(np.abs(Ub - Us)))
            ok += fb == 0 and tb == run.t_end
        assert ok >= len(runs) // 2


def test_batch_rerun_after_reset_is_identical(sv):
    runs, states = _mini_sweep(5, 12)
    P = sv.Params(precision=sv.FP32)
    with sv.Batch(P, runs, states, log_cap=8) as b:
        b.run()
        first = [b.read(i) for i in range(len(runs))]
        b.reset(states)
        b.run()
        for i in range(len(runs)):
            U, t, k, f = b.read(i)
            assert np.array_equal(U, first[i][0], equal_nan=True)
            assert t == first[i][1] and k == first[i][2]


def test_batch_fp64_matches_oracle(sv):
    runs, states = _mini_sweep(7, 6)
    # moderate parameters: the comparison is pointwise
    runs = [replace(r, tau0=max(r.tau0, 0.05) if math.isfinite(r.tau0) else r.tau0,
                    S=min(r.S, 1.0)) for r in runs]
    states = [inputs.waves_1d(1.4, r.n, r.L, inputs.equilibrium_primitive(0.1, r.S),
                              [inputs.Mode(m=r.m, shape=inputs.acoustic_shape(1.4), scale=1e-3)])
              for r in runs]
    P = sv.Params(precision=sv.FP64)
    with sv.Batch(P, runs, states) as b:
        b.run()
        for i, (run, U0) in enumerate(zip(runs, states)):
            U, t, k, f = b.read(i)
            Po = oracle_params(P, S=run.S, tau0=run.tau0, tau_rho=run.tau_rho, tau_T=run.tau_T,
                               Q_rho=run.Q_rho, Q_T=run.Q_T, I_rho=run.I_rho, I_T=run.I_T,
                               limiter=P.limiter)
            ref, tr, kr, rc = O.run(Po, U0, run.n, run.L / run.n, run.t_end)
            assert rc == 0 and f == 0
            assert k == kr and t == tr
            # minmod amplifies rounding noise in active media; these runs are short
            assert rel_linf(U, ref) <= 1e-10, (i, rel_linf(U, ref))


@pytest.mark.parametrize("m", [1, 2, 3])
def test_logged_mode_grows_at_eq8_rate(sv, m):
    """Eigenmode of mode m on L = 1 (N = 512 m: 512 cells per wavelength),
    tau0 0.1, S 1, amplitude 1e-4: the batch's logged a_m(t) grows at Im omega
    within 2% and turns at Re omega within 1%.  (A float state cannot follow
    much smaller amplitudes: each step changes rho by ~dt k |rho'|, which must
    stay above float's unit roundoff at rho ~ 1.)"""
    N = 512 * m
    Po = O.Params(tau0=0.1, limiter=O.VANLEER)
    k = 2 * math.pi * m
    w = D.growing_acoustic_root(Po, k)
    t_end = math.log(30.0) / w.imag
    md = D.eigenmode(Po, k, w)
    U0 = inputs.waves_1d(1.4, N, 1.0, inputs.equilibrium_primitive(Po.Ck, Po.S),
                         [inputs.Mode(m=m, shape=md["prim"], scale=1e-4)])
    run = Run(n=N, t_end=t_end, S=1.0, tau0=0.1, m=m)
    P = sv.Params(precision=sv.FP32, limiter=sv.VANLEER)
    with sv.Batch(P, [run, replace(run, m=0)], [U0, U0], log_cap=40) as b:
        b.run()
        t, a = b.mode_log(0)
        assert len(b.mode_log(1)[0]) == 0
    assert len(t) >= 30 and t[0] == 0.0 and t[-1] == pytest.approx(t_end)
    growth = np.polyfit(t, np.log(np.abs(a)), 1)[0]
    # u = U[1]/U[0] ~ exp(i k x - i w t): a_m ~ exp(-i w t)
    freq = -np.polyfit(t, np.unwrap(np.angle(a)), 1)[0]
    assert abs(growth - w.imag) <= 0.02 * w.imag
    assert abs(freq - w.real) <= 0.01 * abs(w.real)


@pytest.mark.parametrize("m,amp", [(1, 1e-6), (3, 1e-6), (2, 1e-8)])
def test_logged_mode_small_amplitude_perturbation_layout(sv, m, amp):
    """The same eigenmode runs at amplitudes a float state cannot follow, in
    the perturbation layout SV_FP32_PS (its rounding scales with the
    perturbation): growth within 2% and frequency within 1% of eq. 8."""
    N = 512 * m
    Po = O.Params(tau0=0.1, limiter=O.VANLEER)
    k = 2 * math.pi * m
    w = D.growing_acoustic_root(Po, k)
    t_end = math.log(30.0) / w.imag
    md = D.eigenmode(Po, k, w)
    U0 = inputs.waves_1d(1.4, N, 1.0, inputs.equilibrium_primitive(Po.Ck, Po.S),
                         [inputs.Mode(m=m, shape=md["prim"], scale=amp)])
    run = Run(n=N, t_end=t_end, S=1.0, tau0=0.1, m=m)
    P = sv.Params(precision=sv.FP32_PS, limiter=sv.VANLEER)
    with sv.Batch(P, [run], [U0], log_cap=40) as b:
        b.run()
        t, a = b.mode_log(0)
        assert b.read(0, state=False)[3] == 0
    growth = np.polyfit(t, np.log(np.abs(a)), 1)[0]
    freq = -np.polyfit(t, np.unwrap(np.angle(a)), 1)[0]
    assert abs(growth - w.imag) <= 0.02 * w.imag
    assert abs(freq - w.real) <= 0.01 * abs(w.real)


def test_stability_map_signs(sv):
    """Runs on either side of the S1 boundary (Q/I exponents 0): the logged
    fundamental decays below S1 and grows above it."""
    S1 = -0.4 * 0.1 / (-1.0 + 0.4 * -1.5)
    runs, states = [], []
    for S in (0.3 * S1, 3.0 * S1, 20.0 * S1):
        Po = O.Params(S=S, tau0=0.05, limiter=O.VANLEER)
        w = D.growing_acoustic_root(Po, 2 * math.pi)
        md = D.eigenmode(Po, 2 * math.pi, w)
        U0 = inputs.waves_1d(1.4, 512, 1.0, inputs.equilibrium_primitive(0.1, S),
                             [inputs.Mode(m=1, shape=md["prim"], scale=1e-4)])
        runs.append(Run(n=512, t_end=3.0, S=S, tau0=0.05, m=1))
        states.append(U0)
    P = sv.Params(precision=sv.FP32, limiter=sv.VANLEER)
    with sv.Batch(P, runs, states, log_cap=32) as b:
        b.run()
        rates = []
        for i in range(3):
            t, a = b.mode_log(i)
            rates.append(np.polyfit(t, np.log(np.abs(a)), 1)[0])
    assert rates[0] < 0 < rates[1] < rates[2]


def test_flags_are_per_run(sv):
    runs, states = _mini_sweep(9, 4)
    bad = states[1].copy()
    bad[0, 5] = -1.0
    states[1] = bad
    P = sv.Params(precision=sv.FP32)
    with sv.Batch(P, runs, states, max_steps=20) as b:
        b.run()
        flags = [b.read(i, state=False)[3] for i in range(4)]
    assert flags[1] & sv.FLAG_NONPHYS
    for i in (0, 2, 3):
        assert flags[i] in (0, sv.FLAG_MAXSTEPS)


def test_batch_fp64_full_range_matches_oracle(sv):
    """FP64 batch against the oracle at 1e-12 on 24 runs drawn from the whole
    ranges of the stability sweep (N in [256, 16384], tau0 log-uniform down to
    1e-3 where the source cap c_tau min tau sets dt, S up to 2, every eq. 6
    exponent of either sign), van Leer, over each run's first ~20 steps: short
    enough that the unstable draws have not yet amplified rounding noise."""
    raw = inputs.sweep_runs(31, 20)
    # and four draws from the corner of those ranges where the cap binds
    # (coarse grids, tau0 near 1e-3)
    raw += [replace(r, tau0=1e-3 * (1.0 + 0.1 * i))
            for i, r in enumerate(inputs.sweep_runs(32, 4, n_lo=256, n_hi=320))]
    P = sv.Params(precision=sv.FP64, limiter=1)
    runs, states, params = [], [], []
    shape = inputs.acoustic_shape(1.4)
    for r in raw:
        U0 = inputs.waves_1d(1.4, r.N, 1.0, inputs.equilibrium_primitive(0.1, r.S),
                             [inputs.Mode(m=r.m, shape=shape, scale=1e-3)])
        Po = oracle_params(P, S=r.S, tau0=r.tau0, tau_rho=r.tau_rho, tau_T=r.tau_T,
                           Q_rho=r.Q_rho, Q_T=r.Q_T, I_rho=r.I_rho, I_T=r.I_T)
        t_end = 20.5 * O.dt_cfl(Po, U0, r.N, 1.0 / r.N)
        while O.run(Po, U0, r.N, 1.0 / r.N, t_end)[3] != 0:
            t_end *= 0.5                     # the most unstable draw blows up within ~24 steps
        runs.append(Run(n=r.N, t_end=t_end, S=r.S, tau0=r.tau0, tau_rho=r.tau_rho,
                        tau_T=r.tau_T, Q_rho=r.Q_rho, Q_T=r.Q_T, I_rho=r.I_rho, I_T=r.I_T,
                        m=r.m))
        states.append(U0)
        params.append(Po)
    # the draws reach the regimes this test is for: a binding source cap and
    # strongly unstable media (e-folding within a few wave periods)
    capped = sum(O.dt_cfl(Po, U0, run.n, 1.0 / run.n)
                 < 0.9 * O.dt_cfl(oracle_params(P, **{**Po.__dict__, "c_tau": 1e30}), U0, run.n,
                                  1.0 / run.n)
                 for Po, U0, run in zip(params, states, runs))
    growth = [D.max_growth(Po, 2 * math.pi * run.m)[0] / (2 * math.pi * run.m * math.sqrt(1.4))
              for Po, run in zip(params, runs)]
    assert capped >= 3 and max(growth) > 0.2 and min(growth) < 0
    with sv.Batch(P, runs, states) as b:
        b.run()
        for i, (run, U0, Po) in enumerate(zip(runs, states, params)):
            U, t, k, f = b.read(i)
            ref, tr, kr, rc = O.run(Po, U0, run.n, run.L / run.n, run.t_end)
            assert rc == 0 and f == 0, (i, rc, f)
            assert k == kr and t == tr, (i, k, kr, t, tr)
            assert_fp64_parity(U, ref)
