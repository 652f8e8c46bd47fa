"""The 1D perturbation layout SV_FP32_PS against the FP64 oracle, through the C ABI.

The device holds float perturbations about the uniform equilibrium (rho = p =
1, v = 0, E_nu = C_k + S) and the step forms every flux difference and source
so that the equilibrium part cancels before rounding.  Its rounding therefore
scales with the perturbation: one step is checked against the oracle relative
to the perturbation's size (where the full-state float policy is ~1000 times
further off), and the one-wavelength linear-stage run stays close to the oracle
where the full-state float run is swamped by amplified rounding noise."""
import math

import numpy as np
import pytest

from gpu_util import need_gpu, oracle_params
from oracle import dispersion as D
from oracle import orc as O
from paper_1805_03442_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sv():
    return need_gpu()


def _ref(P):
    ev0 = P.Ck + P.S
    return np.array([1.0, 0.0, 1.0 / (P.gamma - 1.0) + ev0, ev0])


def _perturbed(P, N, seed, amp):
    """ref + d with d float-representable and exactly recoverable in double."""
    rng = np.random.default_rng(seed)
    x = (np.arange(N) + 0.5) / N
    d = np.stack([amp * np.sin(2 * np.pi * (f + 1) * x + rng.uniform(0, 2 * np.pi))
                  + 0.1 * amp * rng.standard_normal(N) for f in range(4)])
    d = d.astype(np.float32).astype(np.float64)
    U = _ref(P)[:, None] + d
    assert np.array_equal((U - _ref(P)[:, None]).astype(np.float32).astype(np.float64), d)
    return U, d


def _one_step(sv, P, U0, N, h):
    with sv.Solver(P, (N,), (N * h,)) as s:
        s.write_state(U0)
        dt = s.dt()
        s.step(1)
        U, _ = s.read_state()
        assert s.status() == 0
    return U, dt


@pytest.mark.parametrize("N", [7, 1000, 4099])
@pytest.mark.parametrize("params", [dict(tau0=0.3),
                                    dict(tau0=0.05, S=0.7, Q_rho=0.4, Q_T=-0.3, I_rho=0.2, I_T=0.5),
                                    dict(tau0=math.inf, S=0.0)])
def test_one_step_relative_to_the_perturbation(sv, N, params):
    h = 1.0 / N
    out = {}
    for prec in ("FP32_PS", "FP32"):
        P = sv.Params(precision=getattr(sv, prec), **params)
        U0, d = _perturbed(P, N, seed=N, amp=1e-3)
        U, dt = _one_step(sv, P, U0, N, h)
        ref, rc = O.step(oracle_params(P), U0, N, h, dt)
        assert rc == 0
        scale = np.max(np.abs(d), axis=1)
        out[prec] = np.max(np.max(np.abs(U - ref), axis=1) / scale)
    # float rounding of perturbation-sized terms: a few 1e-7 of the perturbation
    assert out["FP32_PS"] <= 2e-6, out
    # the full-state float policy rounds the O(1) background (~1e-4 of a 1e-3 perturbation)
    assert out["FP32"] >= 30 * out["FP32_PS"], out


@pytest.mark.parametrize("limiter", [0, 1])
def test_linear_stage_tracks_the_oracle(sv, limiter):
    """One-wavelength growing eigenmode (tau0 0.08, S = 1, amplitude 1e-4) to
    the end of the linear stage (the fundamental grown 100 times): the full
    state in float is off by more than the signal there; the perturbation
    layout stays within a few per cent of the signal."""
    N = 1024
    P = sv.Params(precision=sv.FP32_PS, tau0=0.08, limiter=limiter)
    Po = oracle_params(P)
    w = D.growing_acoustic_root(Po, 2 * math.pi)
    md = D.eigenmode(Po, 2 * math.pi, w)
    U0 = inputs.waves_1d(P.gamma, N, 1.0, inputs.equilibrium_primitive(P.Ck, P.S),
                         [inputs.Mode(m=1, shape=md["prim"], scale=1e-4)])
    t_lin = math.log(100.0) / w.imag
    with sv.Solver(P, (N,)) as s:
        s.write_state(U0)
        rc, _ = s.run_to(t_lin)
        U, t = s.read_state()
    ref, tr, _, _ = O.run(Po, U0, N, 1.0 / N, t_lin)
    assert t == tr == t_lin
    v, vr = U[1] / U[0], ref[1] / ref[0]
    signal = np.max(np.abs(vr))
    assert 0.009 < signal < 0.012
    assert np.max(np.abs(v - vr)) <= 0.05 * signal


def test_conservation_and_equilibrium(sv):
    N = 10007
    P = sv.Params(precision=sv.FP32_PS, tau0=0.1)
    U0, d = _perturbed(P, N, seed=3, amp=1e-3)
    with sv.Solver(P, (N,)) as s:
        s.write_state(U0)
        c0 = s.conservation()
        s.step(200)
        c1 = s.conservation()
        assert s.status() == 0
    assert c0[0] == pytest.approx(math.fsum(U0[0]), rel=1e-14)
    for f in (0, 1):                 # mass and momentum: float sums of perturbations
        assert abs(c1[f] - c0[f]) <= 1e-9 * N
    # the uniform equilibrium is exactly zero in the layout: it stays exactly put
    with sv.Solver(P, (N,)) as s:
        Ue = np.repeat(_ref(P)[:, None], N, axis=1)
        s.write_state(Ue)
        s.step(50)
        U, _ = s.read_state()
    assert np.array_equal(U, Ue)


def test_rejected_with_heun(sv):
    with pytest.raises(sv.SvError):
        sv.Solver(sv.Params(precision=sv.FP32_PS, method=sv.HEUN), (1024,))


@pytest.mark.parametrize("N", [1000, 5000])
@pytest.mark.parametrize("bc", [(1, 1), (2, 2), (1, 2)])
def test_walls_and_outflow_against_fp64(sv, N, bc):
    """Wall ghosts (reversed momentum) and outflow copies of perturbations, on
    the sliding warps (1000 cells) and the block tiles (5000): against the
    FP64 kernels at the same time, relative to the perturbation."""
    out = {}
    for prec in ("FP32_PS", "FP64"):
        P = sv.Params(precision=getattr(sv, prec), tau0=0.3)
        U0, d = _perturbed(P, N, seed=N + bc[0], amp=1e-3)
        with sv.Solver(P, (N,), (1.0,), bc=bc) as s:
            s.write_state(U0)
            rc, _ = s.run_to(0.05)
            U, t = s.read_state()
            assert rc == 0 and t == 0.05
        out[prec] = U
    err = np.max(np.abs(out["FP32_PS"] - out["FP64"]), axis=1)
    assert np.all(err <= 3e-4 * np.max(np.abs(d), axis=1)), err


@pytest.mark.parametrize("N", [2000, 5000])
def test_driven_boundary_against_fp64(sv, N):
    """The driven boundary's ghost states (full states in double, minus the
    reference) on both kernels: against the FP64 kernels, relative to the
    wave the boundary drives in."""
    from test_gpu_driven import setup
    out = {}
    for prec in ("FP32_PS", "FP64"):
        P = sv.Params(precision=getattr(sv, prec), S=0.5, tau0=0.0135)
        w, k, base, amp = setup(oracle_params(P))
        U0 = np.repeat(base[:, None], N, axis=1)
        with sv.Solver(P, (N,), (1.0,), bc=(sv.BC_DRIVEN, sv.BC_OUTFLOW)) as s:
            s.set_drive(w, k, base, amp)
            s.write_state(U0)
            rc, _ = s.run_to(0.1)
            U, t = s.read_state()
            assert rc == 0 and t == 0.1
        out[prec] = U
    wave = np.max(np.abs(out["FP64"] - U0), axis=1)
    err = np.max(np.abs(out["FP32_PS"] - out["FP64"]), axis=1)
    assert np.all(wave > 0) and np.all(err <= 1e-3 * wave), (err, wave)
