"""The perturbation layout SV_FP32_PS in 2D (packed plane pairs) and 3D (one
cell per thread) against the FP64 oracle, through the C ABI: one step
relative to the perturbation's size, the uniform equilibrium exactly at rest,
and the 2D active-sector problem (walls, outflow, frozen medium outside the
sector, pulsating source) against the FP64 kernels."""
import math

import numpy as np
import pytest

from gpu_util import need_gpu, oracle_params
from oracle import orc as O
from paper_1805_03442_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sv():
    return need_gpu()


def _ref(P, dim):
    ev0 = P.Ck + P.S
    r = np.zeros(dim + 3)
    r[0], r[-2], r[-1] = 1.0, 1.0 / (P.gamma - 1.0) + ev0, ev0
    return r


def _perturbed(P, n, seed, amp):
    """ref + d, d smooth plus noise, float-representable and recoverable."""
    dim = len(n)
    cells = int(np.prod(n))
    rng = np.random.default_rng(seed)
    grids = np.meshgrid(*[(np.arange(m) + 0.5) / m for m in n], indexing="ij")
    d = []
    for f in range(dim + 3):
        phase = sum((a + f + 1) * g for a, g in enumerate(grids))
        w = amp * np.sin(2 * np.pi * phase + rng.uniform(0, 2 * np.pi))
        d.append((w + 0.1 * amp * rng.standard_normal(w.shape)).T.reshape(-1))   # x fastest
    d = np.array(d).astype(np.float32).astype(np.float64)
    U = _ref(P, dim)[:, None] + d
    assert np.array_equal((U - _ref(P, dim)[:, None]).astype(np.float32).astype(np.float64), d)
    assert U.shape == (dim + 3, cells)
    return U, d


@pytest.mark.parametrize("n", [(37, 29), (130, 70), (17, 9, 11), (33, 20, 9)])
@pytest.mark.parametrize("params", [dict(tau0=0.3),
                                    dict(tau0=0.05, S=0.7, Q_rho=0.4, Q_T=-0.3, I_rho=0.2, I_T=0.5),
                                    dict(tau0=math.inf, S=0.0)])
def test_one_step_relative_to_the_perturbation(sv, n, params):
    h = 1.0 / n[0]
    L = tuple(m * h for m in n)
    out = {}
    for prec in ("FP32_PS", "FP32"):
        P = sv.Params(precision=getattr(sv, prec), **params)
        U0, d = _perturbed(P, n, seed=sum(n), amp=1e-3)
        with sv.Solver(P, n, L) as s:
            s.write_state(U0)
            dt = s.dt()
            s.step(1)
            U, _ = s.read_state()
            assert s.status() == 0
        ref, rc = O.step(oracle_params(P), U0, n, h, dt)
        assert rc == 0
        scale = np.max(np.abs(d), axis=1)
        out[prec] = np.max(np.max(np.abs(U.reshape(ref.shape) - ref), axis=1) / scale)
    assert out["FP32_PS"] <= 2e-6, out
    assert out["FP32"] >= 30 * out["FP32_PS"], out


@pytest.mark.parametrize("n", [(64, 48), (16, 12, 10)])
def test_equilibrium_exactly_at_rest(sv, n):
    P = sv.Params(precision=sv.FP32_PS, tau0=0.1)
    cells = int(np.prod(n))
    Ue = np.repeat(_ref(P, len(n))[:, None], cells, axis=1)
    with sv.Solver(P, n) as s:
        s.write_state(Ue)
        s.step(20)
        U, _ = s.read_state()
        c = s.conservation()
    assert np.array_equal(U.reshape(Ue.shape), Ue)
    assert c[0] == cells and c[-1] == pytest.approx(cells * Ue[-1, 0], rel=1e-15)


def test_sector_problem_against_fp64(sv):
    """The active sector at 120 cells across, to t = 0.3: the pulsating source,
    the frozen medium around the sector and the wall/outflow sides in the
    layout, against the FP64 kernels on the same set-up."""
    pb = inputs.sector_problem(120)
    n, L = (pb.nx, pb.ny), (pb.nx * pb.h, pb.ny * pb.h)
    lo, hi, dlo, dhi = pb.maps
    out = {}
    for prec in ("FP32_PS", "FP64"):
        P = sv.Params(precision=getattr(sv, prec), S=1.0, tau0=0.0135)
        U0 = inputs.sector_rest_state(P.gamma, P.Ck, P.S, pb.nx, pb.ny)
        with sv.Solver(P, n, L, bc=pb.bc) as s:
            s.set_medium2d(lo, hi, dlo, dhi, pb.omega, pb.amp)
            s.write_state(U0)
            rc, steps = s.run_to(0.3)
            U, t = s.read_state()
            assert rc == 0 and t == 0.3
        out[prec] = U
    dev = np.max(np.abs(out["FP64"] - U0), axis=1)
    err = np.max(np.abs(out["FP32_PS"] - out["FP64"]), axis=1)
    # relative to the perturbation the source has put into each field (fields
    # it barely moves are measured against a thousandth of the largest)
    scale = np.maximum(dev, 1e-3 * np.max(dev))
    assert np.all(err <= 1e-4 * scale), (err, dev)
