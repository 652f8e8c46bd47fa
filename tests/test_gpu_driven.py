"""The driven boundary (forced source of the paper's Sec. 3) on the GPU:
FP64 parity with the oracle, and the spatial growth of eq. 8 in FP32 / FP64."""
import math

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


def setup(P_orc, amp=1e-4):
    w = 2 * math.pi / 0.1 * 1.18
    k = D.spatial_root(P_orc, w)
    md = D.eigenmode(P_orc, k, w)
    base = D.equilibrium(P_orc)
    return w, k, base, amp * md["cons"]


def test_fp64_driven_matches_oracle(sv):
    N = 2000
    P = sv.Params(precision=sv.FP64, S=0.5, tau0=0.0135, limiter=sv.VANLEER)
    Po = oracle_params(P)
    w, k, base, amp = setup(Po)
    U0 = np.repeat(base[:, None], N, axis=1)
    with sv.Solver(P, (N,), (1.0,), bc=(sv.BC_DRIVEN, sv.BC_OUTFLOW)) as s:
        s.set_drive(w, k, base, amp)
        s.write_state(U0)
        s.run_to(0.1)
        U, t = s.read_state()
    ref, tr, kr, rc = O.run_driven(Po, U0, N, 1.0 / N, 0.1, O.drive(w, k, base, amp))
    assert rc == 0 and t == tr
    assert_fp64_parity(U, ref)


@pytest.mark.parametrize("prec", ["FP64", "FP32"])
def test_spatial_growth_on_gpu(sv, prec):
    N = 2000
    P = sv.Params(precision=getattr(sv, prec), S=0.5, tau0=0.0135)
    w, k, base, amp = setup(oracle_params(P))
    Tp = 2 * math.pi / w
    acc = np.zeros(N, dtype=complex)
    with sv.Solver(P, (N,), (1.0,), bc=(sv.BC_DRIVEN, sv.BC_OUTFLOW)) as s:
        s.set_drive(w, k, base, amp)
        s.write_state(np.repeat(base[:, None], N, axis=1))
        s.run_to(1.0)
        for i in range(32):
            s.run_to(1.0 + (i + 1) * Tp / 32)
            U, t = s.read_state()
            acc += (U[1] / U[0]) * np.exp(1j * w * t)
    a = acc / 16
    x = inputs.cell_centres(N, 1.0)
    sel = (x > 0.1) & (x < 0.5)
    growth = np.polyfit(x[sel], np.log(np.abs(a[sel])), 1)[0]
    kr = np.polyfit(x[sel], np.unwrap(np.angle(a[sel])), 1)[0]
    assert abs(growth + k.imag) <= 0.02 * abs(k.imag)
    assert abs(kr - k.real) <= 0.005 * k.real
