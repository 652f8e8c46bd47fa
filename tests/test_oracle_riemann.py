"""Pins of the exact frozen-limit Riemann solver: Rankine-Hugoniot jump
conditions across shocks, isentropic invariants across rarefactions, pressure
and velocity continuity at the contact, and the textbook Sod star state."""
import math

import numpy as np
import pytest

from oracle.riemann import Riemann

G = 1.4

CASES = [
    (1.0, 0.0, 1.0, 0.125, 0.0, 0.1),        # Sod: rarefaction left, shock right
    (1.0, -2.0, 0.4, 1.0, 2.0, 0.4),         # two rarefactions
    (1.0, 0.0, 1000.0, 1.0, 0.0, 0.01),      # strong shock (blast-wave left half)
    (5.99924, 19.5975, 460.894, 5.99242, -6.19633, 46.0950),  # two shocks
    (0.5, 0.3, 0.7, 1.7, -0.2, 2.5),
]


def _cons_flux(rho, u, p):
    E = p / (G - 1) + 0.5 * rho * u * u
    return np.array([rho, rho * u, E]), np.array([rho * u, rho * u * u + p, u * (E + p)])


@pytest.mark.parametrize("case", CASES)
def test_jump_conditions(case):
    R = Riemann(G, *case)
    rsL, rsR = R.star_densities()
    lh, lt, c, rt, rh = R.wave_speeds()
    sides = [(R.L, rsL, lh, lt), (R.R, rsR, rh, rt)]
    for (rK, uK, pK), rs, head, tail in sides:
        if R.pstar > pK:                      # shock: U_s [U] = [F]
            s = head
            U1, F1 = _cons_flux(rK, uK, pK)
            U2, F2 = _cons_flux(rs, R.ustar, R.pstar)
            assert np.allclose(s * (U2 - U1), F2 - F1, rtol=1e-10, atol=1e-10 * max(1, abs(F1).max()))
        else:                                 # rarefaction: isentrope + invariant
            assert R.pstar / rs ** G == pytest.approx(pK / rK ** G, rel=1e-12)
            cK = math.sqrt(G * pK / rK)
            cs = math.sqrt(G * R.pstar / rs)
            sgn = 1.0 if (rK, uK, pK) == R.L else -1.0
            assert uK + sgn * 2 * cK / (G - 1) == pytest.approx(R.ustar + sgn * 2 * cs / (G - 1), rel=1e-12, abs=1e-12)
            # fan is continuous at head and tail
            prim_head = R.sample(head + (1e-12 if sgn > 0 else -1e-12))
            assert prim_head[2] == pytest.approx(pK, rel=1e-8)
    # contact: pressure and velocity continuous
    a = R.sample(c - 1e-9)
    b = R.sample(c + 1e-9)
    assert a[1] == pytest.approx(b[1], rel=1e-8, abs=1e-8)
    assert a[2] == pytest.approx(b[2], rel=1e-8)


def test_sod_star_state():
    """Sod's tube (rho, u, p) = (1, 0, 1) | (0.125, 0, 0.1), gamma 1.4: the
    tabulated exact star state p* = 0.30313, u* = 0.92745."""
    R = Riemann(G, 1.0, 0.0, 1.0, 0.125, 0.0, 0.1)
    assert R.pstar == pytest.approx(0.30313, abs=1e-5)
    assert R.ustar == pytest.approx(0.92745, abs=1e-5)


def test_passive_scalar_jumps_only_at_contact():
    R = Riemann(G, 1.0, 0.0, 1.0, 0.125, 0.0, 0.1, evL=0.3, evR=0.9)
    c = R.ustar
    xi = np.linspace(-2, 2, 401)
    ev = R.sample_array(xi)[3]
    assert np.all(ev[xi < c] == 0.3) and np.all(ev[xi > c] == 0.9)
