"""Pins of the oracle's pointwise pieces (pressure, flux, source, HLL, limiter)
and of the dispersion relation, against facts fixed by the paper and by the
mathematics rather than by the oracle itself."""
import itertools
import math

import numpy as np
import pytest

from oracle import dispersion as D
from oracle import orc as O
from paper_1805_03442_gb300 import inputs


def _state(gamma, rho, vel, p, ev):
    return inputs.prim_to_cons(gamma, np.array([rho]), [np.array([v]) for v in vel],
                               np.array([p]), np.array([ev]))[:, 0]


@pytest.mark.parametrize("dim", [1, 2, 3])
def test_pressure_round_trip(orc, dim):
    P = O.Params()
    vel = [0.3, -0.7, 0.11][:dim]
    u = _state(P.gamma, 1.7, vel, 0.8, 0.45)
    assert O.pressure(P, u) == pytest.approx(0.8, rel=1e-14)


def test_flux_of_rest_state_is_pressure_only(orc):
    P = O.Params()
    u = _state(P.gamma, 2.0, [0.0, 0.0], 1.3, 0.4)
    for axis in (0, 1):
        F = O.flux(P, u, axis)
        expect = np.zeros(5)
        expect[1 + axis] = 1.3
        assert np.array_equal(F, expect)


def test_flux_galilean_mass_and_energy(orc):
    """F = (rho u, rho u^2 + p, u (E + p), u E_nu): mass flux = momentum,
    energy flux = u (E + p) with E from eq. 5."""
    P = O.Params()
    rho, u, p, ev = 1.5, -0.4, 0.9, 0.3
    U = _state(P.gamma, rho, [u], p, ev)
    F = O.flux(P, U)
    E = p / 0.4 + 0.5 * rho * u * u + rho * ev
    assert F[0] == pytest.approx(rho * u, rel=1e-15)
    assert F[1] == pytest.approx(rho * u * u + p, rel=1e-15)
    assert F[2] == pytest.approx(u * (E + p), rel=1e-14)
    assert F[3] == pytest.approx(u * rho * ev, rel=1e-15)


def test_source_vanishes_at_equilibrium_and_frozen(orc):
    for P in (O.Params(), O.Params(S=0.3, tau0=2.0, Q_rho=0.5, Q_T=-0.3, I_rho=0.2, I_T=0.7)):
        Y = O.source(P, D.equilibrium(P))
        assert np.max(np.abs(Y)) < 1e-13 / P.tau0
    Pf = O.Params().frozen()
    u = _state(Pf.gamma, 1.3, [0.2], 0.7, 0.9)
    assert np.array_equal(O.source(Pf, u), np.zeros(4))


def test_source_pump_sink_balance_and_relaxation_sign(orc):
    """Hotter-than-equilibrium gas relaxes E_nu up (C_k T > e_nu) and the pump
    always adds rho Q to E_nu; with Q and I of equal exponents rho (Q - I) = 0."""
    P = O.Params(S=0.5, tau0=1.0)
    u = _state(P.gamma, 1.0, [0.0], 10.0, 0.0)   # T = 10, e_nu = 0
    Y = O.source(P, u)
    assert Y[2] == 0.0
    assert Y[3] > 0.0
    # with e_nu = C_k T + Q tau the vibrational source vanishes (steady state of eq. 4)
    T = 1.7
    tau = P.tau0 * T ** P.tau_T
    u = _state(P.gamma, 1.0, [0.0], T, P.Ck * T + (P.S / P.tau0) * tau)
    assert abs(O.source(P, u)[3]) < 1e-14


# -------------------------------------------------------------- HLL (eq. 13)

def test_hll_consistency(orc):
    P = O.Params()
    u = _state(P.gamma, 1.2, [0.3], 0.9, 0.5)
    assert np.allclose(O.hll(P, u, u), O.flux(P, u), rtol=1e-15, atol=1e-15)


def test_hll_supersonic_branches(orc):
    P = O.Params()
    uL = _state(P.gamma, 1.0, [3.0], 1.0, 0.2)
    uR = _state(P.gamma, 0.5, [2.5], 0.8, 0.3)
    assert np.array_equal(O.hll(P, uL, uR), O.flux(P, uL))       # 0 < S_L
    uL = _state(P.gamma, 1.0, [-3.0], 1.0, 0.2)
    uR = _state(P.gamma, 0.5, [-2.5], 0.8, 0.3)
    assert np.array_equal(O.hll(P, uL, uR), O.flux(P, uR))       # S_R < 0


def test_hll_is_the_single_intermediate_state_flux(orc):
    """In the subsonic branch the HLL flux is the flux of the single state U*
    between S_L and S_R: F = F_L + S_L (U* - U_L) = F_R + S_R (U* - U_R) with
    U* = (S_R U_R - S_L U_L - F_R + F_L) / (S_R - S_L) (integral conservation
    over the Riemann fan), and S_L, S_R are the Davis estimates."""
    P = O.Params()
    uL = _state(P.gamma, 1.0, [0.2], 1.0, 0.2)
    uR = _state(P.gamma, 0.4, [-0.1], 0.3, 0.6)
    cL, cR = math.sqrt(1.4 * 1.0 / 1.0), math.sqrt(1.4 * 0.3 / 0.4)
    SL, SR = min(0.2 - cL, -0.1 - cR), max(0.2 + cL, -0.1 + cR)
    FL, FR = O.flux(P, uL), O.flux(P, uR)
    Ustar = (SR * uR - SL * uL - FR + FL) / (SR - SL)
    F = O.hll(P, uL, uR)
    assert np.allclose(F, FL + SL * (Ustar - uL), rtol=1e-13, atol=1e-14)
    assert np.allclose(F, FR + SR * (Ustar - uR), rtol=1e-13, atol=1e-14)


def test_hll_mirror_symmetry(orc):
    P = O.Params()
    uL = _state(P.gamma, 1.3, [0.25], 1.1, 0.2)
    uR = _state(P.gamma, 0.6, [-0.4], 0.5, 0.7)
    mir = np.array([1, -1, 1, 1])
    F = O.hll(P, uL, uR)
    Fm = O.hll(P, uR * mir, uL * mir)
    assert np.allclose(Fm, -F * mir, rtol=1e-13, atol=1e-14)


# -------------------------------------------------------------- limiter

@pytest.mark.parametrize("a,b,mm,vl,mc", [
    (1.0, 2.0, 1.0, 4.0 / 3.0, 1.5),
    (-3.0, -1.0, -1.0, -1.5, -2.0),
    (1.0, -2.0, 0.0, 0.0, 0.0),
    (0.0, 5.0, 0.0, 0.0, 0.0),
    (2.0, 2.0, 2.0, 2.0, 2.0),
    (1.0, 10.0, 1.0, 20.0 / 11.0, 2.0),
])
def test_limiters(orc, a, b, mm, vl, mc):
    assert O.limiter(O.MINMOD, a, b) == pytest.approx(mm, abs=1e-15)
    assert O.limiter(O.VANLEER, a, b) == pytest.approx(vl, abs=1e-15)
    assert O.limiter(O.MC, a, b) == pytest.approx(mc, abs=1e-15)


# -------------------------------------------------------------- eq. 8

PARAM_SETS = [
    O.Params(tau0=0.1),
    O.Params(S=0.5, tau0=0.3, tau_T=-2.0),
    O.Params(S=0.8, tau0=0.05, Q_rho=0.4, Q_T=0.6, I_rho=-0.3, I_T=0.2),
    O.Params(S=1.2, tau0=1.0, tau_rho=-0.5, tau_T=-1.0, Q_rho=-0.2, Q_T=0.3, I_rho=0.5, I_T=-0.4),
]


def _jacobian(fn, U0):
    n = len(U0)
    J = np.zeros((n, n))
    for j in range(n):
        eps = 1e-6 * max(1.0, abs(U0[j]))
        e = np.zeros(n)
        e[j] = eps
        J[:, j] = (fn(U0 + e) - fn(U0 - e)) / (2 * eps)
    return J


@pytest.mark.parametrize("P", PARAM_SETS)
@pytest.mark.parametrize("k", [2 * math.pi, 20.0, 0.7])
def test_quartic_equals_linearised_oracle(orc, P, k):
    """Route 1: roots of eq. 8 (quartic in omega).  Route 2: omega = i eig(-ikA + J),
    A and J the Jacobians of the oracle's flux and source at equilibrium.  They
    agree only if the oracle's eqs. 1-7 and the dispersion relation agree."""
    U0 = D.equilibrium(P)
    A = _jacobian(lambda u: O.flux(P, u), U0)
    J = _jacobian(lambda u: O.source(P, u), U0)
    ev = 1j * np.linalg.eigvals(-1j * k * A + J)
    r = D.roots(P, k)
    scale = max(1.0, np.max(np.abs(r)))
    best = min(np.max(np.abs(ev[list(perm)] - r)) for perm in itertools.permutations(range(4)))
    assert best < 1e-7 * scale


@pytest.mark.parametrize("P", PARAM_SETS)
def test_eigenmode_is_null_vector(orc, P):
    k = 2 * math.pi
    U0 = D.equilibrium(P)
    A = _jacobian(lambda u: O.flux(P, u), U0)
    J = _jacobian(lambda u: O.source(P, u), U0)
    w = D.growing_acoustic_root(P, k)
    v = D.eigenmode(P, k, w)["cons"]
    res = (-1j * k * A + J) @ v + 1j * w * v
    assert np.max(np.abs(res)) < 1e-7 * np.max(np.abs(v)) * max(1, abs(w))


def test_high_frequency_plateau():
    """delta >> 1: omega^2 (A - i delta) ~ k^2 c0^2 (B - i delta) gives
    Im omega -> (B - A) / (2 tau0)."""
    P = O.Params(tau0=0.1)
    c = D.constants(P)
    w = D.growing_acoustic_root(P, 2e4)
    assert w.imag == pytest.approx((c["B"] - c["A"]) / (2 * P.tau0), rel=2e-3)


def test_low_frequency_limit():
    """delta << 1: omega ~ k c0 sqrt(B/A) (1 + i delta (B - A) / (2AB)), i.e.
    Im omega ~ k^2 c0^2 tau0 (B - A) / (2 A^2)."""
    P = O.Params(tau0=0.1)
    c = D.constants(P)
    k = 0.02
    w = D.growing_acoustic_root(P, k)
    assert w.real == pytest.approx(k * math.sqrt(1.4 * c["B"] / c["A"]), rel=1e-4)
    assert w.imag == pytest.approx(k * k * 1.4 * P.tau0 * (c["B"] - c["A"]) / (2 * c["A"] ** 2), rel=2e-3)


@pytest.mark.parametrize("tau_rho,tau_T", [(-1.0, -1.5), (-1.0, -2.0), (-0.5, -1.0)])
def test_S1_boundary(tau_rho, tau_T):
    """The printed boundary S1 = -gamma_1 C_k / (tau_rho + gamma_1 tau_T) separates
    damped (S < S1) from unstable (S > S1) sound waves (Q/I exponents 0)."""
    S1 = -0.4 * 0.1 / (tau_rho + 0.4 * tau_T)
    k = 2 * math.pi
    lo = O.Params(S=0.9 * S1, tau0=0.05, tau_rho=tau_rho, tau_T=tau_T)
    hi = O.Params(S=1.1 * S1, tau0=0.05, tau_rho=tau_rho, tau_T=tau_T)
    at = O.Params(S=S1, tau0=0.05, tau_rho=tau_rho, tau_T=tau_T)
    assert D.growing_acoustic_root(lo, k).imag < 0
    assert D.growing_acoustic_root(hi, k).imag > 0
    c = D.constants(at)
    assert c["B"] - c["A"] == pytest.approx(0.0, abs=1e-15)


def test_increment_trends():
    """The increment grows as tau_rho, tau_T, I_rho, I_T decrease and as Q_rho,
    Q_T increase (the trend statement after the base parameters)."""
    k = 2 * math.pi
    base = dict(S=0.5, tau0=0.1)
    g0 = D.growing_acoustic_root(O.Params(**base), k).imag
    for name, delta in (("tau_rho", -0.2), ("tau_T", -0.2), ("I_rho", -0.2), ("I_T", -0.2),
                        ("Q_rho", +0.2), ("Q_T", +0.2)):
        shifted = getattr(O.Params(), name) + delta
        g = D.growing_acoustic_root(O.Params(**base, **{name: shifted}), k).imag
        assert g > g0, name


def test_derived_regression_roots():
    """Derived (not printed) values for gamma 1.4, C_k 0.1, tau_rho -1, tau_T -1.5,
    S 1, tau0 0.1, k 2 pi: omega = +-8.385226 + 1.210120 i, -6.820241 i, 0."""
    r = np.sort_complex(D.roots(O.Params(tau0=0.1), 2 * math.pi))
    assert r[0].real == pytest.approx(-8.385226, abs=2e-6)
    assert r[-1].real == pytest.approx(8.385226, abs=2e-6)
    assert r[-1].imag == pytest.approx(1.210120, abs=2e-6)
    assert min(r, key=lambda w: w.imag).imag == pytest.approx(-6.820241, abs=2e-6)
