"""Linear theory of Sec. 2.2: the dispersion relation of eq. 8 and its eigenmode.

TEST INFRASTRUCTURE ONLY.

Eq. 8, with gamma_1 = gamma - 1, delta = omega tau0, c0^2 = gamma R T0 and
A = 1 + (C_k + S (tau_T + Q_T)) gamma_1,
B = 1 + (C_k + S (tau_T - tau_rho + Q_T - Q_rho)) gamma_1 / gamma,
reads omega^2 [(A - i delta) + i (1 - i delta) X] = k^2 c0^2 [(B - i delta) + i (1 - i delta) Z].

Units: rho0 = p0 = R = T0 = 1, tau0 free, Q0 = I0 = S / tau0.  In these units
the right-hand coefficient is Z = b / delta with
b = (gamma_1/gamma) S [(I_T - I_rho) - (Q_T - Q_rho)], as printed.  The printed
left-hand coefficient gamma_1 (I0 I_T - Q0 Q_T) / (delta R) equals
gamma_1 S (I_T - Q_T) / (tau0 delta); linearising eqs. 1-4 gives
a / delta with a = gamma_1 S (I_T - Q_T), i.e. the printed form holds when the
time unit is tau0 (tau0 = 1, the paper's normalisation).  We keep tau0 free, so
we use X = a / delta.  Multiplying by delta:

    omega^2 [delta (A - i delta) + i a (1 - i delta)]
        = k^2 c0^2 [delta (B - i delta) + i b (1 - i delta)],

a quartic in omega for real k.  Growth: Im omega > 0 (equivalently Im k < 0 for
real omega, the statement under eq. 8).
"""
from __future__ import annotations

import math

import numpy as np


def constants(P) -> dict:
    g = P.gamma
    g1 = g - 1.0
    A = 1.0 + (P.Ck + P.S * (P.tau_T + P.Q_T)) * g1
    B = 1.0 + (P.Ck + P.S * (P.tau_T - P.tau_rho + P.Q_T - P.Q_rho)) * g1 / g
    a = g1 * P.S * (P.I_T - P.Q_T)
    b = (g1 / g) * P.S * ((P.I_T - P.I_rho) - (P.Q_T - P.Q_rho))
    return dict(A=A, B=B, a=a, b=b, c0sq=g, g1=g1)


def quartic(P, k: float) -> np.ndarray:
    """Coefficients (highest power first) of the corrected eq. 8 as a polynomial in omega."""
    c = constants(P)
    t = P.tau0
    K = k * k * c["c0sq"]
    A, B, a, b = c["A"], c["B"], c["a"], c["b"]
    # LHS: -i t^2 w^4 + t (A + a) w^3 + i a w^2
    # RHS: K (-i t^2 w^2 + t (B + b) w + i b)
    return np.array([-1j * t * t,
                     t * (A + a),
                     1j * a + 1j * K * t * t,
                     -K * t * (B + b),
                     -1j * K * b], dtype=complex)


def roots(P, k: float) -> np.ndarray:
    """All four omega roots for real k, sorted by Im omega (largest last)."""
    if math.isinf(P.tau0):
        c0 = math.sqrt(P.gamma)
        return np.array([-k * c0, 0.0, 0.0, k * c0], dtype=complex)
    r = np.roots(quartic(P, k))
    return r[np.argsort(r.imag)]


def growing_acoustic_root(P, k: float, direction: int = +1) -> complex:
    """The acoustic root travelling in `direction` (sign of Re omega / k)."""
    r = roots(P, k)
    acoustic = [w for w in r if direction * w.real > 1e-9 * abs(k)]
    return max(acoustic, key=lambda w: abs(w.real))


def max_growth(P, k: float) -> tuple[float, complex]:
    """max Im omega over all roots (the stability classifier) and that root."""
    r = roots(P, k)
    w = r[-1]
    return float(w.imag), complex(w)


def eigenmode(P, k: float, omega: complex) -> dict:
    """Complex amplitudes of the linear wave exp(i k x - i omega t) about the
    equilibrium rho0 = 1, u0 = 0, p0 = T0 = 1, with velocity amplitude 1.

    From the linearised continuity and momentum equations (eqs. 1-2):
    rho' = (k / omega) u', p' = (omega / k) u', T' = p' - rho' (eq. 7);
    from eq. 4 with eq. 6 (specific e_nu = E_nu / rho, e_nue = C_k T):
    (1 - i omega tau0) e' = C_k T' + S [(tau_rho + Q_rho) rho' + (tau_T + Q_T) T'].
    Returns primitive amplitudes (rho, u, p, e_nu) and conserved ones
    (rho, m, E, E_nu) with e_nu0 = C_k + S (steady state of eq. 4)."""
    u = 1.0 + 0j
    rho = k / omega * u
    p = omega / k * u
    T = p - rho
    e = (P.Ck * T + P.S * ((P.tau_rho + P.Q_rho) * rho + (P.tau_T + P.Q_T) * T)) \
        / (1.0 - 1j * omega * P.tau0)
    ev0 = P.Ck + P.S
    Ev = ev0 * rho + e
    E = p / (P.gamma - 1.0) + Ev
    return dict(prim=np.array([rho, u, p, e]), cons=np.array([rho, u, E, Ev]))


def equilibrium(P, dim: int = 1) -> np.ndarray:
    """Uniform equilibrium state (rho, m.., E, E_nu) with rho0 = p0 = 1, v = 0."""
    ev0 = P.Ck + P.S
    u = np.zeros(dim + 3)
    u[0] = 1.0
    u[1 + dim] = 1.0 / (P.gamma - 1.0) + ev0
    u[2 + dim] = ev0
    return u


def spatial_root(P, omega: float) -> complex:
    """Spatial problem (real omega, Sec. 3 forced source): eq. 8 is a quadratic
    in k: k^2 = omega^2 [delta (A - i delta) + i a (1 - i delta)]
                / (c0^2 [delta (B - i delta) + i b (1 - i delta)]), delta = omega tau0.
    Returns the root with Re k > 0 (the wave travelling away from the source);
    Im k < 0 means amplification with distance."""
    c = constants(P)
    d = omega * P.tau0
    lhs = omega * omega * (d * (c["A"] - 1j * d) + 1j * c["a"] * (1 - 1j * d))
    rhs = c["c0sq"] * (d * (c["B"] - 1j * d) + 1j * c["b"] * (1 - 1j * d))
    k = np.sqrt(lhs / rhs)
    return complex(k if k.real > 0 else -k)
