"""Pins of the oracle's positivity guard (a reading of the paper: the limiter
text after eq. 14 says nothing about positivity).

The guard has two parts:
  (a) if an extrapolated state U_j +- Theta_j h/2 is non-physical (rho <= 0 or
      p <= 0), every slope of cell j is zero;
  (b) if a face state U^L or U^R (eq. 14 at the half step) is non-physical,
      that face's HLL flux (eq. 13) takes the cell values U_l, U_r instead.

Each case below is a hand-built six-cell periodic state in the frozen limit
(no source) whose flow is supersonic to the right everywhere, so that every
HLL flux is the upwind flux F(U^L) (S_L > 0).  The cells are arranged so that,
with the guard, cell j reduces to the first-order upwind update

    U_j^{n+1} = U_j - (dt/h) (F(U_j) - F(U_{j-1})),

which is evaluated here in exact rational arithmetic from the definition of
the Euler flux (eq. 15's F with the passive E_nu).  Without the guard the
cell's slopes or face states enter and the result moves by O(1): removing
either part of the guard from the oracle fails one of these tests.
"""
from fractions import Fraction as Fr
import math

import numpy as np
import pytest

from oracle import orc as O

GAMMA = Fr(7, 5)


def cons(rho, m, p, ev):
    """Conserved state (rho, rho v, E, E_nu) from rho, rho v, p, E_nu (eq. 5)."""
    rho, m, p, ev = map(Fr, (rho, m, p, ev))
    return (rho, m, p / (GAMMA - 1) + m * m / (2 * rho) + ev, ev)


def pressure(u):
    rho, m, E, ev = u
    return (GAMMA - 1) * (E - m * m / (2 * rho) - ev)


def flux(u):
    rho, m, E, ev = u
    v, p = m / rho, pressure(u)
    return (m, m * v + p, v * (E + p), v * ev)


def sound_speed(u):
    return math.sqrt(float(GAMMA * pressure(u) / u[0]))


def upwind(uj, ujm, r):
    Fj, Fm = flux(uj), flux(ujm)
    return [uj[f] - r * (Fj[f] - Fm[f]) for f in range(4)]


def minmod(a, b):
    if a * b <= 0:
        return Fr(0)
    return a if abs(a) < abs(b) else b


# frozen limit with zero closure exponents: the source vanishes for any state,
# physical or not
FROZEN = dict(tau0=math.inf, S=0.0, tau_rho=0.0, tau_T=0.0)

A = cons(1, 12, 5, Fr(1, 2))
B = cons(1, 11, Fr(1, 10), Fr(1, 2))
C = cons(1, 10, 5, Fr(1, 2))
# case (a): the minus-side extrapolation of cell 3 has p < 0
CASE_A = dict(cells=[A, A, A, B, C, C], j=3, r=Fr(1, 100))

A2 = cons(1, 10, Fr(5, 2), Fr(1, 2))
B2 = cons(1, 10, Fr(1, 5), Fr(1, 2))
C2 = cons(1, 10, 1, Fr(1, 2))
D2 = cons(1, 10, Fr(9, 5), Fr(1, 2))
# case (b): cell 3's slopes survive, but its half-step face states have p < 0
CASE_B = dict(cells=[A2, A2, B2, C2, D2, D2], j=3, r=Fr(1, 2))


def _array(cells):
    return np.array([[float(x) for x in c] for c in cells]).T.copy()


def _step(case):
    U = _array(case["cells"])
    N = U.shape[1]
    h = 1.0 / N
    Un, rc = O.step(O.Params(**FROZEN), U, (N,), h, float(case["r"]) * h)
    return Un, rc


def test_case_a_preconditions():
    """Cell 3 has a nonzero momentum slope and a zero energy slope, so its
    minus-side state carries more kinetic energy than its total energy holds."""
    cells, j = CASE_A["cells"], CASE_A["j"]
    theta = [minmod(cells[j][f] - cells[j - 1][f], cells[j + 1][f] - cells[j][f])
             for f in range(4)]
    assert theta == [0, -1, 0, 0]
    minus = tuple(cells[j][f] - theta[f] / 2 for f in range(4))
    plus = tuple(cells[j][f] + theta[f] / 2 for f in range(4))
    assert pressure(minus) < 0 < pressure(plus)
    # the cells left of j and right of j + 1 are uniform pairs: zero slopes there
    assert cells[j - 2] == cells[j - 1] and cells[j + 1] == cells[(j + 2) % 6]
    for u in cells:                               # supersonic everywhere
        assert float(u[1] / u[0]) - sound_speed(u) > 5.0


def test_case_a_slopes_dropped(orc):
    """Guard (a): with the slopes of cell 3 dropped, its half-step state is U_3
    itself and both of its faces are upwind faces between unextrapolated cells,
    so U_3 moves by the first-order upwind update."""
    Un, _ = _step(CASE_A)
    j, cells = CASE_A["j"], CASE_A["cells"]
    expect = np.array([float(x) for x in upwind(cells[j], cells[j - 1], CASE_A["r"])])
    # (1.01, 11.279, 65.3015, 0.505)
    assert np.allclose(expect, [1.01, 11.279, 65.3015, 0.505], rtol=1e-15, atol=0)
    scale = np.max(np.abs(expect))
    assert np.max(np.abs(Un[:, j] - expect)) <= 1e-15 * scale


def test_case_b_preconditions():
    """Cell 3 keeps its energy slope (both extrapolations physical), but its
    half step lowers the energy of both face states below their kinetic plus
    vibrational energy."""
    cells, j, r = CASE_B["cells"], CASE_B["j"], CASE_B["r"]
    theta = [minmod(cells[j][f] - cells[j - 1][f], cells[j + 1][f] - cells[j][f])
             for f in range(4)]
    assert theta == [0, 0, 2, 0]
    plus = tuple(cells[j][f] + theta[f] / 2 for f in range(4))
    minus = tuple(cells[j][f] - theta[f] / 2 for f in range(4))
    assert pressure(plus) > 0 and pressure(minus) > 0
    Fp, Fm = flux(plus), flux(minus)
    half = tuple(cells[j][f] - r / 2 * (Fp[f] - Fm[f]) for f in range(4))
    face_l = tuple(half[f] + theta[f] / 2 for f in range(4))    # U^L of face j + 1/2
    face_r = tuple(half[f] - theta[f] / 2 for f in range(4))    # U^R of face j - 1/2
    assert pressure(face_l) < 0 and pressure(face_r) < 0
    for u in cells:
        assert float(u[1] / u[0]) - sound_speed(u) > 5.0


def test_case_b_faces_fall_back(orc):
    """Guard (b): both faces of cell 3 fall back to the cell values, so U_3
    moves by the first-order upwind update although its slopes are kept."""
    Un, rc = _step(CASE_B)
    assert rc != 0          # cells next to the jump leave the physical range (r = 1/2)
    j, cells = CASE_B["j"], CASE_B["cells"]
    expect = np.array([float(x) for x in upwind(cells[j], cells[j - 1], CASE_B["r"])])
    assert np.allclose(expect, [1.0, 9.6, 39.0, 0.5], rtol=1e-15, atol=0)
    scale = np.max(np.abs(expect))
    assert np.max(np.abs(Un[:, j] - expect)) <= 1e-15 * scale


@pytest.mark.parametrize("case", [CASE_A, CASE_B])
def test_guard_cases_mirror(orc, case):
    """The mirrored state (x -> -x, v -> -v) gives the mirrored result: the
    guard acts the same way on a left-moving flow."""
    U = _array(case["cells"])
    N = U.shape[1]
    h = 1.0 / N
    P = O.Params(**FROZEN)
    dt = float(case["r"]) * h
    mir = np.array([1, -1, 1, 1])[:, None]
    A_, _ = O.step(P, U, (N,), h, dt)
    B_, _ = O.step(P, (U * mir)[:, ::-1].copy(), (N,), h, dt)
    assert np.array_equal((B_ * mir)[:, ::-1], A_)


def embed_nd(case, reps, dim, axis, other):
    """The case's six cells tiled reps times along axis (0 = x) of a dim-D
    grid, uniform over the other axes (sizes `other`, in axis order) with zero
    transverse momentum.  Returns (U of shape (dim + 3, ncell), x fastest; the
    grid size tuple n)."""
    line = np.tile(_array(case["cells"]), (1, reps))        # rho, m, E, E_nu
    m = line.shape[1]
    rest = iter(other)
    n = tuple(m if a == axis else next(rest) for a in range(dim))
    shape = tuple(reversed(n))                              # numpy order: x last
    bshape = [1] * dim
    bshape[dim - 1 - axis] = m
    U = np.zeros((dim + 3,) + shape)
    U[0] = line[0].reshape(bshape)
    U[1 + axis] = line[1].reshape(bshape)
    U[dim + 1] = line[2].reshape(bshape)
    U[dim + 2] = line[3].reshape(bshape)
    return U.reshape(dim + 3, -1).copy(), n


@pytest.mark.parametrize("dim,axis", [(2, 0), (2, 1), (3, 0), (3, 1), (3, 2)])
@pytest.mark.parametrize("name", ["a", "b"])
def test_guard_cases_embedded_nd(orc, name, dim, axis):
    """The 2D / 3D oracle on the case laid along one axis of the grid: the
    transverse fluxes are uniform and cancel, so every line along that axis
    takes the 1D result, and the guarded cells take the exact upwind value."""
    case = CASE_A if name == "a" else CASE_B
    reps = 2
    U, n = embed_nd(case, reps, dim, axis, (3, 2)[: dim - 1])
    h = 1.0 / n[axis]
    dt = float(case["r"]) * h
    Un, rc = O.step(O.Params(**FROZEN), U, n, h, dt)
    U1, rc1 = O.step(O.Params(**FROZEN), np.tile(_array(case["cells"]), (1, reps)),
                     (6 * reps,), h, dt)
    assert (rc != 0) == (rc1 != 0)
    want, _ = embed_nd(dict(cells=[tuple(U1[:, i]) for i in range(6)]), reps, dim, axis,
                       (3, 2)[: dim - 1])
    # the 1D result of both copies is the same (periodic tiling)
    assert np.array_equal(U1[:, :6], U1[:, 6:])
    assert np.max(np.abs(Un - want)) <= 1e-14 * np.max(np.abs(want))
    j = case["j"]
    expect = np.array([float(x) for x in upwind(case["cells"][j], case["cells"][j - 1],
                                                case["r"])])
    shape = (dim + 3,) + tuple(reversed(n))
    sel = [slice(None)] * (dim + 1)
    sel[dim - axis] = j
    got = Un.reshape(shape)[tuple(sel)].reshape(dim + 3, -1)
    exp_nd = np.zeros(dim + 3)
    exp_nd[0], exp_nd[1 + axis], exp_nd[dim + 1], exp_nd[dim + 2] = expect
    assert np.max(np.abs(got - exp_nd[:, None])) <= 1e-15 * np.max(np.abs(expect))
