"""ctypes binding of the plain C oracle (``orc_muscl.c``).

TEST INFRASTRUCTURE ONLY (tests, smoke check, CPU-baseline leg of the benchmark).

The C file follows Sec. 2.3 of the paper: eq. 13 (HLL), eq. 14 with xi = 0
(piecewise-linear face states), eq. 15 (update with the source Y), eq. 16
(time step), with eqs. 5-7 for pressure, closures and temperature.  ``build()``
compiles it with gcc -O2 -ffp-contract=off (no fast-math), with OpenMP when the
compiler has it.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
from dataclasses import dataclass, field, fields

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liborc.so")
_SRC = os.path.join(_HERE, "orc_muscl.c")

MINMOD, VANLEER, MC = 0, 1, 2
PERIODIC, REFLECT, OUTFLOW, DRIVEN = 0, 1, 2, 3


class _CDrive(ctypes.Structure):
    _fields_ = [("omega", ctypes.c_double), ("k_re", ctypes.c_double), ("k_im", ctypes.c_double),
                ("base", ctypes.c_double * 4), ("amp_re", ctypes.c_double * 4),
                ("amp_im", ctypes.c_double * 4)]


def drive(omega: float, k: complex, base, amp) -> _CDrive:
    """Prescribed boundary wave U = base + Re(amp e^{i(k x - omega t)})."""
    d = _CDrive()
    d.omega, d.k_re, d.k_im = float(omega), float(complex(k).real), float(complex(k).imag)
    for f in range(4):
        d.base[f] = float(base[f])
        d.amp_re[f] = float(complex(amp[f]).real)
        d.amp_im[f] = float(complex(amp[f]).imag)
    return d


def build(force: bool = False) -> str:
    """Compile liborc.so in-tree (oracle/_build).  Returns its path."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_SO)
            and os.path.getmtime(_SO) >= max(os.path.getmtime(_SRC),
                                             os.path.getmtime(os.path.join(_HERE, "orc.h")))):
        return _SO
    base = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
            "-shared", _SRC, "-o", _SO + ".tmp", "-lm"]
    try:
        subprocess.run(base[:1] + ["-fopenmp"] + base[1:], check=True,
                       capture_output=True, text=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True, capture_output=True, text=True)
    os.replace(_SO + ".tmp", _SO)
    return _SO


class _CParams(ctypes.Structure):
    _fields_ = [(n, ctypes.c_double) for n in
                ("gamma", "Ck", "S", "tau0", "tau_rho", "tau_T", "Q_rho", "Q_T",
                 "I_rho", "I_T", "cfl", "c_tau")] + [("limiter", ctypes.c_int)]


@dataclass
class Params:
    """Model and scheme parameters.  Defaults: the paper's 1D runs of Sec. 3
    (gamma = 1.4, C_k = 0.1, tau_rho = -1, tau_T = -1.5, Q/I exponents 0) with
    S = 1 (the nonlinear-stage run) and tau0 = 0.08."""
    gamma: float = 1.4
    Ck: float = 0.1
    S: float = 1.0
    tau0: float = 0.08        # math.inf: frozen limit (Q = I = 0, 1/tau = 0)
    tau_rho: float = -1.0
    tau_T: float = -1.5
    Q_rho: float = 0.0
    Q_T: float = 0.0
    I_rho: float = 0.0
    I_T: float = 0.0
    cfl: float = 0.4
    c_tau: float = 0.5
    limiter: int = MINMOD

    def c(self) -> _CParams:
        return _CParams(*[getattr(self, f.name) for f in fields(self)])

    def frozen(self) -> "Params":
        d = {f.name: getattr(self, f.name) for f in fields(self)}
        d["tau0"] = math.inf
        d["S"] = 0.0
        return Params(**d)


_lib = None


def lib():
    global _lib
    if _lib is None:
        L = ctypes.CDLL(build())
        dp = ctypes.POINTER(ctypes.c_double)
        lp = ctypes.POINTER(ctypes.c_long)
        pp = ctypes.POINTER(_CParams)
        L.orc_pressure.argtypes = [pp, ctypes.c_int, dp]
        L.orc_pressure.restype = ctypes.c_double
        L.orc_flux.argtypes = [pp, ctypes.c_int, ctypes.c_int, dp, dp]
        L.orc_source.argtypes = [pp, ctypes.c_int, dp, dp]
        L.orc_hll.argtypes = [pp, ctypes.c_int, ctypes.c_int, dp, dp, dp]
        L.orc_limiter.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_double]
        L.orc_limiter.restype = ctypes.c_double
        L.orc_physical.argtypes = [pp, ctypes.c_int, dp]
        L.orc_step.argtypes = [pp, ctypes.c_int, lp, ctypes.c_double, ctypes.c_double, dp, dp]
        L.orc_step_cell.argtypes = [pp, ctypes.c_int, lp, ctypes.c_double, ctypes.c_double,
                                    dp, ctypes.c_long, dp]
        L.orc_dt.argtypes = [pp, ctypes.c_int, lp, ctypes.c_double, dp]
        L.orc_dt.restype = ctypes.c_double
        L.orc_run.argtypes = [pp, ctypes.c_int, lp, ctypes.c_double, dp, ctypes.c_double,
                              ctypes.c_double, ctypes.c_long, dp, lp]
        L.orc_threads.restype = ctypes.c_int
        L.orc_set_threads.argtypes = [ctypes.c_int]
        L.orc_step_bc1.argtypes = [pp, ctypes.c_long, ctypes.c_double, ctypes.c_double, ctypes.c_int,
                                   ctypes.c_int, dp, dp]
        L.orc_run_bc1.argtypes = [pp, ctypes.c_long, ctypes.c_double, ctypes.c_int, ctypes.c_int,
                                  dp, ctypes.c_double, ctypes.c_double, ctypes.c_long, dp, lp]
        L.orc_step_heun.argtypes = [pp, ctypes.c_int, lp, ctypes.c_double, ctypes.c_double, dp, dp]
        L.orc_run_heun.argtypes = [pp, ctypes.c_int, lp, ctypes.c_double, dp, ctypes.c_double,
                                   ctypes.c_double, ctypes.c_long, dp, lp]
        L.orc_run_bc1d.argtypes = [pp, ctypes.c_long, ctypes.c_double, ctypes.c_int, ctypes.c_int,
                                   ctypes.POINTER(_CDrive), dp, ctypes.c_double, ctypes.c_double,
                                   ctypes.c_long, dp, lp]
        mp = ctypes.POINTER(_CMedium2)
        ip = ctypes.POINTER(ctypes.c_int)
        L.orc_step2m.argtypes = [pp, ctypes.c_long, ctypes.c_long, ctypes.c_double, ctypes.c_double,
                                 ip, mp, ctypes.c_double, dp, dp]
        L.orc_run2m.argtypes = [pp, ctypes.c_long, ctypes.c_long, ctypes.c_double, ip, mp, dp,
                                ctypes.c_double, ctypes.c_double, ctypes.c_long, dp, lp]
        _lib = L
    return _lib


class _CMedium2(ctypes.Structure):
    _fields_ = [("act_lo", ctypes.POINTER(ctypes.c_int)), ("act_hi", ctypes.POINTER(ctypes.c_int)),
                ("drv_lo", ctypes.POINTER(ctypes.c_int)), ("drv_hi", ctypes.POINTER(ctypes.c_int)),
                ("omega", ctypes.c_double), ("amp", ctypes.c_double)]


class Medium2:
    """Map of the active medium and driven cells of a 2D problem: per row j,
    pump on for act_lo[j] <= i < act_hi[j] (None: everywhere), driven cells
    drv_lo[j] <= i < drv_hi[j] (None: none), pulsation omega, amplitude amp."""

    def __init__(self, act_lo=None, act_hi=None, drv_lo=None, drv_hi=None, omega=0.0, amp=0.0):
        conv = lambda a: None if a is None else np.ascontiguousarray(a, dtype=np.intc)
        self.act_lo, self.act_hi = conv(act_lo), conv(act_hi)
        self.drv_lo, self.drv_hi = conv(drv_lo), conv(drv_hi)
        self.omega, self.amp = float(omega), float(amp)

    def c(self) -> _CMedium2:
        ptr = lambda a: None if a is None else a.ctypes.data_as(ctypes.POINTER(ctypes.c_int))
        return _CMedium2(ptr(self.act_lo), ptr(self.act_hi), ptr(self.drv_lo), ptr(self.drv_hi),
                         self.omega, self.amp)


def _dp(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _shape(n) -> tuple[int, ctypes.Array]:
    n = tuple(int(x) for x in (n if hasattr(n, "__len__") else (n,)))
    arr = (ctypes.c_long * 3)(*(list(n) + [1] * (3 - len(n))))
    return len(n), arr


def _vec(u) -> np.ndarray:
    return np.ascontiguousarray(u, dtype=np.float64)


# ---------------------------------------------------------------- pointwise

def pressure(P: Params, u) -> float:
    u = _vec(u)
    return lib().orc_pressure(ctypes.byref(P.c()), len(u) - 3, _dp(u))


def flux(P: Params, u, axis: int = 0) -> np.ndarray:
    u = _vec(u)
    F = np.zeros_like(u)
    lib().orc_flux(ctypes.byref(P.c()), len(u) - 3, axis, _dp(u), _dp(F))
    return F


def source(P: Params, u) -> np.ndarray:
    u = _vec(u)
    Y = np.zeros_like(u)
    lib().orc_source(ctypes.byref(P.c()), len(u) - 3, _dp(u), _dp(Y))
    return Y


def hll(P: Params, uL, uR, axis: int = 0) -> np.ndarray:
    uL, uR = _vec(uL), _vec(uR)
    F = np.zeros_like(uL)
    lib().orc_hll(ctypes.byref(P.c()), len(uL) - 3, axis, _dp(uL), _dp(uR), _dp(F))
    return F


def limiter(kind: int, a: float, b: float) -> float:
    return lib().orc_limiter(kind, a, b)


def physical(P: Params, u) -> bool:
    u = _vec(u)
    return bool(lib().orc_physical(ctypes.byref(P.c()), len(u) - 3, _dp(u)))


# ---------------------------------------------------------------- grid

def step(P: Params, U: np.ndarray, n, h: float, dt: float) -> tuple[np.ndarray, int]:
    """One MUSCL-Hancock step; U is (nf, ncell) field-major.  Returns (Unew, rc)."""
    dim, na = _shape(n)
    U = np.ascontiguousarray(U, dtype=np.float64)
    out = np.empty_like(U)
    rc = lib().orc_step(ctypes.byref(P.c()), dim, na, h, dt, _dp(U), _dp(out))
    return out, rc


def step_cell(P: Params, U: np.ndarray, n, h: float, dt: float, idx: int) -> np.ndarray:
    dim, na = _shape(n)
    U = np.ascontiguousarray(U, dtype=np.float64)
    out = np.empty(dim + 3)
    lib().orc_step_cell(ctypes.byref(P.c()), dim, na, h, dt, _dp(U), int(idx), _dp(out))
    return out


def dt_cfl(P: Params, U: np.ndarray, n, h: float) -> float:
    dim, na = _shape(n)
    U = np.ascontiguousarray(U, dtype=np.float64)
    return lib().orc_dt(ctypes.byref(P.c()), dim, na, h, _dp(U))


def run(P: Params, U: np.ndarray, n, h: float, t_end: float, t0: float = 0.0,
        max_steps: int = 1 << 40) -> tuple[np.ndarray, float, int, int]:
    """Advance to t_end (last step clamped).  Returns (U, t, steps, rc)."""
    dim, na = _shape(n)
    U = np.array(U, dtype=np.float64, order="C", copy=True)
    t = ctypes.c_double()
    k = ctypes.c_long()
    rc = lib().orc_run(ctypes.byref(P.c()), dim, na, h, _dp(U), t0, t_end, max_steps,
                       ctypes.byref(t), ctypes.byref(k))
    return U, t.value, k.value, rc


def threads() -> int:
    return int(lib().orc_threads())


def set_threads(n: int) -> None:
    """OpenMP threads of the array loops (timing only)."""
    lib().orc_set_threads(int(n))


def step_bc1(P: Params, U: np.ndarray, N: int, h: float, dt: float, bc_lo: int, bc_hi: int):
    """One 1D step with boundary conditions (PERIODIC / REFLECT / OUTFLOW per side)."""
    U = np.ascontiguousarray(U, dtype=np.float64)
    out = np.empty_like(U)
    rc = lib().orc_step_bc1(ctypes.byref(P.c()), int(N), h, dt, bc_lo, bc_hi, _dp(U), _dp(out))
    return out, rc


def run_bc1(P: Params, U: np.ndarray, N: int, h: float, t_end: float, bc_lo: int, bc_hi: int,
            t0: float = 0.0, max_steps: int = 1 << 40):
    U = np.array(U, dtype=np.float64, order="C", copy=True)
    t = ctypes.c_double()
    k = ctypes.c_long()
    rc = lib().orc_run_bc1(ctypes.byref(P.c()), int(N), h, bc_lo, bc_hi, _dp(U), t0, t_end,
                           max_steps, ctypes.byref(t), ctypes.byref(k))
    return U, t.value, k.value, rc


def run_driven(P: Params, U: np.ndarray, N: int, h: float, t_end: float, drv: _CDrive,
               bc_hi: int = OUTFLOW, t0: float = 0.0, max_steps: int = 1 << 40):
    """1D run with the driven boundary at x = 0 and bc_hi at x = L."""
    U = np.array(U, dtype=np.float64, order="C", copy=True)
    t = ctypes.c_double()
    k = ctypes.c_long()
    rc = lib().orc_run_bc1d(ctypes.byref(P.c()), int(N), h, DRIVEN, bc_hi, ctypes.byref(drv),
                            _dp(U), t0, t_end, max_steps, ctypes.byref(t), ctypes.byref(k))
    return U, t.value, k.value, rc


def _bc4(bc):
    return (ctypes.c_int * 4)(*[int(b) for b in bc])


def step2m(P: Params, U: np.ndarray, nx: int, ny: int, h: float, dt: float, bc,
           medium: "Medium2 | None" = None, t: float = 0.0):
    """One 2D step with boundaries bc = (x_lo, x_hi, y_lo, y_hi), the medium
    map and driven cells of `medium`, from time t.  Returns (Unew, rc)."""
    U = np.ascontiguousarray(U, dtype=np.float64)
    out = np.empty_like(U)
    m = medium.c() if medium is not None else None
    rc = lib().orc_step2m(ctypes.byref(P.c()), int(nx), int(ny), h, dt, _bc4(bc),
                          ctypes.byref(m) if m is not None else None, t, _dp(U), _dp(out))
    return out, rc


def run2m(P: Params, U: np.ndarray, nx: int, ny: int, h: float, t_end: float, bc,
          medium: "Medium2 | None" = None, t0: float = 0.0, max_steps: int = 1 << 40):
    """2D run to t_end (last step clamped).  Returns (U, t, steps, rc)."""
    U = np.array(U, dtype=np.float64, order="C", copy=True)
    t = ctypes.c_double()
    k = ctypes.c_long()
    m = medium.c() if medium is not None else None
    rc = lib().orc_run2m(ctypes.byref(P.c()), int(nx), int(ny), h, _bc4(bc),
                         ctypes.byref(m) if m is not None else None, _dp(U), t0, t_end, max_steps,
                         ctypes.byref(t), ctypes.byref(k))
    return U, t.value, k.value, rc


def step_heun(P: Params, U: np.ndarray, n, h: float, dt: float):
    """One Heun (SSP-RK2) step of the same spatial operator; periodic grid."""
    dim, na = _shape(n)
    U = np.ascontiguousarray(U, dtype=np.float64)
    out = np.empty_like(U)
    rc = lib().orc_step_heun(ctypes.byref(P.c()), dim, na, h, dt, _dp(U), _dp(out))
    return out, rc


def run_heun(P: Params, U: np.ndarray, n, h: float, t_end: float, t0: float = 0.0,
             max_steps: int = 1 << 40):
    dim, na = _shape(n)
    U = np.array(U, dtype=np.float64, order="C", copy=True)
    t = ctypes.c_double()
    k = ctypes.c_long()
    rc = lib().orc_run_heun(ctypes.byref(P.c()), dim, na, h, _dp(U), t0, t_end, max_steps,
                            ctypes.byref(t), ctypes.byref(k))
    return U, t.value, k.value, rc
