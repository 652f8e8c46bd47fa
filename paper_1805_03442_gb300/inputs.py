"""Seeded synthetic inputs for the solver and for its tests.

This module holds no arithmetic of the numerical method: it only lays out
initial states (primitive fields turned into the conserved variables of eq. 5)
and draws seeded random numbers.  Both the CUDA path and the CPU oracle take
what it produces as input.

Conserved layout: field-major float64 array of shape (nf, n_z, n_y, n_x)
flattened to (nf, ncell), fields (rho, rho*v_1 .. rho*v_d, E, E_nu),
x fastest.  Cell centres sit at x_j = (j + 1/2) h.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np


def equilibrium_primitive(Ck: float, S: float) -> tuple[float, float, float]:
    """(rho0, p0, e_nu0): rho0 = p0 = 1 and the specific vibrational energy at
    the steady state of the relaxation equation, e_nu0 = C_k + S (R = T0 = 1)."""
    return 1.0, 1.0, Ck + S


def prim_to_cons(gamma: float, rho, vel, p, ev) -> np.ndarray:
    """Primitive (rho, velocity components, p, specific e_nu) -> conserved
    (rho, rho v.., E, E_nu) with E = p/(gamma-1) + rho |v|^2 / 2 + rho e_nu (eq. 5)."""
    rho = np.asarray(rho, dtype=np.float64)
    vel = [np.asarray(v, dtype=np.float64) for v in vel]
    kin = sum(v * v for v in vel)
    Ev = rho * np.asarray(ev, dtype=np.float64)
    E = np.asarray(p, dtype=np.float64) / (gamma - 1.0) + 0.5 * rho * kin + Ev
    out = [rho] + [rho * v for v in vel] + [E, Ev]
    return np.ascontiguousarray(np.stack([np.broadcast_to(a, rho.shape) for a in out]).reshape(len(out), -1))


def cell_centres(n: int, L: float) -> np.ndarray:
    h = L / n
    return (np.arange(n) + 0.5) * h


# ------------------------------------------------------------------ 1D waves

@dataclass
class Mode:
    """One periodic wave: integer wavenumber index m (k = 2 pi m / L), complex
    primitive amplitudes (rho, u, p, e_nu) multiplying exp(i k x), and a scale."""
    m: int
    shape: np.ndarray          # complex (4,): rho, u, p, e_nu
    scale: complex = 1.0


def acoustic_shape(gamma: float, rho0: float = 1.0, p0: float = 1.0) -> np.ndarray:
    """Right-running frozen acoustic wave per unit density amplitude:
    u' = c rho'/rho0, p' = c^2 rho', e_nu' = 0, with c = sqrt(gamma p0 / rho0)."""
    c = math.sqrt(gamma * p0 / rho0)
    return np.array([1.0, c / rho0, c * c, 0.0], dtype=complex)


def waves_1d(gamma: float, N: int, L: float, base, modes: list[Mode]) -> np.ndarray:
    """Conserved (4, N) state: base primitive (rho0, p0, e_nu0) plus sum of modes,
    as point values at cell centres."""
    rho0, p0, ev0 = base
    pert = np.zeros((4, N))
    if all(0 < md.m < N // 2 for md in modes):
        # sum of Re(a e^{i 2 pi m (j + 1/2) / N}) by one inverse real FFT per field
        spec = np.zeros((4, N // 2 + 1), dtype=complex)
        for md in modes:
            shift = np.exp(1j * math.pi * md.m / N)          # cell centres at (j + 1/2) h
            spec[:, md.m] += md.scale * np.asarray(md.shape) * shift * (N / 2.0)
        pert = np.fft.irfft(spec, n=N, axis=1)
    else:
        x = cell_centres(N, L)
        for md in modes:
            ph = np.exp(1j * (2.0 * math.pi * md.m / L) * x)
            for f in range(4):
                pert[f] += np.real(md.scale * md.shape[f] * ph)
    return prim_to_cons(gamma, rho0 + pert[0], [pert[1]], p0 + pert[2], ev0 + pert[3])


def random_phase_modes(seed: int, shape: np.ndarray, n_modes: int, m0: int,
                       amp: float, m_step: int = 1) -> list[Mode]:
    """n_modes waves with m_i = m0 + i*m_step (i = 0..n_modes-1), amplitudes
    amp * m_0 / m_i (a k^-1 spectrum) and seeded uniform random phases."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n_modes):
        m = m0 + i * m_step
        phase = rng.uniform(0.0, 2.0 * math.pi)
        out.append(Mode(m=m, shape=shape, scale=amp * (m0 / m) * np.exp(1j * phase)))
    return out


def double_tube_1d(gamma: float, N: int, L: float, outer, inner) -> np.ndarray:
    """Periodic 'double shock tube': primitive (rho, u, p, e_nu) `outer` for
    x < L/4 or x >= 3L/4 and `inner` in between."""
    x = cell_centres(N, L)
    ins = (x >= 0.25 * L) & (x < 0.75 * L)
    prim = [np.where(ins, inner[f], outer[f]) for f in range(4)]
    return prim_to_cons(gamma, prim[0], [prim[1]], prim[2], prim[3])


def random_states(dim: int, ncell: int, seed: int, gamma: float = 1.4,
                  smooth: bool = False) -> np.ndarray:
    """Random physical states: rho in [0.5, 2], |v_a| <= 0.5, p in [0.5, 2],
    e_nu in [0.1, 1.2].  `smooth` adds a cumulative-sum correlation so that the
    limiter sees both smooth runs and extrema."""
    rng = np.random.default_rng(seed)

    def draw(lo, hi):
        if smooth:
            w = np.cumsum(rng.normal(0.0, 1.0, ncell))
            w = (w - w.min()) / max(w.max() - w.min(), 1e-12)
            return lo + (hi - lo) * w
        return rng.uniform(lo, hi, ncell)

    rho = draw(0.5, 2.0)
    vel = [draw(-0.5, 0.5) for _ in range(dim)]
    p = draw(0.5, 2.0)
    ev = draw(0.1, 1.2)
    return prim_to_cons(gamma, rho, vel, p, ev)


# ------------------------------------------------------------------ batched sweep

@dataclass
class SweepRun:
    N: int
    tau0: float
    S: float
    tau_rho: float
    tau_T: float
    Q_rho: float
    Q_T: float
    I_rho: float
    I_T: float
    m: int
    t_end: float


def sweep_runs(seed: int, nruns: int, n_lo: int = 256, n_hi: int = 16384,
               gamma: float = 1.4, periods: float = 5.0) -> list[SweepRun]:
    """Stability-map sweep: N uniform in [n_lo, n_hi], tau0 log-uniform in
    [1e-3, 1e1], S uniform in [0, 2], exponents tau_rho in [-2, 0],
    tau_T in [-2.5, 0], Q/I exponents in [-1, 1], mode m in 1..8 on L = 1, and
    t_end = `periods` frozen-sound periods of mode m (2 pi / (k c))."""
    rng = np.random.default_rng(seed)
    c = math.sqrt(gamma)
    runs = []
    for _ in range(nruns):
        N = int(rng.integers(n_lo, n_hi + 1))
        m = int(rng.integers(1, 9))
        runs.append(SweepRun(
            N=N, tau0=float(10.0 ** rng.uniform(-3.0, 1.0)), S=float(rng.uniform(0.0, 2.0)),
            tau_rho=float(rng.uniform(-2.0, 0.0)), tau_T=float(rng.uniform(-2.5, 0.0)),
            Q_rho=float(rng.uniform(-1.0, 1.0)), Q_T=float(rng.uniform(-1.0, 1.0)),
            I_rho=float(rng.uniform(-1.0, 1.0)), I_T=float(rng.uniform(-1.0, 1.0)),
            m=m, t_end=periods / (m * c)))
    return runs


# ------------------------------------------------------------------ 2D / 3D

def plane_wave_2d(gamma: float, nx: int, ny: int, L: float, base, mx: int, my: int,
                  amp: float, noise: float, seed: int) -> np.ndarray:
    """Conserved (5, ny*nx): a frozen acoustic plane wave of integer mode
    (mx, my) (direction atan2(my, mx)), density amplitude `amp`, plus seeded
    white noise of relative size `noise` on density and pressure."""
    rho0, p0, ev0 = base
    c = math.sqrt(gamma * p0 / rho0)
    x = cell_centres(nx, L)[None, :]
    y = cell_centres(ny, L)[:, None]
    kx, ky = 2 * math.pi * mx / L, 2 * math.pi * my / L
    kk = math.hypot(kx, ky)
    w = amp * np.cos(kx * x + ky * y)
    rng = np.random.default_rng(seed)
    rho = rho0 + w + noise * rng.standard_normal((ny, nx))
    p = p0 + c * c * w + noise * rng.standard_normal((ny, nx))
    vx = c / rho0 * w * kx / kk
    vy = c / rho0 * w * ky / kk
    return prim_to_cons(gamma, rho, [vx, vy], p, np.full((ny, nx), ev0))


def random_field_3d(gamma: float, n: int, L: float, base, amp: float, seed: int,
                    slope: float = -2.0) -> np.ndarray:
    """Conserved (6, n^3): isotropic seeded random perturbations of density and of
    the three velocity components with power spectrum ~ k^slope, each scaled to
    rms `amp` (velocities in units of the sound speed); pressure follows the
    density adiabatically at first order (p' = c^2 rho')."""
    rho0, p0, ev0 = base
    c = math.sqrt(gamma * p0 / rho0)
    rng = np.random.default_rng(seed)
    k1 = np.fft.fftfreq(n, d=1.0 / n)
    kx, ky, kz = np.meshgrid(k1, k1, np.fft.rfftfreq(n, d=1.0 / n), indexing="ij")
    kk = np.sqrt(kx * kx + ky * ky + kz * kz)
    amp_k = np.where(kk > 0, np.power(np.maximum(kk, 1e-30), slope / 2.0), 0.0)

    def field():
        z = (rng.standard_normal(kk.shape) + 1j * rng.standard_normal(kk.shape)) * amp_k
        f = np.fft.irfftn(z, s=(n, n, n), axes=(0, 1, 2))
        return amp * f / max(np.sqrt(np.mean(f * f)), 1e-300)

    drho = field()
    v = [c * field() for _ in range(3)]
    # axes (i, j, k) of the FFT grid are mapped to (z, y, x): x fastest
    return prim_to_cons(gamma, rho0 + drho, v, p0 + c * c * drho, np.full(drho.shape, ev0))


# ------------------------------------------------------------------ 2D active sector

def row_intervals(mask: np.ndarray) -> tuple[np.ndarray, np.ndarray]:
    """Per row j of a (ny, nx) boolean mask whose true cells are contiguous in
    every row: int32 arrays (lo, hi) with mask[j, lo[j]:hi[j]] the true cells
    (lo = hi = 0 for an empty row).  Raises if a row is not one interval."""
    ny, nx = mask.shape
    lo = np.zeros(ny, dtype=np.int32)
    hi = np.zeros(ny, dtype=np.int32)
    for j in range(ny):
        idx = np.flatnonzero(mask[j])
        if idx.size:
            if idx[-1] - idx[0] + 1 != idx.size:
                raise ValueError(f"row {j} of the mask is not one interval")
            lo[j], hi[j] = idx[0], idx[-1] + 1
    return lo, hi


def sector_maps(nx: int, ny: int, h: float, apex, half_angle: float, r_src: float,
                axis: float = 0.0):
    """The 2D active-sector geometry as per-row cell intervals: the active
    medium is the cells whose centre lies within `half_angle` (radians) of the
    ray from `apex` = (x0, y0) in direction `axis`; the driven source is the
    cells whose centre lies within `r_src` of the apex.  Returns
    (act_lo, act_hi, drv_lo, drv_hi), int32 arrays of ny entries."""
    x = (np.arange(nx) + 0.5) * h
    y = (np.arange(ny) + 0.5) * h
    X, Y = np.meshgrid(x, y)
    dx, dy = X - apex[0], Y - apex[1]
    along = dx * math.cos(axis) + dy * math.sin(axis)
    across = -dx * math.sin(axis) + dy * math.cos(axis)
    active = (along > 0.0) & (np.abs(across) <= math.tan(half_angle) * along)
    driven = dx * dx + dy * dy <= r_src * r_src
    return row_intervals(active) + row_intervals(driven)


def sector_rest_state(gamma: float, Ck: float, S: float, nx: int, ny: int) -> np.ndarray:
    """Conserved (5, ny*nx) rest state rho = p = 1, v = 0, specific vibrational
    energy C_k + S: the steady state of the active medium, and of the frozen
    medium outside it."""
    one = np.ones((ny, nx))
    return prim_to_cons(gamma, one, [0.0 * one, 0.0 * one], one, np.full((ny, nx), Ck + S))


@dataclass
class SectorProblem:
    """The paper's 2D active-sector problem as set up here (Sec. 3; domain,
    source and sizes are not given there): a pulsating source at `apex` on the
    mid-line near the left boundary, the active medium in the 30-degree sector
    opening towards +x (frozen medium elsewhere), a solid wall at x = Lx (G1)
    reached by the front near t = 1, free outflow on the other three sides."""
    nx: int
    ny: int
    h: float
    apex: tuple
    half_angle: float
    r_src: float
    omega: float
    amp: float
    bc: tuple
    maps: tuple


def sector_problem(nx: int, wavelength: float = 0.1, amp: float = 1e-3,
                   gamma: float = 1.4) -> SectorProblem:
    """Domain [0, Lx] x [0, Ly] with Lx = x0 + c0 (t = 1 to reach the wall),
    Ly = Lx, x0 = 2 wavelengths; nx cells across, h = Lx / nx; the source a
    disc of radius wavelength / 4 pulsating at omega = 2 pi c0 / wavelength."""
    c0 = math.sqrt(gamma)
    x0 = 2.0 * wavelength
    Lx = x0 + c0
    h = Lx / nx
    ny = nx
    apex = (x0, 0.5 * ny * h)
    half = math.radians(15.0)
    r_src = 0.25 * wavelength
    maps = sector_maps(nx, ny, h, apex, half, r_src)
    OUT, WALL = 2, 1
    return SectorProblem(nx=nx, ny=ny, h=h, apex=apex, half_angle=half, r_src=r_src,
                         omega=2.0 * math.pi * c0 / wavelength, amp=amp,
                         bc=(OUT, WALL, OUT, OUT), maps=maps)
