"""ctypes binding of libsv.so (include/sv.h): argument marshalling only.

Every step of the solver runs in the library's CUDA kernels.  PyTorch is used
for device memory (the solver's device block is a torch uint8 tensor) and for
the stream the work is enqueued on.  There is no CPU fallback: if libsv.so is
missing or no CUDA device is present, constructing a Solver raises.
"""
from __future__ import annotations

import ctypes
import math
import os
from dataclasses import dataclass, fields

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libsv.so")

SV_OK, SV_EINVAL, SV_ENOMEM, SV_ECUDA, SV_ENONPHYS, SV_EDT, SV_EMAXSTEPS = 0, -1, -2, -3, -4, -5, -7
SV_ESIZE, SV_ESTALL = -8, -9
NOALLOC_MAX_CELLS = (1 << 29) - 1
FLAG_NONPHYS, FLAG_DT, FLAG_MAXSTEPS, FLAG_STALL = 1, 2, 4, 8
LAUNCH_AUTO, LAUNCH_PER_STEP, LAUNCH_PERSISTENT = 0, 1, 2
MINMOD, VANLEER, MC = 0, 1, 2
FP32, FP64, FP32_P64, FP32_PC, FP32_PS = 0, 1, 2, 3, 4
BC_PERIODIC, BC_REFLECT, BC_OUTFLOW, BC_DRIVEN = 0, 1, 2, 3
HANCOCK, HEUN = 0, 1

EXPORTS = ("sv_required_bytes", "sv_init", "sv_write_state", "sv_read_state", "sv_dt_cfl",
           "sv_step", "sv_run_to", "sv_time", "sv_conservation", "sv_status",
           "sv_state_device", "sv_free", "sv_strerror", "sv_batch_required_bytes",
           "sv_batch_init", "sv_batch_reset", "sv_batch_run", "sv_batch_sync", "sv_batch_read",
           "sv_batch_mode_log", "sv_batch_free", "sv_step1d_noalloc", "sv_set_drive",
           "sv_set_launch", "sv_get_launch", "sv_set_wait_limit", "sv_measure_fp64_peak",
           "sv_write_state_f32", "sv_read_state_f32", "sv_num_configs", "sv_get_config", "sv_config_desc",
           "sv_set_config", "sv_autotune", "sv_batch_num_configs", "sv_batch_set_config",
           "sv_batch_get_config", "sv_set_medium2d")


class SvError(RuntimeError):
    def __init__(self, code: int, what: str):
        self.code = code
        super().__init__(f"{what}: {code} ({strerror(code)})")


class _Params(ctypes.Structure):
    _fields_ = [(n, ctypes.c_double) for n in
                ("gamma", "Ck", "S", "tau0", "tau_rho", "tau_T", "Q_rho", "Q_T", "I_rho", "I_T",
                 "cfl", "c_tau")] + [("limiter", ctypes.c_int), ("precision", ctypes.c_int),
                                     ("method", ctypes.c_int)]


class _Run(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("L", ctypes.c_double), ("t_end", ctypes.c_double),
                ("S", ctypes.c_double), ("tau0", ctypes.c_double), ("tau_rho", ctypes.c_double),
                ("tau_T", ctypes.c_double), ("Q_rho", ctypes.c_double), ("Q_T", ctypes.c_double),
                ("I_rho", ctypes.c_double), ("I_T", ctypes.c_double), ("mode", ctypes.c_int)]


class _Drive(ctypes.Structure):
    _fields_ = [("omega", ctypes.c_double), ("k_re", ctypes.c_double), ("k_im", ctypes.c_double),
                ("base", ctypes.c_double * 4), ("amp_re", ctypes.c_double * 4),
                ("amp_im", ctypes.c_double * 4)]


class _Grid(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int), ("n", ctypes.c_int64 * 3), ("L", ctypes.c_double * 3),
                ("bc", ctypes.c_int * 4)]


class _Medium2d(ctypes.Structure):
    _fields_ = [("active_lo", ctypes.POINTER(ctypes.c_int32)),
                ("active_hi", ctypes.POINTER(ctypes.c_int32)),
                ("driven_lo", ctypes.POINTER(ctypes.c_int32)),
                ("driven_hi", ctypes.POINTER(ctypes.c_int32)),
                ("omega", ctypes.c_double), ("amp", ctypes.c_double)]


@dataclass
class Params:
    """sv_params.  Defaults: gamma 1.4, C_k 0.1, tau_rho -1, tau_T -1.5, Q/I
    exponents 0 (the 1D runs of the paper), S 1, tau0 0.08, CFL 0.4."""
    gamma: float = 1.4
    Ck: float = 0.1
    S: float = 1.0
    tau0: float = 0.08
    tau_rho: float = -1.0
    tau_T: float = -1.5
    Q_rho: float = 0.0
    Q_T: float = 0.0
    I_rho: float = 0.0
    I_T: float = 0.0
    cfl: float = 0.4
    c_tau: float = 0.5
    limiter: int = MINMOD
    precision: int = FP32
    method: int = HANCOCK

    def c(self) -> _Params:
        return _Params(*[getattr(self, f.name) for f in fields(self)])


_lib = None


def lib() -> ctypes.CDLL:
    """Load libsv.so (built by paper_1805_03442_gb300.build); raises if absent."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is not built; run paper_1805_03442_gb300.build.build()")
    L = ctypes.CDLL(LIB_PATH)
    vp, dp = ctypes.c_void_p, ctypes.POINTER(ctypes.c_double)
    L.sv_required_bytes.argtypes = [ctypes.POINTER(_Params), ctypes.POINTER(_Grid),
                                    ctypes.POINTER(ctypes.c_size_t)]
    L.sv_init.argtypes = [ctypes.POINTER(_Params), ctypes.POINTER(_Grid), vp, vp, ctypes.c_size_t,
                          ctypes.POINTER(vp)]
    L.sv_write_state.argtypes = [vp, dp, ctypes.c_double]
    L.sv_read_state.argtypes = [vp, dp, dp]
    fp = ctypes.POINTER(ctypes.c_float)
    L.sv_write_state_f32.argtypes = [vp, fp, ctypes.c_double]
    L.sv_read_state_f32.argtypes = [vp, fp, dp]
    L.sv_dt_cfl.argtypes = [vp, dp]
    L.sv_step.argtypes = [vp, ctypes.c_int64]
    L.sv_run_to.argtypes = [vp, ctypes.c_double, ctypes.c_int64, ctypes.POINTER(ctypes.c_int64)]
    L.sv_time.argtypes = [vp, dp, ctypes.POINTER(ctypes.c_int64)]
    L.sv_conservation.argtypes = [vp, dp]
    L.sv_status.argtypes = [vp, ctypes.POINTER(ctypes.c_uint32)]
    L.sv_state_device.argtypes = [vp, ctypes.POINTER(vp), ctypes.POINTER(ctypes.c_int)]
    L.sv_free.argtypes = [vp]
    L.sv_free.restype = None
    L.sv_strerror.argtypes = [ctypes.c_int]
    L.sv_strerror.restype = ctypes.c_char_p
    rp = ctypes.POINTER(_Run)
    L.sv_batch_required_bytes.argtypes = [ctypes.POINTER(_Params), rp, ctypes.c_int64, ctypes.c_int,
                                          ctypes.POINTER(ctypes.c_size_t)]
    L.sv_batch_init.argtypes = [ctypes.POINTER(_Params), rp, ctypes.c_int64, dp, ctypes.c_int,
                                ctypes.c_int64, vp, vp, ctypes.c_size_t, ctypes.POINTER(vp)]
    L.sv_batch_reset.argtypes = [vp, dp]
    L.sv_batch_run.argtypes = [vp]
    L.sv_batch_sync.argtypes = [vp]
    L.sv_batch_read.argtypes = [vp, ctypes.c_int64, dp, dp, ctypes.POINTER(ctypes.c_int64),
                                ctypes.POINTER(ctypes.c_uint32)]
    L.sv_batch_mode_log.argtypes = [vp, ctypes.c_int64, dp, dp, dp, ctypes.c_int64,
                                    ctypes.POINTER(ctypes.c_int64)]
    L.sv_batch_free.argtypes = [vp]
    L.sv_batch_free.restype = None
    L.sv_set_drive.argtypes = [vp, ctypes.POINTER(_Drive)]
    L.sv_set_launch.argtypes = [vp, ctypes.c_int]
    L.sv_set_wait_limit.argtypes = [vp, ctypes.c_int]
    L.sv_measure_fp64_peak.argtypes = [vp, ctypes.POINTER(ctypes.c_double)]
    L.sv_set_medium2d.argtypes = [vp, ctypes.POINTER(_Medium2d)]
    L.sv_get_launch.argtypes = [vp, ctypes.POINTER(ctypes.c_int)]
    ip = ctypes.POINTER(ctypes.c_int)
    L.sv_num_configs.argtypes = [vp, ip]
    L.sv_get_config.argtypes = [vp, ip, ctypes.c_char_p, ctypes.c_size_t]
    L.sv_config_desc.argtypes = [vp, ctypes.c_int, ctypes.c_char_p, ctypes.c_size_t]
    L.sv_set_config.argtypes = [vp, ctypes.c_int]
    L.sv_autotune.argtypes = [vp, ctypes.c_int, ip, dp]
    L.sv_batch_num_configs.argtypes = [vp, ip]
    L.sv_batch_set_config.argtypes = [vp, ctypes.c_int]
    L.sv_batch_get_config.argtypes = [vp, ip, ctypes.c_char_p, ctypes.c_size_t]
    L.sv_step1d_noalloc.argtypes = [ctypes.POINTER(_Params), ctypes.c_int64, ctypes.c_double, vp, vp,
                                    dp, ctypes.POINTER(ctypes.c_uint32), vp]
    _lib = L
    return L


def strerror(code: int) -> str:
    try:
        return lib().sv_strerror(code).decode()
    except RuntimeError:
        return "?"


def _check(rc: int, what: str) -> int:
    if rc != SV_OK:
        raise SvError(rc, what)
    return rc


def _dp(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def grid(n, L=None, bc=(BC_PERIODIC, BC_PERIODIC)) -> _Grid:
    """sv_grid for cells per axis n, lengths L (default: h = 1 / n[0]) and
    boundary conditions bc = (x_lo, x_hi) or (x_lo, x_hi, y_lo, y_hi)."""
    n = tuple(int(x) for x in (n if hasattr(n, "__len__") else (n,)))
    if L is None:
        L = tuple(float(x) / n[0] for x in n)          # h = 1 / n[0]
    L = tuple(float(x) for x in (L if hasattr(L, "__len__") else (L,)))
    g = _Grid()
    g.dim = len(n)
    for a in range(3):
        g.n[a] = n[a] if a < len(n) else 1
        g.L[a] = L[a] if a < len(L) else 1.0
    bc = tuple(int(b) for b in bc) + (BC_PERIODIC,) * (4 - len(bc))
    for i in range(4):
        g.bc[i] = bc[i]
    return g


def step1d_noalloc(params: Params, n: int, L: float, u_in: int, u_out: int, stream=None,
                   wait: bool = True):
    """sv_step1d_noalloc: one 1D step from the caller's device buffer u_in to
    u_out (device addresses, 4 * n elements of the params' precision), for
    callers that cannot allocate device memory.  Returns (dt taken, flags)
    when `wait`, else None (asynchronous)."""
    import torch
    st = stream if stream is not None else torch.cuda.current_stream()
    dt, fl = ctypes.c_double(), ctypes.c_uint32()
    rc = lib().sv_step1d_noalloc(ctypes.byref(params.c()), int(n), float(L), ctypes.c_void_p(u_in),
                                 ctypes.c_void_p(u_out), ctypes.byref(dt) if wait else None,
                                 ctypes.byref(fl) if wait else None,
                                 ctypes.c_void_p(st.cuda_stream))
    _check(rc, "sv_step1d_noalloc")
    return (dt.value, fl.value) if wait else None


def measure_fp64_peak(stream=None) -> float:
    """sv_measure_fp64_peak: the device's FP64 FMA throughput in TFLOP/s (the
    roofline denominator of the FP64 step kernels)."""
    import torch
    st = stream if stream is not None else torch.cuda.current_stream()
    out = ctypes.c_double()
    _check(lib().sv_measure_fp64_peak(ctypes.c_void_p(st.cuda_stream), ctypes.byref(out)),
           "sv_measure_fp64_peak")
    return out.value


class Solver:
    """One periodic grid advanced by the fused MUSCL-Hancock kernels.

    n: cells per axis (tuple of 1-3 ints), L: lengths per axis (equal cell size).
    memory="torch" backs the solver's device block by a torch uint8 tensor;
    memory="library" lets libsv allocate it.  stream: a torch.cuda.Stream, or
    None for torch's current stream.  bc: boundary conditions (BC_*) at x = 0
    and x = L of a 1D grid."""

    def __init__(self, params: Params, n, L=None, stream=None, memory: str = "torch",
                 bc=(BC_PERIODIC, BC_PERIODIC)):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("no CUDA device: the solver has no CPU path")
        self.params = params
        self.g = grid(n, L, bc)
        self.dim = self.g.dim
        self.n = tuple(self.g.n[a] for a in range(self.dim))
        self.nf = self.dim + 3
        self.ncell = int(np.prod(self.n))
        self._stream = stream if stream is not None else torch.cuda.current_stream()
        pc = params.c()
        nbytes = ctypes.c_size_t()
        _check(lib().sv_required_bytes(ctypes.byref(pc), ctypes.byref(self.g), ctypes.byref(nbytes)),
               "sv_required_bytes")
        self.device_bytes = nbytes.value
        self._mem = None
        dev_ptr = None
        if memory == "torch":
            self._mem = torch.empty(self.device_bytes, dtype=torch.uint8, device="cuda")
            dev_ptr = self._mem.data_ptr()
        h = ctypes.c_void_p()
        _check(lib().sv_init(ctypes.byref(pc), ctypes.byref(self.g),
                             ctypes.c_void_p(self._stream.cuda_stream), dev_ptr,
                             self.device_bytes, ctypes.byref(h)), "sv_init")
        self._h = h

    # ------------------------------------------------------------ lifecycle
    def close(self):
        if getattr(self, "_h", None):
            lib().sv_free(self._h)
            self._h = None
        self._mem = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # ------------------------------------------------------------ I/O
    def write_state(self, U: np.ndarray, t: float = 0.0):
        U = np.ascontiguousarray(U, dtype=np.float64).reshape(self.nf, self.ncell)
        _check(lib().sv_write_state(self._h, _dp(U), float(t)), "sv_write_state")

    def write_state_ptr(self, host_ptr: int, t: float = 0.0):
        """Upload from a host address (e.g. a pinned torch tensor's data_ptr)."""
        _check(lib().sv_write_state(self._h, ctypes.cast(host_ptr, ctypes.POINTER(ctypes.c_double)),
                                    float(t)), "sv_write_state")

    def read_state(self) -> tuple[np.ndarray, float]:
        U = np.empty((self.nf, self.ncell))
        t = ctypes.c_double()
        _check(lib().sv_read_state(self._h, _dp(U), ctypes.byref(t)), "sv_read_state")
        return U, t.value

    def read_state_ptr(self, host_ptr: int) -> float:
        t = ctypes.c_double()
        _check(lib().sv_read_state(self._h, ctypes.cast(host_ptr, ctypes.POINTER(ctypes.c_double)),
                                   ctypes.byref(t)), "sv_read_state")
        return t.value

    # float host buffers (sv_write_state_f32 / sv_read_state_f32): half the bytes
    def write_state_f32(self, U: np.ndarray, t: float = 0.0):
        U = np.ascontiguousarray(U, dtype=np.float32).reshape(self.nf, self.ncell)
        _check(lib().sv_write_state_f32(self._h, U.ctypes.data_as(ctypes.POINTER(ctypes.c_float)),
                                        float(t)), "sv_write_state_f32")

    def read_state_f32(self) -> tuple[np.ndarray, float]:
        U = np.empty((self.nf, self.ncell), dtype=np.float32)
        t = ctypes.c_double()
        _check(lib().sv_read_state_f32(self._h, U.ctypes.data_as(ctypes.POINTER(ctypes.c_float)),
                                       ctypes.byref(t)), "sv_read_state_f32")
        return U, t.value

    def write_state_ptr_f32(self, host_ptr: int, t: float = 0.0):
        _check(lib().sv_write_state_f32(self._h, ctypes.cast(host_ptr, ctypes.POINTER(ctypes.c_float)),
                                        float(t)), "sv_write_state_f32")

    def read_state_ptr_f32(self, host_ptr: int) -> float:
        t = ctypes.c_double()
        _check(lib().sv_read_state_f32(self._h, ctypes.cast(host_ptr, ctypes.POINTER(ctypes.c_float)),
                                       ctypes.byref(t)), "sv_read_state_f32")
        return t.value

    # ------------------------------------------------------------ stepping
    def dt(self) -> float:
        d = ctypes.c_double()
        _check(lib().sv_dt_cfl(self._h, ctypes.byref(d)), "sv_dt_cfl")
        return d.value

    def step(self, nsteps: int = 1):
        _check(lib().sv_step(self._h, int(nsteps)), "sv_step")

    def run_to(self, t_end: float, max_steps: int = 1 << 62, check: bool = True) -> tuple[int, int]:
        k = ctypes.c_int64()
        rc = lib().sv_run_to(self._h, float(t_end), int(max_steps), ctypes.byref(k))
        if check and rc not in (SV_OK,):
            raise SvError(rc, "sv_run_to")
        return rc, k.value

    def set_drive(self, omega: float, k: complex, base, amp):
        """Driven boundary (bc[0] = BC_DRIVEN): ghost cells at x < 0 hold
        base + Re(amp e^{i(k x - omega t)}) (conserved variables)."""
        d = _Drive()
        d.omega, d.k_re, d.k_im = float(omega), float(complex(k).real), float(complex(k).imag)
        for f in range(4):
            d.base[f] = float(base[f])
            d.amp_re[f] = float(complex(amp[f]).real)
            d.amp_im[f] = float(complex(amp[f]).imag)
        _check(lib().sv_set_drive(self._h, ctypes.byref(d)), "sv_set_drive")

    def set_medium2d(self, active_lo=None, active_hi=None, driven_lo=None, driven_hi=None,
                     omega: float = 0.0, amp: float = 0.0):
        """2D medium map (per row j: active medium for active_lo[j] <= i <
        active_hi[j], frozen elsewhere; None: active everywhere) and driven
        cells (per row: driven_lo[j] <= i < driven_hi[j] hold the pulsating
        source of amplitude amp and angular frequency omega; None: none)."""
        keep = []

        def ptr(a):
            if a is None:
                return None
            a = np.ascontiguousarray(a, dtype=np.int32)
            keep.append(a)
            return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))
        m = _Medium2d(ptr(active_lo), ptr(active_hi), ptr(driven_lo), ptr(driven_hi),
                      float(omega), float(amp))
        _check(lib().sv_set_medium2d(self._h, ctypes.byref(m)), "sv_set_medium2d")

    def set_launch(self, mode: int):
        """LAUNCH_AUTO, LAUNCH_PER_STEP or LAUNCH_PERSISTENT (1D MUSCL-Hancock)."""
        _check(lib().sv_set_launch(self._h, int(mode)), "sv_set_launch")

    def set_wait_limit(self, polls: int):
        """sv_set_wait_limit: the persistent loop's barrier waits give up after
        `polls` polls (0: the default limit); a failure-path test hook."""
        _check(lib().sv_set_wait_limit(self._h, int(polls)), "sv_set_wait_limit")

    @property
    def launch(self) -> int:
        """The launch mode the next steps use (LAUNCH_PER_STEP or LAUNCH_PERSISTENT)."""
        m = ctypes.c_int()
        _check(lib().sv_get_launch(self._h, ctypes.byref(m)), "sv_get_launch")
        return m.value

    # ------------------------------------------------------------ launch configurations
    def configs(self) -> list[str]:
        """Descriptions of the solver's launch configurations (same results,
        different speed)."""
        n = ctypes.c_int()
        _check(lib().sv_num_configs(self._h, ctypes.byref(n)), "sv_num_configs")
        out = []
        for i in range(n.value):
            buf = ctypes.create_string_buffer(256)
            _check(lib().sv_config_desc(self._h, i, buf, 256), "sv_config_desc")
            out.append(buf.value.decode())
        return out

    @property
    def config(self) -> int:
        i = ctypes.c_int()
        _check(lib().sv_get_config(self._h, ctypes.byref(i), None, 0), "sv_get_config")
        return i.value

    def set_config(self, index: int):
        _check(lib().sv_set_config(self._h, int(index)), "sv_set_config")

    def autotune(self, steps: int = 10, cold: bool = False) -> tuple[int, list[float]]:
        """Time every configuration on the current state (restored after each
        trial) and keep the fastest; cold: each timed step after an L2-evicting
        write.  Returns (index, microseconds per step of each configuration)."""
        n = len(self.configs())
        us = (ctypes.c_double * n)()
        best = ctypes.c_int()
        k = -int(steps) if cold else int(steps)
        _check(lib().sv_autotune(self._h, k, ctypes.byref(best), us), "sv_autotune")
        return best.value, list(us)

    def time(self) -> tuple[float, int]:
        t, k = ctypes.c_double(), ctypes.c_int64()
        _check(lib().sv_time(self._h, ctypes.byref(t), ctypes.byref(k)), "sv_time")
        return t.value, k.value

    def conservation(self) -> np.ndarray:
        out = np.empty(self.nf)
        _check(lib().sv_conservation(self._h, _dp(out)), "sv_conservation")
        return out

    def status(self) -> int:
        f = ctypes.c_uint32()
        _check(lib().sv_status(self._h, ctypes.byref(f)), "sv_status")
        return f.value

    def state_device(self):
        """(device pointer, element bytes) of the current state buffer."""
        p, e = ctypes.c_void_p(), ctypes.c_int()
        _check(lib().sv_state_device(self._h, ctypes.byref(p), ctypes.byref(e)), "sv_state_device")
        return p.value, e.value


class Batch:
    """A batched sweep of independent 1D periodic runs, advanced by one
    persistent launch (sv_batch_*).

    runs: sequence of objects with attributes n, L (optional, default 1),
    t_end, S, tau0, tau_rho, tau_T, Q_rho, Q_T, I_rho, I_T, m (logged mode);
    states: list of (4, n) float64 initial states in the same order.
    `params` supplies gamma, C_k, cfl, c_tau, limiter and precision."""

    def __init__(self, params: Params, runs, states, log_cap: int = 64,
                 max_steps: int = 10 ** 6, stream=None, memory: str = "torch"):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("no CUDA device: the batch has no CPU path")
        self.params = params
        self.nruns = len(runs)
        arr = (_Run * self.nruns)()
        for i, r in enumerate(runs):
            arr[i] = _Run(int(r.n), float(getattr(r, "L", 1.0)), float(r.t_end), float(r.S),
                          float(r.tau0), float(r.tau_rho), float(r.tau_T), float(r.Q_rho),
                          float(r.Q_T), float(r.I_rho), float(r.I_T), int(getattr(r, "m", 0)))
        self._runs = arr
        self.n = [int(r.n) for r in runs]
        self.log_cap = int(log_cap)
        self._stream = stream if stream is not None else torch.cuda.current_stream()
        host = self._concat(states)
        pc = params.c()
        nbytes = ctypes.c_size_t()
        _check(lib().sv_batch_required_bytes(ctypes.byref(pc), arr, self.nruns, self.log_cap,
                                             ctypes.byref(nbytes)), "sv_batch_required_bytes")
        self.device_bytes = nbytes.value
        self._mem = None
        dev_ptr = None
        if memory == "torch":
            self._mem = torch.empty(self.device_bytes, dtype=torch.uint8, device="cuda")
            dev_ptr = self._mem.data_ptr()
        h = ctypes.c_void_p()
        _check(lib().sv_batch_init(ctypes.byref(pc), arr, self.nruns, _dp(host), self.log_cap,
                                   int(max_steps), ctypes.c_void_p(self._stream.cuda_stream),
                                   dev_ptr, self.device_bytes, ctypes.byref(h)), "sv_batch_init")
        self._h = h
        self._initial = host

    def reset_initial(self):
        """Upload the initial states given at construction again (times, step
        counts and flags back to zero)."""
        _check(lib().sv_batch_reset(self._h, _dp(self._initial)), "sv_batch_reset")

    def _concat(self, states) -> np.ndarray:
        parts = []
        for U, n in zip(states, self.n):
            U = np.asarray(U, dtype=np.float64).reshape(4, n)
            parts.append(U.reshape(-1))
        return np.ascontiguousarray(np.concatenate(parts))

    def close(self):
        if getattr(self, "_h", None):
            lib().sv_batch_free(self._h)
            self._h = None
        self._mem = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def reset(self, states):
        host = self._concat(states)
        _check(lib().sv_batch_reset(self._h, _dp(host)), "sv_batch_reset")

    def configs(self) -> list[str]:
        """Descriptions of the batch's launch configurations (block size per run)."""
        n = ctypes.c_int()
        _check(lib().sv_batch_num_configs(self._h, ctypes.byref(n)), "sv_batch_num_configs")
        cur = self.config
        out = []
        for i in range(n.value):
            _check(lib().sv_batch_set_config(self._h, i), "sv_batch_set_config")
            buf = ctypes.create_string_buffer(256)
            _check(lib().sv_batch_get_config(self._h, None, buf, 256), "sv_batch_get_config")
            out.append(buf.value.decode())
        _check(lib().sv_batch_set_config(self._h, cur), "sv_batch_set_config")
        return out

    @property
    def config(self) -> int:
        i = ctypes.c_int()
        _check(lib().sv_batch_get_config(self._h, ctypes.byref(i), None, 0), "sv_batch_get_config")
        return i.value

    def set_config(self, index: int):
        _check(lib().sv_batch_set_config(self._h, int(index)), "sv_batch_set_config")

    def run(self):
        _check(lib().sv_batch_run(self._h), "sv_batch_run")

    def sync(self):
        _check(lib().sv_batch_sync(self._h), "sv_batch_sync")

    def read(self, i: int, state: bool = True):
        U = np.empty((4, self.n[i])) if state else None
        t, k, f = ctypes.c_double(), ctypes.c_int64(), ctypes.c_uint32()
        _check(lib().sv_batch_read(self._h, i, _dp(U) if state else None, ctypes.byref(t),
                                   ctypes.byref(k), ctypes.byref(f)), "sv_batch_read")
        return U, t.value, k.value, f.value

    def mode_log(self, i: int):
        cap = self.log_cap
        t, re, im = np.empty(cap), np.empty(cap), np.empty(cap)
        c = ctypes.c_int64()
        _check(lib().sv_batch_mode_log(self._h, i, _dp(t), _dp(re), _dp(im), cap, ctypes.byref(c)),
               "sv_batch_mode_log")
        n = c.value
        return t[:n], re[:n] + 1j * im[:n]
