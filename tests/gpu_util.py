"""Helpers shared by the GPU tests: build-once fixtures and error measures."""
import numpy as np
import pytest


def need_gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1805_03442_gb300 import build
    build.build()
    from paper_1805_03442_gb300 import sv
    return sv


def rel_linf(a: np.ndarray, b: np.ndarray) -> float:
    """max over fields of max|a - b| / max(max|b|, 1).

    Every field is either O(1) (density, total and vibrational energy) or a
    perturbation driven by O(1) fluxes (momentum, whose flux carries p ~ 1), so
    errors are measured against max(|field|, 1): rounding in an O(1) flux shows
    up at the same absolute level in every field."""
    a = np.asarray(a).reshape(a.shape[0], -1)
    b = np.asarray(b).reshape(b.shape[0], -1)
    out = 0.0
    for f in range(b.shape[0]):
        scale = max(np.max(np.abs(b[f])), 1.0)
        out = max(out, float(np.max(np.abs(a[f] - b[f])) / scale))
    return out


def field_rel_linf(a: np.ndarray, b: np.ndarray, floor: float = 1e-6) -> dict:
    """Per field f: max|a_f - b_f| / max|b_f|, the error relative to the
    field's own size, for every field whose max|b_f| >= floor (a momentum
    field of a small wave is gated on its own scale this way, not on the O(1)
    scale that rel_linf uses).  Returns {field index: error}."""
    a = np.asarray(a).reshape(a.shape[0], -1)
    b = np.asarray(b).reshape(b.shape[0], -1)
    out = {}
    for f in range(b.shape[0]):
        scale = float(np.max(np.abs(b[f])))
        if scale >= floor:
            out[f] = float(np.max(np.abs(a[f] - b[f])) / scale)
    return out


def assert_fp64_parity(a: np.ndarray, b: np.ndarray, tol: float = 1e-12,
                       small_tol: float = 1e-9, o1: float = 0.1) -> None:
    """FP64 GPU against the FP64 oracle, two ways:
    * rel_linf <= tol: every field's error on the O(1) scale of the fluxes
      that update it;
    * each field relative to its own size (field_rel_linf, fields >= 1e-6):
      <= tol for fields of size >= o1, <= small_tol for smaller ones.  A small
      field -- the momentum of a 1e-3 wave -- is updated by an O(1) flux
      (m^2/rho + p with p ~ 1) whose rounding (~1e-16 per step) it takes on at
      its own scale: over K steps about K 1e-16 / max|m|, e.g. 2e-10 for the
      6000-step linear-stage run with max|m| = 1.3e-3."""
    r = rel_linf(a, b)
    assert r <= tol, f"rel_linf {r:.3e} > {tol:.0e}"
    bb = np.asarray(b).reshape(b.shape[0], -1)
    for f, e in field_rel_linf(a, b).items():
        lim = tol if np.max(np.abs(bb[f])) >= o1 else small_tol
        assert e <= lim, f"field {f}: {e:.3e} of its own size > {lim:.0e}"


def primitives(U: np.ndarray, dim: int, gamma: float = 1.4) -> dict:
    rho = U[0]
    vel = [U[1 + a] / rho for a in range(dim)]
    kin = sum(U[1 + a] * v for a, v in enumerate(vel))
    p = (gamma - 1.0) * (U[1 + dim] - 0.5 * kin - U[2 + dim])
    return {"rho": rho, "v": vel[0], "p": p, "ev": U[2 + dim] / rho}


def oracle_params(P, **over):
    """The oracle's parameter record with the same values as an sv.Params."""
    from oracle import orc as O
    d = dict(gamma=P.gamma, Ck=P.Ck, S=P.S, tau0=P.tau0, tau_rho=P.tau_rho, tau_T=P.tau_T,
             Q_rho=P.Q_rho, Q_T=P.Q_T, I_rho=P.I_rho, I_T=P.I_T, cfl=P.cfl, c_tau=P.c_tau,
             limiter=P.limiter)
    d.update(over)
    return O.Params(**d)
