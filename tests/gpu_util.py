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
