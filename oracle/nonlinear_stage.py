"""The nonlinear stage of the one-wavelength eigenmode run, on the oracle.

TEST INFRASTRUCTURE ONLY (a study of the oracle's own solutions; the product
path never imports it).

The run: one wavelength on L = 1, the growing acoustic eigenmode of eq. 8 at
amplitude 1e-4 on the uniform equilibrium (gamma 1.4, C_k 0.1, tau_rho -1,
tau_T -1.5, Q/I exponents 0, S = 1, tau0 = 0.08: the parameters of the
paper's 1D runs, Sec. 3), advanced for up to 20 wave periods.  The question is
whether what happens after the linear growth -- shock formation and then the
loss of positivity (p < 0) that ends every run of these parameters -- is a
property of the model's solution or of the scheme: it is the model's if the
time of that collapse and the shock statistics before it converge as the
scheme's free choices change (CFL number, the source time-step factor c_tau,
the limiter, the grid).

For each setting the oracle runs to t = 5, t = 10 and then to 20 periods or
to the step that leaves the physical range (the oracle's step returns
non-zero), and reports at t = 5 and t = 10 the shocks of the velocity field
(count, mean spacing, mean velocity jump, mean max pressure ratio across
them), max rho, min p, and the collapse time.

    python oracle/nonlinear_stage.py [--quick] [--jobs J]
    python oracle/nonlinear_stage.py --golden tests/golden/nonlinear_stage.json

--quick runs the N = 1024 settings only; --golden writes the statistics of
the two settings the GPU comparison uses (minmod and van Leer, N = 1024,
CFL 0.4).  Each setting runs in its own
process (spawned, one oracle thread each).
"""
from __future__ import annotations

import argparse
import itertools
import json
import math
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def shocks(U: np.ndarray, gamma: float = 1.4, thresh: float = 0.05) -> dict:
    """Shocks of a periodic 1D state: maximal runs of faces where the velocity
    drops by more than thresh / 10 per cell, kept if the whole run drops by
    more than thresh.  Returns count, mean spacing (in units of L = 1), mean
    velocity jump and mean pressure ratio across them."""
    N = U.shape[1]
    rho, m, E, Ev = U
    u = m / rho
    p = (gamma - 1.0) * (E - 0.5 * m * u - Ev)
    du = np.roll(u, -1) - u                   # face j + 1/2
    steep = du < -thresh / 10.0
    if steep.all() or not steep.any():
        return {"count": 0, "spacing": None, "jump": None, "p_ratio": None}
    start = int(np.argmin(steep))             # a face that is not steep: runs do not wrap
    order = [(start + i) % N for i in range(N)]
    runs, cur = [], []
    for j in order:
        if steep[j]:
            cur.append(j)
        elif cur:
            runs.append(cur)
            cur = []
    if cur:
        runs.append(cur)
    found = []
    for r in runs:
        jump = float(np.sum(du[r]))
        if jump < -thresh:
            a, b = r[0], (r[-1] + 1) % N          # cells before and after the run
            centre = (r[0] + 0.5 * len(r)) % N
            found.append((centre, -jump, float(max(p[a], p[b]) / min(p[a], p[b]))))
    if not found:
        return {"count": 0, "spacing": None, "jump": None, "p_ratio": None}
    c = sorted(x[0] for x in found)
    gaps = [(c[(i + 1) % len(c)] - c[i]) % N or N for i in range(len(c))]
    return {"count": len(found), "spacing": float(np.mean(gaps)) / N,
            "jump": float(np.mean([x[1] for x in found])),
            "p_ratio": float(np.mean([x[2] for x in found]))}


def snapshot(U: np.ndarray, gamma: float = 1.4) -> dict:
    rho, m, E, Ev = U
    p = (gamma - 1.0) * (E - 0.5 * m * m / rho - Ev)
    out = shocks(U, gamma)
    out.update({"max_rho": float(np.max(rho)), "min_p": float(np.min(p)),
                "max_u": float(np.max(np.abs(m / rho)))})
    return out


def run_setting(setting: dict) -> dict:
    from oracle import dispersion as D
    from oracle import orc as O
    from paper_1805_03442_gb300 import inputs
    O.set_threads(1)
    N, cfl, c_tau, lim = setting["N"], setting["cfl"], setting["c_tau"], setting["limiter"]
    P = O.Params(tau0=0.08, S=1.0, cfl=cfl, c_tau=c_tau, limiter=lim)
    k = 2 * math.pi
    w = D.growing_acoustic_root(P, k)
    md = D.eigenmode(P, k, w)
    U = inputs.waves_1d(P.gamma, N, 1.0, inputs.equilibrium_primitive(P.Ck, P.S),
                        [inputs.Mode(m=1, shape=md["prim"], scale=1e-4)])
    t_end = 20 * 2 * math.pi / w.real
    out = dict(setting)
    out["t_end"] = t_end
    t, steps = 0.0, 0
    for mark in (5.0, 10.0, t_end):
        U, t, n, rc = O.run(P, U, N, 1.0 / N, mark, t0=t)
        steps += n
        if rc != 0:
            out["collapse_t"] = t
            out["steps"] = steps
            out["at_collapse"] = snapshot(U, P.gamma)
            return out
        if mark < t_end:
            out[f"t{int(mark)}"] = snapshot(U, P.gamma)
    out["collapse_t"] = None
    out["steps"] = steps
    out["at_end"] = snapshot(U, P.gamma)
    return out


SETTINGS = [dict(N=N, cfl=cfl, c_tau=ct, limiter=lim)
            for N, cfl, ct, lim in itertools.product((1024, 2048), (0.4, 0.2), (0.5, 0.1), (0, 1))]


# the settings whose oracle statistics tests/golden/nonlinear_stage.json holds
GOLDEN = [dict(N=1024, cfl=0.4, c_tau=0.5, limiter=0), dict(N=1024, cfl=0.4, c_tau=0.5, limiter=1)]


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--quick", action="store_true")
    ap.add_argument("--jobs", type=int, default=os.cpu_count() or 1)
    ap.add_argument("--json", default="")
    ap.add_argument("--golden", default="",
                    help="write the oracle's statistics of the GOLDEN settings to this file")
    a = ap.parse_args(argv)
    todo = [s for s in SETTINGS if not a.quick or s["N"] == 1024]
    if a.golden:
        todo = GOLDEN
    import concurrent.futures as cf
    import multiprocessing as mp
    with cf.ProcessPoolExecutor(max_workers=a.jobs, mp_context=mp.get_context("spawn")) as ex:
        res = list(ex.map(run_setting, todo))
    if a.golden:
        with open(a.golden, "w") as f:
            json.dump({"source": "oracle/nonlinear_stage.py --golden (FP64 oracle, one thread)",
                       "setup": "one-wavelength growing eigenmode of eq. 8, amplitude 1e-4, N = "
                                "1024, tau0 0.08, S 1, the paper's Sec. 3 parameters",
                       "runs": res}, f, indent=1)
        return
    names = {0: "minmod", 1: "van Leer"}
    print("| N | CFL | c_tau | limiter | collapse t | shocks t=5 (count / spacing / jump) "
          "| shocks t=10 (count / spacing / jump) | max rho t=10 |")
    print("|---|---|---|---|---|---|---|---|")

    def fmt(s):
        if not s or not s.get("count"):
            return "0"
        return f"{s['count']} / {s['spacing']:.3f} / {s['jump']:.3f}"
    for r in res:
        ct = f"{r['collapse_t']:.3f}" if r["collapse_t"] is not None else "none"
        print(f"| {r['N']} | {r['cfl']} | {r['c_tau']} | {names[r['limiter']]} | {ct} | "
              f"{fmt(r.get('t5'))} | {fmt(r.get('t10'))} | "
              f"{r.get('t10', {}).get('max_rho', float('nan')):.3f} |")
    if a.json:
        with open(a.json, "w") as f:
            json.dump(res, f, indent=1)


if __name__ == "__main__":
    main()
