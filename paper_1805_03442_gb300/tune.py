"""Autotuner for the launch configurations of the solver kernels.

Every solver kernel comes in a few launch configurations that compute bitwise
the same states and differ only in speed (``sv.h``: block-tile register budget
or sliding warps in 1D, planes per block in 2D/3D, block size per run in the
batched sweep).  This module picks one by timing them on the device and
remembers the choice in a JSON cache, keyed by the device and by the problem's
class (dimension, precision, limiter, source variant, grid size to the nearest
power of two), so that later solvers of the same class start tuned.

Cache layout::

    {"<device>": {"<key>": {"config": "<description>", "us": [..], "when": <unix time>}}}

The description, not the index, is stored: if the library's list of
configurations changes, a stale entry no longer matches and is tuned again.
"""
from __future__ import annotations

import json
import math
import os
import time

_HERE = os.path.dirname(os.path.abspath(__file__))
DEFAULT_CACHE = os.path.join(_HERE, "_build", "tune_cache.json")


def device_name() -> str:
    """Name and compute capability of the current CUDA device."""
    import torch
    i = torch.cuda.current_device()
    major, minor = torch.cuda.get_device_capability(i)
    return f"{torch.cuda.get_device_name(i)} sm_{major}{minor}"


def source_kind(params) -> str:
    """The source variant the kernels compile for these parameters."""
    if math.isinf(params.tau0):
        return "frozen"
    if params.Q_rho == params.Q_T == params.I_rho == params.I_T == 0.0:
        return "qi0"
    return "general"


def solver_key(params, n) -> str:
    """Problem class of a solver: dimension, precision, method, limiter, source
    variant and log2 of the cell count (rounded)."""
    n = tuple(int(x) for x in (n if hasattr(n, "__len__") else (n,)))
    cells = 1
    for x in n:
        cells *= x
    return (f"solver/{len(n)}d/prec{params.precision}/method{params.method}/lim{params.limiter}/"
            f"{source_kind(params)}/2^{round(math.log2(max(cells, 1)))}")


def batch_key(params) -> str:
    return f"batch/prec{params.precision}/lim{params.limiter}"


class Cache:
    """The JSON file of tuned choices (created on first store)."""

    def __init__(self, path: str | None = None):
        self.path = path or DEFAULT_CACHE
        self.data: dict = {}
        if os.path.exists(self.path):
            try:
                with open(self.path) as f:
                    self.data = json.load(f)
            except (OSError, ValueError):
                self.data = {}

    def get(self, device: str, key: str) -> dict | None:
        return self.data.get(device, {}).get(key)

    def put(self, device: str, key: str, config: str, us: list[float]):
        self.data.setdefault(device, {})[key] = {
            "config": config, "us": [None if not math.isfinite(u) else u for u in us],
            "when": time.time()}
        os.makedirs(os.path.dirname(os.path.abspath(self.path)), exist_ok=True)
        tmp = self.path + ".tmp"
        with open(tmp, "w") as f:
            json.dump(self.data, f, indent=1, sort_keys=True)
        os.replace(tmp, self.path)


def tune_solver(solver, key: str, device: str, cache: Cache | None = None, steps: int = 10,
                force: bool = False, cold: bool = False) -> dict:
    """Give `solver` the cached configuration of its class, or time all of its
    configurations (``solver.autotune``) and cache the fastest.  cold: time
    each step after an L2-evicting write (its own cache entry, key + "/cold"),
    for runs measured that way.  Returns
    ``{"config": description, "index": i, "us": [...], "cached": bool}``."""
    cache = cache or Cache()
    if cold:
        key = key + "/cold"
    descs = solver.configs()
    hit = None if force else cache.get(device, key)
    if hit is not None and hit.get("config") in descs:
        i = descs.index(hit["config"])
        solver.set_config(i)
        return {"config": descs[i], "index": i, "us": hit.get("us"), "cached": True}
    if len(descs) == 1:
        solver.set_config(0)
        return {"config": descs[0], "index": 0, "us": None, "cached": False}
    best, us = solver.autotune(steps, cold=True) if cold else solver.autotune(steps)
    cache.put(device, key, descs[best], us)
    return {"config": descs[best], "index": best, "us": us, "cached": False}


def tune_batch(make_batch, key: str, device: str, cache: Cache | None = None,
               force: bool = False) -> dict:
    """Choose the batch launch configuration.  `make_batch()` returns a fresh
    small batch (a sample of the real runs with shortened end times) whose
    ``run()`` / ``sync()`` are timed once per configuration.  Returns
    ``{"config": description, "index": i, "us": [...], "cached": bool}``; the
    index is for the caller's own batch, whose configurations are the same."""
    cache = cache or Cache()
    hit = None if force else cache.get(device, key)
    with make_batch() as b:
        descs = b.configs()
        if hit is not None and hit.get("config") in descs:
            return {"config": hit["config"], "index": descs.index(hit["config"]),
                    "us": hit.get("us"), "cached": True}
        times = []
        for i in range(len(descs)):
            b.set_config(i)
            b.reset_initial()
            b.run()
            b.sync()                     # warm-up: graph capture and first launch
            b.reset_initial()
            t0 = time.perf_counter()
            b.run()
            b.sync()
            times.append(1e6 * (time.perf_counter() - t0))
    best = min(range(len(times)), key=lambda i: times[i])
    cache.put(device, key, descs[best], times)
    return {"config": descs[best], "index": best, "us": times, "cached": False}
