"""Host logic of the autotuner (paper_1805_03442_gb300/tune.py): cache keys,
cache hits and misses, stale entries, and the batch chooser, against fake
solvers and batches (no GPU)."""
import json
import math

from paper_1805_03442_gb300 import tune
from paper_1805_03442_gb300.sv import Params, FP64, VANLEER


class FakeSolver:
    def __init__(self, descs, times, cold_times=None):
        self.descs, self.times = descs, times
        self.cold_times = cold_times or times
        self.config, self.tuned = 0, 0

    def configs(self):
        return list(self.descs)

    def set_config(self, i):
        assert 0 <= i < len(self.descs)
        self.config = i

    def autotune(self, steps, cold=False):
        self.tuned += 1
        self.cold = cold
        times = self.cold_times if cold else self.times
        best = min(range(len(times)), key=lambda i: times[i])
        self.config = best
        return best, list(times)


class FakeBatch:
    """Context manager whose run() time is set by its configuration."""
    cost = {0: 3e-3, 1: 1e-3}

    def __init__(self, log):
        self.log, self.cfg = log, 0

    def __enter__(self):
        return self

    def __exit__(self, *a):
        return False

    def configs(self):
        return ["batch A", "batch B"]

    def set_config(self, i):
        self.cfg = i

    def reset_initial(self):
        self.log.append(("reset", self.cfg))

    def run(self):
        import time
        time.sleep(self.cost[self.cfg])
        self.log.append(("run", self.cfg))

    def sync(self):
        pass


def test_keys_separate_problem_classes():
    P = Params()
    assert tune.source_kind(P) == "qi0"
    assert tune.source_kind(Params(tau0=math.inf)) == "frozen"
    assert tune.source_kind(Params(Q_rho=0.5)) == "general"
    k1 = tune.solver_key(P, (1 << 22,))
    assert k1.startswith("solver/1d/") and k1.endswith("/2^22")
    assert tune.solver_key(P, (3000000,)) == k1            # same power of two
    assert tune.solver_key(P, (1 << 20,)) != k1
    assert tune.solver_key(Params(precision=FP64), (1 << 22,)) != k1
    assert tune.solver_key(Params(limiter=VANLEER), (1 << 22,)) != k1
    assert tune.solver_key(P, (64, 64)).startswith("solver/2d/")
    assert tune.batch_key(P) != tune.batch_key(Params(precision=FP64))


def test_miss_then_hit(tmp_path):
    path = tmp_path / "c.json"
    s = FakeSolver(["a", "b", "c"], [5.0, 2.0, 3.0])
    r = tune.tune_solver(s, "k", "dev", tune.Cache(str(path)))
    assert r == {"config": "b", "index": 1, "us": [5.0, 2.0, 3.0], "cached": False}
    assert s.tuned == 1 and s.config == 1
    stored = json.loads(path.read_text())
    assert stored["dev"]["k"]["config"] == "b"
    # a new solver of the same class takes the stored choice without timing
    s2 = FakeSolver(["a", "b", "c"], [5.0, 2.0, 3.0])
    r2 = tune.tune_solver(s2, "k", "dev", tune.Cache(str(path)))
    assert r2["cached"] and r2["index"] == 1 and s2.tuned == 0 and s2.config == 1
    # another device or class is tuned on its own
    s3 = FakeSolver(["a", "b", "c"], [1.0, 2.0, 3.0])
    assert not tune.tune_solver(s3, "k", "dev2", tune.Cache(str(path)))["cached"]
    assert s3.config == 0


def test_stale_entry_is_retuned(tmp_path):
    path = tmp_path / "c.json"
    c = tune.Cache(str(path))
    c.put("dev", "k", "old config that no longer exists", [1.0])
    s = FakeSolver(["x", "y"], [4.0, 1.0])
    r = tune.tune_solver(s, "k", "dev", tune.Cache(str(path)))
    assert not r["cached"] and r["config"] == "y" and s.tuned == 1
    assert json.loads(path.read_text())["dev"]["k"]["config"] == "y"


def test_force_and_single_config(tmp_path):
    path = tmp_path / "c.json"
    s = FakeSolver(["a", "b"], [2.0, 1.0])
    tune.tune_solver(s, "k", "dev", tune.Cache(str(path)))
    s.times = [0.5, 1.0]
    r = tune.tune_solver(s, "k", "dev", tune.Cache(str(path)), force=True)
    assert r["index"] == 0 and s.tuned == 2
    one = FakeSolver(["only"], [1.0])
    r1 = tune.tune_solver(one, "k1", "dev", tune.Cache(str(path)))
    assert r1["index"] == 0 and one.tuned == 0          # nothing to choose, nothing timed


def test_infinite_times_stored_as_null(tmp_path):
    path = tmp_path / "c.json"
    s = FakeSolver(["a", "b"], [math.inf, 1.0])
    tune.tune_solver(s, "k", "dev", tune.Cache(str(path)))
    assert json.loads(path.read_text())["dev"]["k"]["us"] == [None, 1.0]


def test_corrupt_cache_is_ignored(tmp_path):
    path = tmp_path / "c.json"
    path.write_text("{not json")
    s = FakeSolver(["a", "b"], [2.0, 1.0])
    assert tune.tune_solver(s, "k", "dev", tune.Cache(str(path)))["index"] == 1


def test_batch_chooser(tmp_path):
    path = tmp_path / "c.json"
    log = []
    r = tune.tune_batch(lambda: FakeBatch(log), "bk", "dev", tune.Cache(str(path)))
    assert r["config"] == "batch B" and r["index"] == 1 and not r["cached"]
    # each configuration: reset, warm-up run, reset, timed run
    assert [e for e in log if e[0] == "run"] == [("run", 0), ("run", 0), ("run", 1), ("run", 1)]
    log.clear()
    r2 = tune.tune_batch(lambda: FakeBatch(log), "bk", "dev", tune.Cache(str(path)))
    assert r2["cached"] and r2["index"] == 1 and not log


def test_cold_tuning_has_its_own_entry(tmp_path):
    """Tuning with L2 flushed before every step (the benchmark's conditions) is
    cached apart from back-to-back tuning, and each keeps its own pick."""
    path = tmp_path / "c.json"
    descs = ["tiles", "sliding"]
    s = FakeSolver(descs, [2.0, 1.0], cold_times=[1.0, 2.0])
    warm = tune.tune_solver(s, "k", "dev", tune.Cache(str(path)))
    assert warm["config"] == "sliding" and not s.cold
    cold = tune.tune_solver(s, "k", "dev", tune.Cache(str(path)), cold=True)
    assert cold["config"] == "tiles" and s.cold and not cold["cached"]
    data = json.loads(path.read_text())["dev"]
    assert data["k"]["config"] == "sliding" and data["k/cold"]["config"] == "tiles"
    s2 = FakeSolver(descs, [5.0, 5.0])
    assert tune.tune_solver(s2, "k", "dev", tune.Cache(str(path)), cold=True)["config"] == "tiles"
    assert s2.tuned == 0
