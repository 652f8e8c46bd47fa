"""Host logic of the benchmark's roofline objects (no GPU): the DRAM traffic
reported for each 1D launch configuration, and the ALU roofline of the FP64
lines against the FP64 rate derived from GB300's unit counts and clock."""
import os
import sys

import pytest

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import bench  # noqa: E402

TILE3 = "1D: 512-cell block tiles, 2 cells per thread, 78 registers, 3 blocks/SM"
TILE2 = "1D: 512-cell block tiles, 2 cells per thread, 2 blocks/SM"
TILE4 = "1D: 512-cell block tiles, 2 cells per thread, 64 registers, 4 blocks/SM"
WIDE = "1D: 1024-cell block tiles, 4 cells per thread, 2 blocks/SM"
SLIDE = "1D: warps sliding over 64-cell chunks, 2 cells per thread"


def test_traffic_per_configuration():
    n = 1 << 22
    got = {c: bench.traffic_of("1d", n, "fp32", c) for c in (TILE3, TILE2, TILE4, WIDE, SLIDE)}
    assert got[TILE3] == 86.8e6 and got[TILE2] == 87.2e6 and got[TILE4] == 86.5e6
    assert got[SLIDE] == 91.7e6 and got[WIDE] is None        # no capture of the 1024-cell tiles
    # every capture lies between the algorithmic read (67.1 MB) and read + write (134.2 MB)
    alg = 2 * 4 * 4 * n
    assert all(alg / 2 < v < alg for v in got.values() if v is not None)
    # other workloads, sizes and precisions report null
    assert bench.traffic_of("1d", n // 2, "fp32", TILE3) is None
    assert bench.traffic_of("1d", n, "fp32_ps", TILE3) is None
    assert bench.traffic_of("2d", n, "fp32", TILE3) is None


def test_fp64_roofline():
    # 2 FMA lanes per SM per clock x 2 flops x 152 SMs x 2.07 GHz
    assert bench.FP64_PEAK_TFLOPS == pytest.approx(1.25856, rel=1e-12)
    r = bench.fp64_roofline(1, 1 << 22, 3.59e-3, 0.011)
    assert r["bound"] == "alu" and r["unit"] == "TFLOP/s" and r["traffic"] is None
    assert r["flops_per_launch"] == pytest.approx(681.4 * (1 << 22))
    assert r["achieved"] == pytest.approx(681.4 * (1 << 22) / 3.59e-3 / 1e12)
    assert r["frac"] == pytest.approx(r["achieved"] / r["peak"]) and 0 < r["frac"] < 1
    # flops per cell grow with the dimension (more fluxes, more fields)
    f = bench.FP64_FLOPS_PER_CELL
    assert f[1] < f[2] < f[3]
