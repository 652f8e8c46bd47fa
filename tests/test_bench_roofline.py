"""Host logic of the benchmark's roofline objects (no GPU): the DRAM traffic
reported for each 1D launch configuration and the 3D line, and the ALU roofline of the FP64
lines against the FP64 rate the library's probe measures."""
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
    assert got[TILE3] == 89.7e6 and got[TILE2] == 89.9e6 and got[TILE4] == 90.0e6
    assert got[SLIDE] == 91.6e6 and got[WIDE] == 86.2e6
    # back to back the launch moves nearly the algorithmic bytes (its own write-back included)
    assert 0.9 < bench.TRAFFIC_B2B_1D_FP32_N22 / (2 * 4 * 4 * n) <= 1.0
    # every capture lies between the algorithmic read (67.1 MB) and read + write (134.2 MB)
    alg = 2 * 4 * 4 * n
    assert all(alg / 2 < v < alg for v in got.values() if v is not None)
    # other workloads, sizes and precisions report null
    assert bench.traffic_of("1d", n // 2, "fp32", TILE3) is None
    assert bench.traffic_of("1d", n, "fp32_ps", TILE3) is None
    assert bench.traffic_of("2d", n, "fp32", TILE3) is None


def test_traffic_3d():
    """The 3D FP32 line at 512^3 reports the capture of its 128-plane
    segments: more than the algorithmic 48 B per cell (halo columns and rows
    read by two tiles), less than half again as much; other segment lengths,
    sizes and precisions report null."""
    n = 512 ** 3
    seg128 = "2D/3D: marching segments of 128 planes per block"
    v = bench.traffic_of("3d", n, "fp32", seg128)
    assert v == 7567.1e6 and 1.0 < v / (2 * 6 * 4 * n) < 1.5
    assert bench.traffic_of("3d", n, "fp32", "2D/3D: marching segments of 256 planes per block") is None
    assert bench.traffic_of("3d", 256 ** 3, "fp32", seg128) is None
    assert bench.traffic_of("3d", n, "fp32_pc", seg128) is None


def test_fp64_roofline():
    peak = 1.2524                                # TFLOP/s, as the probe measures it on GB300
    r = bench.fp64_roofline(1, 1 << 22, 2.31e-3, 0.017, peak)
    assert r["bound"] == "alu" and r["unit"] == "TFLOP/s" and r["traffic"] is None
    assert r["peak"] == peak and "measured" in r["peak_src"]
    assert r["flops_per_launch"] == pytest.approx(422.9 * (1 << 22))
    assert r["achieved"] == pytest.approx(422.9 * (1 << 22) / 2.31e-3 / 1e12)
    assert r["frac"] == pytest.approx(r["achieved"] / r["peak"]) and 0 < r["frac"] < 1
    # flops per cell grow with the dimension (more fluxes, more fields)
    f = bench.FP64_FLOPS_PER_CELL
    assert f[1] < f[2] < f[3]
