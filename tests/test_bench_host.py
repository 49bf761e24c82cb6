"""Host-side arithmetic of bench.py that the reported figures rest on, checked without a GPU:
the sampled GEMM's depth after repeated draws are merged, the algorithmic work per stage that the
roofline divides by, the measured-traffic figure, and the workload the line names."""
import argparse
import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import bench  # noqa: E402

torch = pytest.importorskip("torch")


def test_gemm_depth_counts_distinct_draws():
    """Column unit: the number of distinct drawn columns.  Block unit: the columns of the distinct
    drawn blocks (a block drawn twice is one run of n_k columns)."""
    off = np.array([0, 3, 7, 12, 20], dtype=np.int64)  # n_k = 3, 4, 5, 8
    r = {"idx": torch.tensor([5, 1, 5, 5, 19, 0, 1], dtype=torch.int32), "unit": 0}
    assert bench.gemm_depth(r, off) == 4  # {0, 1, 5, 19}
    r = {"idx": torch.tensor([2, 0, 2, 3, 3, 3], dtype=torch.int32), "unit": 1}
    assert bench.gemm_depth(r, off) == 3 + 5 + 8  # blocks {0, 2, 3}


def test_stage_work_of_the_bench_product():
    """The fused statistics pass reads M and N once (FP32) and writes x, y (n each) and five K-long
    block statistics in FP64; the apply's flops are 2 m p times the GEMM's depth."""
    w = bench.WORKLOAD
    nk = np.diff(bench.offsets_of(w))
    work = bench.stage_work(w, 8192, nk, "OPL", depth=6175)
    m, n, p, K = 8192, 65536, 8192, 1024
    assert work["stats_f"]["bytes"] == 4 * (m * n + n * p) + 8 * (2 * n + 5 * K) == 4_296_056_832
    assert work["gram_f"]["bytes"] == 4 * (m * n + n * p)
    assert work["apply"]["flops"] == 2.0 * m * p * 6175
    assert bench.stage_work(w, 8192, nk, "OPL")["apply"]["flops"] == 2.0 * m * p * 8192
    # the measured DRAM bytes of one launch (scaled from the profiling case's m + p = 4096 to 16384)
    # lie within 3% above the algorithmic bytes: no wasted re-reads beyond the windows' edge boxes
    assert 1.0 <= bench.TRAFFIC["stats_f"] / work["stats_f"]["bytes"] < 1.03


def test_bench_workload_is_the_named_configuration():
    """Default bench: M 8192 x 65536, N 65536 x 8192, K = 1024 blocks of 16..128 columns, c = K/8
    blocks, L = c n / K = 8192 draws; the profiling case keeps n, K and the blocks with m = p = 2048."""
    args = argparse.Namespace(small=False, profile_case=False)
    w = bench.workload(args)
    off = bench.offsets_of(w)
    nk = np.diff(off)
    assert (w["m"], w["n"], w["p"], w["K"]) == (8192, 65536, 8192, 1024)
    assert off[0] == 0 and off[-1] == w["n"] and nk.size == w["K"]
    assert nk.min() >= 16 and nk.max() <= 128
    assert w["c_blocks"] == w["K"] // 8
    assert "L=8192 outer products" in bench.workload_name(args)
    prof = bench.workload(argparse.Namespace(small=False, profile_case=True))
    assert (prof["m"], prof["p"]) == (2048, 2048)
    assert np.array_equal(bench.offsets_of(prof), off)
