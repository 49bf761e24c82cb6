"""The N > 1 path on the CPU: replicas over torch.distributed with the gloo backend, two ranks.

bench.py --gpus N runs one independent product per rank per step (no collective on the data path):
the ranks share only a barrier around the timed region and the maximum of their elapsed times, and
each rank draws its data with seed + 1000 * rank and its sample with stream id (rank << 8) | purpose.
These tests run that host logic as two gloo processes (127.0.0.1) and check it against one process.
"""
import json
import os
import socket
import subprocess
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
torch = pytest.importorskip("torch")


def _free_port():
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _replica_worker(rank, world, port, outdir):
    sys.path.insert(0, ROOT)
    import torch.distributed as dist

    import bench
    import oracle
    import synthetic as S
    from paper_2105_04940_gb300 import pipeline as PL

    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        bench.barrier(world)
        # the timed value: the slowest rank's elapsed time
        elapsed = bench.max_over_ranks(10.0 * (rank + 1), world, torch.device("cpu"))
        # this rank's product: data seed + 1000 * rank, sample stream (rank << 8) | MAIN
        w = bench.SMALL
        off = bench.offsets_of(w)
        M, N = S.scaled_gaussian(32, w["n"], 32, off, w["sigma"], seed=w["data_seed"] + 1000 * rank)
        sid = PL.stream_id(rank, oracle.PURPOSE_MAIN)
        x, y = oracle.col_row_sq_norms(M, N)
        st = oracle.block_stats(x, y, off)
        p = oracle.p_col_opt(st["w"], st["a"], off)
        ck = oracle.apportion(oracle.g_hat(st["a"]), np.diff(off), 256)
        idx, _ = oracle.sample_alg2(p, off, ck, seed=7, sid=sid)
        np.save(os.path.join(outdir, f"idx{rank}.npy"), idx)
        with open(os.path.join(outdir, f"r{rank}.json"), "w") as fh:
            json.dump({"elapsed": elapsed, "sid": sid, "m00": float(M[0, 0])}, fh)
        bench.barrier(world)
    finally:
        dist.destroy_process_group()


def test_two_gloo_replicas(tmp_path):
    import torch.multiprocessing as mp

    port = _free_port()
    mp.start_processes(_replica_worker, args=(2, port, str(tmp_path)), nprocs=2, join=True, start_method="spawn")
    r = [json.load(open(tmp_path / f"r{k}.json")) for k in range(2)]
    idx = [np.load(tmp_path / f"idx{k}.npy") for k in range(2)]
    # both ranks see the maximum elapsed time
    assert r[0]["elapsed"] == r[1]["elapsed"] == 20.0
    # independent replicas: different data and different sample streams
    assert r[0]["sid"] != r[1]["sid"]
    assert r[0]["m00"] != r[1]["m00"]
    assert not np.array_equal(idx[0], idx[1])
    # a replica's draws do not depend on the number of ranks: rank 1's stream alone gives the same
    sys.path.insert(0, ROOT)
    import bench
    import oracle
    import synthetic as S
    from paper_2105_04940_gb300 import pipeline as PL
    w = bench.SMALL
    off = bench.offsets_of(w)
    M, N = S.scaled_gaussian(32, w["n"], 32, off, w["sigma"], seed=w["data_seed"] + 1000)
    x, y = oracle.col_row_sq_norms(M, N)
    st = oracle.block_stats(x, y, off)
    p = oracle.p_col_opt(st["w"], st["a"], off)
    ck = oracle.apportion(oracle.g_hat(st["a"]), np.diff(off), 256)
    alone, _ = oracle.sample_alg2(p, off, ck, seed=7, sid=PL.stream_id(1, oracle.PURPOSE_MAIN))
    np.testing.assert_array_equal(alone, idx[1])


def test_reference_arm_under_torchrun_two_ranks():
    """bench.py --impl reference launched like the multi-GPU bench: rank 0 alone prints one line."""
    port = _free_port()
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(port), os.path.join(ROOT, "bench.py"),
           "--impl", "reference", "--gpus", "2", "--small", "--steps", "1", "--warmup", "0"]
    env = dict(os.environ, OMP_NUM_THREADS="1")
    r = subprocess.run(cmd, capture_output=True, text=True, timeout=600, cwd=ROOT, env=env)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    out = json.loads(lines[0])
    assert out["impl"] == "reference" and out["n_gpus"] == 2
    assert out["cpu_baseline"]["kind"] == "oracle" and out["value"] > 0
