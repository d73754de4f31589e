"""The N > 1 path of bench.py on the CPU: world-size-2 gloo ranks.

Nothing is sharded (replicas only): each rank simulates its own seed's batch, and the
only collective is the timing's barrier and max over ranks.  These tests run the same
helpers bench.py uses under torchrun, with the gloo backend instead of NCCL.
"""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port), "WORLD_SIZE": str(world),
                       "RANK": str(rank), "LOCAL_RANK": str(rank), "BENCH_BACKEND": "gloo"})
    sys.path.insert(0, ROOT)
    import numpy as np
    import torch.distributed as dist

    import bench
    from paper_2208_14567_gb300 import inputs as I
    w, r, local = bench.dist_setup()
    bench.barrier(w)
    m = bench.max_over_ranks(float(10 * (r + 1)), w, "cpu")
    batch = I.dyad_batch(64, 6, 8, seed=r)  # the per-rank workload of the bench
    sums = [None] * w
    dist.all_gather_object(sums, float(np.asarray(batch.pos, dtype=np.float64).sum()))
    with open(os.path.join(out_dir, f"rank{r}.json"), "w") as f:
        json.dump({"world": w, "rank": r, "local": local, "max": m, "pos_sums": sums}, f)
    dist.destroy_process_group()


def test_rank_helpers_two_gloo_ranks(tmp_path):
    """dist_setup, barrier and max_over_ranks on two ranks: every rank reads the maximum,
    and the ranks' batches differ (weak scaling: each rank adds its own work)."""
    import torch.multiprocessing as mp
    port = free_port()
    mp.start_processes(_rank_main, args=(2, port, str(tmp_path)), nprocs=2, start_method="spawn")
    res = [json.load(open(tmp_path / f"rank{r}.json")) for r in range(2)]
    for r, d in enumerate(res):
        assert d["world"] == 2 and d["rank"] == r and d["local"] == r
        assert d["max"] == 20.0
    assert res[0]["pos_sums"] == res[1]["pos_sums"]
    assert res[0]["pos_sums"][0] != res[0]["pos_sums"][1]


def test_reference_arm_under_torchrun_prints_once(tmp_path):
    """bench.py --impl reference launched as the harness launches it for N = 2 (torchrun,
    rendezvous on 127.0.0.1): rank 0 alone times the oracle and prints one JSON line, the
    other rank exits 0 without work."""
    pytest.importorskip("torch")
    env = dict(os.environ, BENCH_BACKEND="gloo", OMP_NUM_THREADS="1")
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(free_port()), os.path.join(ROOT, "bench.py"),
           "--impl", "reference", "--gpus", "2", "--steps", "2", "--warmup", "3", "--ref-sample", "2000"]
    r = subprocess.run(cmd, cwd=str(tmp_path), env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1, r.stdout
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["value"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["e2e"]["h2d_bytes_per_step"] == 0
    # the reference arm describes the same configuration as the GPU arm's line
    sys.path.insert(0, ROOT)
    import bench
    args = type("A", (), {"T": 200, "config": 3, "headline_batch": 0})()
    assert d["config"] == bench.config_dict(bench.headline_config(args), args, 2)
    assert d["steps"] == 2 and d["ms_per_step"] > 0
