"""The multi-rank paths of bench.py on the CPU: two gloo ranks for the
max-over-ranks timing and the per-rank shards, and the reference arm under
torchrun (rank 0 prints the one JSON line, the other rank exits quietly)."""
import json
import os
import socket
import subprocess
import sys

import numpy as np
import torch
import torch.distributed as tdist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _ranks(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    tdist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        t = bench.max_over_ranks(10.0 * (rank + 1), tdist, torch.device("cpu"))
        tree, A2, lam, Q, Ef = bench.make_workload(32, rank)
        shard = torch.from_numpy(np.concatenate([A2.ravel(), Ef.ravel()]))
        shards = [torch.empty_like(shard) for _ in range(world)]
        tdist.all_gather(shards, shard)
        out[rank] = (t, bool(torch.equal(shards[0], shards[1])), float(np.abs(tree.p).sum()))
    finally:
        tdist.destroy_process_group()


def test_two_gloo_ranks_take_the_max_time_and_own_shards():
    world = 2
    with mp.get_context("spawn").Manager() as man:
        out = man.dict()
        mp.spawn(_ranks, args=(world, free_port(), out), nprocs=world, join=True)
        res = dict(out)
    assert res[0][0] == res[1][0] == 20.0          # both ranks see the slowest time
    assert res[0][1] is False                      # shards differ by rank
    assert res[0][2] == res[1][2]                  # the same tree everywhere
    assert bench.job_value(2, 1 << 20, 10, 2000.0) == 2 * (1 << 20) * 10 / 2.0


def test_reference_arm_prints_one_line_on_rank_zero():
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(free_port()), os.path.join(ROOT, "bench.py"),
           "--impl", "reference", "--gpus", "2", "--steps", "1", "--warmup", "3", "--ref-points", "4",
           "--points", "64"]
    r = subprocess.run(cmd, capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [x for x in r.stdout.splitlines() if x.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["value"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["e2e"]["h2d_bytes_per_step"] == 0
