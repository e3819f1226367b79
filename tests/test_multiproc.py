"""The multi-rank path of bench.py on CPU: two gloo ranks (torch.distributed,
127.0.0.1).  The method has no exchange step, so ranks are replicas; what must
hold is the job-level bookkeeping -- the slowest rank sets the time (max over
ranks), work adds up over ranks, every rank meets the barriers, and only rank
0 runs the reference arm's oracle and prints."""
from __future__ import annotations

import json
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank: int, world: int, port: int, out_dir: str) -> None:
    os.environ.update({"RANK": str(rank), "LOCAL_RANK": str(rank), "WORLD_SIZE": str(world),
                       "MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port)})
    sys.path.insert(0, ROOT)
    import bench

    w, r, local = bench.dist_env()
    dist = bench.init_dist(w, "gloo")
    assert dist is not None and dist.get_world_size() == world and r == rank and local == rank
    per_rank_ms = [3.0, 5.0][rank]
    bench.barrier(dist)
    slowest = bench.reduce_max(dist, per_rank_ms)
    total = bench.reduce_sum(dist, 10.0 * (rank + 1))
    bench.barrier(dist)
    # rank != 0 leaves the reference arm at once, without touching the oracle
    ret = None
    if rank == 1:
        class A:  # bench's argparse namespace, minimal
            workload, steps, warmup = "grid2d_256", 1, 3
        ret = bench.reference_arm(A)
    with open(os.path.join(out_dir, f"rank{rank}.json"), "w") as f:
        json.dump({"slowest": slowest, "total": total, "ret": ret}, f)
    dist.destroy_process_group()


def test_two_gloo_ranks(tmp_path):
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp

    port = _free_port()
    mp.spawn(_rank_main, args=(2, port, str(tmp_path)), nprocs=2, join=True)
    got = [json.load(open(tmp_path / f"rank{r}.json")) for r in range(2)]
    for g in got:
        assert g["slowest"] == 5.0  # max over ranks: the slowest rank's time
        assert g["total"] == 30.0   # work summed over ranks
    assert got[1]["ret"] == 0        # non-zero ranks exit the reference arm with status 0
