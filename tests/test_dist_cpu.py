"""The benchmark's multi-rank plumbing on CPU: two gloo ranks (one process each, as torchrun
launches one per GPU). Each rank times its own batch; the job's time is the slowest rank's and
its throughput counts every rank's units. Ranks draw distinct synthetic batches. The reference
arm does its work on rank 0 only."""
from __future__ import annotations

import json
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), WORLD_SIZE=str(world),
                      RANK=str(rank), LOCAL_RANK=str(rank))
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    w, r, lr = bench.rank_info()
    local_seconds = 1.0 + rank  # rank 1 is the slower one
    slowest = bench.max_over_ranks(local_seconds, w, "cpu")
    rate = bench.job_rate(w, 256 * 10, slowest)
    seed = bench.rank_seed(3000, r)
    # the reference arm returns at once on every rank but 0
    ref = None
    if r != 0:
        import argparse
        ref = bench.run_reference(argparse.Namespace(seed=3000, poses=256, cpu_sample=1, steps=1, warmup=0,
                                                     gpus=w))
    dist.barrier()
    dist.destroy_process_group()
    with open(os.path.join(out_dir, f"rank{rank}.json"), "w") as fh:
        json.dump({"world": w, "rank": r, "local": lr, "slowest": slowest, "rate": rate, "seed": seed,
                   "ref": ref}, fh)


def test_two_gloo_ranks(tmp_path):
    world = 2
    mp.start_processes(_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True,
                       start_method="spawn")
    res = [json.load(open(tmp_path / f"rank{r}.json")) for r in range(world)]
    assert [x["rank"] for x in res] == [0, 1] and all(x["world"] == 2 for x in res)
    assert all(x["slowest"] == 2.0 for x in res)           # both ranks see the slowest time
    assert all(x["rate"] == 2 * 2560 / 2.0 for x in res)   # every rank's units over it
    assert res[0]["seed"] != res[1]["seed"]                # distinct batches
    assert res[1]["ref"] is None
