"""The benchmark's multi-rank path on the CPU: two gloo ranks join through
bench.py's own helpers (the GPU arm differs only in using NCCL), take the max
of their timings, aggregate whole-job throughput, and the reference arm's
non-zero rank does no work."""
from __future__ import annotations

import argparse
import importlib.util
import json
import os
import socket

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank: int, world: int, port: int, out_dir: str):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), WORLD_SIZE=str(world),
                      RANK=str(rank), LOCAL_RANK=str(rank))
    bench = _bench()
    args = argparse.Namespace(impl="reference")
    w, r, local = bench.dist_setup(args, backend="gloo")
    bench.barrier(w)
    slowest = bench.max_over_ranks(1.0 + rank, w)          # the ranks' own step times
    total = bench.sum_over_ranks(10.0 * (1 + rank), w)      # the ranks' copied bytes
    value = bench.job_throughput(w, 2.0e12, slowest)        # 2 TFLOP of work on every rank
    reference = bench.run_reference(args, w, r) if r != 0 else "rank 0 not run here"
    bench.barrier(w)
    import torch.distributed as dist
    dist.destroy_process_group()
    with open(os.path.join(out_dir, f"rank{rank}.json"), "w") as f:
        json.dump({"world": w, "rank": r, "slowest": slowest, "value": value, "total": total,
                   "reference": reference}, f)


def test_two_gloo_ranks_take_the_max_and_aggregate(tmp_path):
    world = 2
    mp.start_processes(_rank, args=(world, _free_port(), str(tmp_path)), nprocs=world,
                       start_method="spawn")
    results = [json.load(open(tmp_path / f"rank{r}.json")) for r in range(world)]
    for r, res in enumerate(results):
        assert res["world"] == world and res["rank"] == r
        assert res["slowest"] == 2.0                  # max over ranks of 1.0 and 2.0
        assert res["total"] == 30.0                   # sum over ranks of 10 and 20
        assert res["value"] == pytest.approx(2.0)     # 2 ranks x 2 TFLOP / 2 s
    assert results[1]["reference"] is None            # non-zero ranks exit without work
