"""Row-partitioned gemm (one process per GPU, rank r computing rows [r0, r1)
of C with B replicated; the paper's row-block distribution, Section III-C,
with no exchange since a row of C reads only its own row of A): the
partition's host logic, and the path over two gloo ranks on the CPU, where
each rank computes its block with the FP64 oracle standing in for its GPU
and the blocks are gathered and compared with the whole product."""
from __future__ import annotations

import json
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

from paper_1804_10694_gb300.partition import TILE_ROWS, row_blocks


@pytest.mark.parametrize("M", [0, 1, 255, 256, 257, 1060, 4099, 8192, 10 * 256 + 3])
@pytest.mark.parametrize("world", [1, 2, 3, 4, 8])
def test_blocks_cover_rows_once_on_tile_edges(M, world):
    blocks = row_blocks(M, world)
    assert len(blocks) == world
    cursor = 0
    for r0, r1 in blocks:
        assert r0 == cursor and r1 >= r0          # contiguous, in rank order
        assert r0 % TILE_ROWS == 0 or r0 == M     # starts on a tile edge
        cursor = r1
    assert cursor == M                            # every row exactly once
    tiles = [-(-(r1 - r0) // TILE_ROWS) for r0, r1 in blocks]
    assert max(tiles) - min(tiles) <= 1           # balanced to within one tile


def test_blocks_reject_bad_arguments():
    with pytest.raises(ValueError):
        row_blocks(100, 0)
    with pytest.raises(ValueError):
        row_blocks(-1, 2)


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank: int, world: int, port: int, out_dir: str):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), WORLD_SIZE=str(world),
                      RANK=str(rank), LOCAL_RANK=str(rank))
    import torch
    import torch.distributed as dist
    import oracle
    import workloads as W
    dist.init_process_group("gloo")
    M, N, K = 1300, 96, 200
    # every rank draws the same inputs (B replicated; A and C whole, each rank
    # reads only its rows)
    A, B, C0 = W.uniform(M, K, 71), W.uniform(K, N, 72), W.uniform(M, N, 73)
    r0, r1 = row_blocks(M, world)[rank]
    mine = oracle.gemm_f64(r1 - r0, N, K, 1.5, np.ascontiguousarray(A[r0:r1]), B, 0.5,
                           np.ascontiguousarray(C0[r0:r1]))
    # gather the blocks (padded to the largest) on every rank
    rows = max(b - a for a, b in row_blocks(M, world))
    pad = np.zeros((rows, N))
    pad[:r1 - r0] = mine
    parts = [torch.zeros(rows, N, dtype=torch.float64) for _ in range(world)]
    dist.all_gather(parts, torch.from_numpy(pad))
    whole = np.concatenate([p.numpy()[:b - a] for p, (a, b) in zip(parts, row_blocks(M, world))])
    ref = oracle.gemm_f64(M, N, K, 1.5, A, B, 0.5, C0)
    dist.destroy_process_group()
    with open(os.path.join(out_dir, f"rank{rank}.json"), "w") as f:
        json.dump({"block": [r0, r1], "equal": bool(np.array_equal(whole, ref))}, f)


def test_two_gloo_ranks_assemble_the_whole_product(tmp_path):
    world = 2
    mp.start_processes(_rank, args=(world, _free_port(), str(tmp_path)), nprocs=world,
                       start_method="spawn")
    res = [json.load(open(tmp_path / f"rank{r}.json")) for r in range(world)]
    assert [r["block"] for r in res] == [[0, 768], [768, 1300]]   # 6 tiles: 3 + 3 (the last partial)
    assert all(r["equal"] for r in res)


# ------------------------------------------------ grouped gemm by problems
def test_problem_shares_cover_every_problem_once_balanced():
    """Largest-first greedy shares of the 512 grouped problems: every
    problem on exactly one rank, indices ascending within a share, and no
    rank more than the largest problem's flops above the average (the
    greedy bound); with one rank, all problems in order."""
    import workloads as W
    from paper_1804_10694_gb300.partition import problem_shares
    shapes = W.grouped_shapes()
    flops = [2 * m * n * k for (m, n, k) in shapes]
    assert problem_shares(shapes, 1) == [list(range(len(shapes)))]
    for world in (2, 3, 4, 8):
        shares = problem_shares(shapes, world)
        assert sorted(i for s in shares for i in s) == list(range(len(shapes)))
        assert all(s == sorted(s) for s in shares)
        loads = [sum(flops[i] for i in s) for s in shares]
        assert max(loads) - sum(loads) / world <= max(flops)
    # more ranks than problems: the extra ranks are idle
    assert problem_shares([(8, 8, 8), (4, 4, 4)], 3) == [[0], [1], []]
    with pytest.raises(ValueError):
        problem_shares(shapes, 0)


def _rank_problems(rank: int, world: int, port: int, out_dir: str):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), WORLD_SIZE=str(world),
                      RANK=str(rank), LOCAL_RANK=str(rank))
    import torch
    import torch.distributed as dist
    import oracle
    from paper_1804_10694_gb300.partition import problem_shares
    dist.init_process_group("gloo")
    rng = np.random.default_rng(9)
    shapes = [tuple(int(x) for x in rng.integers(1, 40, 3)) for _ in range(9)]
    data = [tuple(rng.uniform(-1, 1, sh).astype(np.float32) for sh in ((m, k), (k, n), (m, n)))
            for (m, n, k) in shapes]
    mine = problem_shares(shapes, world)[rank]
    # each rank computes its problems (the FP64 oracle standing in for its
    # GPU's grouped launch) and the results are gathered on every rank
    flat = np.concatenate([oracle.gemm_f64(*shapes[i], 1.5, data[i][0], data[i][1], 0.5, data[i][2]).ravel()
                           for i in mine] or [np.zeros(0)])
    total = sum(m * n for (m, n, k) in shapes)
    buf = np.zeros(total)
    buf[:flat.size] = flat
    parts = [torch.zeros(total, dtype=torch.float64) for _ in range(world)]
    dist.all_gather(parts, torch.from_numpy(buf))
    got = {}
    for r, share in enumerate(problem_shares(shapes, world)):
        off = 0
        for i in share:
            m, n, _ = shapes[i]
            got[i] = parts[r].numpy()[off:off + m * n].reshape(m, n)
            off += m * n
    equal = all(np.array_equal(got[i], oracle.gemm_f64(*shapes[i], 1.5, data[i][0], data[i][1], 0.5,
                                                         data[i][2])) for i in range(len(shapes)))
    dist.destroy_process_group()
    with open(os.path.join(out_dir, f"prob{rank}.json"), "w") as f:
        json.dump({"share": mine, "equal": bool(equal)}, f)


def test_two_gloo_ranks_split_a_grouped_gemm_by_problems(tmp_path):
    world = 2
    mp.start_processes(_rank_problems, args=(world, _free_port(), str(tmp_path)), nprocs=world,
                       start_method="spawn")
    res = [json.load(open(tmp_path / f"prob{r}.json")) for r in range(world)]
    assert sorted(res[0]["share"] + res[1]["share"]) == list(range(9))
    assert all(r["equal"] for r in res)
