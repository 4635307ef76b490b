"""Row-partitioned gemm over several processes, one GPU each.

The paper distributes a computation by blocks of rows, one block per node,
and exchanges data only where a block reads a neighbour's rows (Section
III-C: the distribute, send and receive commands, Fig. 3(c); Section V-A:
each distributed loop becomes a condition on the process rank).  A gemm row of C
reads one row of A and all of B, so the partition needs no exchange at all:
rank r computes rows [r0, r1) of C = alpha * A * B + beta * C from rows
[r0, r1) of A, its own copy of B (replicated: the caller places it, for
instance by a broadcast once) and rows [r0, r1) of C.

Block boundaries fall on 256-row edges, the height of a CTA pair's output
tile, so that no output tile is split between ranks, and the blocks are
balanced to within one such tile.  Each rank's call is an ordinary gemm on
row views of A and C (leading dimensions unchanged), so its result is the
single-GPU result on those rows.

A grouped gemm (independent problems) is partitioned by problems instead:
each rank runs a grouped plan over its share, the shares balanced by flops
(problem_shares).  A problem's result does not depend on the other problems
of its launch, so every rank's results are the single-GPU grouped results.
"""
from __future__ import annotations

TILE_ROWS = 256   # rows of a CTA pair's output tile


def row_blocks(M: int, world: int, align: int = TILE_ROWS) -> list[tuple[int, int]]:
    """[r0, r1) of every rank: whole `align`-row tiles, as even as possible
    (the first ranks take one tile more when the count does not divide), the
    last block ending at M.  Ranks past the tile count get empty blocks."""
    if world < 1 or M < 0 or align < 1:
        raise ValueError("world >= 1, M >= 0 and align >= 1")
    tiles = -(-M // align)
    base, extra = divmod(tiles, world)
    out, t = [], 0
    for r in range(world):
        n = base + (1 if r < extra else 0)
        r0, r1 = min(M, t * align), min(M, (t + n) * align)
        out.append((r0, r1))
        t += n
    return out


def gemm_rows(A, B, C, alpha: float = 1.0, beta: float = 0.0, rank: int = 0, world: int = 1,
              mode="auto", select="default", stream=None):
    """This rank's share of C <- alpha*A@B + beta*C (torch CUDA tensors, row
    major; A and C hold all M rows, B is the full K x N matrix).  Rows of C
    outside the rank's block are not touched.  Returns (r0, r1)."""
    from . import gemm
    M = A.shape[0]
    if C.shape[0] != M:
        raise ValueError("A and C must have the same number of rows")
    r0, r1 = row_blocks(M, world)[rank]
    if r1 > r0:
        gemm(A[r0:r1], B, C[r0:r1], alpha, beta, mode=mode, select=select, stream=stream)
    return r0, r1


def problem_shares(shapes, world: int) -> list[list[int]]:
    """Problem indices of every rank for a grouped gemm of `shapes` ((M, N, K)
    each): largest-first greedy balancing of 2 M N K flops (each problem, in
    decreasing flops, ties by index, goes to the rank with the fewest flops so
    far, ties to the lowest rank), so that no rank's flops exceed the average
    by more than the largest problem's.  Indices ascend within a share; ranks
    past the problem count get empty shares."""
    if world < 1:
        raise ValueError("world >= 1")
    flops = [2 * int(m) * int(n) * int(k) for (m, n, k) in shapes]
    order = sorted(range(len(flops)), key=lambda i: (-flops[i], i))
    load = [0] * world
    shares = [[] for _ in range(world)]
    for i in order:
        r = min(range(world), key=lambda q: (load[q], q))
        shares[r].append(i)
        load[r] += flops[i]
    return [sorted(s) for s in shares]


def gemm_grouped_problems(shapes, As, Bs, Cs, alphas, betas, rank: int = 0, world: int = 1,
                          mode="bf16x3", stream=None, block_n=None, kb=None):
    """This rank's share of a grouped gemm: C_i <- alpha_i A_i B_i + beta_i C_i
    for the problems i of problem_shares(shapes, world)[rank] (torch CUDA
    tensors, tight row-major), in one grouped launch (eager; the plan is
    destroyed after it, which waits for the launch).  Other problems' C are
    not touched.  block_n / kb: the grouped plan's tile width and fold length
    (default: its own choice for the share).  Returns the share's indices."""
    from . import GroupedPlan
    mine = problem_shares(shapes, world)[rank]
    if mine:
        plan = GroupedPlan([shapes[i] for i in mine], mode=mode, block_n=block_n, kb=kb)
        try:
            plan.execute([As[i] for i in mine], [Bs[i] for i in mine], [Cs[i] for i in mine],
                         [alphas[i] for i in mine], [betas[i] for i in mine], stream=stream, graph=False)
        finally:
            plan.destroy()
    return mine
