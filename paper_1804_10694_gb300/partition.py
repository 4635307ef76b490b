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
