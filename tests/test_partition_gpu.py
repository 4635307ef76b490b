"""The row-partitioned gemm's ranks run through the library on one GPU, one
after the other (they never wait on each other): each rank writes exactly its
own block of rows of C, and the blocks together equal the FP64 oracle's
whole result (bit for bit on integer inputs)."""
import numpy as np
import pytest
import torch

import oracle
import workloads as W
from gpu_helpers import TOL, dev
from paper_1804_10694_gb300.partition import gemm_rows, row_blocks

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("world", [2, 3])
@pytest.mark.parametrize("gen", ["uniform", "int"])
def test_ranks_write_their_rows_and_assemble_the_product(world, gen):
    M, N, K = 1300, 520, 900
    f = W.uniform if gen == "uniform" else W.integers
    A, B, C0 = f(M, K, 81), f(K, N, 82), f(M, N, 83)
    ref = oracle.gemm_f64(M, N, K, 1.5, A, B, 0.5, C0)
    dA, dB, dC = dev(A), dev(B), dev(C0)
    for rank in range(world):
        before = dC.clone()
        r0, r1 = gemm_rows(dA, dB, dC, 1.5, 0.5, rank=rank, world=world, mode="bf16x3")
        torch.cuda.synchronize()
        assert (r0, r1) == row_blocks(M, world)[rank]
        after = dC.cpu().numpy()
        untouched = np.ones(M, bool)
        untouched[r0:r1] = False
        assert np.array_equal(after[untouched], before.cpu().numpy()[untouched])
    got = dC.cpu().numpy()
    if gen == "int":
        assert np.array_equal(got, ref.astype(np.float32))
    else:
        assert oracle.rel_frob(got, ref) <= TOL


@pytest.mark.parametrize("world", [2, 3])
def test_grouped_problem_shares_match_the_whole_group(world):
    """A grouped gemm split by problems (problem_shares): the ranks' grouped
    launches (same tile width and fold length), one after the other on one
    GPU, give for every problem the bits of the whole group's launch, and
    each problem matches the FP64 oracle; a rank touches only its own
    problems' C."""
    import paper_1804_10694_gb300 as pkg
    from paper_1804_10694_gb300.partition import gemm_grouped_problems, problem_shares
    shapes = W.grouped_shapes()[:48]
    data = [(W.uniform(m, k, 900 + 3 * i), W.uniform(k, n, 901 + 3 * i), W.uniform(m, n, 902 + 3 * i))
            for i, (m, n, k) in enumerate(shapes)]
    G = len(shapes)
    alphas, betas = [1.5] * G, [0.5] * G
    As = [dev(a) for a, _, _ in data]
    Bs = [dev(b) for _, b, _ in data]
    whole = [dev(c) for _, _, c in data]
    plan = pkg.GroupedPlan(shapes, mode="bf16x3", block_n=128, kb=4)
    plan.execute(As, Bs, whole, alphas, betas, graph=False)
    torch.cuda.synchronize()
    plan.destroy()
    split = [dev(c) for _, _, c in data]
    for rank in range(world):
        before = [c.clone() for c in split]
        mine = gemm_grouped_problems(shapes, As, Bs, split, alphas, betas, rank=rank, world=world,
                                     block_n=128, kb=4)
        torch.cuda.synchronize()
        assert mine == problem_shares(shapes, world)[rank]
        for i in range(G):
            if i not in mine:
                assert torch.equal(split[i], before[i])
    pkg.device_error()
    for i, (m, n, k) in enumerate(shapes):
        got = split[i].cpu().numpy()
        assert np.array_equal(got.view(np.uint32), whole[i].cpu().numpy().view(np.uint32)), i
        ref = oracle.gemm_f64(m, n, k, 1.5, data[i][0], data[i][1], 0.5, data[i][2])
        assert oracle.rel_frob(got, ref) <= TOL, i
