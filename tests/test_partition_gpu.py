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
