"""Operands and results of more than 2^31 elements, through the C ABI.

Sizes are 64-bit at the boundary and each of M, N, K fits in 31 bits, but
their products do not: an element offset past 2^31 - 1 must be formed in 64
bits by the packing pass (reads of A, writes of its planes), the tensor-core
epilogue (loads and stores of C) and the SIMT kernel.  Two problems take
each side past it: A of 2.2 * 10^9 elements (2 200 000 x 1000) and C of
2.2 * 10^9 elements (2 200 000 x 1000).  Their entries are integer closed
forms (workloads.int_pattern), exact in FP32, bf16 and tf32, and every
partial sum is an integer below 2^24, so every mode gives the definition's
value exactly (Tiramisu Section I; a schedule does not change the result,
Section III).  Sampled rows -- the first ones, the middle, both sides of the
first row that starts past 2^31 elements, 200 random rows past it and the
last 300 rows, which end in a partial tile -- are compared bit for bit with
the FP64 oracle, which rebuilds those rows of A and C from the same closed
forms on the host."""
import numpy as np
import pytest
import torch

import oracle
import paper_1804_10694_gb300 as pkg
import workloads as W
from gpu_helpers import MODES

pytestmark = pytest.mark.gpu

TWO31 = 2 ** 31
ALPHA, BETA = 1.5, 0.5
# (a, b, m, off) of workloads.int_pattern for A, B and C
PAT_A, PAT_B, PAT_C = (1, 3, 17, 8), (5, 7, 13, 6), (1, 1, 5, 2)
M_BIG = 2_200_000
NEED_BYTES = 48 * 2 ** 30   # inputs, the largest plan's planes and temporaries


def _need_memory():
    free, _ = torch.cuda.mem_get_info()
    if free < NEED_BYTES:
        pytest.skip(f"needs {NEED_BYTES >> 30} GiB of free device memory, {free >> 30} GiB free")


def _fill(X: torch.Tensor, pat, chunk_elems: int = 1 << 26) -> torch.Tensor:
    """X's entries (i, k) = int_pattern(i, k), computed on the device a block
    of rows at a time (no full-size temporaries)."""
    rows, cols = X.shape
    chunk_rows = max(1, chunk_elems // max(cols, 1))
    k = torch.arange(cols, device="cuda", dtype=torch.int64)[None, :]
    for r0 in range(0, rows, chunk_rows):
        r1 = min(rows, r0 + chunk_rows)
        i = torch.arange(r0, r1, device="cuda", dtype=torch.int64)[:, None]
        X[r0:r1] = W.int_pattern(i, k, *pat).to(torch.float32)
    return X


def _device_matrix(rows: int, cols: int, pat) -> torch.Tensor:
    return _fill(torch.empty(rows, cols, dtype=torch.float32, device="cuda"), pat)


def _host_rows(rows: np.ndarray, cols: int, pat) -> np.ndarray:
    i = rows.astype(np.int64)[:, None]
    k = np.arange(cols, dtype=np.int64)[None, :]
    return np.ascontiguousarray(W.int_pattern(i, k, *pat).astype(np.float32))


def _sample_rows(M: int, row_len: int) -> np.ndarray:
    first_past = TWO31 // row_len + 1   # the first row whose first element lies past 2^31 - 1
    assert first_past < M - 300
    rows = {0, 1, 127, 128, M // 2, first_past - 1, first_past}
    rows.update(range(M - 300, M))
    rows.update(np.random.default_rng(7).integers(first_past, M, 200).tolist())
    return np.array(sorted(rows), dtype=np.int64)


def _check(M: int, N: int, K: int, row_len: int):
    _need_memory()
    A = _device_matrix(M, K, PAT_A)
    B = _device_matrix(K, N, PAT_B)
    C = torch.empty(M, N, dtype=torch.float32, device="cuda")
    rows = _sample_rows(M, row_len)
    # the oracle on the sampled rows: row i of the result depends on row i of
    # A and of C only, so the rows form a problem of their own
    A_rows, C0_rows = _host_rows(rows, K, PAT_A), _host_rows(rows, N, PAT_C)
    B_host = _host_rows(np.arange(K), N, PAT_B)
    ref = oracle.gemm_f64(len(rows), N, K, ALPHA, A_rows, B_host, BETA, C0_rows).astype(np.float32)
    idx = torch.from_numpy(rows).cuda()
    for mode in MODES:
        _fill(C, PAT_C)
        with pkg.Plan(M, N, K, mode=mode) as plan:
            plan.execute(A, B, C, ALPHA, BETA)
            torch.cuda.synchronize()
        pkg.device_error()
        got = C.index_select(0, idx).cpu().numpy()
        bad = np.count_nonzero(got.view(np.uint32) != ref.view(np.uint32))
        assert bad == 0, (mode, M, N, K, bad)


def test_operand_past_2_31_elements():
    """A is 2 200 000 x 1000 (its planes likewise, with the padded pitch):
    the pack's reads and writes pass 2^31 elements; C is 2 200 000 x 72 (a
    partial 32-column chunk in the epilogue)."""
    _check(M_BIG, 72, 1000, row_len=1000)


def test_result_past_2_31_elements():
    """C is 2 200 000 x 1000 (beta != 0: read and written past 2^31
    elements); K = 40 is one partial k-chunk."""
    _check(M_BIG, 1000, 40, row_len=1000)
