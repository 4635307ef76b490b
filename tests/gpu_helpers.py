"""Shared helpers of the GPU parity tests: copy seeded storage arrays to the
device, call the library through the C ABI, bring results back."""
from __future__ import annotations

import functools

import numpy as np
import torch

import oracle
import paper_1804_10694_gb300 as pkg
import workloads as W

MODES = ("simt", "bf16x3", "tf32x3", "bf16x6")
TOL = 1e-5   # relative Frobenius error bound for every result


def dev(a: np.ndarray) -> torch.Tensor:
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def run_gemm(mode, M, N, K, alpha, A, B, beta, C0, config_id=None, select="default"):
    """A, B, C0: numpy storage arrays (second dimension = leading dimension).
    Returns the whole C storage array after the call."""
    dA, dB = dev(A), dev(B)
    dC = dev(C0)
    lda, ldb, ldc = A.shape[1], B.shape[1], C0.shape[1]
    if config_id is None:
        pkg.gemm_f32_ex(M, N, K, alpha, dA.data_ptr(), lda, dB.data_ptr(), ldb, beta,
                        dC.data_ptr(), ldc, mode, select, torch.cuda.current_stream().cuda_stream)
    else:
        plan = pkg.Plan(M, N, K, lda, ldb, ldc, mode=mode, config_id=config_id)
        plan.execute_ptrs(alpha, dA.data_ptr(), dB.data_ptr(), beta, dC.data_ptr())
        torch.cuda.synchronize()
        plan.destroy()
    torch.cuda.synchronize()
    return dC.cpu().numpy()


def check_padding_untouched(before: np.ndarray, after: np.ndarray, N: int):
    """Columns N..ld-1 of C are outside the matrix: they must keep their bytes."""
    if before.shape[1] > N:
        assert np.array_equal(before[:, N:].view(np.uint32), after[:, N:].view(np.uint32))


@functools.lru_cache(maxsize=8)
def square_inputs(n: int, config_index: int, gen: str = "uniform"):
    sa, sb, sc = W.seeds(config_index)
    f = {"uniform": W.uniform, "wide": W.wide_range, "int": W.integers}[gen]
    return f(n, n, sa + n), f(n, n, sb + n), f(n, n, sc + n)
