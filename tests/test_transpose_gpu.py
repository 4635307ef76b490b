"""Transposed operand layouts (BLAS TN / NT / TT).  The packing pass reads
each layout directly, producing the same planes as for the untransposed
matrices, so results must equal the untransposed gemm bit for bit, and meet
the oracle bound."""
from __future__ import annotations

import numpy as np
import pytest
import torch

import oracle
import paper_1804_10694_gb300 as pkg
import workloads as W
from gpu_helpers import TOL, check_padding_untouched, dev, run_gemm

pytestmark = pytest.mark.gpu


def run_t(ta, tb, mode, M, N, K, alpha, As, Bs, beta, C0, select="default"):
    """As, Bs: storage arrays of A (K x M when ta) and B (N x K when tb)."""
    dA, dB, dC = dev(As), dev(Bs), dev(C0)
    pkg.gemm_f32_t(ta, tb, M, N, K, alpha, dA.data_ptr(), As.shape[1], dB.data_ptr(), Bs.shape[1], beta,
                   dC.data_ptr(), C0.shape[1], mode, select, torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    return dC.cpu().numpy()


@pytest.mark.parametrize("mode", ["bf16x3", "tf32x3", "bf16x6", "simt"])
@pytest.mark.parametrize("ta,tb", [(1, 0), (0, 1), (1, 1)])
def test_transposes_match_untransposed_bitwise(mode, ta, tb):
    M, N, K = 333, 270, 515
    A, B = W.uniform(M, K, 201), W.uniform(K, N, 202)
    C0 = W.uniform(M, N, 203, ld=N + 2)
    # stored layouts with padded leading dimensions (NaN padding must not be read)
    As = W._with_ld(np.ascontiguousarray(A.T), M + 3, np.nan) if ta else A
    Bs = W._with_ld(np.ascontiguousarray(B.T), K + 1, np.nan) if tb else B
    got = run_t(ta, tb, mode, M, N, K, 1.5, As, Bs, 0.5, C0)
    base = run_gemm(mode, M, N, K, 1.5, A, B, 0.5, C0)
    assert np.array_equal(got.view(np.uint32), base.view(np.uint32))
    assert oracle.rel_frob(got, oracle.gemm_f64(M, N, K, 1.5, A, B, 0.5, C0)) <= TOL
    check_padding_untouched(C0, got, N)


@pytest.mark.parametrize("mode", ["bf16x3", "tf32x3", "bf16x6", "simt"])
def test_transposed_integer_inputs_bit_exact(mode):
    M, N, K = 300, 200, 700
    A, B, C0 = W.integers(M, K, 204), W.integers(K, N, 205), W.integers(M, N, 206)
    ref = oracle.gemm_f64(M, N, K, 1.5, A, B, 0.5, C0).astype(np.float32)
    got = run_t(1, 1, mode, M, N, K, 1.5, np.ascontiguousarray(A.T), np.ascontiguousarray(B.T), 0.5, C0)
    assert np.array_equal(got, ref)


@pytest.mark.parametrize("mode", ["bf16x3", "tf32x3", "bf16x6"])
def test_transposed_block_scaling(mode):
    """Blocks of 128 rows of A are 128 columns of the stored A^T: the
    transposing pack must scale them as blocks (tiny and mixed blocks)."""
    M, N, K = 300, 200, 500
    A = W.uniform(M, K, 207)
    A[128:256] = W.scaled(A[128:256], -100)
    B = W.scaled(W.uniform(K, N, 208), -20)
    ref = oracle.gemm_f64(M, N, K, 1.0, A, B, 0.0, None)
    got = run_t(1, 1, mode, M, N, K, 1.0, np.ascontiguousarray(A.T), np.ascontiguousarray(B.T), 0.0,
                np.zeros((M, N), np.float32))
    assert oracle.rel_frob(got, ref) <= TOL


def test_transposed_plan_and_model_selection():
    M, N, K = 640, 384, 1024
    A, B, C0 = W.uniform(M, K, 209), W.uniform(K, N, 210), W.uniform(M, N, 211)
    At, Bt = dev(np.ascontiguousarray(A.T)), dev(np.ascontiguousarray(B.T))
    ref = oracle.gemm_f64(M, N, K, 1.0, A, B, 1.0, C0)
    for sel in ("default", "exhaustive"):
        plan = pkg.Plan(M, N, K, mode="bf16x3", select=sel, trans_a=True, trans_b=True)
        dC = dev(C0)
        plan.execute(At, Bt, dC, 1.0, 1.0)
        torch.cuda.synchronize()
        assert oracle.rel_frob(dC.cpu().numpy(), ref) <= TOL
        plan.destroy()


@pytest.mark.parametrize("ta,tb", [(1, 0), (0, 1), (1, 1)])
def test_simt_transposes_on_ragged_and_unaligned_shapes(ta, tb):
    """The SIMT kernel's partial tiles and scalar loads with transposed
    layouts: odd leading dimensions, edges in every dimension."""
    for (M, N, K) in [(129, 131, 37), (1, 300, 9), (257, 1, 130), (5, 7, 3)]:
        A, B = W.uniform(M, K, 220 + M), W.uniform(K, N, 221 + N)
        C0 = W.uniform(M, N, 222, ld=N + 1)
        As = W._with_ld(np.ascontiguousarray(A.T), M + 1, np.nan) if ta else A
        Bs = W._with_ld(np.ascontiguousarray(B.T), K + 3, np.nan) if tb else B
        got = run_t(ta, tb, "simt", M, N, K, 1.5, As, Bs, -0.5, C0)
        assert oracle.rel_frob(got, oracle.gemm_f64(M, N, K, 1.5, A, B, -0.5, C0)) <= TOL, (M, N, K)
        check_padding_untouched(C0, got, N)
