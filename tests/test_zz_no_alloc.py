"""The allocation-free entry point, gemm_f32_bf16x3_noalloc, called through the
C ABI.  It exists for callers that cannot allocate device memory (a stream
capture where allocation is illegal, a framework allocator that owns device
memory, a path that cannot afford cudaMalloc's synchronisation); its scratch
is a fixed static device array.  Its result must agree with the regular
BF16x3 entry point, gemm_f32_ex, and with the FP64 oracle, on two calls in a
row (the second call must not see stale scratch from the first: the larger
problem runs first, so the smaller one's block maxima and pack counters lie
where the first call left packed planes), its error word must read clear
afterwards, and an oversized problem must be refused without touching C.

This file is named to be collected last, so that a run stopping at its first
failure has already run every other test."""
import ctypes

import numpy as np
import pytest
import torch

import oracle
import paper_1804_10694_gb300 as pkg
import workloads as W

pytestmark = pytest.mark.gpu

TOL = 1e-5
BF16X3 = 2


def _call_noalloc(lib, M, N, K, alpha, dA, dB, beta, dC, stream):
    return lib.gemm_f32_bf16x3_noalloc(M, N, K, ctypes.c_float(alpha), dA.data_ptr(), dA.stride(0),
                                       dB.data_ptr(), dB.stride(0), ctypes.c_float(beta),
                                       dC.data_ptr(), dC.stride(0), stream)


def _call_regular(lib, M, N, K, alpha, dA, dB, beta, dC, stream):
    return lib.gemm_f32_ex(M, N, K, ctypes.c_float(alpha), dA.data_ptr(), dA.stride(0),
                           dB.data_ptr(), dB.stride(0), ctypes.c_float(beta), dC.data_ptr(),
                           dC.stride(0), BF16X3, 0, stream)


def test_noalloc_matches_regular_entry_point_on_consecutive_calls():
    lib = pkg.load()
    stream = torch.cuda.current_stream().cuda_stream
    # two different problems in a row, the larger first: the second call's
    # block maxima and pack counters sit (about 750 KB into the array) where
    # the first call wrote packed planes, so they must be cleared by the call
    cases = [((1024, 777, 2000), (1.0, 0.0), 202), ((300, 260, 333), (1.5, 0.5), 101)]
    for (M, N, K), (alpha, beta), seed in cases:
        hA, hB, hC0 = W.uniform(M, K, seed), W.uniform(K, N, seed + 1), W.uniform(M, N, seed + 2)
        A, B, C0 = (torch.from_numpy(x).cuda() for x in (hA, hB, hC0))
        c_regular, c_noalloc = C0.clone(), C0.clone()
        assert _call_regular(lib, M, N, K, alpha, A, B, beta, c_regular, stream) == 0, \
            lib.gemm_last_error()
        assert _call_noalloc(lib, M, N, K, alpha, A, B, beta, c_noalloc, stream) == 0, \
            lib.gemm_last_error()
        torch.cuda.synchronize()
        got, reg = c_noalloc.cpu().numpy(), c_regular.cpu().numpy().astype(np.float64)
        assert oracle.rel_frob(got, reg) <= TOL, (M, N, K)
        assert oracle.rel_frob(got, oracle.gemm_f64(M, N, K, alpha, hA, hB, beta, hC0)) <= TOL, (M, N, K)
    # no pipeline wait gave up: the path's own error word, read through
    # gemm_device_error, is clear
    assert lib.gemm_device_error() == 0, lib.gemm_last_error()


def test_noalloc_rejects_problems_beyond_its_scratch():
    lib = pkg.load()
    M = N = K = 4096          # needs 128 MiB of scratch, the fixed maximum is 64 MiB
    A = torch.zeros(1, device="cuda")
    C = torch.full((4, 4), 7.0, device="cuda")
    st = lib.gemm_f32_bf16x3_noalloc(M, N, K, ctypes.c_float(1.0), A.data_ptr(), K, A.data_ptr(), N,
                                     ctypes.c_float(0.0), C.data_ptr(), N, None)
    assert st == 1
    assert b"scratch" in lib.gemm_last_error()
    torch.cuda.synchronize()
    assert torch.all(C == 7.0)
