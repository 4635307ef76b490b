"""Parity of the fused-split variant, where the gemm kernel splits A itself
instead of reading packed planes (only B is packed).  It runs the same
split arithmetic, block exponents and MMA sequence as the packed variant
with the same tile configuration, so the two must agree bit for bit; each
result must also meet the oracle bound on its own."""
from __future__ import annotations

import math

import numpy as np
import pytest
import torch

import oracle
import paper_1804_10694_gb300 as pkg
import workloads as W
from gpu_helpers import TOL, check_padding_untouched, dev

pytestmark = pytest.mark.gpu

KEYS = ("block_n", "split_k", "kb", "group_m")


def fused_ids(mode):
    return [i for i in range(pkg.config_count(mode)) if pkg.config_get(mode, i)["fused"]]


def packed_twin(mode, cid):
    c = pkg.config_get(mode, cid)
    for i in range(pkg.config_count(mode)):
        d = pkg.config_get(mode, i)
        if not d["fused"] and d["cluster"] == 1 and all(d[k] == c[k] for k in KEYS):
            return i
    raise AssertionError(c)


def pick(mode, block_n, split_k, kb=4, group_m=16):
    for i in fused_ids(mode):
        c = pkg.config_get(mode, i)
        if (c["block_n"], c["split_k"], c["kb"], c["group_m"]) == (block_n, split_k, kb, group_m):
            return i
    raise AssertionError((block_n, split_k, kb, group_m))


def run_cfg(mode, cid, M, N, K, alpha, A, B, beta, C0, a_offset=0):
    """Run one configuration; A may start a_offset floats into its buffer
    (a misaligned base address when a_offset % 4 != 0)."""
    lda, ldb, ldc = A.shape[1], B.shape[1], C0.shape[1]
    flat = np.zeros(A.size + a_offset, np.float32)
    flat[a_offset:] = A.ravel()
    dA = dev(flat)
    dB, dC = dev(B), dev(C0)
    plan = pkg.Plan(M, N, K, lda, ldb, ldc, mode=mode, config_id=cid)
    plan.execute_ptrs(alpha, dA.data_ptr() + 4 * a_offset, dB.data_ptr(), beta, dC.data_ptr())
    torch.cuda.synchronize()
    plan.destroy()
    return dC.cpu().numpy()


@pytest.mark.parametrize("mode", ["bf16x3", "tf32x3"])
def test_fused_table_mirrors_packed(mode):
    ids = fused_ids(mode)
    assert len(ids) * 3 == pkg.config_count(mode)   # single-CTA packed, pairs, fused
    assert len({packed_twin(mode, i) for i in ids}) == len(ids)


@pytest.mark.parametrize("mode", ["bf16x3", "tf32x3"])
def test_every_fused_configuration_matches_packed_bitwise(mode):
    M, N, K = 1000, 300, 700
    A = W.uniform(M, K, 91, ld=K + 4)
    B, C0 = W.uniform(K, N, 92, ld=N + 3), W.uniform(M, N, 93, ld=N + 1)
    ref = oracle.gemm_f64(M, N, K, 1.5, A, B, 0.5, C0)
    for cid in fused_ids(mode):
        got = run_cfg(mode, cid, M, N, K, 1.5, A, B, 0.5, C0)
        twin = run_cfg(mode, packed_twin(mode, cid), M, N, K, 1.5, A, B, 0.5, C0)
        assert np.array_equal(got.view(np.uint32), twin.view(np.uint32)), pkg.config_get(mode, cid)
        assert oracle.rel_frob(got, ref) <= TOL
        check_padding_untouched(C0, got, N)


@pytest.mark.parametrize("mode", ["bf16x3", "tf32x3"])
@pytest.mark.parametrize("lda_pad,a_offset", [(1, 0), (0, 1), (3, 0), (0, 2)])
def test_fused_unaligned_a(mode, lda_pad, a_offset):
    """Rows of A not 16-byte aligned (odd lda or a shifted base): the kernel
    copies A four bytes at a time; K = 333 also leaves a partial 16-byte unit
    at the end of every row on the aligned path."""
    M, N, K = 517, 200, 333
    A = W.uniform(M, K, 94, ld=K + lda_pad)
    B, C0 = W.uniform(K, N, 95), W.uniform(M, N, 96)
    ref = oracle.gemm_f64(M, N, K, 1.0, A, B, 0.25, C0)
    for bn, sk in ((64, 1), (128, 1), (128, 2)):
        cid = pick(mode, bn, sk)
        got = run_cfg(mode, cid, M, N, K, 1.0, A, B, 0.25, C0, a_offset=a_offset)
        twin = run_cfg(mode, packed_twin(mode, cid), M, N, K, 1.0, A, B, 0.25, C0)
        assert np.array_equal(got.view(np.uint32), twin.view(np.uint32)), (bn, sk)
        assert oracle.rel_frob(got, ref) <= TOL


@pytest.mark.parametrize("mode", ["bf16x3", "tf32x3"])
def test_fused_integer_inputs_bit_exact(mode):
    M, N, K = 700, 260, 900
    A, B, C0 = W.integers(M, K, 97), W.integers(K, N, 98), W.integers(M, N, 99)
    ref = oracle.gemm_f64(M, N, K, 1.5, A, B, 0.5, C0).astype(np.float32)
    for bn, sk in ((64, 1), (128, 1), (64, 3)):
        got = run_cfg(mode, pick(mode, bn, sk), M, N, K, 1.5, A, B, 0.5, C0)
        assert np.array_equal(got, ref), (bn, sk)


@pytest.mark.parametrize("mode", ["bf16x3", "tf32x3"])
def test_fused_block_scaling(mode):
    """Operand blocks outside the safe range are scaled by the kernel itself
    (exponent from the max-only pass): tiny products near 2^-120 and a
    product that overflows FP32 before alpha."""
    M, N, K = 300, 200, 500
    base_a, base_b = W.uniform(M, K, 41), W.uniform(K, N, 42)
    cases = [(W.scaled(base_a, -100), W.scaled(base_b, -20), 1.0),
             (W.scaled(base_a, 64), W.scaled(base_b, 64), math.ldexp(1.0, -20))]
    # one block of A tiny, the others not: per-block exponents differ
    mixed = base_a.copy()
    mixed[128:256] = W.scaled(base_a[128:256], -90)
    cases.append((mixed, base_b, 1.0))
    C0 = np.zeros((M, N), np.float32)
    for A, B, alpha in cases:
        ref = oracle.gemm_f64(M, N, K, alpha, A, B, 0.0, None)
        for bn, sk in ((64, 1), (128, 2)):
            cid = pick(mode, bn, sk)
            got = run_cfg(mode, cid, M, N, K, alpha, A, B, 0.0, C0)
            twin = run_cfg(mode, packed_twin(mode, cid), M, N, K, alpha, A, B, 0.0, C0)
            assert np.isfinite(got).all()
            assert np.array_equal(got.view(np.uint32), twin.view(np.uint32))
            assert oracle.rel_frob(got, ref) <= TOL


@pytest.mark.parametrize("M,N,K", W.CONV_SHAPES)
def test_fused_conv_shapes(M, N, K):
    sa, sb, _ = W.seeds(W.CONFIG_CONV)
    A, B = W.uniform(M, K, sa), W.uniform(K, N, sb)
    C0 = np.zeros((M, N), np.float32)
    ref = oracle.gemm_f64(M, N, K, 1.0, A, B, 0.0, None)
    for mode in ("bf16x3", "tf32x3"):
        for bn, sk in ((64, 1), (128, 1), (128, 3)):
            cid = pick(mode, bn, sk)
            got = run_cfg(mode, cid, M, N, K, 1.0, A, B, 0.0, C0)
            assert oracle.rel_frob(got, ref) <= TOL, (mode, bn, sk)
            twin = run_cfg(mode, packed_twin(mode, cid), M, N, K, 1.0, A, B, 0.0, C0)
            assert np.array_equal(got.view(np.uint32), twin.view(np.uint32)), (mode, bn, sk)


def test_fused_wide_range_2048():
    n = 2048
    sa, sb, sc = W.seeds(W.CONFIG_WIDE)
    A, B, C0 = W.wide_range(n, n, sa + 7), W.wide_range(n, n, sb + 7), W.wide_range(n, n, sc + 7)
    ref = oracle.gemm_f64(n, n, n, 1.0, A, B, 0.5, C0)
    for mode in ("bf16x3", "tf32x3"):
        cid = pick(mode, 128, 1)
        got = run_cfg(mode, cid, n, n, n, 1.0, A, B, 0.5, C0)
        assert oracle.rel_frob(got, ref) <= TOL
        twin = run_cfg(mode, packed_twin(mode, cid), n, n, n, 1.0, A, B, 0.5, C0)
        assert np.array_equal(got.view(np.uint32), twin.view(np.uint32))
