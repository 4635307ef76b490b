"""GPU parity of the six-product mode (BF16X6) against the CPU oracle, through
the C ABI.

Each FP32 operand is split in three bf16 planes, hi + mid + lo (exact for
normal values), and the product keeps the six plane products whose indices
sum to at most two.  The dropped products (mid*lo, lo*mid, lo*lo) are below
2^-23 of |a||b|, so what remains is the rounding of the FP32 accumulation:
the mode is meant to be as accurate as a plain single-precision gemm.

Bar: relative Frobenius error against the FP64 definition at most FACTOR
times that of the definition evaluated in FP32 by the oracle (k increasing,
every product and sum rounded; the factor covers a different summation
order), and never above the three-product modes' 1e-5; bit-exact on integer
inputs; packed planes bit-identical to the oracle's three-way split."""
import numpy as np
import pytest
import torch

import oracle
import paper_1804_10694_gb300 as pkg
import workloads as W
from gpu_helpers import TOL, check_padding_untouched, dev, run_gemm

pytestmark = pytest.mark.gpu

MODE = "bf16x6"
FACTOR = 2.0


@pytest.fixture(autouse=True, scope="module")
def _device():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    pkg.load()
    yield
    pkg.device_error()


def fp32_bound(M, N, K, alpha, A, B, beta, C0, ref) -> float:
    """FACTOR x the error of the FP32 evaluation of the same problem."""
    f32 = oracle.gemm_f32_seq(M, N, K, alpha, A, B, beta, C0)
    return FACTOR * max(oracle.rel_frob(f32, ref), 2.0 ** -24)


# ------------------------------------------------------------- split/pack
@pytest.mark.parametrize("transpose", [False, True])
@pytest.mark.parametrize("gen", ["uniform", "wide", "tiny"])
def test_split_pack_three_planes_bit_exact(transpose, gen):
    from oracle import split
    rows, cols = (300, 77) if not transpose else (77, 300)
    if gen == "uniform":
        X = W.uniform(rows, cols, 5, ld=cols + 3)
    elif gen == "wide":
        X = W.wide_range(rows, cols, 6, ld=cols + 3, lo=-40, hi=40)
    else:
        X = W.scaled(W.uniform(rows, cols, 7), -120)
        X = W._with_ld(X, cols + 3, np.nan)
    planes, amax = pkg.split_pack(dev(X)[:, :cols], mode=MODE, transpose=transpose)
    torch.cuda.synchronize()
    P = planes.float().cpu().numpy()
    assert P.shape[0] == 3
    logical = X[:, :cols]
    src = logical.T.copy() if transpose else logical
    prow, K = src.shape
    hi, mid, lo, exps = split.split_rows(src, prow, K, "bf16x6")
    got_exps = [split.block_exponent(np.array([v], np.int32).view(np.float32)[0])
                for v in amax.cpu().numpy()]
    assert list(exps) == got_exps
    for p, ref in enumerate((hi, mid, lo)):
        assert np.array_equal(P[p, :, :K].view(np.uint32), ref.view(np.uint32)), p
    assert not P[:, :, K:].any()          # pitch padding is zero


# ------------------------------------------------------------ accuracy
SHAPES = [(300, 260, 333, 0), (129, 257, 1060, 1), (1060, 1060, 1060, 0), (1, 1, 1, 0),
          (5, 3, 7, 3), (128, 128, 64, 0), (260, 65, 97, 3), (64, 777, 4099, 1)]


@pytest.mark.parametrize("M,N,K,pad", SHAPES)
@pytest.mark.parametrize("alpha,beta", W.ALPHA_BETA)
def test_fp32_level_accuracy(M, N, K, pad, alpha, beta):
    A = W.uniform(M, K, 21, ld=K + pad)
    B = W.uniform(K, N, 22, ld=N + pad)
    C0 = W.uniform(M, N, 23, ld=N + pad)
    ref = oracle.gemm_f64(M, N, K, alpha, A, B, beta, C0)
    got = run_gemm(MODE, M, N, K, alpha, A, B, beta, C0)
    err = oracle.rel_frob(got, ref)
    assert err <= fp32_bound(M, N, K, alpha, A, B, beta, C0, ref), (M, N, K, err)
    assert err <= TOL
    check_padding_untouched(C0, got, N)


@pytest.mark.parametrize("K", [256, 1060, 4099])
def test_more_accurate_than_three_products(K):
    """The third plane removes the split error that dominates BF16X3."""
    M, N = 256, 192
    A, B = W.uniform(M, K, 24), W.uniform(K, N, 25)
    ref = oracle.gemm_f64(M, N, K, 1.0, A, B, 0.0, None)
    z = np.zeros((M, N), np.float32)
    e6 = oracle.rel_frob(run_gemm(MODE, M, N, K, 1.0, A, B, 0.0, z), ref)
    e3 = oracle.rel_frob(run_gemm("bf16x3", M, N, K, 1.0, A, B, 0.0, z), ref)
    assert e6 * 3.0 < e3, (e6, e3)


def test_wide_range_and_scaled_blocks():
    M, N, K = 600, 500, 700
    A = W.wide_range(M, K, 26, lo=-30, hi=30)
    B = W.wide_range(K, N, 27, lo=-30, hi=30)
    A[128:256] = W.scaled(A[128:256], -110)
    B[:, 256:384] = W.scaled(np.ascontiguousarray(B[:, 256:384]), 60)   # |b| < 2^90: sums stay finite
    C0 = W.uniform(M, N, 28)
    ref = oracle.gemm_f64(M, N, K, 1.0, A, B, 0.5, C0)
    got = run_gemm(MODE, M, N, K, 1.0, A, B, 0.5, C0)
    err = oracle.rel_frob(got, ref)
    assert err <= fp32_bound(M, N, K, 1.0, A, B, 0.5, C0, ref), err


@pytest.mark.parametrize("alpha,beta", W.ALPHA_BETA)
def test_integer_inputs_bit_exact(alpha, beta):
    M, N, K = 700, 650, 1100
    A, B, C0 = W.integers(M, K, 1), W.integers(K, N, 2), W.integers(M, N, 3)
    ref = oracle.gemm_f64(M, N, K, alpha, A, B, beta, C0)
    got = run_gemm(MODE, M, N, K, alpha, A, B, beta, C0)
    assert np.array_equal(got, ref.astype(np.float32))


# --------------------------------------------------- schedule invariance
def test_every_configuration():
    """All 144 BF16X6 configurations (packed ones only: single CTAs and CTA
    pairs) at a shape with several tiles and ragged edges; integer inputs
    give identical bits."""
    M, N, K = 520, 390, 700
    A, B, C0 = W.uniform(M, K, 31), W.uniform(K, N, 32), W.uniform(M, N, 33)
    Ai, Bi, Ci = W.integers(M, K, 34), W.integers(K, N, 35), W.integers(M, N, 36)
    ref = oracle.gemm_f64(M, N, K, 1.5, A, B, 0.5, C0)
    bound = fp32_bound(M, N, K, 1.5, A, B, 0.5, C0, ref)
    refi = oracle.gemm_f64(M, N, K, 1.5, Ai, Bi, 0.5, Ci).astype(np.float32)
    n = pkg.config_count(MODE)
    assert n == 144
    for cid in range(n):
        cfg = pkg.config_get(MODE, cid)
        assert cfg["fused"] == 0 and cfg["stages"] == 2
        got = run_gemm(MODE, M, N, K, 1.5, A, B, 0.5, C0, config_id=cid)
        assert oracle.rel_frob(got, ref) <= bound, cfg
        assert np.array_equal(run_gemm(MODE, M, N, K, 1.5, Ai, Bi, 0.5, Ci, config_id=cid), refi), cfg


def test_fused_configurations_are_rejected():
    with pytest.raises(pkg.GemmError):
        pkg.Plan(256, 256, 256, mode=MODE, config_id=144)
    with pytest.raises(pkg.GemmError):
        pkg.config_get(MODE, 144)


# ------------------------------------------------------------- full size
def test_8192_against_fp32_evaluation():
    """The 8192^3 problem in its default launch configuration against the
    FP32 bar (at most FACTOR times the error of the oracle's sequential FP32
    evaluation), on one row of every 128-row tile plus the last row (the
    sequential FP32 evaluation is too slow on a CPU for all 8192 rows; the
    whole matrix is checked against the FP64 oracle at 1e-5 in
    test_gemm_gpu's full-size tests)."""
    n = 8192
    sa, sb, sc = W.seeds(W.CONFIG_SWEEP)
    A, B, C0 = W.uniform(n, n, sa), W.uniform(n, n, sb), W.uniform(n, n, sc)
    got = run_gemm(MODE, n, n, n, 1.0, A, B, 0.5, C0)
    rng = np.random.default_rng(3)
    rows = sorted({int(t * 128 + rng.integers(128)) for t in range(n // 128)} | {n - 1})
    ref = oracle.gemm_f64_rows(rows, n, n, 1.0, A, B, 0.5, C0)
    f32 = oracle.gemm_f32_seq(len(rows), n, n, 1.0, np.ascontiguousarray(A[rows]), B, 0.5,
                              np.ascontiguousarray(C0[rows]))
    err = oracle.rel_frob(np.ascontiguousarray(got[rows]), ref)
    assert err <= FACTOR * oracle.rel_frob(f32, ref), err
