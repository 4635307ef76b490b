"""GPU parity of the compensated epilogue (GEMM_OPT_COMPENSATED) against the
CPU oracle, through the C ABI.

The tensor core accumulates the products of a fold (kb k-chunks) in TMEM;
the epilogue adds these per-fold partial sums into FP32 registers.  With the
option a fold is one k-chunk and every addition is Knuth's TwoSum (the
rounded sum and its exact error), the errors summed apart and added back
once.  The tests pin that mechanism with a constructed case whose nonzero
fold partials are 2^24, 1, 1, -2^24 (exact result 2: a plain FP32 running
sum loses both ones, the compensated one keeps them),
check every mode against the FP64 definition (relative Frobenius error
<= 1e-5; the six-product mode against twice the error of the oracle's FP32
evaluation), bit-exactness on integer inputs, the mapping of fused-split and
CTA-pair configurations to the single-CTA packed kernel, and that on a long
K the compensated sum is more accurate than the plain one with the same
tiles and folds."""
import numpy as np
import pytest
import torch

import oracle
import paper_1804_10694_gb300 as pkg
import workloads as W
from gpu_helpers import TOL, check_padding_untouched, dev

pytestmark = pytest.mark.gpu

TC_MODES = ("bf16x3", "tf32x3", "bf16x6")


@pytest.fixture(autouse=True, scope="module")
def _device():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    pkg.load()
    yield
    pkg.device_error()


def _config(mode, block_n=128, split_k=1, kb=4, group_m=16, fused=0, cluster=1):
    for cid in range(pkg.config_count(mode)):
        c = pkg.config_get(mode, cid)
        if (c["block_n"], c["split_k"], c["kb"], c["group_m"], c["fused"], c["cluster"]) == \
                (block_n, split_k, kb, group_m, fused, cluster):
            return cid
    raise AssertionError("configuration not in the table")


def run_plan(mode, M, N, K, alpha, A, B, beta, C0, compensated, config_id=None):
    """A, B, C0: storage arrays (second dimension = leading dimension)."""
    dA, dB, dC = dev(A), dev(B), dev(C0)
    plan = pkg.Plan(M, N, K, A.shape[1], B.shape[1], C0.shape[1], mode=mode, config_id=config_id,
                    compensated=compensated)
    info = plan.info()
    plan.execute_ptrs(alpha, dA.data_ptr(), dB.data_ptr(), beta, dC.data_ptr())
    torch.cuda.synchronize()
    plan.destroy()
    pkg.device_error()
    return dC.cpu().numpy(), info


@pytest.mark.parametrize("mode", TC_MODES)
def test_fold_errors_are_kept(mode):
    """Fold partials 2^24, 1, 1, -2^24: the plain register sum rounds
    2^24 + 1 back to 2^24 (ties to even) twice and ends at 0; the
    compensated sum returns the exact 2 in every output."""
    chunk = 32 if mode == "tf32x3" else 64
    kb = 4
    F = kb * chunk                       # k-elements per fold
    M, N, K = 200, 100, 4 * F            # ragged tiles: masked rows and columns
    A = np.zeros((M, K), np.float32)
    B = np.zeros((K, N), np.float32)
    A[:, 0], B[0, :] = 2.0 ** 12, 2.0 ** 12          # fold 0: 2^24
    A[:, F], B[F, :] = 1.0, 1.0                      # fold 1: 1
    A[:, 2 * F], B[2 * F, :] = 1.0, 1.0              # fold 2: 1
    A[:, 3 * F], B[3 * F, :] = -(2.0 ** 12), 2.0 ** 12   # fold 3: -2^24
    C0 = np.zeros((M, N), np.float32)
    ref = oracle.gemm_f64(M, N, K, 1.0, A, B, 0.0, None)
    assert np.all(ref == 2.0)
    cid = _config(mode, kb=kb)
    plain, _ = run_plan(mode, M, N, K, 1.0, A, B, 0.0, C0, False, cid)
    comp, _ = run_plan(mode, M, N, K, 1.0, A, B, 0.0, C0, True, cid)
    assert np.all(plain == 0.0)
    assert np.all(comp == 2.0)


@pytest.mark.parametrize("mode", TC_MODES)
@pytest.mark.parametrize("shape,pad", [((777, 300, 1500), 3), ((1060, 1060, 1060), 0), ((130, 64, 4099), 1)])
def test_matches_oracle(mode, shape, pad):
    M, N, K = shape
    A = W.uniform(M, K, 11, ld=K + pad)
    B = W.uniform(K, N, 12, ld=N + pad)
    C0 = W.uniform(M, N, 13, ld=N + pad)
    ref = oracle.gemm_f64(M, N, K, 1.5, A, B, 0.5, C0)
    got, _ = run_plan(mode, M, N, K, 1.5, A, B, 0.5, C0, True)
    err = oracle.rel_frob(got[:, :N], ref)
    assert err <= TOL, err
    check_padding_untouched(C0, got, N)
    if mode == "bf16x6":
        f32 = oracle.gemm_f32_seq(M, N, K, 1.5, A, B, 0.5, C0)
        assert err <= 2.0 * max(oracle.rel_frob(f32, ref), 2.0 ** -24), err


@pytest.mark.parametrize("mode", TC_MODES)
@pytest.mark.parametrize("split_k", [1, 3])
def test_integer_inputs_bit_exact(mode, split_k):
    M, N, K = 513, 260, 2000
    A, B, C0 = W.integers(M, K, 21), W.integers(K, N, 22), W.integers(M, N, 23)
    ref = oracle.gemm_f64(M, N, K, 1.0, A, B, 0.5, C0).astype(np.float32)
    got, _ = run_plan(mode, M, N, K, 1.0, A, B, 0.5, C0, True, _config(mode, split_k=split_k))
    assert np.array_equal(got, ref)


@pytest.mark.parametrize("mode", ("bf16x3", "tf32x3"))
def test_other_configurations_run_the_narrow_tile(mode):
    """A wider, CTA-pair or fused-split configuration asked for with the
    option runs the single-CTA packed 128 x 64 tile with the same split-K and
    raster group: the same result bits as that configuration asked for
    directly."""
    M, N, K = 700, 520, 900
    A, B, C0 = W.uniform(M, K, 31), W.uniform(K, N, 32), W.uniform(M, N, 33)
    single = _config(mode, block_n=64, split_k=1, kb=4, group_m=16)
    want, info = run_plan(mode, M, N, K, 1.25, A, B, 0.5, C0, True, single)
    assert info["config_id"] == single
    for other in (_config(mode, block_n=128, split_k=1, kb=4, group_m=16),
                  _config(mode, block_n=256, split_k=1, kb=4, group_m=16, cluster=2),
                  _config(mode, block_n=128, split_k=1, kb=4, group_m=16, fused=1)):
        got, info = run_plan(mode, M, N, K, 1.25, A, B, 0.5, C0, True, other)
        assert info["config_id"] == single
        assert np.array_equal(got, want)


@pytest.mark.parametrize("mode", ("tf32x3", "bf16x6"))
def test_more_accurate_than_plain_fold_sum(mode):
    """K = 8192: with the same tiles, the compensated epilogue (folds of one
    k-chunk, summed with TwoSum) has a smaller error against the FP64
    definition than the plain one (folds of 4 chunks, plain FP32 sum)."""
    M, N, K = 1024, 1024, 8192
    A, B = W.uniform(M, K, 41), W.uniform(K, N, 42)
    C0 = np.zeros((M, N), np.float32)
    ref = oracle.gemm_f64(M, N, K, 1.0, A, B, 0.0, None)
    cid = _config(mode, block_n=64, kb=4)
    plain, _ = run_plan(mode, M, N, K, 1.0, A, B, 0.0, C0, False, cid)
    comp, _ = run_plan(mode, M, N, K, 1.0, A, B, 0.0, C0, True, cid)
    e_plain, e_comp = oracle.rel_frob(plain, ref), oracle.rel_frob(comp, ref)
    print(f"{mode} K=8192 rel_frob: plain fold sum {e_plain:.3e}, compensated {e_comp:.3e}")
    assert e_comp < e_plain <= TOL
