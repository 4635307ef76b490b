"""GPU parity of the CTA-pair configurations (256-row output tiles on a pair
of SMs, one tcgen05 cta_group::2 operation over both) against the FP64
oracle, through the C ABI.

Edge cases particular to pairs: a matrix whose last 256-row tile leaves the
second CTA's rows partly or wholly outside M (the peer loads a zero-filled
box and stores nothing), tiles whose second half of columns lies past N,
splits of K and unaligned leading dimensions.  Integer inputs are
bit-exact (a schedule must not change the answer, Tiramisu Section III)."""
import numpy as np
import pytest
import oracle
import paper_1804_10694_gb300 as pkg
import workloads as W
from gpu_helpers import TOL, check_padding_untouched, run_gemm

pytestmark = pytest.mark.gpu


def pair_ids(mode, **want):
    return [i for i in range(pkg.config_count(mode))
            if pkg.config_get(mode, i)["cluster"] == 2
            and all(pkg.config_get(mode, i)[k] == v for k, v in want.items())]


def single_twin(mode, cid):
    """The single-CTA configuration with the same width, split, fold and group."""
    c = pkg.config_get(mode, cid)
    for i in range(pkg.config_count(mode)):
        d = pkg.config_get(mode, i)
        if d["cluster"] == 1 and not d["fused"] and all(
                d[k] == c[k] for k in ("block_n", "split_k", "kb", "group_m")):
            return i
    return None


SHAPES = [
    (300, 65, 129, 0),     # last pair tile: CTA 0 rows 256..299, CTA 1 wholly past M; N < BN/2 + 2
    (129, 700, 1000, 3),   # one pair tile, 1 row in CTA 1; unaligned leading dimensions
    (777, 513, 333, 1),    # ragged everywhere
    (256, 256, 64, 0),     # exactly one tile, one k-chunk
    (1, 1, 1, 0),
    (2048, 1024, 700, 0),  # several waves of tiles
]


@pytest.mark.parametrize("mode", ["bf16x3", "tf32x3", "bf16x6"])
@pytest.mark.parametrize("M,N,K,pad", SHAPES)
def test_pair_configurations_against_oracle(mode, M, N, K, pad):
    A = W.uniform(M, K, 601, ld=K + pad)
    B = W.uniform(K, N, 602, ld=N + pad)
    C0 = W.uniform(M, N, 603, ld=N + pad)
    ref = oracle.gemm_f64(M, N, K, 1.5, A, B, 0.5, C0)
    ids = pair_ids(mode, group_m=16, kb=4) + pair_ids(mode, split_k=3, kb=2, group_m=1)
    assert ids
    for cid in ids:
        got = run_gemm(mode, M, N, K, 1.5, A, B, 0.5, C0, config_id=cid)
        err = oracle.rel_frob(got, ref)
        assert err <= TOL, (pkg.config_get(mode, cid), err)
        check_padding_untouched(C0, got, N)


@pytest.mark.parametrize("mode", ["bf16x3", "tf32x3", "bf16x6"])
def test_pair_integer_inputs_bit_exact(mode):
    M, N, K = 700, 650, 1100
    A, B, C0 = W.integers(M, K, 611), W.integers(K, N, 612), W.integers(M, N, 613)
    ref = oracle.gemm_f64(M, N, K, 1.5, A, B, 0.5, C0).astype(np.float32)
    for cid in pair_ids(mode, kb=4, group_m=16):
        got = run_gemm(mode, M, N, K, 1.5, A, B, 0.5, C0, config_id=cid)
        assert np.array_equal(got, ref), pkg.config_get(mode, cid)


def test_pair_agrees_with_single_cta_twin():
    """A pair tile and a single-CTA tile accumulate the same products in the
    same k order and fold at the same chunks: their results agree to far
    below the error bound (and, where the tensor core's accumulation does
    not depend on the tile height, bit for bit)."""
    M, N, K = 1000, 768, 2000
    A, B, C0 = W.uniform(M, K, 621), W.uniform(K, N, 622), W.uniform(M, N, 623)
    for cid in pair_ids("bf16x3", block_n=128, group_m=16):
        twin = single_twin("bf16x3", cid)
        p = run_gemm("bf16x3", M, N, K, 1.0, A, B, 0.0, C0, config_id=cid)
        s = run_gemm("bf16x3", M, N, K, 1.0, A, B, 0.0, C0, config_id=twin)
        assert oracle.rel_frob(p, s.astype(np.float64)) <= 1e-6, pkg.config_get("bf16x3", cid)


def test_pair_wide_range_and_scaling():
    """Per-block exponents: A's blocks are 128 rows, one per CTA of a pair;
    B's are 128 columns, one per epilogue warpgroup of a 256-wide tile."""
    M, N, K = 600, 520, 900
    A = W.wide_range(M, K, 631)
    B = W.wide_range(K, N, 632)
    A[:128] = W.scaled(A[:128], -90)          # one block of rows far below the safe range
    B[:, 256:384] = W.scaled(B[:, 256:384], 70)
    C0 = W.uniform(M, N, 633)
    ref = oracle.gemm_f64(M, N, K, 1.0, A, B, 0.0, C0)
    for cid in pair_ids("bf16x3", kb=4, group_m=16, split_k=1):
        got = run_gemm("bf16x3", M, N, K, 1.0, A, B, 0.0, C0, config_id=cid)
        assert oracle.rel_frob(got, ref) <= TOL, pkg.config_get("bf16x3", cid)


def test_pair_large_square_whole_matrix():
    """4096^3 on the 256 x 256 pair tile and on the 256 x 128 one (several
    waves of units on every pair of SMs), the whole result against the
    oracle."""
    n = 4096
    sa, sb, sc = W.seeds(W.CONFIG_SWEEP)
    A, B, C0 = W.uniform(n, n, sa), W.uniform(n, n, sb), W.uniform(n, n, sc)
    P = oracle.product_f64(n, n, n, A, B)
    ref = oracle.axpby_f64(1.5, P, 0.5, C0)
    for bn in (256, 128):
        cid = pair_ids("bf16x3", block_n=bn, split_k=1, kb=4, group_m=16)[0]
        got = run_gemm("bf16x3", n, n, n, 1.5, A, B, 0.5, C0, config_id=cid)
        assert oracle.rel_frob(got, ref) <= TOL, bn
    pkg.device_error()


def test_default_picks_pairs_and_host_panel_pipeline_runs_them():
    """4096 x 2048 x 1024: the default tile choice takes the 256 x 256 pair
    tile (its estimate: 2 waves of pair units against 4 of 128 x 128 units
    and 7 of 128 x 64 units).  Through
    gemm_f32_host with page-locked buffers the row-panel pipeline runs it:
    panels of an even number of 128-row tiles, each launch starting at an
    even 128-row block; unaligned ldc, padding untouched."""
    import torch
    M, N, K = 4096, 2048, 1024
    cid = pkg.config_default("bf16x3", M, N, K)
    c = pkg.config_get("bf16x3", cid)
    assert c["cluster"] == 2 and c["block_n"] == 256, c
    A, B, C0 = W.uniform(M, K, 651, ld=K + 4), W.uniform(K, N, 652), W.uniform(M, N, 653, ld=N + 2)
    ref = oracle.gemm_f64(M, N, K, 1.5, A, B, 0.5, C0)
    lib = pkg.load()
    hA, hB = torch.from_numpy(A).pin_memory(), torch.from_numpy(B).pin_memory()
    hC = torch.from_numpy(C0.copy()).pin_memory()
    st = lib.gemm_f32_host(M, N, K, 1.5, hA.data_ptr(), K + 4, hB.data_ptr(), N, 0.5, hC.data_ptr(),
                           N + 2, pkg.MODES["bf16x3"], None)
    assert st == 0, lib.gemm_last_error()
    got = hC.numpy()
    assert oracle.rel_frob(got, ref) <= TOL
    check_padding_untouched(C0, got, N)
