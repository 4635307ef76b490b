"""Parity of the direct convolution (3x3 and other odd R x S filters, as an
implicit gemm) with the convolution oracle, and with the gemm path on an
explicitly formed patch matrix (same split, same MMAs: bit for bit).  Two
paths: packed (bf16 modes, C a multiple of 16: the image split once into
planes, 16-channel im2col boxes of them) and fused-split (the FP32 patches
staged and split inside the kernel)."""
from __future__ import annotations

import math

import numpy as np
import pytest
import torch

import oracle
from oracle import conv
import paper_1804_10694_gb300 as pkg
import workloads as W
from gpu_helpers import TOL

pytestmark = pytest.mark.gpu


def run_conv(x, f, alpha, beta, out0, mode="bf16x3", config_id=None):
    n, H, Wd, C = x.shape
    R, S, _, K = f.shape
    plan = pkg.ConvPlan(n, H, Wd, C, K, R, S, mode=mode, config_id=config_id)
    dx, df, do = (torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in (x, f, out0))
    plan.execute(dx, df, do, alpha, beta)
    torch.cuda.synchronize()
    cid = plan.info()["config_id"]
    plan.destroy()
    return do.cpu().numpy(), cid


def patches(x, R=3, S=3):
    """Patch matrix, row = output pixel, column = (r, s, c)."""
    n, H, Wd, C = x.shape
    pr, ps = R // 2, S // 2
    pad = np.zeros((n, H + 2 * pr, Wd + 2 * ps, C), np.float32)
    pad[:, pr:pr + H, ps:ps + Wd] = x
    cols = [pad[:, r:r + H, s:s + Wd, :].reshape(-1, C) for r in range(R) for s in range(S)]
    return np.ascontiguousarray(np.concatenate(cols, axis=1))


def fused_ids(mode, **want):
    out = []
    for i in range(pkg.config_count(mode)):
        c = pkg.config_get(mode, i)
        if c["fused"] and all(c[k] == v for k, v in want.items()):
            out.append(i)
    return out


def packed_ids(mode, **want):
    out = []
    for i in range(pkg.config_count(mode)):
        c = pkg.config_get(mode, i)
        if not c["fused"] and c["cluster"] == 1 and all(c[k] == v for k, v in want.items()):
            out.append(i)
    return out


def path_config(path, mode="bf16x3"):
    """None (the default path) or the first fused configuration of the
    default tile shape."""
    return None if path == "default" else fused_ids(mode, block_n=64, group_m=16, kb=4, split_k=1)[0]


@pytest.mark.parametrize("mode", ["bf16x3", "tf32x3"])
def test_small_images_match_oracle(mode):
    x = W.conv_image(2, 9, 13, 8, 101)
    f = W.conv_filter(8, 12, 102)
    out0 = W.conv_image(2, 9, 13, 12, 103)
    ref = conv.conv3x3_f64(x, f, 1.5, 0.5, out0)
    got, _ = run_conv(x, f, 1.5, 0.5, out0, mode)
    assert oracle.rel_frob(got.reshape(-1, 12), ref.reshape(-1, 12)) <= TOL


@pytest.mark.parametrize("mode", ["bf16x3", "tf32x3"])
def test_integer_images_bit_exact(mode):
    x = W.conv_image(1, 17, 11, 12, 104, kind="integers")
    f = W.conv_filter(12, 20, 105, kind="integers")
    out0 = W.conv_image(1, 17, 11, 20, 106, kind="integers")
    ref = conv.conv3x3_f64(x, f, 1.5, 0.5, out0).astype(np.float32)
    got, _ = run_conv(x, f, 1.5, 0.5, out0, mode)
    assert np.array_equal(got, ref)


@pytest.mark.parametrize("mode", ["bf16x3", "tf32x3"])
def test_every_fused_configuration_equals_gemm_on_patch_matrix(mode):
    """The patch matrix the kernel gathers, formed explicitly and run through
    the gemm with the same configuration, gives the same bits (uniform data:
    both use exponent 0)."""
    x = W.conv_image(2, 11, 7, 16, 107)
    f = W.conv_filter(16, 40, 108)
    out0 = W.conv_image(2, 11, 7, 40, 109)
    P = patches(x)
    M, Kd, K = P.shape[0], P.shape[1], 40
    dP, dB = torch.from_numpy(P).cuda(), torch.from_numpy(f.reshape(Kd, K).copy()).cuda()
    ref = conv.conv3x3_f64(x, f, 1.0, -0.5, out0).reshape(-1, K)
    for cid in fused_ids(mode):
        got, _ = run_conv(x, f, 1.0, -0.5, out0, mode, config_id=cid)
        dC = torch.from_numpy(out0.reshape(-1, K).copy()).cuda()
        plan = pkg.Plan(M, K, Kd, mode=mode, config_id=cid)
        plan.execute(dP, dB, dC, 1.0, -0.5)
        torch.cuda.synchronize()
        plan.destroy()
        assert np.array_equal(got.reshape(-1, K).view(np.uint32), dC.cpu().numpy().view(np.uint32)), \
            pkg.config_get(mode, cid)
        assert oracle.rel_frob(got.reshape(-1, K), ref) <= TOL


@pytest.mark.parametrize("mode,C", [("bf16x3", 64), ("tf32x3", 32), ("bf16x3", 128)])
def test_im2col_staging_equals_gemm_on_patch_matrix(mode, C):
    """Channel counts whose chunks are whole taps are staged by TMA's im2col
    mode (offsets per tap, zero outside the image, rows wrapping across image
    rows and images); same bits as the gemm on the formed patch matrix."""
    x = W.conv_image(2, 7, 10, C, 150 + C)
    f = W.conv_filter(C, 24, 151)
    out0 = W.conv_image(2, 7, 10, 24, 152)
    P = patches(x)
    M, Kd, K = P.shape[0], P.shape[1], 24
    dP, dB = torch.from_numpy(P).cuda(), torch.from_numpy(f.reshape(Kd, K).copy()).cuda()
    for cid in fused_ids(mode, group_m=16, kb=4)[::3]:
        got, _ = run_conv(x, f, 1.5, 0.5, out0, mode, config_id=cid)
        dC = torch.from_numpy(out0.reshape(-1, K).copy()).cuda()
        plan = pkg.Plan(M, K, Kd, mode=mode, config_id=cid)
        plan.execute(dP, dB, dC, 1.5, 0.5)
        torch.cuda.synchronize()
        plan.destroy()
        assert np.array_equal(got.reshape(-1, K).view(np.uint32), dC.cpu().numpy().view(np.uint32)), \
            pkg.config_get(mode, cid)


def test_degenerate_images():
    # 1x1 images: only the centre tap sees data; a one-pixel-wide image; C = 4, K = 1
    for (n, H, Wd, C, K) in [(3, 1, 1, 4, 5), (1, 7, 1, 8, 3), (2, 5, 6, 4, 1)]:
        x = W.conv_image(n, H, Wd, C, 110 + H)
        f = W.conv_filter(C, K, 120 + Wd)
        out0 = np.zeros((n, H, Wd, K), np.float32)
        ref = conv.conv3x3_f64(x, f)
        got, _ = run_conv(x, f, 1.0, 0.0, out0)
        assert oracle.rel_frob(got.reshape(-1, K), ref.reshape(-1, K)) <= TOL, (n, H, Wd, C, K)


def test_whole_image_exponent_keeps_tiny_inputs():
    """One power-of-two exponent for the whole image: inputs near 2^-100
    keep their low parts."""
    x = W.scaled(W.conv_image(1, 20, 20, 8, 130), -100)
    f = W.conv_filter(8, 16, 131)
    ref = conv.conv3x3_f64(x, f)
    got, _ = run_conv(x, f, 1.0, 0.0, np.zeros((1, 20, 20, 16), np.float32))
    assert oracle.rel_frob(got.reshape(-1, 16), ref.reshape(-1, 16)) <= TOL


@pytest.mark.parametrize("layer", W.CONV3X3_LAYERS)
def test_full_size_layers_sampled_pixels(layer):
    n, H, Wd, C, K = layer
    x = W.conv_image(n, H, Wd, C, 140)
    f = W.conv_filter(C, K, 141)
    got, cid = run_conv(x, f, 1.0, 0.0, np.zeros((n, H, Wd, K), np.float32))
    rng = np.random.default_rng(7)
    pix = sorted(set(rng.choice(n * H * Wd, 96, replace=False).tolist()) |
                 {0, Wd - 1, (H - 1) * Wd, H * Wd - 1})
    ref = conv.conv3x3_pixels_f64(pix, x, f)
    assert oracle.rel_frob(got.reshape(-1, K)[pix], ref) <= TOL


def test_misaligned_image_is_rejected():
    plan = pkg.Conv3x3Plan(1, 4, 4, 4, 4)
    buf = torch.zeros(1 + 4 * 4 * 4, device="cuda")
    f = torch.zeros(3, 3, 4, 4, device="cuda")
    out = torch.zeros(1, 4, 4, 4, device="cuda")
    lib = pkg.load()
    st = lib.gemm_plan_execute(plan._h, 1.0, buf.data_ptr() + 4, f.data_ptr(), 0.0, out.data_ptr(), None)
    assert st == 2   # GEMM_ERR_ALIGNMENT
    plan.destroy()


# ------------------------------------------------- other odd filter sizes
RS = [(1, 1), (5, 5), (7, 3), (3, 9), (11, 11)]


@pytest.mark.parametrize("R,S", RS)
@pytest.mark.parametrize("mode,C", [("bf16x3", 8), ("bf16x3", 64), ("tf32x3", 32), ("bf16x3", 16),
                                    ("bf16x3", 48), ("tf32x3", 16)])
@pytest.mark.parametrize("path", ["default", "fused"])
def test_rs_filters_match_oracle(R, S, mode, C, path):
    """Default path: packed for the bf16 mode with C = 16, 48, 64 (the last
    chunk is partial when R*S*C is not a multiple of 64: its boxes past K are
    neither loaded nor multiplied).  Fused path: gathered (C = 8), staged by
    im2col in 32-channel boxes (whole-tap chunks) and in 16-channel boxes."""
    x = W.conv_image(2, 13, 9, C, 160 + R)
    f = W.conv_filter(C, 20, 161 + S, R=R, S=S)
    out0 = W.conv_image(2, 13, 9, 20, 162)
    ref = conv.conv_f64(x, f, 1.5, 0.5, out0)
    got, _ = run_conv(x, f, 1.5, 0.5, out0, mode, config_id=path_config(path, mode))
    assert oracle.rel_frob(got.reshape(-1, 20), ref.reshape(-1, 20)) <= TOL, (R, S)


@pytest.mark.parametrize("R,S,C", [(5, 5, 16), (11, 11, 16), (7, 7, 64)])
def test_rs_integer_images_bit_exact(R, S, C):
    x = W.conv_image(1, 15, 12, C, 163, kind="integers")
    f = W.conv_filter(C, 24, 164, kind="integers", R=R, S=S)
    out0 = W.conv_image(1, 15, 12, 24, 165, kind="integers")
    ref = conv.conv_f64(x, f, 1.5, 0.5, out0).astype(np.float32)
    got, _ = run_conv(x, f, 1.5, 0.5, out0)
    assert np.array_equal(got, ref)


@pytest.mark.parametrize("R,S,C", [(5, 5, 64), (7, 3, 64), (11, 11, 64), (5, 5, 12), (5, 5, 16),
                                   (3, 3, 48), (11, 11, 16), (3, 3, 32)])
def test_rs_equals_gemm_on_patch_matrix(R, S, C):
    x = W.conv_image(2, 9, 11, C, 166)
    f = W.conv_filter(C, 40, 167, R=R, S=S)
    out0 = W.conv_image(2, 9, 11, 40, 168)
    P = patches(x, R, S)
    M, Kd, K = P.shape[0], P.shape[1], 40
    dP, dB = torch.from_numpy(P).cuda(), torch.from_numpy(f.reshape(Kd, K).copy()).cuda()
    for cid in fused_ids("bf16x3", group_m=16, kb=4)[::4]:
        got, _ = run_conv(x, f, 1.0, -0.5, out0, config_id=cid)
        dC = torch.from_numpy(out0.reshape(-1, K).copy()).cuda()
        plan = pkg.Plan(M, K, Kd, mode="bf16x3", config_id=cid)
        plan.execute(dP, dB, dC, 1.0, -0.5)
        torch.cuda.synchronize()
        plan.destroy()
        assert np.array_equal(got.reshape(-1, K).view(np.uint32), dC.cpu().numpy().view(np.uint32)), \
            (R, S, C, pkg.config_get("bf16x3", cid))


@pytest.mark.parametrize("R", W.CONV_FILTER_SIZES[::2])
def test_paper_conv_layer_sampled_pixels(R):
    """The paper's Conv layer: 32 images of 512 x 512 x 16, 16 output
    features, R x R filters; sampled pixels including image corners."""
    n, H, Wd, C, K = W.CONV_PAPER_LAYER
    x = W.conv_image(n, H, Wd, C, 170)
    f = W.conv_filter(C, K, 171, R=R, S=R)
    got, _ = run_conv(x, f, 1.0, 0.0, np.zeros((n, H, Wd, K), np.float32))
    rng = np.random.default_rng(R)
    hw = H * Wd
    pix = sorted(set(rng.choice(n * hw, 64, replace=False).tolist()) |
                 {0, Wd - 1, (H - 1) * Wd, hw - 1, (n - 1) * hw, n * hw - 1})
    ref = conv.conv_pixels_f64(pix, x, f)
    assert oracle.rel_frob(got.reshape(-1, K)[pix], ref) <= TOL, R


@pytest.mark.parametrize("path", ["default", "fused"])
@pytest.mark.parametrize("mode,C,R", [("bf16x3", 16, 3), ("bf16x3", 48, 5), ("tf32x3", 16, 3), ("bf16x3", 8, 3)])
def test_infinite_pixel_reaches_only_its_windows(mode, C, R, path):
    """An Inf pixel makes exactly the outputs whose window holds it
    non-finite: the unloaded part of a partial last chunk is split as zeros
    (fused) or not multiplied (packed), never taken from taps past the
    filter or from stale shared memory."""
    x = W.conv_image(1, 12, 10, C, 180)
    x[0, 5, 5, 3] = np.inf
    f = W.conv_filter(C, 16, 181, R=R, S=R)
    ref = conv.conv_f64(x, f).reshape(-1, 16)
    got, _ = run_conv(x, f, 1.0, 0.0, np.zeros((1, 12, 10, 16), np.float32), mode,
                      config_id=path_config(path, mode))
    got = got.reshape(-1, 16)
    assert np.array_equal(np.isfinite(got), np.isfinite(ref))
    rows = np.isfinite(ref).all(axis=1)
    assert rows.sum() > 0 and oracle.rel_frob(got[rows], ref[rows]) <= TOL


# ----------------------------------------------------------- packed path
def test_packed_path_is_the_default_where_it_applies():
    for mode, C, fused in [("bf16x3", 16, False), ("bf16x3", 48, False), ("bf16x6", 32, False),
                           ("tf32x3", 16, False), ("tf32x3", 64, False),
                           ("bf16x3", 8, True), ("bf16x3", 12, True), ("tf32x3", 24, True)]:
        plan = pkg.ConvPlan(1, 6, 5, C, 8, 3, 3, mode=mode)
        cid = plan.info()["config_id"]
        plan.destroy()
        assert pkg.config_get(mode, cid)["fused"] == int(fused), (mode, C)


@pytest.mark.parametrize("mode", ["bf16x3", "bf16x6", "tf32x3"])
@pytest.mark.parametrize("R,S,C", [(3, 3, 16), (5, 5, 16), (3, 3, 48), (7, 3, 64), (1, 1, 32)])
def test_packed_configurations_equal_gemm_on_patch_matrix(mode, R, S, C):
    """The packed kernel multiplies the split image's planes through im2col
    boxes; the gemm on the formed patch matrix, same configuration, splits
    the same values and issues the same MMAs in the same order (uniform data:
    exponent 0 for both): same bits, for tile widths 64 and 128, folds and
    split-K."""
    x = W.conv_image(2, 9, 11, C, 190 + C)
    f = W.conv_filter(C, 40, 191, R=R, S=S)
    out0 = W.conv_image(2, 9, 11, 40, 192)
    P = patches(x, R, S)
    M, Kd, K = P.shape[0], P.shape[1], 40
    dP, dB = torch.from_numpy(P).cuda(), torch.from_numpy(f.reshape(Kd, K).copy()).cuda()
    ref = conv.conv_f64(x, f, 1.0, -0.5, out0).reshape(-1, K)
    for cid in packed_ids(mode)[::5]:
        got, _ = run_conv(x, f, 1.0, -0.5, out0, mode, config_id=cid)
        dC = torch.from_numpy(out0.reshape(-1, K).copy()).cuda()
        plan = pkg.Plan(M, K, Kd, mode=mode, config_id=cid)
        plan.execute(dP, dB, dC, 1.0, -0.5)
        torch.cuda.synchronize()
        plan.destroy()
        assert np.array_equal(got.reshape(-1, K).view(np.uint32), dC.cpu().numpy().view(np.uint32)), \
            (R, S, C, pkg.config_get(mode, cid))
        assert oracle.rel_frob(got.reshape(-1, K), ref) <= TOL


@pytest.mark.parametrize("mode", ["bf16x3", "tf32x3"])
@pytest.mark.parametrize("shift", [-100, 60])
def test_packed_image_exponent_rescales(shift, mode):
    """An image outside [2^-48, 2^48) takes the whole-image exponent: the
    second split pass re-splits it scaled, so tiny inputs keep their low
    parts and large ones do not overflow the products."""
    x = W.scaled(W.conv_image(1, 20, 20, 16, 193), shift)
    f = W.conv_filter(16, 16, 194)
    ref = conv.conv_f64(x, f)
    got, cid = run_conv(x, f, 1.0, 0.0, np.zeros((1, 20, 20, 16), np.float32), mode)
    assert not pkg.config_get(mode, cid)["fused"]
    assert oracle.rel_frob(got.reshape(-1, 16), ref.reshape(-1, 16)) <= TOL


@pytest.mark.parametrize("R,C", [(3, 16), (11, 16), (5, 32)])
def test_packed_bf16x6_integer_and_uniform(R, C):
    xi = W.conv_image(2, 10, 13, C, 195, kind="integers")
    fi = W.conv_filter(C, 24, 196, kind="integers", R=R, S=R)
    oi = W.conv_image(2, 10, 13, 24, 197, kind="integers")
    got, _ = run_conv(xi, fi, 1.5, 0.5, oi, "bf16x6")
    assert np.array_equal(got, conv.conv_f64(xi, fi, 1.5, 0.5, oi).astype(np.float32))
    x = W.conv_image(2, 10, 13, C, 198)
    f = W.conv_filter(C, 24, 199, R=R, S=R)
    ref = conv.conv_f64(x, f).reshape(-1, 24)
    e6 = oracle.rel_frob(run_conv(x, f, 1.0, 0.0, np.zeros((2, 10, 13, 24), np.float32), "bf16x6")[0]
                         .reshape(-1, 24), ref)
    e3 = oracle.rel_frob(run_conv(x, f, 1.0, 0.0, np.zeros((2, 10, 13, 24), np.float32), "bf16x3")[0]
                         .reshape(-1, 24), ref)
    assert e6 <= TOL and e6 * 3.0 < e3, (e6, e3)


@pytest.mark.parametrize("mode", ["bf16x3", "bf16x6", "tf32x3"])
@pytest.mark.parametrize("n,H,Wd,C,K,R", [(3, 5, 7, 32, 200, 3), (1, 1, 1, 16, 8, 5), (2, 1, 9, 64, 130, 3),
                                          (1, 17, 3, 48, 64, 7)])
def test_packed_wide_outputs_and_small_images(mode, n, H, Wd, C, K, R):
    """Several output-channel tiles (K = 200, 130), 1x1 and one-row images
    (taps almost all in the padding), 64-channel boxes next to 16-channel
    ones."""
    x = W.conv_image(n, H, Wd, C, 200 + C)
    f = W.conv_filter(C, K, 201, R=R, S=R)
    out0 = W.conv_image(n, H, Wd, K, 202)
    ref = conv.conv_f64(x, f, 1.5, 0.5, out0).reshape(-1, K)
    got, cid = run_conv(x, f, 1.5, 0.5, out0, mode)
    assert not pkg.config_get(mode, cid)["fused"]
    assert oracle.rel_frob(got.reshape(-1, K), ref) <= TOL


@pytest.mark.parametrize("mode", ["bf16x3", "tf32x3", "bf16x6"])
@pytest.mark.parametrize("path", ["packed", "fused"])
def test_plan_state_is_clean_between_executions(mode, path):
    """The image exponent, B's block maxima and counters and the dynamic tile
    order's unit counter are cleared by the last CTA of each execution's gemm
    launch: one plan run on an image that needs scaling (2^-100), then an
    ordinary one, then the first again gives the bits of a fresh plan each
    time."""
    if mode == "bf16x6" and path == "fused":
        pytest.skip("BF16X6 convolutions run packed only")
    n, H, Wd, C, K = 2, 20, 24, 32, 48
    base = W.conv_image(n, H, Wd, C, 111)
    images = [W.scaled(base, -100), base]
    f = W.conv_filter(C, K, 112)
    out0 = W.conv_image(n, H, Wd, K, 113)
    cid = None if path == "packed" else fused_ids(mode, block_n=64, group_m=16, kb=4, split_k=1)[0]
    fresh = [run_conv(x, f, 1.5, 0.5, out0, mode, cid)[0] for x in images]
    plan = pkg.ConvPlan(n, H, Wd, C, K, 3, 3, mode=mode, config_id=cid)
    df = torch.from_numpy(f).cuda()
    for i in (0, 1, 0, 1):
        dx = torch.from_numpy(np.ascontiguousarray(images[i])).cuda()
        do = torch.from_numpy(out0.copy()).cuda()
        plan.execute(dx, df, do, 1.5, 0.5)
        torch.cuda.synchronize()
        assert np.array_equal(do.cpu().numpy(), fresh[i]), i
    plan.destroy()
    pkg.device_error()


@pytest.mark.parametrize("mode", ["bf16x3", "tf32x3", "bf16x6"])
@pytest.mark.parametrize("K,R", [(16, 3), (32, 5), (7, 3)])
def test_few_output_features_narrow_tile(mode, K, R):
    """A default packed plan with at most 32 output features runs 128 x 32
    tiles, two CTAs a SM: within 1e-5 of the convolution oracle (ragged
    pixel count, K not a multiple of the tile), bit-exact on integers."""
    n, H, Wd, C = 2, 21, 37, 16
    x = W.conv_image(n, H, Wd, C, 131)
    f = W.conv_filter(C, K, 132, R=R, S=R)
    out0 = W.conv_image(n, H, Wd, K, 133)
    ref = conv.conv_f64(x, f, 1.5, 0.5, out0)
    got, _ = run_conv(x, f, 1.5, 0.5, out0, mode)
    assert oracle.rel_frob(got.reshape(-1, K), ref.reshape(-1, K)) <= TOL
    xi = W.conv_image(n, H, Wd, C, 134, kind="integers")
    fi = W.conv_filter(C, K, 135, kind="integers", R=R, S=R)
    zi = np.zeros((n, H, Wd, K), np.float32)
    refi = conv.conv_f64(xi, fi, 1.0, 0.0, zi).astype(np.float32)
    goti, _ = run_conv(xi, fi, 1.0, 0.0, zi, mode)
    assert np.array_equal(goti, refi)
    pkg.device_error()
