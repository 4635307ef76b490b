"""Pins of the convolution oracle against what the definition fixes (no GPU):
filters whose result is known in closed form, an independently built patch
matrix times the gemm oracle, and exact rational brute force."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from oracle import conv
import workloads as W


def test_identity_filter_returns_the_image():
    x = W.conv_image(2, 5, 7, 3, 1)
    f = np.zeros((3, 3, 3, 3), np.float32)
    f[1, 1] = np.eye(3)
    assert np.array_equal(conv.conv3x3_f64(x, f), x.astype(np.float64))


def test_corner_tap_shifts_the_image_with_zero_border():
    """Tap (r, s) = (0, 0) reads in[h - 1, w - 1]: the output is the image
    shifted down and right, zero in the first row and column.  A swapped
    tap order or a wrong padding fails here."""
    x = W.conv_image(1, 6, 4, 2, 2)
    f = np.zeros((3, 3, 2, 2), np.float32)
    f[0, 0] = np.eye(2)
    got = conv.conv3x3_f64(x, f)
    want = np.zeros_like(got)
    want[:, 1:, 1:, :] = x[:, :-1, :-1, :]
    assert np.array_equal(got, want)
    f = np.zeros((3, 3, 2, 2), np.float32)
    f[2, 1] = np.eye(2)          # reads in[h + 1, w]: shifted up
    got = conv.conv3x3_f64(x, f)
    want = np.zeros_like(got)
    want[:, :-1, :, :] = x[:, 1:, :, :]
    assert np.array_equal(got, want)


def _patches(x):
    """Patch matrix built by explicit loops: row = output pixel, column =
    (r, s, c) in that order."""
    n, H, Wd, C = x.shape
    P = np.zeros((n * H * Wd, 9 * C), np.float32)
    for b in range(n):
        for h in range(H):
            for w in range(Wd):
                row = (b * H + h) * Wd + w
                for r in range(3):
                    for s in range(3):
                        hh, ww = h + r - 1, w + s - 1
                        if 0 <= hh < H and 0 <= ww < Wd:
                            P[row, (r * 3 + s) * C:(r * 3 + s + 1) * C] = x[b, hh, ww]
    return P


def test_equals_patch_matrix_times_filter_matrix():
    x = W.conv_image(2, 9, 11, 5, 3)
    f = W.conv_filter(5, 7, 4)
    out0 = W.uniform(2 * 9 * 11, 7, 5).reshape(2, 9, 11, 7)
    P = _patches(x)
    ref = oracle.gemm_f64(P.shape[0], 7, 9 * 5, 1.5, P, f.reshape(45, 7), 0.5, out0.reshape(-1, 7))
    got = conv.conv3x3_f64(x, f, 1.5, 0.5, out0).reshape(-1, 7)
    assert np.abs(got - ref).max() <= 1e-12 * np.abs(ref).max()


def test_pixels_form_matches_whole_output():
    x = W.conv_image(1, 13, 10, 4, 6)
    f = W.conv_filter(4, 3, 7)
    out0 = W.uniform(130, 3, 8).reshape(1, 13, 10, 3)
    full = conv.conv3x3_f64(x, f, 2.0, -1.0, out0).reshape(-1, 3)
    pix = [0, 9, 10, 64, 129]
    assert np.allclose(conv.conv3x3_pixels_f64(pix, x, f, 2.0, -1.0, out0), full[pix], rtol=0, atol=1e-12)


def test_exact_brute_force_on_integers():
    x = W.conv_image(1, 4, 3, 2, 9, kind="integers")
    f = W.conv_filter(2, 3, 10, kind="integers")
    out0 = W.conv_image(1, 4, 3, 3, 11, kind="integers")
    ex = conv.conv3x3_exact(x, f, 1.5, 0.5, out0)
    got = conv.conv3x3_f64(x, f, 1.5, 0.5, out0)
    for b in range(1):
        for h in range(4):
            for w in range(3):
                for k in range(3):
                    assert float(ex[b][h][w][k]) == got[b, h, w, k]


# ------------------------------------------------- other odd filter sizes
@pytest.mark.parametrize("R,S", [(1, 1), (5, 5), (7, 3), (3, 9), (11, 11)])
def test_centre_tap_is_identity_for_every_size(R, S):
    x = W.conv_image(2, 6, 13, 3, 21)
    f = np.zeros((R, S, 3, 3), np.float32)
    f[R // 2, S // 2] = np.eye(3)
    assert np.array_equal(conv.conv_f64(x, f), x.astype(np.float64))


@pytest.mark.parametrize("R,S,r,s", [(5, 5, 0, 0), (5, 5, 4, 1), (7, 3, 6, 2), (11, 11, 2, 9)])
def test_off_centre_tap_shifts_by_its_offset(R, S, r, s):
    """Tap (r, s) reads in[h + r - (R-1)/2, w + s - (S-1)/2], zero outside."""
    x = W.conv_image(1, 12, 14, 2, 22)
    f = np.zeros((R, S, 2, 2), np.float32)
    f[r, s] = np.eye(2)
    got = conv.conv_f64(x, f)
    dh, dw = r - R // 2, s - S // 2
    want = np.zeros_like(got)
    H, Wd = 12, 14
    for h in range(H):
        for w in range(Wd):
            if 0 <= h + dh < H and 0 <= w + dw < Wd:
                want[0, h, w] = x[0, h + dh, w + dw]
    assert np.array_equal(got, want)


def test_one_by_one_filter_is_a_pixel_matrix_product():
    x = W.conv_image(3, 5, 4, 6, 23)
    f = W.conv_filter(6, 5, 24, R=1, S=1)
    want = (x.reshape(-1, 6).astype(np.float64) @ f[0, 0].astype(np.float64)).reshape(3, 5, 4, 5)
    assert np.array_equal(conv.conv_f64(x, f), want)


@pytest.mark.parametrize("R,S", [(5, 5), (9, 7), (11, 11)])
def test_box_filter_equals_window_sums_of_the_integral_image(R, S):
    """All-ones filter on one channel: each output is the sum of the image
    over its R x S window (zero outside), read off a summed-area table."""
    x = W.conv_image(1, 17, 15, 1, 25, kind="integers")
    f = np.ones((R, S, 1, 1), np.float32)
    got = conv.conv_f64(x, f)[0, :, :, 0]
    H, Wd = 17, 15
    img = x[0, :, :, 0].astype(np.float64)
    I = np.zeros((H + 1, Wd + 1))
    I[1:, 1:] = img.cumsum(0).cumsum(1)
    for h in range(H):
        for w in range(Wd):
            h1, h2 = max(0, h - R // 2), min(H, h + R // 2 + 1)
            w1, w2 = max(0, w - S // 2), min(Wd, w + S // 2 + 1)
            assert got[h, w] == I[h2, w2] - I[h1, w2] - I[h2, w1] + I[h1, w1]


def _patches_rs(x, R, S):
    n, H, Wd, C = x.shape
    P = np.zeros((n * H * Wd, R * S * C), np.float32)
    for b in range(n):
        for h in range(H):
            for w in range(Wd):
                row = (b * H + h) * Wd + w
                for r in range(R):
                    for s in range(S):
                        hh, ww = h + r - R // 2, w + s - S // 2
                        if 0 <= hh < H and 0 <= ww < Wd:
                            P[row, (r * S + s) * C:(r * S + s + 1) * C] = x[b, hh, ww]
    return P


@pytest.mark.parametrize("R,S", [(5, 5), (7, 3)])
def test_rs_equals_patch_matrix_times_filter_matrix(R, S):
    x = W.conv_image(2, 8, 9, 3, 26)
    f = W.conv_filter(3, 4, 27, R=R, S=S)
    out0 = W.uniform(2 * 8 * 9, 4, 28).reshape(2, 8, 9, 4)
    P = _patches_rs(x, R, S)
    ref = oracle.gemm_f64(P.shape[0], 4, R * S * 3, 1.5, P, f.reshape(R * S * 3, 4), 0.5, out0.reshape(-1, 4))
    got = conv.conv_f64(x, f, 1.5, 0.5, out0).reshape(-1, 4)
    assert np.abs(got - ref).max() <= 1e-12 * np.abs(ref).max()
    pix = [0, 17, 71, 143]
    assert np.allclose(conv.conv_pixels_f64(pix, x, f, 1.5, 0.5, out0), got[pix], rtol=0, atol=1e-12)


def test_rs_exact_brute_force():
    x = W.conv_image(1, 5, 4, 2, 29)
    f = W.conv_filter(2, 2, 30, R=5, S=3)
    ex = conv.conv_exact(x, f)
    got = conv.conv_f64(x, f)
    for h in range(5):
        for w in range(4):
            for k in range(2):
                assert abs(float(ex[0][h][w][k]) - got[0, h, w, k]) <= 1e-15 * max(1.0, abs(got[0, h, w, k]))
