"""Pins of the convolution oracle against what the definition fixes (no GPU):
filters whose result is known in closed form, an independently built patch
matrix times the gemm oracle, and exact rational brute force."""
from __future__ import annotations

import numpy as np

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
