"""FP64 oracle for the direct 3x3 convolution (stride 1, zero padding 1) --
test infrastructure only; see the package docstring.

The paper benchmarks convolutions (its Conv and VGG layers, Section VI); as
a gemm, a 3x3 convolution is the product of the image's patch matrix with the
filter matrix.  The oracle is the definition written out:

    out[n, h, w, k] = alpha * sum_{r, s, c} in[n, h + r - 1, w + s - 1, c] * f[r, s, c, k]
                      + beta * out0[n, h, w, k]

with in[...] = 0 outside the image.  Images are NHWC (channels contiguous),
the filter is RSCK (r: row tap, s: column tap, c: input channel, k: output
channel).  Accumulation is in float64, one filter tap at a time (nine shifted
channel products, each a library matrix product).  ``conv3x3_exact`` is an
independent restatement in exact rationals for tiny cases.
"""
from __future__ import annotations

from fractions import Fraction

import numpy as np


def conv3x3_f64(inp: np.ndarray, f: np.ndarray, alpha: float = 1.0, beta: float = 0.0,
                out0: np.ndarray | None = None) -> np.ndarray:
    """The whole output, float64."""
    x = np.asarray(inp, np.float64)
    w = np.asarray(f, np.float64)
    n, H, W, C = x.shape
    assert w.shape[:3] == (3, 3, C), w.shape
    K = w.shape[3]
    pad = np.zeros((n, H + 2, W + 2, C))
    pad[:, 1:H + 1, 1:W + 1, :] = x
    acc = np.zeros((n, H, W, K))
    for r in range(3):
        for s in range(3):
            patch = pad[:, r:r + H, s:s + W, :].reshape(-1, C)
            acc += (patch @ w[r, s]).reshape(n, H, W, K)
    out = float(alpha) * acc
    if beta != 0.0:
        out += float(beta) * np.asarray(out0, np.float64)
    return out


def conv3x3_pixels_f64(pixels, inp: np.ndarray, f: np.ndarray, alpha: float = 1.0,
                       beta: float = 0.0, out0: np.ndarray | None = None) -> np.ndarray:
    """Output rows of the listed pixels (flat index n*H*W + h*W + w), float64,
    shape [len(pixels), K]: for large images, checked pixel by pixel."""
    x = np.asarray(inp, np.float64)
    w = np.asarray(f, np.float64)
    n, H, W, C = x.shape
    K = w.shape[3]
    out = np.zeros((len(pixels), K))
    for i, p in enumerate(pixels):
        b, rem = divmod(int(p), H * W)
        h, col = divmod(rem, W)
        for r in range(3):
            for s in range(3):
                hh, ww = h + r - 1, col + s - 1
                if 0 <= hh < H and 0 <= ww < W:
                    out[i] += x[b, hh, ww, :] @ w[r, s]
    out *= float(alpha)
    if beta != 0.0:
        out += float(beta) * np.asarray(out0, np.float64).reshape(-1, K)[list(pixels)]
    return out


def conv3x3_exact(inp: np.ndarray, f: np.ndarray, alpha: float = 1.0, beta: float = 0.0,
                  out0: np.ndarray | None = None):
    """Exact rational result for tiny cases (pure Python loops over every
    output element, tap and channel)."""
    n, H, W, C = inp.shape
    K = f.shape[3]
    a, bt = Fraction(float(alpha)), Fraction(float(beta))
    out = [[[[Fraction(0)] * K for _ in range(W)] for _ in range(H)] for _ in range(n)]
    for b in range(n):
        for h in range(H):
            for col in range(W):
                for k in range(K):
                    s_ = Fraction(0)
                    for r in range(3):
                        for s in range(3):
                            hh, ww = h + r - 1, col + s - 1
                            if not (0 <= hh < H and 0 <= ww < W):
                                continue
                            for c in range(C):
                                s_ += Fraction(float(inp[b, hh, ww, c])) * Fraction(float(f[r, s, c, k]))
                    v = a * s_
                    if bt != 0:
                        v += bt * Fraction(float(out0[b, h, col, k]))
                    out[b][h][col][k] = v
    return out
