"""FP64 oracle for the direct convolution (stride 1, "same" zero padding,
odd filter sizes R x S; the 3x3 case has padding 1) -- test infrastructure
only; see the package docstring.

The paper benchmarks convolutions (its Conv and VGG layers, Section VI, with
filter sizes specialised from 3x3 to 11x11); as a gemm, a convolution is the
product of the image's patch matrix with the filter matrix.  The oracle is
the definition written out, with pR = (R - 1) / 2 and pS = (S - 1) / 2:

    out[n, h, w, k] = alpha * sum_{r, s, c} in[n, h + r - pR, w + s - pS, c] * f[r, s, c, k]
                      + beta * out0[n, h, w, k]

with in[...] = 0 outside the image.  Images are NHWC (channels contiguous),
the filter is RSCK (r: row tap, s: column tap, c: input channel, k: output
channel).  Accumulation is in float64, one filter tap at a time (R*S shifted
channel products, each a library matrix product).  ``conv_exact`` is an
independent restatement in exact rationals for tiny cases.
"""
from __future__ import annotations

from fractions import Fraction

import numpy as np


def _taps(f: np.ndarray, C: int) -> tuple[int, int, int, int]:
    R, S = int(f.shape[0]), int(f.shape[1])
    assert R % 2 == 1 and S % 2 == 1 and f.shape[2] == C, f.shape
    return R, S, (R - 1) // 2, (S - 1) // 2


def conv_f64(inp: np.ndarray, f: np.ndarray, alpha: float = 1.0, beta: float = 0.0,
             out0: np.ndarray | None = None) -> np.ndarray:
    """The whole output, float64."""
    x = np.asarray(inp, np.float64)
    w = np.asarray(f, np.float64)
    n, H, W, C = x.shape
    R, S, pr, ps = _taps(w, C)
    K = w.shape[3]
    pad = np.zeros((n, H + 2 * pr, W + 2 * ps, C))
    pad[:, pr:pr + H, ps:ps + W, :] = x
    acc = np.zeros((n, H, W, K))
    for r in range(R):
        for s in range(S):
            patch = pad[:, r:r + H, s:s + W, :].reshape(-1, C)
            acc += (patch @ w[r, s]).reshape(n, H, W, K)
    out = float(alpha) * acc
    if beta != 0.0:
        out += float(beta) * np.asarray(out0, np.float64)
    return out


def conv_pixels_f64(pixels, inp: np.ndarray, f: np.ndarray, alpha: float = 1.0,
                    beta: float = 0.0, out0: np.ndarray | None = None) -> np.ndarray:
    """Output rows of the listed pixels (flat index n*H*W + h*W + w), float64,
    shape [len(pixels), K]: for large images, checked pixel by pixel."""
    x = np.asarray(inp, np.float64)
    w = np.asarray(f, np.float64)
    n, H, W, C = x.shape
    R, S, pr, ps = _taps(w, C)
    K = w.shape[3]
    out = np.zeros((len(pixels), K))
    for i, p in enumerate(pixels):
        b, rem = divmod(int(p), H * W)
        h, col = divmod(rem, W)
        for r in range(R):
            for s in range(S):
                hh, ww = h + r - pr, col + s - ps
                if 0 <= hh < H and 0 <= ww < W:
                    out[i] += x[b, hh, ww, :] @ w[r, s]
    out *= float(alpha)
    if beta != 0.0:
        out += float(beta) * np.asarray(out0, np.float64).reshape(-1, K)[list(pixels)]
    return out


def conv_exact(inp: np.ndarray, f: np.ndarray, alpha: float = 1.0, beta: float = 0.0,
               out0: np.ndarray | None = None):
    """Exact rational result for tiny cases (pure Python loops over every
    output element, tap and channel)."""
    n, H, W, C = inp.shape
    R, S, pr, ps = _taps(np.asarray(f), C)
    K = f.shape[3]
    a, bt = Fraction(float(alpha)), Fraction(float(beta))
    out = [[[[Fraction(0)] * K for _ in range(W)] for _ in range(H)] for _ in range(n)]
    for b in range(n):
        for h in range(H):
            for col in range(W):
                for k in range(K):
                    s_ = Fraction(0)
                    for r in range(R):
                        for s in range(S):
                            hh, ww = h + r - pr, col + s - ps
                            if not (0 <= hh < H and 0 <= ww < W):
                                continue
                            for c in range(C):
                                s_ += Fraction(float(inp[b, hh, ww, c])) * Fraction(float(f[r, s, c, k]))
                    v = a * s_
                    if bt != 0:
                        v += bt * Fraction(float(out0[b, h, col, k]))
                    out[b][h][col][k] = v
    return out


# the 3x3 names (padding 1)
def conv3x3_f64(inp, f, alpha=1.0, beta=0.0, out0=None):
    assert f.shape[:2] == (3, 3), f.shape
    return conv_f64(inp, f, alpha, beta, out0)


def conv3x3_pixels_f64(pixels, inp, f, alpha=1.0, beta=0.0, out0=None):
    assert f.shape[:2] == (3, 3), f.shape
    return conv_pixels_f64(pixels, inp, f, alpha, beta, out0)


def conv3x3_exact(inp, f, alpha=1.0, beta=0.0, out0=None):
    assert f.shape[:2] == (3, 3), f.shape
    return conv_exact(inp, f, alpha, beta, out0)
