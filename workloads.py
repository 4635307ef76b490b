"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle.

This module only draws numbers: it holds none of the gemm arithmetic (no
products, sums, splits or scaling), so both the CUDA path and the CPU oracle may
take their inputs from here without sharing any of the method's code.

Workloads (the paper measures sgemm on 1060x1060 matrices and on the matrix
products that implement convolutions, Section VI-A; the synthetic stand-ins
below keep those shapes and draw entries from fixed distributions):

* ``uniform``      -- iid uniform[-1, 1] drawn in float64, rounded to float32.
* ``wide_range``   -- sign * 2**u, u ~ U[-10, 10] continuous, sign a fair coin.
* ``wide_range_int_exp`` -- the same with integer u (entries exact in bf16).
* ``integers``     -- iid integers in [-8, 8] inclusive (products exact in fp32).
* ``grouped_shapes`` -- M, N, K each round(exp(U(ln 32, ln 1024))), clamped.

Seeds follow ``seed = 1000 * config_index + {0: A, 1: B, 2: C}``.
"""
from __future__ import annotations

import math

import numpy as np

# Square sweep (includes sizes that are not tile multiples: 1060 = 8*128 + 36,
# 4099 is prime) and the three conv-as-gemm shapes of 3x3 convolutions on
# 224x224 images (M = output pixels, N = output channels, K = 9 * in channels).
SQUARE_SWEEP = (1024, 1060, 2048, 4099, 8192)
CONV_SHAPES = ((50176, 64, 576), (12544, 128, 1152), (3136, 256, 2304))
# the 3x3 convolution layers behind CONV_SHAPES (batch, H, W, C in, K out):
# M = batch*H*W output pixels, N = K, K_gemm = 9*C
CONV3X3_LAYERS = ((1, 224, 224, 64, 64), (1, 112, 112, 128, 128), (1, 56, 56, 256, 256))
# the paper's Conv benchmark: 512 x 512 images, 16 input and output features,
# batch 32, filters specialised from 3x3 to 11x11 (batch, H, W, C, K)
CONV_PAPER_LAYER = (32, 512, 512, 16, 16)
CONV_FILTER_SIZES = (3, 5, 7, 9, 11)
ALPHA_BETA = ((1.0, 0.0), (1.5, 0.5))

CONFIG_SMALL = 0      # 512^3, alpha 1.5, beta 0.5
CONFIG_SWEEP = 1      # square sweep
CONFIG_WIDE = 2       # 8192^3 wide range + integer variant
CONFIG_GROUPED = 3    # 512 grouped problems
CONFIG_CONV = 4       # conv-as-gemm shapes


def seeds(config_index: int) -> tuple[int, int, int]:
    """Seeds for (A, B, C) of one workload configuration."""
    base = 1000 * config_index
    return base, base + 1, base + 2


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def uniform(rows: int, cols: int, seed: int, ld: int | None = None,
            pad_value: float = np.nan) -> np.ndarray:
    """rows x cols float32 matrix, iid uniform[-1, 1], stored with leading
    dimension ``ld`` (>= cols).  Padding columns hold ``pad_value`` (NaN by
    default) so that a kernel which reads outside the logical matrix poisons
    its result.  Returns the full rows x ld storage array."""
    vals = _rng(seed).uniform(-1.0, 1.0, size=(rows, cols)).astype(np.float32)
    return _with_ld(vals, ld, pad_value)


def wide_range(rows: int, cols: int, seed: int, ld: int | None = None,
               lo: float = -10.0, hi: float = 10.0,
               pad_value: float = np.nan) -> np.ndarray:
    """sign * 2**u with u ~ U[lo, hi] continuous (float64, then float32)."""
    g = _rng(seed)
    u = g.uniform(lo, hi, size=(rows, cols))
    sign = np.where(g.integers(0, 2, size=(rows, cols)) == 0, -1.0, 1.0)
    vals = (sign * np.exp2(u)).astype(np.float32)
    return _with_ld(vals, ld, pad_value)


def wide_range_int_exp(rows: int, cols: int, seed: int, ld: int | None = None,
                       lo: int = -10, hi: int = 10,
                       pad_value: float = np.nan) -> np.ndarray:
    """sign * 2**u with integer u uniform in [lo, hi]."""
    g = _rng(seed)
    u = g.integers(lo, hi + 1, size=(rows, cols)).astype(np.float64)
    sign = np.where(g.integers(0, 2, size=(rows, cols)) == 0, -1.0, 1.0)
    vals = (sign * np.exp2(u)).astype(np.float32)
    return _with_ld(vals, ld, pad_value)


def integers(rows: int, cols: int, seed: int, ld: int | None = None,
             lo: int = -8, hi: int = 8, pad_value: float = np.nan) -> np.ndarray:
    """iid integers in [lo, hi] inclusive, as float32."""
    vals = _rng(seed).integers(lo, hi + 1, size=(rows, cols)).astype(np.float32)
    return _with_ld(vals, ld, pad_value)


def int_pattern(i, k, a: int, b: int, m: int, off: int):
    """Integer entries (a*i + b*k) mod m - off at row indices i and column
    indices k (broadcastable integer arrays, numpy or torch alike; the caller
    converts to float32).  With m <= 17 they are exact in FP32, bf16 and tf32:
    closed-form inputs for problems too large to draw and copy from the host,
    whose rows can be rebuilt one at a time for the oracle."""
    return (a * i + b * k) % m - off


def scaled(arr: np.ndarray, log2_scale: int) -> np.ndarray:
    """Multiply by an exact power of two (input shaping for range tests)."""
    return (arr.astype(np.float64) * math.ldexp(1.0, log2_scale)).astype(np.float32)


def _with_ld(vals: np.ndarray, ld: int | None, pad_value: float) -> np.ndarray:
    rows, cols = vals.shape
    if ld is None or ld == cols:
        return np.ascontiguousarray(vals)
    if ld < cols:
        raise ValueError("leading dimension smaller than row length")
    out = np.full((rows, ld), pad_value, dtype=np.float32)
    out[:, :cols] = vals
    return out


def grouped_shapes(count: int = 512, seed: int = 4000, lo: int = 32,
                   hi: int = 1024) -> list[tuple[int, int, int]]:
    """(M, N, K) triples, each dimension round(exp(U(ln lo, ln hi))) clamped
    to [lo, hi], dimensions independent."""
    g = _rng(seed)
    u = g.uniform(math.log(lo), math.log(hi), size=(count, 3))
    dims = np.clip(np.rint(np.exp(u)), lo, hi).astype(np.int64)
    return [tuple(int(x) for x in row) for row in dims]


def training_shapes(count: int, seed: int, lo: int = 32, hi: int = 65536,
                    max_mnk_log2: float = 37.0,
                    max_elems: int = 2 ** 27) -> list[tuple[int, int, int]]:
    """Shapes for autotuner timing runs: log-uniform M, N, K in [lo, hi] with
    M*N*K <= 2**max_mnk_log2 and every operand at most max_elems elements
    (rejection sampled), plus conv-like skinny shapes (large M, N in
    {16..512}, K = 9 * channels)."""
    g = _rng(seed)
    out: list[tuple[int, int, int]] = []
    n_skinny = count // 5
    while len(out) < count - n_skinny:
        m, n, k = (int(x) for x in np.rint(np.exp(g.uniform(math.log(lo), math.log(hi), size=3))))
        if (math.log2(float(m) * float(n) * float(k)) <= max_mnk_log2
                and max(m * k, k * n, m * n) <= max_elems):
            out.append((m, n, k))
    chans = (16, 32, 64, 128, 256, 512)
    while len(out) < count:
        cin = int(g.choice(chans))
        cout = int(g.choice(chans))
        side = int(g.choice((7, 14, 28, 56, 112, 224)))
        m = side * side * int(g.choice((1, 2, 4)))
        k = 9 * cin
        if math.log2(float(m) * cout * k) <= max_mnk_log2 and m * k <= max_elems:
            out.append((m, cout, k))
    return out


def conv_image(batch: int, H: int, W: int, C: int, seed: int, kind: str = "uniform") -> np.ndarray:
    """NHWC float32 image: iid uniform[-1, 1], or integers in [-8, 8]."""
    rng = _rng(seed)
    if kind == "integers":
        return rng.integers(-8, 9, size=(batch, H, W, C)).astype(np.float32)
    return rng.uniform(-1.0, 1.0, size=(batch, H, W, C)).astype(np.float32)


def conv_filter(C: int, K: int, seed: int, kind: str = "uniform", R: int = 3, S: int = 3) -> np.ndarray:
    """RSCK float32 R x S filter (3x3 by default): iid uniform[-1, 1], or
    integers in [-8, 8]."""
    rng = _rng(seed)
    if kind == "integers":
        return rng.integers(-8, 9, size=(R, S, C, K)).astype(np.float32)
    return rng.uniform(-1.0, 1.0, size=(R, S, C, K)).astype(np.float32)
