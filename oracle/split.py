"""Oracle for the operand split of the split-precision products (numpy, slow,
element by element in vectorised form) -- test infrastructure only.

The paper packs operands before the gemm main loop ("array packing", Section I
and Section VI-A).  Here packing also splits each FP32 value into a high and a
low part of lower precision, so that three tensor-core products
hi*hi + hi*lo + lo*hi recover FP32 accuracy (Henry, Tang & Heinecke, ARITH 2019,
for bf16; the tf32 form is the same with 11-bit significands).  Readings taken
where the paper is silent (it does not describe this method at all):

* Block scaling: A is scaled per block of 128 rows (all of K), B per block of
  128 columns (all of K).  The block exponent is e = floor(log2(max |x|)),
  clamped to [-126, 126], for blocks whose max lies outside [2**-48, 2**48);
  e = 0 for blocks inside that range (there no product, no sum of up to
  2**31 products and no low part of a significant element leaves the normal
  range, so scaling brings nothing), for all-zero blocks and for blocks
  holding a non-finite value.  The scaled value is x * 2**-e, one FP32
  multiply.
* hi = RN(x'), lo = RN(x' - hi) with RN round-to-nearest-even to bf16 (8-bit
  significand) or tf32 (11-bit significand); x' - hi is an FP32 subtraction.
  A non-finite x' gives hi = x', lo = 0.
* The BF16x6 mode splits in three: hi, mid = RN(x' - hi), lo =
  RN((x' - hi) - mid); hi + mid + lo = x' exactly for normal x' (8 + 8 + 8
  significant bits cover FP32's 24).

All rounding here is written from the IEEE definition on the bit pattern.
"""
from __future__ import annotations

import numpy as np

BLOCK = 128  # rows of A / columns of B sharing one exponent


def _bits(x: np.ndarray) -> np.ndarray:
    return np.ascontiguousarray(x, dtype=np.float32).view(np.uint32)


def round_bf16(x: np.ndarray) -> np.ndarray:
    """Round FP32 values to the nearest bf16 value (ties to even), returned as
    FP32.  NaN stays NaN, +-Inf stays, overflow past the largest bf16 gives
    +-Inf (as IEEE rounding does)."""
    u = _bits(x).astype(np.uint64)
    keep = (u >> 16) & 1
    r = ((u + 0x7FFF + keep) & 0xFFFF0000).astype(np.uint32)
    out = r.view(np.float32).copy()
    nan = np.isnan(x)
    out[nan] = np.float32(np.nan)
    return out


def round_tf32(x: np.ndarray) -> np.ndarray:
    """Round FP32 values to the nearest tf32 value (10 stored significand bits,
    ties to even), returned as FP32 with the low 13 bits zero."""
    u = _bits(x).astype(np.uint64)
    keep = (u >> 13) & 1
    r = ((u + 0xFFF + keep) & 0xFFFFE000).astype(np.uint32)
    out = r.view(np.float32).copy()
    nan = np.isnan(x)
    out[nan] = np.float32(np.nan)
    return out


SAFE_EXP = 48  # blocks with max |x| in [2**-48, 2**48) are not scaled


def block_exponent(absmax: float) -> int:
    """0 for 0, non-finite or max in [2**-48, 2**48); else floor(log2(absmax))
    clamped to [-126, 126]."""
    a = float(absmax)
    if a == 0.0 or not np.isfinite(a):
        return 0
    bits = int(np.array([a], dtype=np.float32).view(np.uint32)[0])
    e = ((bits >> 23) & 0xFF) - 127          # -127 for a subnormal maximum
    if -SAFE_EXP <= e < SAFE_EXP:
        return 0
    return max(-126, min(126, e))


def pow2(e: int) -> np.float32:
    """2**e as an FP32 value (e within the normal range)."""
    return np.float32(np.ldexp(1.0, e))


def split_values(xs: np.ndarray, rounder) -> tuple[np.ndarray, np.ndarray]:
    """hi = RN(x'), lo = RN(x' - hi) for already-scaled FP32 values x'."""
    xs = np.asarray(xs, dtype=np.float32)
    hi = rounder(xs)
    finite = np.isfinite(xs)
    with np.errstate(invalid="ignore", over="ignore"):
        diff = (xs - hi).astype(np.float32)
    lo = rounder(np.where(finite, diff, np.float32(0.0)).astype(np.float32))
    hi = np.where(finite, hi, xs).astype(np.float32)
    return hi, lo


def split3_values(xs: np.ndarray) -> tuple[np.ndarray, np.ndarray, np.ndarray]:
    """Three-way bf16 split of already-scaled FP32 values (the BF16x6 mode):
    hi = RN(x'), mid = RN(x' - hi), lo = RN((x' - hi) - mid), each
    difference an FP32 subtraction (exact: the remainders have at most 16 and
    8 significant bits).  A non-finite x' gives hi = x', mid = lo = 0."""
    xs = np.asarray(xs, dtype=np.float32)
    finite = np.isfinite(xs)
    with np.errstate(invalid="ignore", over="ignore"):
        hi = round_bf16(xs)
        r1 = np.where(finite, (xs - hi).astype(np.float32), np.float32(0.0)).astype(np.float32)
        mid = round_bf16(r1)
        r2 = (r1 - mid).astype(np.float32)
        lo = round_bf16(r2)
    hi = np.where(finite, hi, xs).astype(np.float32)
    return hi, mid, lo


def split_rows(X: np.ndarray, rows: int, cols: int, precision: str):
    """Split a row-major matrix whose rows are grouped in blocks of 128 (the A
    operand; B is passed transposed, i.e. as N x K).  Returns (hi, lo, exps)
    with hi/lo rows x cols FP32 arrays and one exponent per 128-row block;
    for precision "bf16x6", (hi, mid, lo, exps)."""
    rounder = round_bf16 if precision in ("bf16", "bf16x6") else round_tf32
    X = np.asarray(X, dtype=np.float32)[:rows, :cols]
    nblk = (rows + BLOCK - 1) // BLOCK
    hi = np.zeros((rows, cols), np.float32)
    lo = np.zeros((rows, cols), np.float32)
    lo2 = np.zeros((rows, cols), np.float32)
    exps = np.zeros(nblk, np.int32)
    for b in range(nblk):
        blk = X[b * BLOCK:(b + 1) * BLOCK]
        amax = np.max(np.abs(blk)) if blk.size else np.float32(0.0)
        if blk.size and np.isnan(blk).any():
            amax = np.float32(np.nan)
        e = block_exponent(amax)
        exps[b] = e
        with np.errstate(over="ignore", invalid="ignore"):
            scaled = (blk * pow2(-e)).astype(np.float32)
        if precision == "bf16x6":
            h, l, l2 = split3_values(scaled)
            lo2[b * BLOCK:(b + 1) * BLOCK] = l2
        else:
            h, l = split_values(scaled, rounder)
        hi[b * BLOCK:(b + 1) * BLOCK] = h
        lo[b * BLOCK:(b + 1) * BLOCK] = l
    if precision == "bf16x6":
        return hi, lo, lo2, exps        # hi, mid, lo
    return hi, lo, exps
