// Split arithmetic shared by the packing pass and the fused-split gemm
// kernel, so that both write bit-identical hi/lo values:
//     hi = RN(x'),  lo = RN(x' - hi)
// with RN round-to-nearest-even to bf16 (hardware conversion) or to tf32
// (bit arithmetic; tf32 values are kept in 32-bit containers).  A non-finite
// x' gives hi = x', lo = 0.  The six-product bf16 mode splits in three:
//     hi = RN(x'),  mid = RN(x' - hi),  lo = RN((x' - hi) - mid).
// Every difference is one FP32 subtraction of the rounded x' (__fsub_rn
// keeps it from being fused with the multiply that scaled x).
#pragma once
#include <cuda_bf16.h>

namespace gb {

__device__ __forceinline__ float round_tf32_rne(float x) {
  const unsigned u = __float_as_uint(x);
  if ((u & 0x7F800000u) == 0x7F800000u) return x;   // Inf / NaN unchanged
  const unsigned r = (u + 0xFFFu + ((u >> 13) & 1u)) & 0xFFFFE000u;
  return __uint_as_float(r);
}

struct HiLoBf16 {
  __nv_bfloat16 hi, lo;
};

__device__ __forceinline__ HiLoBf16 split_bf16(float xs) {
  HiLoBf16 o;
  o.hi = __float2bfloat16_rn(xs);
  o.lo = isfinite(xs) ? __float2bfloat16_rn(__fsub_rn(xs, __bfloat162float(o.hi))) : __float2bfloat16_rn(0.0f);
  return o;
}

struct Split3Bf16 {
  __nv_bfloat16 hi, mid, lo;
};

__device__ __forceinline__ Split3Bf16 split3_bf16(float xs) {
  Split3Bf16 o;
  o.hi = __float2bfloat16_rn(xs);
  if (isfinite(xs)) {
    const float r1 = __fsub_rn(xs, __bfloat162float(o.hi));   // exact
    o.mid = __float2bfloat16_rn(r1);
    o.lo = __float2bfloat16_rn(__fsub_rn(r1, __bfloat162float(o.mid)));
  } else {
    o.mid = o.lo = __float2bfloat16_rn(0.0f);
  }
  return o;
}

__device__ __forceinline__ void split_tf32(float xs, float& hi, float& lo) {
  hi = round_tf32_rne(xs);
  lo = isfinite(xs) ? round_tf32_rne(__fsub_rn(xs, hi)) : 0.0f;
}

// |x| as an orderable bit pattern (non-negative floats order like their bits;
// NaN patterns sort above Inf, so a NaN marks the block as non-finite).
__device__ __forceinline__ unsigned abs_bits(float x) { return __float_as_uint(x) & 0x7FFFFFFFu; }

}  // namespace gb
