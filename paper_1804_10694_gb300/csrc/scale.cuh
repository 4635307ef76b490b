// Power-of-two block scaling used by the split pass and undone by the gemm
// epilogue.  All of it is exponent-field arithmetic on FP32 bit patterns.
#pragma once
#include <cstdint>

namespace gb {

// Blocks whose max |x| lies in [2^-kSafeExp, 2^kSafeExp) are not scaled
// (e = 0): without scaling, no product of two such values, no sum of up to
// 2^31 of them and no low part of their significant elements leaves the
// normal range, so a scale would bring no accuracy.  Only blocks outside that
// range (tiny or huge operands) are rescaled.
constexpr int kSafeExp = 48;

// Block exponent from the bit pattern of the block's max |x|: 0 for an
// all-zero block, a block holding Inf/NaN (bit pattern >= 0x7F800000) or a
// block in the safe range; otherwise floor(log2(max)) clamped to [-126, 126].
__host__ __device__ __forceinline__ int block_exponent(unsigned amax_bits) {
  if (amax_bits == 0u || amax_bits >= 0x7F800000u) return 0;
  int e = static_cast<int>((amax_bits >> 23) & 0xFFu) - 127;
  if (e >= -kSafeExp && e < kSafeExp) return 0;
  if (e < -126) e = -126;
  if (e > 126) e = 126;
  return e;
}

// 2^e as an FP32 value for e in [-126, 127] (a normal number), built from bits.
__device__ __forceinline__ float pow2f(int e) {
  return __uint_as_float(static_cast<unsigned>(e + 127) << 23);
}

// x * 2^e for e in [-252, 252], exact unless the result leaves the normal
// range: the factor is applied as two normal powers of two.
__device__ __forceinline__ float scale_pow2(float x, int e) {
  const int e1 = e / 2;
  const int e2 = e - e1;
  return (x * pow2f(e1)) * pow2f(e2);
}

}  // namespace gb
