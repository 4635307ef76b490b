// The gemm epilogue's last step, shared by the tensor-core kernels: undo the
// per-block power-of-two scaling of the operands, apply alpha and beta, and
// store a warp's 32 rows of an output tile (or a split-K partial).
#pragma once
#include <cstdint>

#include "ptx.cuh"
#include "scale.cuh"

namespace gb {

// Per-problem values the epilogue needs.
struct EpiView {
  int M, N;
  float* C;
  int64_t ldc;
  float alpha, beta;
  const unsigned* amaxA;
  const unsigned* amaxB;
  float* partial;
  int split_k;
  int amaxA_stride;         // 1: one exponent per 128-row block; 0: one for all of A
};

// One thread holds S[0 .. EC) = the FP32 sums of row row0 + lane, columns
// col0 .. col0 + EC - 1, in units of 2^-(eA + eB) (e = eA + eB); the warp
// covers rows row0 .. row0 + 31.  Writes alpha * 2^e * S + beta * C to C
// (or alpha * 2^e * S to split ks's partial-sum plane when split_k > 1);
// rows >= M and columns >= N are masked.  buf: this warp's 32 x PITCH float
// staging buffer in shared memory.
template <int EC, int PITCH>
__device__ __forceinline__ void epilogue_store(float (&S)[EC], const EpiView& v, int e, int ks, int row0,
                                               int col0, int lane, float* buf) {
  // undo the block scaling, acc * 2^(eA + eB).  With e != 0 alpha is
  // applied before the power of two, so that a result in range is not
  // lost to an overflow of the unscaled sum (the power of two is exact).
  float alpha = v.alpha;
  float beta = v.beta;
  if (v.split_k > 1 || e != 0) {
#pragma unroll
    for (int i = 0; i < EC; ++i) S[i] = e != 0 ? scale_pow2(alpha * S[i], e) : alpha * S[i];
    alpha = 1.0f;
  }
  // destination: C, or this split's partial-sum plane (the reduction
  // kernel adds beta * C)
  float* dst = v.C;
  int64_t ldd = v.ldc;
  if (v.split_k > 1) {
    dst = v.partial + static_cast<int64_t>(ks) * v.M * v.N;
    ldd = v.N;
    beta = 0.0f;
  }
  // Two store paths, chosen per 32-column chunk and uniform per warp.
  // Aligned rows and a full chunk: each thread stores its own row with
  // float4 accesses (C loads of the chunk issued first).  Otherwise
  // (unaligned ldc, partial chunk or rows): the warp brings the 32x32
  // chunk of C into a padded shared buffer by cp.async (lane = column,
  // every row in flight at once; beta != 0), combines it with its sums
  // there (lane = row), then walks the buffer one row at a time (lane =
  // column), so that every global access of the warp covers 128
  // contiguous bytes of one row whatever the alignment.
  const int nrows = min(32, v.M - row0);
  const bool rows_vec = nrows == 32 && (ldd & 3) == 0 && (reinterpret_cast<uintptr_t>(dst) & 15) == 0;
#pragma unroll
  for (int j = 0; j < EC / 32; ++j) {
    const int cb = col0 + j * 32;
    if (nrows <= 0 || cb >= v.N) break;   // uniform across the warp
    if (rows_vec && cb + 32 <= v.N) {
      float4* c4 = reinterpret_cast<float4*>(dst + static_cast<int64_t>(row0 + lane) * ldd + cb);
      float4 old[8];
      if (beta != 0.0f) {
#pragma unroll
        for (int i = 0; i < 8; ++i) old[i] = c4[i];
      }
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        const float* sv = &S[j * 32 + 4 * i];
        float4 o;
        if (beta != 0.0f) {
          o.x = fmaf(alpha, sv[0], beta * old[i].x);
          o.y = fmaf(alpha, sv[1], beta * old[i].y);
          o.z = fmaf(alpha, sv[2], beta * old[i].z);
          o.w = fmaf(alpha, sv[3], beta * old[i].w);
        } else {
          o.x = alpha * sv[0];
          o.y = alpha * sv[1];
          o.z = alpha * sv[2];
          o.w = alpha * sv[3];
        }
        c4[i] = o;
      }
      continue;
    }
    const bool col_ok = cb + lane < v.N;
    float* base = dst + static_cast<int64_t>(row0) * ldd + cb + lane;
    if (beta != 0.0f) {
      // the chunk of C comes into the buffer by 4-byte cp.async copies
      // (lane = column, each row 128 contiguous bytes), all 32 rows in
      // flight at once, then combines with the row-held sums in place
      const float* src = base;
      uint32_t sdst = smem_u32(&buf[lane]);
#pragma unroll 4
      for (int r = 0; r < 32; ++r) {
        const bool in = col_ok && r < nrows;
        cp_async_4(sdst, in ? src : dst, in ? 4u : 0u);
        src += ldd;
        sdst += PITCH * 4;
      }
      cp_async_commit();
      cp_async_wait_all();
      __syncwarp();
#pragma unroll
      for (int i = 0; i < 32; ++i) {
        float* bp = &buf[lane * PITCH + i];
        *bp = fmaf(alpha, S[j * 32 + i], beta * *bp);
      }
    } else {
#pragma unroll
      for (int i = 0; i < 32; ++i) buf[lane * PITCH + i] = alpha * S[j * 32 + i];
    }
    __syncwarp();
    {
      float* out = base;
#pragma unroll 4
      for (int r = 0; r < 32; ++r) {
        if (col_ok && r < nrows) *out = buf[r * PITCH + lane];
        out += ldd;
      }
    }
    __syncwarp();
  }
}

}  // namespace gb
