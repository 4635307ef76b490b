// Units of work of the persistent tensor-core kernels, the order in which
// output tiles are walked, and the clearing of a plan's per-execution state.
#pragma once
#include "ptx.cuh"

namespace gb {

// One unit of work of a CTA (or CTA pair): an output tile (tm, tn) of
// problem `prob` and the range [c0, c1) of 128-byte k-chunks it covers (all
// of K unless split), ks being the split's index.
struct Work {
  int prob, tm, tn, ks, c0, c1;
};

// Tile t of a tiles_m x tiles_n grid in grouped raster order: groups of
// group_m tile rows, each group walked column by column, so that the CTAs
// running at the same time share rows of A and columns of B in L2.
__device__ __forceinline__ void raster(int t, int tiles_m, int tiles_n, int group_m, int& tm, int& tn) {
  const int group_tiles = group_m * tiles_n;
  const int g = t / group_tiles;
  const int first_m = g * group_m;
  const int rows_in_group = min(tiles_m - first_m, group_m);
  const int r = t % group_tiles;
  tm = first_m + r % rows_in_group;
  tn = r / rows_in_group;
}

// A plan's per-execution state (block maxima, pack counters, the unit
// counter of a dynamic tile order) must be zero when the next execution's
// first kernel starts.  Instead of a memset before every execution, the last
// CTA of the gemm launch to finish clears it: every CTA counts itself done
// on `done` (the word after the state) once all its threads have finished
// with the state, and the CTA that completes the count -- all others have
// then stopped reading -- zeroes the state and then the count.  The count
// is an acquire-release atomic at GPU scope: its release (cumulative over
// the CTA after the barrier) orders the CTA's reads of the state before it,
// and the last CTA's acquire orders every count before its zeroing.  Every
// thread of the CTA calls this, after a CTA barrier that follows its last
// read of the state.  nwords == 0: nothing to clear.
__device__ __forceinline__ void clear_execution_state(unsigned* state, int nwords) {
  if (nwords <= 0) return;   // uniform over the grid
  __shared__ int s_last;
  unsigned* done = state + nwords;
  if (threadIdx.x == 0)
    s_last = atom_add_acq_rel_gpu(done, 1u) == gridDim.x * gridDim.y * gridDim.z - 1 ? 1 : 0;
  __syncthreads();
  if (s_last) {
    for (int i = threadIdx.x; i < nwords; i += blockDim.x) state[i] = 0u;
    if (threadIdx.x == 0) *done = 0u;
  }
}

}  // namespace gb
