// Units of work of the persistent tensor-core kernels and the order in which
// output tiles are walked.
#pragma once

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

}  // namespace gb
