// Instantiations of the wide tensor-core Gram tile with 13 member rows per warp (208 rows)
// for 192 < N <= 208 (the 3D plume workload's 200 members): the converter warps skip the
// rows the 256-row tile would leave empty.
#include "gram_kernel.cuh"

namespace pidk {

cudaError_t launch_gram_wide13(const GramParams& p, int prec, int iso_kind, int grid,
                               size_t smem, cudaStream_t s) {
  return gram_tile_launch<16, 13, true>(p, prec, iso_kind, grid, smem, s);
}

cudaError_t gram_wide13_init(int max_smem) { return gram_tile_init<16, 13, true>(max_smem); }

}  // namespace pidk
