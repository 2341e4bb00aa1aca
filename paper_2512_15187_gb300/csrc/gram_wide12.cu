// Instantiations of the wide tensor-core Gram tile with 12 member rows per warp (192 rows)
// for 128 < N <= 192: the converter warps skip the rows the 256-row tile would leave empty.
#include "gram_kernel.cuh"

namespace pidk {

cudaError_t launch_gram_wide12(const GramParams& p, int prec, int iso_kind, int grid,
                               size_t smem, cudaStream_t s) {
  return gram_tile_launch<16, 12, true>(p, prec, iso_kind, grid, smem, s);
}

cudaError_t gram_wide12_init(int max_smem) { return gram_tile_init<16, 12, true>(max_smem); }

}  // namespace pidk
