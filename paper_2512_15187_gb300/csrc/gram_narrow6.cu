// Instantiations of the narrow tensor-core Gram tile with 6 members per warp: 48 rows for
// 8-warp groups (N <= 48) and 96 rows for 16-warp groups (64 < N <= 96), so that the
// converter warps of a partly filled tile do not map and convert empty rows.
#include "gram_kernel.cuh"

namespace pidk {

cudaError_t launch_gram_narrow6(const GramParams& p, int G, int prec, int iso_kind, int grid,
                                size_t smem, cudaStream_t s) {
  if (G == 8) return gram_tile_launch<8, 6>(p, prec, iso_kind, grid, smem, s);
  if (G == 16) return gram_tile_launch<16, 6>(p, prec, iso_kind, grid, smem, s);
  return cudaErrorInvalidValue;
}

cudaError_t gram_narrow6_init(int max_smem) {
  cudaError_t e = gram_tile_init<8, 6>(max_smem);
  return e == cudaSuccess ? gram_tile_init<16, 6>(max_smem) : e;
}

}  // namespace pidk
