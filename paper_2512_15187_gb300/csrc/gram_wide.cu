// Instantiations of the tensor-core Gram kernel for 128 < N <= 256 (the wide tile of
// gram_kernel.cuh: 16 warps own 256 operand rows, two M = 128 row blocks per K step).
#include "gram_kernel.cuh"

namespace pidk {

cudaError_t launch_gram_wide(const GramParams& p, int prec, int iso_kind, int grid, size_t smem,
                             cudaStream_t s) {
  return gram_tile_launch<16, 16, true>(p, prec, iso_kind, grid, smem, s);
}

cudaError_t gram_wide_init(int max_smem) { return gram_tile_init<16, 16, true>(max_smem); }

}  // namespace pidk
