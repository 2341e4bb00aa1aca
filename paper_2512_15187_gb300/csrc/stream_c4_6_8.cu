// Streaming-pass instantiations for the tile class VEC=4, MPW=6, G=8.
#include "stream_kernel.cuh"

namespace pidk {

cudaError_t launch_stream_c4_6_8(const StreamParams& p, int iso, bool coef, int grid,
                                  size_t smem, cudaStream_t s) {
  return StreamClass<4, 6, 8>::launch(p, iso, coef, grid, smem, s);
}

cudaError_t init_stream_c4_6_8(int smem) { return StreamClass<4, 6, 8>::init(smem); }

}  // namespace pidk
