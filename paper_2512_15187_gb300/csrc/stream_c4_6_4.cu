// Streaming-pass instantiations for the tile class VEC=4, MPW=6, G=4.
#include "stream_kernel.cuh"

namespace pidk {

cudaError_t launch_stream_c4_6_4(const StreamParams& p, int iso, bool coef, int grid,
                                  size_t smem, cudaStream_t s) {
  return StreamClass<4, 6, 4>::launch(p, iso, coef, grid, smem, s);
}

cudaError_t init_stream_c4_6_4(int smem) { return StreamClass<4, 6, 4>::init(smem); }

}  // namespace pidk
