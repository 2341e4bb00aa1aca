// Streaming-pass instantiations for the tile class VEC=1, MPW=28, G=16.
#include "stream_kernel.cuh"

namespace pidk {

cudaError_t launch_stream_c1_28_16(const StreamParams& p, int iso, bool coef, int grid,
                                  size_t smem, cudaStream_t s) {
  return StreamClass<1, 28, 16>::launch(p, iso, coef, grid, smem, s);
}

cudaError_t init_stream_c1_28_16(int smem) { return StreamClass<1, 28, 16>::init(smem); }

}  // namespace pidk
