// Streaming-pass instantiations for the tile class VEC=2, MPW=13, G=16.
#include "stream_kernel.cuh"

namespace pidk {

cudaError_t launch_stream_c2_13_16(const StreamParams& p, int iso, bool coef, int grid,
                                  size_t smem, cudaStream_t s) {
  return StreamClass<2, 13, 16>::launch(p, iso, coef, grid, smem, s);
}

cudaError_t init_stream_c2_13_16(int smem) { return StreamClass<2, 13, 16>::init(smem); }

}  // namespace pidk
