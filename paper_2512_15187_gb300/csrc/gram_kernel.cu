// Instantiations of the tensor-core Gram kernel for N <= 128 with 8 members per warp
// (gram_kernel.cuh), the launch dispatch over tile, group size, precision and isovalue kind,
// and the FP8 operand scale.
#include "gram_kernel.cuh"

namespace pidk {

cudaError_t launch_gram_wide(const GramParams& p, int prec, int iso_kind, int grid, size_t smem,
                             cudaStream_t s);
cudaError_t gram_wide_init(int max_smem);
cudaError_t launch_gram_wide12(const GramParams& p, int prec, int iso_kind, int grid, size_t smem,
                               cudaStream_t s);
cudaError_t gram_wide12_init(int max_smem);
cudaError_t launch_gram_narrow6(const GramParams& p, int G, int prec, int iso_kind, int grid,
                                size_t smem, cudaStream_t s);
cudaError_t gram_narrow6_init(int max_smem);

// mpw: members per warp of the tile (6 or 8 narrow, 12 or 16 wide)
size_t gram_smem_bytes(int G, int mpw, bool wide, int prec, int dF, int dO, int stage_floats) {
  const size_t NG = kGramConvWarps / G;
  const size_t T = wide ? GramShape<true>::T : GramShape<false>::T;
  const size_t plane = static_cast<size_t>(mpw) * G * 128;
  const size_t op_stage = (prec == 2 ? 2 : 1) * (prec == 3 ? 1 : 2) * plane;
  const size_t rb = static_cast<size_t>(G) * T + T;
  return 1024 + NG * (dO * op_stage + static_cast<size_t>(dF) * stage_floats * 4 + 2 * rb * 4 +
                      (static_cast<size_t>(dF) + dO + 5) * 8 + 8) + 16 +
         16 + NG * sizeof(GramLeader);
}

cudaError_t launch_gram(const GramParams& p, int G, int mpw, bool wide, int prec, int iso_kind,
                        int grid, size_t smem, cudaStream_t s) {
  if (wide) {
    if (G != 16) return cudaErrorInvalidValue;
    if (mpw == 16) return launch_gram_wide(p, prec, iso_kind, grid, smem, s);
    if (mpw == 12) return launch_gram_wide12(p, prec, iso_kind, grid, smem, s);
    return cudaErrorInvalidValue;
  }
  if (mpw == 6) return launch_gram_narrow6(p, G, prec, iso_kind, grid, smem, s);
  if (mpw != 8) return cudaErrorInvalidValue;
  if (G == 8) return gram_tile_launch<8, 8>(p, prec, iso_kind, grid, smem, s);
  if (G == 16) return gram_tile_launch<16, 8>(p, prec, iso_kind, grid, smem, s);
  return cudaErrorInvalidValue;
}

cudaError_t gram_kernels_init(int max_smem) {
  cudaError_t e = gram_tile_init<8, 8>(max_smem);
  if (e == cudaSuccess) e = gram_tile_init<16, 8>(max_smem);
  if (e == cudaSuccess) e = gram_narrow6_init(max_smem);
  if (e == cudaSuccess) e = gram_wide12_init(max_smem);
  if (e == cudaSuccess) e = gram_tiled_init(max_smem);
  return e == cudaSuccess ? gram_wide_init(max_smem) : e;
}

// Power-of-two E4M3 operand scale for weighted ensembles: the largest operand is
// u sqrt(w) <= sqrt(max w), mapped at or below 448 (the largest finite E4M3 value).
__global__ void fp8_scale_kernel(const float* w, int64_t M, float* out) {
  __shared__ unsigned int smax;
  if (threadIdx.x == 0) smax = 0u;
  __syncthreads();
  unsigned int local = 0u;
  for (int64_t x = threadIdx.x; x < M; x += blockDim.x) local = max(local, __float_as_uint(w[x]));
  atomicMax(&smax, local);
  __syncthreads();
  if (threadIdx.x == 0) {
    const float r = sqrtf(__uint_as_float(smax));
    float s = 1.0f;
    // largest power of two with r * s <= 448
    if (r > 0.f && isfinite(r)) s = exp2f(floorf(log2f(448.0f / r)));
    *out = s;
  }
}

cudaError_t launch_fp8_scale(const float* w, int64_t M, float* out, cudaStream_t s) {
  fp8_scale_kernel<<<1, 1024, 0, s>>>(w, M, out);
  return cudaGetLastError();
}

}  // namespace pidk
