// Instantiations of the tensor-core Gram kernel for 128 < N <= 256 (the wide tile of
// gram_kernel.cuh: 16 warps own 256 operand rows, two M = 128 row blocks per K step).
#include "gram_kernel.cuh"

namespace pidk {

template <int ISO, int PREC>
static cudaError_t wide_launch_t(const GramParams& p, int grid, size_t smem, cudaStream_t s) {
  if (p.use_tma)
    gram_kernel<16, ISO, PREC, true, true><<<grid, kGramThreads, smem, s>>>(p);
  else
    gram_kernel<16, ISO, PREC, false, true><<<grid, kGramThreads, smem, s>>>(p);
  return cudaGetLastError();
}

cudaError_t launch_gram_wide(const GramParams& p, int prec, int iso_kind, int grid, size_t smem,
                             cudaStream_t s) {
#define PIDK_WIDE_CASE(ISO)                                             \
  if (iso_kind == ISO) {                                                \
    if (prec == 1) return wide_launch_t<ISO, 1>(p, grid, smem, s);      \
    if (prec == 2) return wide_launch_t<ISO, 2>(p, grid, smem, s);      \
    if (prec == 3) return wide_launch_t<ISO, 3>(p, grid, smem, s);      \
  }
  PIDK_WIDE_CASE(ISOK_NONE)
  PIDK_WIDE_CASE(ISOK_NORMAL)
  PIDK_WIDE_CASE(ISOK_STEP)
#undef PIDK_WIDE_CASE
  return cudaErrorInvalidValue;
}

cudaError_t gram_wide_init(int max_smem) {
  cudaError_t e = cudaSuccess;
#define PIDK_WIDE_INIT(ISO, PREC)                                                            \
  if (e == cudaSuccess)                                                                      \
    e = cudaFuncSetAttribute(gram_kernel<16, ISO, PREC, true, true>,                         \
                             cudaFuncAttributeMaxDynamicSharedMemorySize, max_smem);         \
  if (e == cudaSuccess)                                                                      \
    e = cudaFuncSetAttribute(gram_kernel<16, ISO, PREC, false, true>,                        \
                             cudaFuncAttributeMaxDynamicSharedMemorySize, max_smem);
  PIDK_WIDE_INIT(ISOK_NONE, 1) PIDK_WIDE_INIT(ISOK_NONE, 2) PIDK_WIDE_INIT(ISOK_NONE, 3)
  PIDK_WIDE_INIT(ISOK_NORMAL, 1) PIDK_WIDE_INIT(ISOK_NORMAL, 2) PIDK_WIDE_INIT(ISOK_NORMAL, 3)
  PIDK_WIDE_INIT(ISOK_STEP, 1) PIDK_WIDE_INIT(ISOK_STEP, 2) PIDK_WIDE_INIT(ISOK_STEP, 3)
#undef PIDK_WIDE_INIT
  return e;
}

}  // namespace pidk
