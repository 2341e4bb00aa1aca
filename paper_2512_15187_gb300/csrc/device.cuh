// Device-side helpers: inline PTX for mbarriers, TMA bulk-tensor copies, named barriers
// and bounded waits. Every wait in this library is bounded by %globaltimer.
#pragma once

#include <cuda.h>
#include <cstdint>

namespace pidk {

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ uint64_t global_timer_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
               : "memory");
}

__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Wait for the phase with the given parity to complete; false if the bound ran out.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity,
                                                  uint64_t timeout_ns) {
  if (mbar_try_wait(bar, parity)) return true;
  const uint64_t t0 = global_timer_ns();
  while (true) {
#pragma unroll 1
    for (int i = 0; i < 32; ++i)
      if (mbar_try_wait(bar, parity)) return true;
    if (global_timer_ns() - t0 > timeout_ns) return false;
  }
}

// 2D tiled TMA load global -> shared, completion counted on `bar` in bytes.
// x = innermost (cell) coordinate, y = member row. x must be a multiple of 4 (16 bytes).
__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, uint64_t* bar,
                                            int32_t x, int32_t y) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%3, %4}], [%2];" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(smem_u32(bar)), "r"(x), "r"(y)
      : "memory");
}

__device__ __forceinline__ void tma_load_1d(void* dst, const CUtensorMap* map, uint64_t* bar,
                                            int32_t x) {
  asm volatile(
      "cp.async.bulk.tensor.1d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%3}], [%2];" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(smem_u32(bar)), "r"(x)
      : "memory");
}

__device__ __forceinline__ void prefetch_tmap(const CUtensorMap* map) {
  asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(map)) : "memory");
}

__device__ __forceinline__ void named_barrier(uint32_t id, uint32_t nthreads) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(nthreads) : "memory");
}

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ float rcp_approx(float x) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}

__device__ __forceinline__ float ex2_approx(float x) {
  float r;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}

// sqrt(log2 e): the isovalue scale carries it, so that log2(e) a^2 = a'^2 below.
constexpr double kSqrtLog2e = 1.2011224087864498;

// erfc(a) / 2 for a >= 0, given a' = sqrt(log2 e) a, in 16 FP32 operations (two of them
// MUFU). Relative error below 3e-7 down to FP32's smallest normal number (a ~ 9.3); beyond
// that the result flushes to 0. Form after the Chebyshev-fitted erfc of Numerical Recipes
// (2nd ed., Sec. 6.2): with t = 1 / (1 + a/2),
//   erfc(a) / 2 = t * 2^(Q(t) - log2(e) a^2) = t * 2^(Q(t) - a'^2),
// where Q is a degree-9 polynomial whose coefficients were fitted for this library by
// csrc/fit_erfc.py (float64 near-minimax fit on Chebyshev nodes of t).
__device__ __forceinline__ float half_erfc_scaled(float as) {
  const float t = rcp_approx(fmaf(static_cast<float>(0.5 / kSqrtLog2e), as, 1.0f));
  float q = 1.966346219e-01f;
  q = fmaf(q, t, -9.140366267e-01f);
  q = fmaf(q, t, 1.507482838e+00f);
  q = fmaf(q, t, -7.885746771e-01f);
  q = fmaf(q, t, -2.953876851e-01f);
  q = fmaf(q, t, 9.776866458e-02f);
  q = fmaf(q, t, 1.710338295e-02f);
  q = fmaf(q, t, 5.647117482e-01f);
  q = fmaf(q, t, 1.439913215e+00f);
  q = fmaf(q, t, -2.825615422e+00f);
  return t * ex2_approx(fmaf(-as, as, q));
}

// Soft-mask value of one input element (Sec. 3.5); used by the standalone map.
//   mode 1: u = P(F < q), q ~ Normal(mu, sigma): u = erfc(a)/2 with a = (F - mu) / (sigma
//           sqrt 2), from xs = (F - mu) * inv, inv = +-sqrt(log2 e) / (sigma sqrt 2)
//           (negated for the super-level set P(F > q)).
//   mode 2/3: sigma = 0, the indicator of F < t or F > t.
__device__ __forceinline__ float iso_value(float f, int32_t mode, float mu, float inv, float t) {
  if (mode == 1) {
    const float xs = (f - mu) * inv;
    const float h = half_erfc_scaled(fabsf(xs));
    return xs >= 0.f ? h : 1.0f - h;
  }
  if (mode == 2) return f < t ? 1.0f : 0.0f;
  return f > t ? 1.0f : 0.0f;
}

}  // namespace pidk
