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

// 4-byte asynchronous copy global -> shared (any 4-byte aligned addresses); `bytes` = 0
// writes zeros and reads nothing.
__device__ __forceinline__ void cp_async4(void* dst, const void* src, uint32_t bytes) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(smem_u32(dst)), "l"(src),
               "r"(bytes)
               : "memory");
}
// 16-byte copy of which the first `bytes` (0..16) are read and the rest zero-filled; both
// addresses 16-byte aligned. Cached in L2 only.
__device__ __forceinline__ void cp_async16(void* dst, const void* src, uint32_t bytes) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(smem_u32(dst)), "l"(src),
               "r"(bytes)
               : "memory");
}
// Arrive on `bar` once this thread's earlier cp.async copies have landed (the arrival counts
// toward the barrier's expected count).
__device__ __forceinline__ void cp_async_arrive(uint64_t* bar) {
  asm volatile("cp.async.mbarrier.arrive.noinc.shared::cta.b64 [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.wait_all;" ::: "memory");
}

__device__ __forceinline__ void prefetch_tmap(const CUtensorMap* map) {
  asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(map)) : "memory");
}

__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// ---- tcgen05 (5th-generation tensor cores, accumulators in tensor memory) ----

__device__ __forceinline__ void tmem_alloc(uint32_t* smem_dst, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                   smem_u32(smem_dst)),
               "r"(ncols)
               : "memory");
}
__device__ __forceinline__ void tmem_relinquish() {
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols)
               : "memory");
}
__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
// Arrive on `bar` once every tcgen05.mma issued so far by this thread has completed.
__device__ __forceinline__ void tc_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                   smem_u32(bar))
               : "memory");
}
// D[tmem] (+)= A[smem] x B[smem]^T, BF16 or FP16 operands, FP32 accumulate.
__device__ __forceinline__ void umma_f16(uint32_t d_tmem, uint64_t a_desc, uint64_t b_desc,
                                         uint32_t idesc, uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
      "l"(a_desc), "l"(b_desc), "r"(idesc), "r"(accumulate)
      : "memory");
}
// Same for 8-bit (E4M3 / E5M2) operands.
__device__ __forceinline__ void umma_f8(uint32_t d_tmem, uint64_t a_desc, uint64_t b_desc,
                                        uint32_t idesc, uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
      "l"(a_desc), "l"(b_desc), "r"(idesc), "r"(accumulate)
      : "memory");
}
// 32 consecutive FP32 columns of this warp's 32 TMEM lanes (one lane per thread).
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32]) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, "
      "%12, %13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, "
      "%30, %31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]),
        "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]),
        "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

// Shared-memory matrix descriptor of a K-major operand in the 128-byte swizzle layout:
// rows of 128 bytes, 8-row atoms of 1024 bytes (stride between atoms = 1024 B), start
// address 16-byte granular (advancing it by 32 B steps along K inside the atom).
__device__ __forceinline__ uint64_t umma_desc_sw128(uint32_t smem_addr) {
  uint64_t d = 0;
  d |= static_cast<uint64_t>((smem_addr & 0x3FFFFu) >> 4);   // start address
  d |= static_cast<uint64_t>(1) << 16;                        // leading byte offset (unused)
  d |= static_cast<uint64_t>(1024 >> 4) << 32;                // stride byte offset
  d |= static_cast<uint64_t>(1) << 46;                        // descriptor version
  d |= static_cast<uint64_t>(2) << 61;                        // 128-byte swizzle
  return d;
}

// Instruction descriptor: FP32 accumulator, K-major A and B, M x N tile.
//   a_fmt/b_fmt: kind::f16 -> 1 = BF16; kind::f8f6f4 -> 0 = E4M3.
__host__ __device__ constexpr uint32_t umma_idesc(uint32_t fmt, uint32_t M, uint32_t N) {
  return (1u << 4) | (fmt << 7) | (fmt << 10) | ((N >> 3) << 17) | ((M >> 4) << 24);
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

// Order-preserving integer key of a double: for non-NaN a, b, a < b <=> key(a) < key(b) and
// a == b <=> key(a) == key(b) (-0 is folded into +0). GB300 issues FP64 compares at a small
// fraction of the integer rate, so the O(N^2) rank counts compare keys.
__device__ __forceinline__ unsigned long long order_key(double d) {
  const long long b = __double_as_longlong(d + 0.0);
  return b >= 0 ? static_cast<unsigned long long>(b) | 0x8000000000000000ull
                : ~static_cast<unsigned long long>(b);
}

// Order-preserving unsigned key of a float (keys compare as the floats do; 0 is below the
// key of every float, so a zeroed key array is the identity of a maximum taken with atomicMax).
__device__ __forceinline__ unsigned int fkey(float v) {
  const unsigned int b = __float_as_uint(v);
  return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}
__device__ __forceinline__ float fkey_inv(unsigned int k) {
  return __uint_as_float((k & 0x80000000u) ? (k & 0x7fffffffu) : ~k);
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

// Packed FP32 pairs: on the sm_100 family one FFMA2 / FADD2 / FMUL2 instruction does the
// arithmetic of two FP32 lanes with the rounding of the scalar instruction (round to
// nearest even, no flush), so a kernel bound by instruction issue does half the issues.
__device__ __forceinline__ float2 f2(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 f2_fma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 f2_add(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 f2_mul(float2 a, float2 b) { return __fmul2_rn(a, b); }

// half_erfc_scaled for two arguments xs (of either sign: a' = |xs|), with the polynomial on
// packed pairs. Bitwise equal to the scalar function: the polynomial is evaluated with
// negated coefficients, p = -Q(t) at every step (round to nearest is symmetric), so that
// fma(xs, xs, p) = -fma(-a', a', Q) exactly and 2^-(that) is the scalar's 2^(Q - a'^2).
__device__ __forceinline__ float2 half_erfc_scaled2(float2 xs) {
  constexpr float c = static_cast<float>(0.5 / kSqrtLog2e);
  const float2 t = make_float2(rcp_approx(fmaf(c, fabsf(xs.x), 1.0f)),
                               rcp_approx(fmaf(c, fabsf(xs.y), 1.0f)));
  float2 p = f2(-1.966346219e-01f);
  p = f2_fma(p, t, f2(9.140366267e-01f));
  p = f2_fma(p, t, f2(-1.507482838e+00f));
  p = f2_fma(p, t, f2(7.885746771e-01f));
  p = f2_fma(p, t, f2(2.953876851e-01f));
  p = f2_fma(p, t, f2(-9.776866458e-02f));
  p = f2_fma(p, t, f2(-1.710338295e-02f));
  p = f2_fma(p, t, f2(-5.647117482e-01f));
  p = f2_fma(p, t, f2(-1.439913215e+00f));
  p = f2_fma(p, t, f2(2.825615422e+00f));
  const float2 r = f2_fma(xs, xs, p);
  return f2_mul(t, make_float2(ex2_approx(-r.x), ex2_approx(-r.y)));
}

// Normal-isovalue soft masks of two field values (see iso_value, mode 1), bitwise equal to
// two scalar evaluations: xs = (F - mu) * inv, u = h if xs >= 0 else 1 - h.
__device__ __forceinline__ float2 iso_normal2(float2 f, float mu, float inv) {
  const float2 xs = f2_mul(f2_add(f, f2(-mu)), f2(inv));
  const float2 h = half_erfc_scaled2(xs);
  const float2 g = f2_fma(h, f2(-1.0f), f2(1.0f));
  return make_float2(xs.x >= 0.f ? h.x : g.x, xs.y >= 0.f ? h.y : g.y);
}

// The piecewise-linear maps (modes 4-6): a uniform isovalue distribution (Sec. 3.5) and
// the level-centred map of the weather example (Sec. 3.6).
//   mode 4: u = clamp((mu - F) inv, 0, 1)   mode 5: u = clamp((F - mu) inv, 0, 1)
//   mode 6: u = max(0, 1 - |F - mu| inv)
__device__ __forceinline__ float iso_piecewise(float f, int32_t mode, float mu, float inv) {
  if (mode == 6) return fmaxf(0.0f, fmaf(-fabsf(f - mu), inv, 1.0f));
  const float v = mode == 4 ? (mu - f) * inv : (f - mu) * inv;
  return fminf(fmaxf(v, 0.0f), 1.0f);
}

// Soft-mask value of one input element (Sec. 3.5); used by the standalone map.
//   mode 1: u = P(F < q), q ~ Normal(mu, sigma): u = erfc(a)/2 with a = (F - mu) / (sigma
//           sqrt 2), from xs = (F - mu) * inv, inv = +-sqrt(log2 e) / (sigma sqrt 2)
//           (negated for the super-level set P(F > q)).
//   mode 2/3: sigma = 0, the indicator of F < t or F > t; modes 4-6: iso_piecewise.
__device__ __forceinline__ float iso_value(float f, int32_t mode, float mu, float inv, float t) {
  if (mode == 1) {
    const float xs = (f - mu) * inv;
    const float h = half_erfc_scaled(fabsf(xs));
    return xs >= 0.f ? h : 1.0f - h;
  }
  if (mode == 2) return f < t ? 1.0f : 0.0f;
  if (mode == 3) return f > t ? 1.0f : 0.0f;
  return iso_piecewise(f, mode, mu, inv);
}

}  // namespace pidk
