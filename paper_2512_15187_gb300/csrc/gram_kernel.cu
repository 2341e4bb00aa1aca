// Instantiations of the tensor-core Gram kernel for N <= 128 with 8 members per warp
// (gram_kernel.cuh), the launch dispatch over tile, group size, precision and isovalue kind,
// and the per-member E4M3 operand scales.
#include <algorithm>

#include "gram_kernel.cuh"

namespace pidk {

cudaError_t launch_gram_wide(const GramParams& p, int prec, int iso_kind, int grid, size_t smem,
                             cudaStream_t s);
cudaError_t gram_wide_init(int max_smem);
cudaError_t launch_gram_wide12(const GramParams& p, int prec, int iso_kind, int grid, size_t smem,
                               cudaStream_t s);
cudaError_t gram_wide12_init(int max_smem);
cudaError_t launch_gram_wide13(const GramParams& p, int prec, int iso_kind, int grid, size_t smem,
                               cudaStream_t s);
cudaError_t gram_wide13_init(int max_smem);
cudaError_t launch_gram_narrow6(const GramParams& p, int G, int prec, int iso_kind, int grid,
                                size_t smem, cudaStream_t s);
cudaError_t gram_narrow6_init(int max_smem);

// mpw: members per warp of the tile (6 or 8 narrow, 12 or 16 wide)
size_t gram_smem_bytes(int G, int mpw, bool wide, int prec, int dF, int dO, int stage_floats) {
  const size_t NG = kGramConvWarps / G;
  const size_t T = wide ? GramShape<true>::T : GramShape<false>::T;
  const size_t plane = static_cast<size_t>(mpw) * G * 128;
  // K-blocks per operand stage: one for E4M3 (128 cells) and for the wide tile's 16-bit
  // operands (64 cells, its FP32 stage), two for the narrow tile's 16-bit operands
  const size_t op_stage = (prec == 2 ? 2 : 1) * ((prec == 3 || wide) ? 1 : 2) * plane;
  const size_t rb = static_cast<size_t>(G) * T + T;
  return 1024 + NG * (dO * op_stage + static_cast<size_t>(dF) * stage_floats * 4 + 2 * rb * 4 +
                      (static_cast<size_t>(dF) + 2 * dO + 5) * 8 + 8) + 16 +
         16 + NG * sizeof(GramLeader) + kGramConvWarps * kGramMaxMpw * sizeof(float);
}

cudaError_t launch_gram(const GramParams& p, int G, int mpw, bool wide, int prec, int iso_kind,
                        int grid, size_t smem, cudaStream_t s) {
  if (wide) {
    if (G != 16) return cudaErrorInvalidValue;
    if (mpw == 16) return launch_gram_wide(p, prec, iso_kind, grid, smem, s);
    if (mpw == 12) return launch_gram_wide12(p, prec, iso_kind, grid, smem, s);
    if (mpw == 13) return launch_gram_wide13(p, prec, iso_kind, grid, smem, s);
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
  if (e == cudaSuccess) e = gram_wide13_init(max_smem);
  if (e == cudaSuccess) e = gram_tiled_init(max_smem);
  return e == cudaSuccess ? gram_wide_init(max_smem) : e;
}

// ---- Per-member E4M3 operand scales ----
//
// The inclusion u_i subset_p u_j = G_ij / m_i does not change when u_i is multiplied by a
// positive constant (Eq. 9: the scale cancels between the sums of the ratio), so each
// member's operands may carry a power-of-two scale s_i of their own, undone exactly when
// the Gram partials leave the tensor memory (G_ij = G'_ij / (s_i s_j)). Choosing s_i as the
// largest power of two with max_x u_i(x) sqrt(w_x) s_i <= 448 (the largest finite E4M3
// value) puts every member's largest operand in the top binade of E4M3, so a member whose
// values are all small keeps E4M3's full relative precision instead of falling into its
// subnormal range.
//
// One pass finds the per-member maxima (or, in a batch that also streams the same soft
// masks for PID-mean, that streaming pass does, see stream_kernel's MAXU). Soft masks, and
// weighted fields (mapped element by element), reduce the operand u sqrt(w) itself. For unweighted fields it is enough to find
// the field value that the map sends highest, since every isovalue map is monotone in a
// simple function of F (its "proxy"), and to map that one value.

namespace {

// Proxy of a field value: the soft mask of each isovalue mode is a non-decreasing function
// of it (Normal: u = erfc(xs)/2 decreases in xs = (F - mu) inv, whose sign carries the
// direction; sub-level step and uniform maps decrease in F; super-level ones increase;
// the level map decreases in |F - mu|).
__device__ __forceinline__ float iso_proxy(float f, int32_t mode, float mu, float inv) {
  switch (mode) {
    case ISO_NORMAL: return -((f - mu) * inv);
    case ISO_STEP_BELOW:
    case ISO_UNIFORM_BELOW: return -f;
    case ISO_LEVEL: return -fabsf(f - mu);
    default: return f;   // ISO_STEP_ABOVE, ISO_UNIFORM_ABOVE
  }
}

// The soft mask of the field value whose proxy is p, with the arithmetic of iso_value
// (the negations are exact, so the value equals the map of that field value).
__device__ __forceinline__ float iso_from_proxy(float p, int32_t mode, float mu, float inv, float t) {
  switch (mode) {
    case ISO_NORMAL: {
      const float xs = -p;
      const float h = half_erfc_scaled(fabsf(xs));
      return xs >= 0.f ? h : 1.0f - h;
    }
    case ISO_STEP_BELOW: return iso_value(-p, mode, mu, inv, t);
    case ISO_UNIFORM_BELOW: return iso_value(-p, mode, mu, inv, t);
    case ISO_LEVEL: return fmaxf(0.0f, fmaf(p, inv, 1.0f));
    default: return iso_value(p, mode, mu, inv, t);
  }
}

constexpr int kScaleThreads = 256;

// PROXY: unweighted fields (reduce the proxy of F); otherwise reduce u sqrt(w), mapping
// fields element by element. One CTA per (member, segment of seg_cells cells).
template <bool PROXY>
__global__ void __launch_bounds__(kScaleThreads) member_max_kernel(const __grid_constant__ ScaleParams p) {
  const int i = blockIdx.y;
  const int64_t c0 = static_cast<int64_t>(blockIdx.x) * p.seg_cells;
  const int64_t c1 = min(static_cast<int64_t>(p.M), c0 + p.seg_cells);
  const float* row = p.data + static_cast<int64_t>(i) * p.ld;
  const bool field = p.iso_mode != ISO_NONE;
  float best = PROXY ? -__int_as_float(0x7f800000) : 0.0f;
  for (int64_t x = c0 + 4 * static_cast<int64_t>(threadIdx.x); x < c1; x += 4 * kScaleThreads) {
    float f[4], w[4] = {1.f, 1.f, 1.f, 1.f};
    int n = 4;
    if (p.vec_ok && x + 4 <= c1) {
      const float4 a = __ldcs(reinterpret_cast<const float4*>(row + x));
      f[0] = a.x; f[1] = a.y; f[2] = a.z; f[3] = a.w;
      if (!PROXY && p.w) {
        const float4 b = __ldg(reinterpret_cast<const float4*>(p.w + x));
        w[0] = b.x; w[1] = b.y; w[2] = b.z; w[3] = b.w;
      }
    } else {
      n = static_cast<int>(c1 - x < 4 ? c1 - x : 4);
      for (int v = 0; v < n; ++v) {
        f[v] = __ldcs(row + x + v);
        if (!PROXY && p.w) w[v] = __ldg(p.w + x + v);
      }
    }
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      if (v >= n) break;
      float val;
      if constexpr (PROXY) {
        val = iso_proxy(f[v], p.iso_mode, p.iso_mu, p.iso_inv);
      } else {
        const float u = field ? iso_value(f[v], p.iso_mode, p.iso_mu, p.iso_inv, p.iso_t) : f[v];
        val = p.w ? u * sqrtf(w[v]) : u;
      }
      best = fmaxf(best, val);
    }
  }
  // block maximum, then one atomic per CTA
  __shared__ float red[kScaleThreads / 32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) best = fmaxf(best, __shfl_xor_sync(0xffffffffu, best, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = best;
  __syncthreads();
  if (threadIdx.x == 0) {
    float b = red[0];
    for (int k = 1; k < kScaleThreads / 32; ++k) b = fmaxf(b, red[k]);
    atomicMax(p.maxkey + i, fkey(b));
  }
}

// s_i from the maximum: the largest k with v 2^k <= 448 = 1.75 * 2^8, i.e. k = 8 - e when
// the significand of v (in [1, 2)) is at most 1.75, else 7 - e; k is kept within [-63, 63]
// so that every product of two inverse scales is a normal FP32 power of two. A member with
// no positive value (all zeros) takes s_i = 1.
__global__ void member_scale_kernel(const __grid_constant__ ScaleParams p, bool proxy) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= p.N) return;
  float v = fkey_inv(p.maxkey[i]);
  if (proxy) v = iso_from_proxy(v, p.iso_mode, p.iso_mu, p.iso_inv, p.iso_t);
  int k = 0;
  if (v > 0.f && v < __int_as_float(0x7f800000)) {
    const unsigned int b = __float_as_uint(v);
    const int e = static_cast<int>((b >> 23) & 0xffu) - 127;   // -127: subnormal v
    k = ((b & 0x7fffffu) <= 0x600000u ? 8 : 7) - e;
    k = max(-63, min(63, k));
  }
  p.scale[i] = __uint_as_float(static_cast<unsigned int>(127 + k) << 23);
  p.scale[p.N + i] = __uint_as_float(static_cast<unsigned int>(127 - k) << 23);
}

}  // namespace

cudaError_t launch_member_scales_from_keys(const ScaleParams& p, cudaStream_t s) {
  member_scale_kernel<<<(p.N + 255) / 256, 256, 0, s>>>(p, false);
  return cudaGetLastError();
}

cudaError_t launch_member_scales(const ScaleParams& p, int sms, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(p.maxkey, 0, static_cast<size_t>(p.N) * sizeof(unsigned int), s);
  if (e != cudaSuccess) return e;
  ScaleParams q = p;
  // about four CTAs per SM over all members, segments of at least 4096 cells
  const int64_t want = std::max<int64_t>(1, (4LL * sms + p.N - 1) / p.N);
  const int64_t segs = std::max<int64_t>(1, std::min<int64_t>(want, (p.M + 4095) / 4096));
  q.seg_cells = static_cast<int32_t>(((p.M + segs - 1) / segs + 1023) / 1024 * 1024);
  const dim3 grid(static_cast<unsigned>((p.M + q.seg_cells - 1) / q.seg_cells), static_cast<unsigned>(p.N));
  const bool proxy = p.iso_mode != ISO_NONE && p.w == nullptr;
  if (proxy) member_max_kernel<true><<<grid, kScaleThreads, 0, s>>>(q);
  else member_max_kernel<false><<<grid, kScaleThreads, 0, s>>>(q);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  member_scale_kernel<<<(p.N + 255) / 256, 256, 0, s>>>(q, proxy);
  return cudaGetLastError();
}

}  // namespace pidk
