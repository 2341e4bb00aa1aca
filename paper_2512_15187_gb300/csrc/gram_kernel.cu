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

// The value whose maximum a member's scale needs: the proxy of F for unweighted fields
// (PROXY), otherwise u sqrt(w), mapping fields element by element.
template <bool PROXY>
__device__ __forceinline__ float scale_value(const ScaleDesc& d, float f, float w) {
  if constexpr (PROXY) {
    return iso_proxy(f, d.iso_mode, d.iso_mu, d.iso_inv);
  } else {
    const float u = d.iso_mode != ISO_NONE ? iso_value(f, d.iso_mode, d.iso_mu, d.iso_inv, d.iso_t) : f;
    return d.w ? u * sqrtf(w) : u;
  }
}

// The maximum over one CTA's segment [c0, c1) of member i. Aligned rows are read as float4
// with four loads in flight per thread; the rest cell by cell.
template <bool PROXY>
__device__ __forceinline__ float member_segment_max(const ScaleDesc& d, int i, int64_t c0, int64_t c1) {
  constexpr int U = 4;
  const float* row = d.data + static_cast<int64_t>(i) * d.ld;
  const bool use_w = !PROXY && d.w != nullptr;
  float best = PROXY ? -__int_as_float(0x7f800000) : 0.0f;
  int64_t tail = c0;
  if (d.vec_ok) {
    const int64_t n4 = (c1 - c0) >> 2;   // c0 is a multiple of 1024: float4-aligned
    const float4* r4 = reinterpret_cast<const float4*>(row + c0);
    const float4* w4 = use_w ? reinterpret_cast<const float4*>(d.w + c0) : nullptr;
    for (int64_t j0 = threadIdx.x; j0 < n4; j0 += static_cast<int64_t>(U) * kScaleThreads) {
      float4 a[U], b[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int64_t j = j0 + static_cast<int64_t>(u) * kScaleThreads;
        if (j < n4) {
          a[u] = __ldcs(r4 + j);
          b[u] = use_w ? __ldg(w4 + j) : make_float4(1.f, 1.f, 1.f, 1.f);
        } else {
          a[u] = make_float4(0.f, 0.f, 0.f, 0.f);
          b[u] = make_float4(1.f, 1.f, 1.f, 1.f);
        }
      }
#pragma unroll
      for (int u = 0; u < U; ++u) {
        if (j0 + static_cast<int64_t>(u) * kScaleThreads >= n4) break;
        best = fmaxf(best, scale_value<PROXY>(d, a[u].x, b[u].x));
        best = fmaxf(best, scale_value<PROXY>(d, a[u].y, b[u].y));
        best = fmaxf(best, scale_value<PROXY>(d, a[u].z, b[u].z));
        best = fmaxf(best, scale_value<PROXY>(d, a[u].w, b[u].w));
      }
    }
    tail = c0 + 4 * n4;
  }
  for (int64_t x = tail + threadIdx.x; x < c1; x += kScaleThreads)
    best = fmaxf(best, scale_value<PROXY>(d, __ldcs(row + x), use_w ? __ldg(d.w + x) : 1.f));
  return best;
}

// One CTA per (ensemble, member, segment): the CTA's maximum goes to its own slot of the
// ensemble's scale region, so the pass needs no atomics and no cleared keys.
__global__ void __launch_bounds__(kScaleThreads) member_max_kernel(const __grid_constant__ ScaleBatchParams p) {
  const int b = blockIdx.x;
  int e = -1;   // the last descriptor with a max pass that starts at or before this CTA
  for (int k = 0; k < p.n; ++k)
    if (!p.d[k].from_keys && p.d[k].block_begin <= b) e = k;
  if (e < 0) return;
  const ScaleDesc& d = p.d[e];
  const int local = b - d.block_begin;
  const int i = local / d.segs;
  const int sg = local - i * d.segs;
  const int64_t c0 = static_cast<int64_t>(sg) * d.seg_cells;
  const int64_t c1 = min(static_cast<int64_t>(d.M), c0 + d.seg_cells);
  float best = d.proxy ? member_segment_max<true>(d, i, c0, c1) : member_segment_max<false>(d, i, c0, c1);
  __shared__ float red[kScaleThreads / 32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) best = fmaxf(best, __shfl_xor_sync(0xffffffffu, best, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = best;
  __syncthreads();
  if (threadIdx.x == 0) {
    float m = red[0];
    for (int k = 1; k < kScaleThreads / 32; ++k) m = fmaxf(m, red[k]);
    d.scale[2 * kGramTiledMaxN + local] = m;
  }
}

// s_i from the maximum: the largest k with v 2^k <= 448 = 1.75 * 2^8, i.e. k = 8 - e when
// the significand of v (in [1, 2)) is at most 1.75, else 7 - e; k is kept within [-63, 63]
// so that every product of two inverse scales is a normal FP32 power of two. A member with
// no positive value (all zeros) takes s_i = 1. One CTA per ensemble.
__global__ void __launch_bounds__(kScaleThreads) member_scale_kernel(const __grid_constant__ ScaleBatchParams p) {
  const ScaleDesc& d = p.d[blockIdx.x];
  const float* slots = d.scale + 2 * kGramTiledMaxN;
  for (int i = threadIdx.x; i < d.N; i += kScaleThreads) {
    float v;
    if (d.from_keys) {
      v = fkey_inv(reinterpret_cast<const unsigned int*>(slots)[i]);
    } else {
      v = slots[i * d.segs];
      for (int sg = 1; sg < d.segs; ++sg) v = fmaxf(v, slots[i * d.segs + sg]);
      if (d.proxy) v = iso_from_proxy(v, d.iso_mode, d.iso_mu, d.iso_inv, d.iso_t);
    }
    int k = 0;
    if (v > 0.f && v < __int_as_float(0x7f800000)) {
      const unsigned int b = __float_as_uint(v);
      const int e = static_cast<int>((b >> 23) & 0xffu) - 127;   // -127: subnormal v
      k = ((b & 0x7fffffu) <= 0x600000u ? 8 : 7) - e;
      k = max(-63, min(63, k));
    }
    d.scale[i] = __uint_as_float(static_cast<unsigned int>(127 + k) << 23);
    d.scale[d.N + i] = __uint_as_float(static_cast<unsigned int>(127 - k) << 23);
  }
}

}  // namespace

cudaError_t launch_member_scales(const ScaleBatchParams& p, cudaStream_t s) {
  if (p.n <= 0 || p.n > kScaleBatch) return cudaErrorInvalidValue;
  if (p.total_blocks > 0) {
    member_max_kernel<<<p.total_blocks, kScaleThreads, 0, s>>>(p);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  member_scale_kernel<<<p.n, kScaleThreads, 0, s>>>(p);
  return cudaGetLastError();
}

}  // namespace pidk
