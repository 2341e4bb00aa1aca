// The streaming pass of PID-mean / exact full PID (included by the per-class translation
// units stream_c*.cu, each of which instantiates one tile class).
//
// One pass over an ensemble U [N][M]: per tile of T cells the column sum
// s(x) = sum_j c_j u_j(x) is formed on chip, then every member accumulates
//   m_i = sum_x w u_i  and  A_i = sum_x w u_i s.
// With c_j = 1, s = N u_bar (the mean contour of Eq. 15 times N: the 1/N is applied in
// FP64 by the finalisation, so no rounded 1/N enters the FP32 sums) and IN_in = A_i /
// (N m_i), IN_out = A_i / (N m_bar) (Eq. 16). With c_j = 1/(N m_j) the same pass yields
// IN_out of full PID exactly: A_i = (1/N) sum_j G_ij / m_j (Eq. 10 with the sums of
// Eq. 14). The isovalue map of Sec. 3.5 can be applied to each element as it is read.
//
// Work decomposition: groups of G warps share a TMA-fed shared-memory ring of stages; a
// stage holds [N rows][sub*T cells] of one chunk; warp q of a group owns members
// q, q+G, q+2G, ... (MPW of them) and lane l owns VEC consecutive cells of each T-cell
// register tile. Each group processes whole chunks and writes one partial (m_i, A_i) per
// member per chunk; a separate finalisation reduces the chunks in a fixed order.
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "device.cuh"
#include "internal.h"

namespace pidk {

__device__ __forceinline__ const EnsDesc& stream_desc(const StreamParams& p, int e) {
  return p.descs ? p.descs[e] : p.one;
}

// Ensemble owning flat unit u (unit_begin is increasing across the descriptor array).
__device__ __forceinline__ int stream_find_ens(const StreamParams& p, int u) {
  if (p.descs == nullptr) return 0;
  int lo = 0, hi = p.n_ens - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (p.descs[mid].unit_begin <= u) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// First unit whose start lies at or after position w of the launch's work (member-cells,
// counted along the ensembles and their chunks). Group g owns the units starting in
// [W g / groups, W (g+1) / groups): equal work per group to within one unit, whatever the
// mix of ensemble sizes, and contiguous units, so a group meets each ensemble once.
template <typename Params>
__device__ __forceinline__ int unit_at_work(const Params& p, int64_t w) {
  if (w >= p.total_work) return p.total_units;
  const EnsDesc* d = &p.one;
  if (p.descs != nullptr) {
    int lo = 0, hi = p.n_ens - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (p.descs[mid].work_begin <= w) lo = mid; else hi = mid - 1;
    }
    d = p.descs + lo;
  }
  const int64_t per = static_cast<int64_t>(d->N) * d->chunk_cells;
  const int64_t c = (w - d->work_begin + per - 1) / per;
  return d->unit_begin + static_cast<int>(c < d->n_chunks ? c : d->n_chunks);
}

template <int VEC> struct VecT;
template <> struct VecT<1> { using T = float; };
template <> struct VecT<2> { using T = float2; };
template <> struct VecT<4> { using T = float4; };

template <int VEC>
__device__ __forceinline__ void lds_vec(float (&dst)[VEC], const float* src) {
  const typename VecT<VEC>::T v = *reinterpret_cast<const typename VecT<VEC>::T*>(src);
  if constexpr (VEC == 1) {
    dst[0] = v;
  } else if constexpr (VEC == 2) {
    dst[0] = v.x; dst[1] = v.y;
  } else {
    dst[0] = v.x; dst[1] = v.y; dst[2] = v.z; dst[3] = v.w;
  }
}

// VEC floats starting `ro` (0..3) floats after `base` (VEC-aligned, in a row with at least
// 4 floats after the VEC read): aligned vector loads, shifted by the warp-uniform ro.
template <int VEC>
__device__ __forceinline__ void lds_shifted(float (&dst)[VEC], const float* base, int ro) {
  if constexpr (VEC == 1) {
    dst[0] = base[ro];
  } else if constexpr (VEC == 2) {
    if ((ro & 1) == 0) {
      lds_vec<2>(dst, base + ro);
    } else {
      const float2 a = *reinterpret_cast<const float2*>(base + ro - 1);
      const float2 b = *reinterpret_cast<const float2*>(base + ro + 1);
      dst[0] = a.y; dst[1] = b.x;
    }
  } else {
    const float4 a = *reinterpret_cast<const float4*>(base);
    if (ro == 0) {
      dst[0] = a.x; dst[1] = a.y; dst[2] = a.z; dst[3] = a.w;
    } else {
      const float4 b = *reinterpret_cast<const float4*>(base + 4);
      if (ro == 1) { dst[0] = a.y; dst[1] = a.z; dst[2] = a.w; dst[3] = b.x; }
      else if (ro == 2) { dst[0] = a.z; dst[1] = a.w; dst[2] = b.x; dst[3] = b.y; }
      else { dst[0] = a.w; dst[1] = b.x; dst[2] = b.y; dst[3] = b.z; }
    }
  }
}

// Streaming (evict-first) global store of VEC consecutive floats.
template <int VEC>
__device__ __forceinline__ void stg_cs_vec(float* dst, const float (&src)[VEC]) {
  if constexpr (VEC == 1) {
    __stcs(dst, src[0]);
  } else if constexpr (VEC == 2) {
    __stcs(reinterpret_cast<float2*>(dst), make_float2(src[0], src[1]));
  } else {
    __stcs(reinterpret_cast<float4*>(dst), make_float4(src[0], src[1], src[2], src[3]));
  }
}

template <int VEC>
__device__ __forceinline__ void sts_vec(float* dst, const float (&src)[VEC]) {
  if constexpr (VEC == 1) {
    *dst = src[0];
  } else if constexpr (VEC == 2) {
    *reinterpret_cast<float2*>(dst) = make_float2(src[0], src[1]);
  } else {
    *reinterpret_cast<float4*>(dst) = make_float4(src[0], src[1], src[2], src[3]);
  }
}

// Isovalue map kinds compiled into a kernel: none, the Normal isovalue, and the step family
// (sigma = 0 thresholds and the piecewise-linear maps, told apart at run time).
enum IsoKind : int { ISOK_NONE = 0, ISOK_NORMAL = 1, ISOK_STEP = 2 };

// s[v] = sum over r < G of part[r * stride + v], added in order r = 0, 1, ... (packed pairs
// when VEC is even; the order, and so the bits, are those of a scalar loop).
template <int VEC, int G>
__device__ __forceinline__ void sum_partials(float (&s)[VEC], const float* part, int stride) {
  if constexpr (VEC % 2 == 0) {
    float2 a[VEC / 2];
#pragma unroll
    for (int v = 0; v < VEC / 2; ++v) a[v] = f2(0.f);
#pragma unroll
    for (int r = 0; r < G; ++r) {
      float t[VEC];
      lds_vec<VEC>(t, part + r * stride);
#pragma unroll
      for (int v = 0; v < VEC / 2; ++v) a[v] = f2_add(a[v], make_float2(t[2 * v], t[2 * v + 1]));
    }
#pragma unroll
    for (int v = 0; v < VEC / 2; ++v) { s[2 * v] = a[v].x; s[2 * v + 1] = a[v].y; }
  } else {
#pragma unroll
    for (int v = 0; v < VEC; ++v) s[v] = 0.f;
#pragma unroll
    for (int r = 0; r < G; ++r) {
      float t[VEC];
      lds_vec<VEC>(t, part + r * stride);
#pragma unroll
      for (int v = 0; v < VEC; ++v) s[v] += t[v];
    }
  }
}

// Soft-mask value of one element for a compile-time isovalue kind (Sec. 3.5).
//   NORMAL: u = erfc(xs) / 2, xs = (F - mu) * inv with inv = +-sqrt(log2 e) / (sigma sqrt 2)
//   STEP:   u = 1[(F - t) * dir < 0], dir = +1 (F < t) or -1 (F > t)
template <int ISO>
__device__ __forceinline__ float iso_map(float f, float mu, float inv, float t, float dir) {
  if constexpr (ISO == ISOK_NORMAL) {
    const float xs = (f - mu) * inv;
    const float h = half_erfc_scaled(fabsf(xs));
    return xs >= 0.f ? h : 1.0f - h;
  } else if constexpr (ISO == ISOK_STEP) {
    return (f - t) * dir < 0.f ? 1.0f : 0.0f;
  } else {
    return f;
  }
}

// TMA producer cursor of a group. It lives in shared memory: only the group's leader thread
// uses it, so it takes no registers from the converter warps.
struct StreamProducer {
  const EnsDesc* pd;   // descriptor of the ensemble being loaded
  long n_issued;       // stages issued so far
  int iu, u_end;       // unit being loaded, end of the group's run
  int ist, in_st;      // stage within the unit, stages of the unit
  int icell0, slot;    // first cell of the unit, ring slot of the next stage
  int e_begin, e_end, chunk, M, boxes, rows, has_w;
  int ncls;            // residue classes of unaligned rows staged by TMA (0: none)
};
static_assert(sizeof(StreamProducer) <= kStreamProducerBytes, "producer cursor size");

// The isovalue map over a lane's MPW x VEC values, two at a time (packed FP32) for the
// normal kind: pairs of neighbouring cells, or of neighbouring members when VEC = 1.
template <int ISO, int MPW, int VEC>
__device__ __forceinline__ void iso_map_tile(float (&x)[MPW][VEC], float mu, float inv, float t,
                                             float dir, int mode) {
  if constexpr (ISO == ISOK_NORMAL && VEC % 2 == 0) {
#pragma unroll
    for (int k = 0; k < MPW; ++k)
#pragma unroll
      for (int v = 0; v < VEC; v += 2) {
        const float2 u = iso_normal2(make_float2(x[k][v], x[k][v + 1]), mu, inv);
        x[k][v] = u.x;
        x[k][v + 1] = u.y;
      }
  } else if constexpr (ISO == ISOK_NORMAL && MPW % 2 == 0) {
#pragma unroll
    for (int k = 0; k < MPW; k += 2)
#pragma unroll
      for (int v = 0; v < VEC; ++v) {
        const float2 u = iso_normal2(make_float2(x[k][v], x[k + 1][v]), mu, inv);
        x[k][v] = u.x;
        x[k + 1][v] = u.y;
      }
  } else if constexpr (ISO == ISOK_STEP) {
    // the step maps (sigma = 0) or, for the other kinds, the piecewise-linear maps; the
    // branch is uniform across the launch's ensemble
    if (mode <= ISO_STEP_ABOVE) {
#pragma unroll
      for (int k = 0; k < MPW; ++k)
#pragma unroll
        for (int v = 0; v < VEC; ++v) x[k][v] = iso_map<ISO>(x[k][v], mu, inv, t, dir);
    } else {
#pragma unroll
      for (int k = 0; k < MPW; ++k)
#pragma unroll
        for (int v = 0; v < VEC; ++v) x[k][v] = iso_piecewise(x[k][v], mode, mu, inv);
    }
  } else {
#pragma unroll
    for (int k = 0; k < MPW; ++k)
#pragma unroll
      for (int v = 0; v < VEC; ++v) x[k][v] = iso_map<ISO>(x[k][v], mu, inv, t, dir);
  }
}

// Layout of the dynamic shared memory (per CTA):
//   ring  [n_groups][depth][stage_floats]   TMA destinations [rows][sub*T]; the last sub*T
//                                           floats of a stage hold the cell measures
//   red   [n_groups][2][G*T + T]            partial column sums and their total, double-buffered
//   bars  [n_groups][depth]                 "stage full" mbarriers
//   flags [n_groups][2]                     abort flags (bounded wait ran out), one per
//                                           exchange-buffer parity (see below)
// MAXU (soft masks, first pass only): also reduce each member's largest u sqrt(w) into
// the descriptor's umax keys (the per-member E4M3 scales of a Gram over the same masks).
template <int VEC, int MPW, int G, int ISO, bool COEF, bool TMA, bool MAXU = false>
__global__ void __launch_bounds__(kStreamThreads, 1)
stream_kernel(const __grid_constant__ StreamParams p) {
  static_assert(!MAXU || (ISO == ISOK_NONE && !COEF), "maxima of soft masks, first pass");
  static_assert(MPW <= 32, "member coefficients are broadcast from one lane each");
  static_assert(VEC % 2 == 0 || MPW % 2 == 0, "values are processed in packed pairs");
  constexpr int T = 32 * VEC;
  constexpr int NG = kStreamWarps / G;
  constexpr int RB = G * T + T;  // floats per exchange buffer
  extern __shared__ __align__(1024) unsigned char smem[];

  const int warp = threadIdx.x >> 5;
  const int lane = threadIdx.x & 31;
  const int grp = warp / G;
  const int q = warp - grp * G;
  const int depth = p.depth;
  const int SF = p.stage_floats;
  // One register tile per TMA stage (every tile class is planned with sub = 1): the stage
  // width is a compile-time constant, so row offsets fold into the shared-memory loads.
  constexpr int SUB = 1;
  constexpr int TS = SUB * T;
  // Row stride of a stage: TMA stores rows back to back; the cp.async path stores each
  // row's enclosing 16-byte-aligned span (4 floats more), the row's first cell `roff` floats in.
  constexpr int RS = TMA ? TS : TS + 4;
  // Unaligned rows staged by TMA through the residue-class maps (see EnsDesc::tmap_cls)
  // instead of the threads' cp.async copies; the whole launch takes one of the two. The
  // one-cell-per-lane classes keep the cp.async spans (their spans of TS + 4 = 36 cells
  // cost more L2 traffic than the copies save), and compile without the class code.
  const bool CLS = !TMA && VEC > 1 && p.use_tma == 2;

  float* ring = reinterpret_cast<float*>(smem);
  float* red = ring + static_cast<size_t>(NG) * depth * SF;
  uint64_t* bars = reinterpret_cast<uint64_t*>(red + NG * 2 * RB);
  volatile int* flags = reinterpret_cast<volatile int*>(bars + NG * depth);
  StreamProducer* prod = reinterpret_cast<StreamProducer*>(
      (reinterpret_cast<uintptr_t>(flags + 2 * NG) + 15) & ~static_cast<uintptr_t>(15));

  float* my_ring = ring + static_cast<size_t>(grp) * depth * SF;
  float* my_red = red + grp * 2 * RB;
  uint64_t* my_bars = bars + grp * depth;
  const bool leader = (q == 0) && (lane == 0);

  // The ring's stages are filled by the leader's TMA copies (rows 16-byte aligned), or else
  // by every thread's 4-byte cp.async copies (see cpa_issue), each thread arriving once per
  // stage when its copies have landed.
  if (leader) {
    for (int s = 0; s < depth; ++s)
      mbar_init(&my_bars[s], (TMA || CLS) ? 1u : static_cast<uint32_t>(G * 32));
    fence_mbar_init();
  }
  // A warp that gives up on a wait sets the flag of the register tile whose group barrier
  // it arrives at next; all warps of the group read that flag after that barrier, so they
  // leave together (the other parity belongs to the neighbouring barrier).
  if (threadIdx.x < 2 * NG) flags[threadIdx.x] = 0;
  __syncthreads();

  // Each group takes a contiguous run of the flat unit list (an equal share of the work).
  // An ensemble's chunks are consecutive units, so a group looks an ensemble up (and
  // reloads its descriptor) only when it crosses into the next one; the chunks, and so the
  // results, do not depend on which group computes them.
  const int gid = blockIdx.x * NG + grp;
  const int total_groups = gridDim.x * NG;
  const int u_begin = unit_at_work(p, p.total_work * gid / total_groups);
  const int u_end = unit_at_work(p, p.total_work * (gid + 1) / total_groups);

  // ---- producer cursor (leader lane of the group only, in shared memory) ----
  StreamProducer& P = prod[grp];
  auto set_unit = [&](int u) {
    if (u >= P.e_end) {
      const EnsDesc* pd = &stream_desc(p, stream_find_ens(p, u));
      P.pd = pd;
      P.e_begin = pd->unit_begin;
      P.e_end = pd->unit_begin + pd->n_chunks;
      P.chunk = pd->chunk_cells;
      P.M = pd->M;
      P.boxes = pd->n_boxes;
      P.rows = pd->box_rows;
      P.has_w = pd->w != nullptr;
      P.ncls = pd->n_cls;
    }
    P.icell0 = (u - P.e_begin) * P.chunk;
    P.in_st = (min(P.chunk, P.M - P.icell0) + TS - 1) / TS;
  };
  auto issue_next = [&]() {
    if (P.iu >= P.u_end) return;
    const int slot = P.slot;
    P.slot = slot + 1 == depth ? 0 : slot + 1;
    float* dst = my_ring + static_cast<size_t>(slot) * SF;
    const int boxes = P.boxes, rows = P.rows;
    const bool has_w_p = P.has_w != 0;
    const EnsDesc* pd = P.pd;
    const uint32_t bytes = static_cast<uint32_t>(boxes * rows * TS + (has_w_p ? TS : 0)) * 4u;
    mbar_arrive_expect_tx(&my_bars[slot], bytes);
    const int x0 = P.icell0 + P.ist * TS;
    for (int b = 0; b < boxes; ++b)
      tma_load_2d(dst + static_cast<size_t>(b) * rows * TS, &pd->tmap, &my_bars[slot], x0, b * rows);
    if (has_w_p) tma_load_1d(dst + SF - TS, &pd->tmap_w, &my_bars[slot], x0);
    ++P.n_issued;
    if (++P.ist == P.in_st) {
      P.ist = 0;
      if (++P.iu < P.u_end) set_unit(P.iu);
    }
  };
  // Unaligned rows through the class maps: class c's boxes fill the stage rows from
  // c n_boxes box_rows on, each row the 16-byte-aligned span of TS + 4 cells around the
  // stage's cells (its first cell (data + i ld) mod 16 bytes in); cells past M read as 0.
  auto issue_next_cls = [&]() {
    if (P.iu >= P.u_end) return;
    const int slot = P.slot;
    P.slot = slot + 1 == depth ? 0 : slot + 1;
    float* dst = my_ring + static_cast<size_t>(slot) * SF;
    const int boxes = P.boxes, rows = P.rows, nc = P.ncls;
    const bool has_w_p = P.has_w != 0;
    const EnsDesc* pd = P.pd;
    const uint32_t bytes = static_cast<uint32_t>(nc * boxes * rows * RS + (has_w_p ? TS : 0)) * 4u;
    mbar_arrive_expect_tx(&my_bars[slot], bytes);
    const int x0 = P.icell0 + P.ist * TS;
    for (int c = 0; c < nc; ++c) {
      const CUtensorMap* m = c == 0 ? &pd->tmap : &pd->tmap_cls[c - 1];
      for (int b = 0; b < boxes; ++b)
        tma_load_2d(dst + static_cast<size_t>(c * boxes + b) * rows * RS, m, &my_bars[slot], x0,
                    b * rows);
    }
    if (has_w_p) tma_load_1d(dst + SF - TS, &pd->tmap_w, &my_bars[slot], x0);
    ++P.n_issued;
    if (++P.ist == P.in_st) {
      P.ist = 0;
      if (++P.iu < P.u_end) set_unit(P.iu);
    }
  };
  if (leader) {
    P.pd = nullptr;
    P.n_issued = 0;
    P.iu = u_begin;
    P.u_end = u_end;
    P.ist = 0;
    P.in_st = 0;
    P.icell0 = 0;
    P.slot = 0;
    P.e_begin = 0;
    P.e_end = 0;
    if (TMA) {
      if (P.iu < P.u_end) set_unit(P.iu);
      for (int s = 0; s < depth; ++s) issue_next();
    } else if (CLS) {
      if (P.iu < P.u_end) set_unit(P.iu);
      for (int s = 0; s < depth; ++s) issue_next_cls();
    }
  }

  // ---- consumers: every warp of the group ----
  long k_cons = 0;
  int c_slot = 0;
  uint32_t c_par = 0;
  long k_sub = 0;   // register tiles processed (parity of the exchange buffer)
  bool aborted = false;
  uint32_t bad = 0;

  // Descriptor fields of the current ensemble, kept in registers (the asm barriers below
  // clobber memory, so reading them through the descriptor would reload them every tile).
  const EnsDesc* dp = nullptr;
  int N = 0, M = 0, e_begin = 0, e_end = 0, e_chunk = 0;
  bool validate = false, has_w = false;
  float* u_out = nullptr;   // pass 1 of a field: soft masks stored for pass 2
  float iso_mu = 0.f, iso_inv = 0.f, iso_t = 0.f, dir = 1.f, pad = 0.f, my_cf = 0.f;
  int iso_md = 0;
  // Stage row of this warp's k-th member (unaligned rows): srow0 + k sstep. The cp.async
  // spans keep member order (row q + k G); with class maps the member q + k G sits in the
  // slot of class q mod n_cls, at row (q + k G) / n_cls (G is a multiple of n_cls).
  int srow0 = q, sstep = G;
  for (int u = u_begin; u < u_end && !aborted; ++u) {
    if (u >= e_end) {
      dp = &stream_desc(p, stream_find_ens(p, u));
      if constexpr (!TMA) {
        if (CLS) {
          const int nc = dp->n_cls;
          srow0 = (q & (nc - 1)) * dp->n_boxes * dp->box_rows + q / nc;
          sstep = G / nc;
        }
      }
      N = dp->N;
      M = dp->M;
      e_begin = dp->unit_begin;
      e_end = e_begin + dp->n_chunks;
      e_chunk = dp->chunk_cells;
      validate = dp->validate != 0;
      has_w = dp->w != nullptr;
      if constexpr (ISO != ISOK_NONE && !COEF) u_out = dp->u_out;
      iso_mu = dp->iso_mu;
      iso_inv = dp->iso_inv;
      iso_t = dp->iso_t;
      iso_md = dp->iso_mode;
      dir = iso_pad_sign(iso_md);
      // Rows past N read this value, which every isovalue kind maps to exactly 0.
      pad = ISO == ISOK_NONE ? 0.f
                             : (ISO == ISOK_NORMAL ? copysignf(__int_as_float(0x7f800000), iso_inv)
                                                   : dir * __int_as_float(0x7f800000));
      // Column-sum coefficients: lane k holds c_j of this warp's k-th member (pass 2), or
      // every member weighs 1 (pass 1).
      my_cf = 0.f;
      if constexpr (COEF) {
        const int i = q + lane * G;
        if (lane < MPW && i < N) my_cf = dp->coef[i];
      }
    }
    const EnsDesc& d = *dp;
    const int c = u - e_begin;
    const int cell0 = c * e_chunk;
    const int cells = min(e_chunk, M - cell0);
    const int n_st = (cells + TS - 1) / TS;
    float accM[MPW], accA[MPW], accX[MAXU ? MPW : 1];
#pragma unroll
    for (int k = 0; k < MPW; ++k) { accM[k] = 0.f; accA[k] = 0.f; }
#pragma unroll
    for (int k = 0; k < (MAXU ? MPW : 1); ++k) accX[k] = 0.f;

    // Rows that are not 16-byte aligned (no TMA): each stage holds, per member row, the
    // 16-byte-aligned span that encloses the stage's cells, its first cell `ro` floats
    // before the stage's first cell, copied in 16-byte pieces by the warp that owns the row
    // (its lanes take the rows' pieces in turn). A piece reads only the row's cells below M
    // (zero-filling the rest) and pieces wholly past M are skipped: cells past M are masked
    // to zero after they are read. A span starts at most 3 cells before the row's first
    // cell, inside the previous row; only row 0's first piece can start before the data,
    // and it is copied cell by cell from cell 0 on (the cells before are never read).
    // Warp 0 also copies the cell measures with 4-byte copies. Every thread arrives on the
    // stage's barrier once its copies have landed.
    const int boff = static_cast<int>((reinterpret_cast<uintptr_t>(d.data) >> 2) & 3u);
    const int ld3 = static_cast<int>(d.ld & 3);
    // Lane l copies piece l % PR (of the PR = TS / 4 main pieces of a span) of rows
    // r RPI + l / PR for every r; lane k also copies the span's last piece of row k (the
    // classes of 28 and 32 members per warp, and odd member counts, walk the pieces in one
    // strided loop instead).
    constexpr int PR = TS / 4;          // main 16-byte pieces of a span (the last is extra)
    constexpr int RPI = 32 / PR;        // rows per copy instruction

    auto cpa_piece = [&](float* stage, int xs0, int i, int pc) {
      const int ro = (boff + i * ld3) & 3;
      const int first = xs0 - ro + 4 * pc;   // the piece's first cell (row-relative)
      const int left = M - first;
      if (left <= 0) return;
      float* dst = stage + static_cast<size_t>(i) * RS + 4 * pc;
      const float* row = d.data + static_cast<int64_t>(i) * d.ld;
      if (first >= 0 || i > 0) {
        cp_async16(dst, row + first, left >= 4 ? 16u : static_cast<uint32_t>(4 * left));
      } else {
#pragma unroll
        for (int e = 0; e < 4; ++e)
          if (first + e >= 0 && first + e < M) cp_async4(dst + e, row + first + e, 4u);
      }
    };
    auto cpa_issue = [&](int st_i, int slot_i) {
      float* stage = my_ring + static_cast<size_t>(slot_i) * SF;
      const int xs0 = cell0 + st_i * TS;   // the stage's first cell (a multiple of 32)
      if constexpr ((VEC == 1 && MPW > 24) || MPW % RPI != 0) {
        // the widest classes (fewer registers), and member counts that do not fill whole
        // copy instructions: the warp's pieces in one strided loop
        for (int t = lane; t < MPW * (PR + 1); t += 32) {
          const int k = t / (PR + 1), c = t - k * (PR + 1);
          if (q + k * G < N) cpa_piece(stage, xs0, q + k * G, c);
        }
      } else {
        const int sr = lane / PR, pc = lane - sr * PR;
#pragma unroll
        for (int r = 0; r < MPW / RPI; ++r) {
          const int i = q + (r * RPI + sr) * G;
          if (i < N) cpa_piece(stage, xs0, i, pc);
        }
        if (lane < MPW && q + lane * G < N) cpa_piece(stage, xs0, q + lane * G, PR);
      }
      if (q == 0 && has_w) {
        const int xs = xs0 + lane;
#pragma unroll
        for (int v = 0; v < VEC; ++v) {
          const bool in = xs + 32 * v < M;
          cp_async4(stage + SF - TS + lane + 32 * v, d.w + (in ? xs + 32 * v : 0), in ? 4u : 0u);
        }
      }
      cp_async_arrive(&my_bars[slot_i]);
    };
    if constexpr (!TMA) {
      if (!CLS) {
        int sl = c_slot;
        for (int st_i = 0; st_i < depth && st_i < n_st; ++st_i) {
          cpa_issue(st_i, sl);
          if (++sl == depth) sl = 0;
        }
      }
    }

    for (int st = 0; st < n_st && !aborted; ++st, ++k_cons) {
      const int slot = c_slot;          // k_cons % depth
      const uint32_t par = c_par;       // (k_cons / depth) & 1
      if (++c_slot == depth) { c_slot = 0; c_par ^= 1u; }
      const float* sb = my_ring + static_cast<size_t>(slot) * SF;
      if (!mbar_wait_bounded(&my_bars[slot], par, kWaitTimeoutNs)) flags[2 * grp + (k_sub & 1)] = 1;
      for (int j = 0; j < SUB; ++j, ++k_sub) {
        const int x0 = cell0 + st * TS + j * T;     // first cell of this register tile
        const int xl = x0 + lane * VEC;             // first cell of this lane
        const bool full = x0 + T <= M;              // no cell past the end of the ensemble
        float x[MPW][VEC];
        float wv[VEC];

        // the stage in shared memory, filled by TMA or by the threads' cp.async copies
#pragma unroll
        for (int k = 0; k < MPW; ++k) {
          const int i = q + k * G;
          if (i < N) {
            if constexpr (TMA) {
              lds_vec<VEC>(x[k], sb + static_cast<size_t>(i) * TS + j * T + lane * VEC);
            } else {
              // the row's cells start `ro` floats into its span (the same for the warp)
              lds_shifted<VEC>(x[k], sb + static_cast<size_t>(srow0 + k * sstep) * RS + j * T + lane * VEC,
                               (boff + i * ld3) & 3);
            }
          } else {
#pragma unroll
            for (int v = 0; v < VEC; ++v) x[k][v] = pad;
          }
        }
        if (has_w) lds_vec<VEC>(wv, sb + SF - TS + j * T + lane * VEC);

        if (validate) {
#pragma unroll
          for (int v = 0; v < VEC; ++v) {
            if (xl + v < M) {
              if (has_w && (!(wv[v] > 0.f) || !(wv[v] < 3.0e38f))) bad |= ERR_DOMAIN;
#pragma unroll
              for (int k = 0; k < MPW; ++k) {
                if (q + k * G < N) {
                  const float f = x[k][v];
                  if (ISO != ISOK_NONE ? !(fabsf(f) < 3.0e38f) : !(f >= 0.f && f <= 1.f))
                    bad |= ERR_DOMAIN;
                }
              }
            }
          }
        }
        if constexpr (ISO != ISOK_NONE) iso_map_tile<ISO>(x, iso_mu, iso_inv, iso_t, dir, iso_md);
        if constexpr (ISO != ISOK_NONE && !COEF) {
          // The soft masks of this tile, stored once so that pass 2 reads them instead of
          // repeating the isovalue map (rows are round_up(M, 4) floats, 16-byte aligned).
          if (u_out != nullptr) {
            const int64_t ldu = (M + 3) & ~3;
#pragma unroll
            for (int k = 0; k < MPW; ++k) {
              const int i = q + k * G;
              if (i < N) {
                float* dst = u_out + static_cast<int64_t>(i) * ldu + xl;
                if (xl + VEC <= M) {
                  stg_cs_vec<VEC>(dst, x[k]);
                } else {
#pragma unroll
                  for (int v = 0; v < VEC; ++v)
                    if (xl + v < M) __stcs(dst + v, x[k][v]);
                }
              }
            }
          }
        }
        if constexpr (!COEF && VEC == 1) {
          // BF16 operands u sqrt(w) of the row-block-tiled Gram (N > 256: the one-cell-per-lane
          // classes), written from the masks this pass maps anyway (cells past M are never
          // read: the tile kernel's copies zero-fill them).
          // read through the descriptor here, so the pointer holds no register in the loop
          uint16_t* const op_out = dp->op_out;
          if (op_out != nullptr) {
            const int64_t op_ld = dp->op_ld;
            float sw[VEC];
#pragma unroll
            for (int v = 0; v < VEC; ++v) sw[v] = has_w ? sqrtf(wv[v]) : 1.f;
#pragma unroll
            for (int k = 0; k < MPW; ++k) {
              const int i = q + k * G;
              if (i < N) {
                uint16_t* dst = op_out + static_cast<int64_t>(i) * op_ld + xl;
                uint16_t b[VEC];
#pragma unroll
                for (int v = 0; v < VEC; ++v)
                  b[v] = __bfloat16_as_ushort(__float2bfloat16_rn(x[k][v] * sw[v]));
                if (xl + VEC <= M) {
                  if constexpr (VEC == 4) {
                    *reinterpret_cast<uint2*>(dst) = make_uint2(b[0] | (static_cast<uint32_t>(b[1]) << 16),
                                                                b[2] | (static_cast<uint32_t>(b[3]) << 16));
                  } else if constexpr (VEC == 2) {
                    *reinterpret_cast<uint32_t*>(dst) = b[0] | (static_cast<uint32_t>(b[1]) << 16);
                  } else {
                    dst[0] = b[0];
                  }
                } else {
#pragma unroll
                  for (int v = 0; v < VEC; ++v)
                    if (xl + v < M) dst[v] = b[v];
                }
              }
            }
          }
        }
        if (!full) {  // only the ensemble's last tile: cells past M carry no mass
#pragma unroll
          for (int v = 0; v < VEC; ++v) {
            if (xl + v >= M) {
#pragma unroll
              for (int k = 0; k < MPW; ++k) x[k][v] = 0.f;
            }
          }
        }

        // Column sum over this warp's members (padding rows hold zeros) ...
        float s[VEC];
        if constexpr (VEC % 2 == 0) {
          float2 s2[VEC / 2];
#pragma unroll
          for (int v = 0; v < VEC / 2; ++v) s2[v] = f2(0.f);
#pragma unroll
          for (int k = 0; k < MPW; ++k) {
            if constexpr (COEF) {
              const float2 cfk = f2(__shfl_sync(0xffffffffu, my_cf, k));
#pragma unroll
              for (int v = 0; v < VEC / 2; ++v)
                s2[v] = f2_fma(cfk, make_float2(x[k][2 * v], x[k][2 * v + 1]), s2[v]);
            } else {
#pragma unroll
              for (int v = 0; v < VEC / 2; ++v)
                s2[v] = f2_add(s2[v], make_float2(x[k][2 * v], x[k][2 * v + 1]));
            }
          }
#pragma unroll
          for (int v = 0; v < VEC / 2; ++v) { s[2 * v] = s2[v].x; s[2 * v + 1] = s2[v].y; }
        } else {
          float2 s2 = f2(0.f);
#pragma unroll
          for (int k = 0; k < MPW; k += 2) {
            if constexpr (COEF) {
              const float2 cfk = make_float2(__shfl_sync(0xffffffffu, my_cf, k),
                                             __shfl_sync(0xffffffffu, my_cf, k + 1));
              s2 = f2_fma(cfk, make_float2(x[k][0], x[k + 1][0]), s2);
            } else {
              s2 = f2_add(s2, make_float2(x[k][0], x[k + 1][0]));
            }
          }
          s[0] = s2.x + s2.y;
        }
        // ... then across the G warps of the group: every warp posts its partial; either
        // every warp adds the G partials (xchg 0), or warp r first totals the cells
        // [r T/G, (r+1) T/G) and every warp then reads the totals (xchg 1). Both add the
        // partials in warp order, so both give the same bits.
        float* rb = my_red + static_cast<int>(k_sub & 1) * RB;
        if constexpr (G > 1) {
          sts_vec<VEC>(rb + q * T + lane * VEC, s);
          named_barrier(1 + grp, G * 32);
        } else {
          __syncwarp();
        }
        if (flags[2 * grp + (k_sub & 1)]) { aborted = true; break; }
        if constexpr (TMA) {
          if (leader && j == SUB - 1) issue_next();  // every warp has read this slot: refill it
        } else if (CLS) {
          if (leader && j == SUB - 1) issue_next_cls();  // every warp has read this slot
        } else {
          if (j == SUB - 1 && st + depth < n_st) cpa_issue(st + depth, slot);
        }
        if constexpr (G > 2) {
          if (p.xchg == 1) {
            constexpr int cpw = T / G;
            if (lane < cpw) {
              const int cc = q * cpw + lane;
              float acc = 0.f;
#pragma unroll
              for (int r = 0; r < G; ++r) acc += rb[r * T + cc];
              rb[G * T + cc] = acc;
            }
            named_barrier(1 + grp, G * 32);
            lds_vec<VEC>(s, rb + G * T + lane * VEC);
          } else {
            sum_partials<VEC, G>(s, rb + lane * VEC, T);
          }
        } else if constexpr (G == 2) {
          sum_partials<VEC, G>(s, rb + lane * VEC, T);
        }
        // Per-member accumulation: m_i += w u_i, A_i += w u_i s. The branches on the
        // weights and on padding rows (i >= N: zeros, nothing to add) are uniform across
        // the warp; the arithmetic of each member is the same on every path. (The
        // one-cell-per-lane classes keep a single loop: the duplicated code costs them
        // registers.)
        if constexpr (VEC == 1) {
#pragma unroll
          for (int k = 0; k < MPW; ++k) {
            const float t = has_w ? wv[0] * x[k][0] : x[k][0];
            accM[k] += t;
            accA[k] = fmaf(t, s[0], accA[k]);
          }
        } else if (has_w) {
#pragma unroll
          for (int k = 0; k < MPW; ++k) {
            if (q + k * G < N) {
#pragma unroll
              for (int v = 0; v < VEC; ++v) {
                const float t = wv[v] * x[k][v];
                accM[k] += t;
                accA[k] = fmaf(t, s[v], accA[k]);
              }
            }
          }
        } else {
#pragma unroll
          for (int k = 0; k < MPW; ++k) {
            if (q + k * G < N) {
#pragma unroll
              for (int v = 0; v < VEC; ++v) {
                accM[k] += x[k][v];
                accA[k] = fmaf(x[k][v], s[v], accA[k]);
              }
            }
          }
        }
        if constexpr (MAXU && VEC == 1) {
          // the operand u sqrt(w), rounded as the Gram kernels round it
          const float sw = has_w ? sqrtf(wv[0]) : 1.f;
#pragma unroll
          for (int k = 0; k < MPW; ++k) accX[k] = fmaxf(accX[k], has_w ? x[k][0] * sw : x[k][0]);
        } else if constexpr (MAXU) {
          // the operand u sqrt(w), rounded as the Gram kernels round it
          if (has_w) {
            float sw[VEC];
#pragma unroll
            for (int v = 0; v < VEC; ++v) sw[v] = sqrtf(wv[v]);
#pragma unroll
            for (int k = 0; k < MPW; ++k)
              if (q + k * G < N)
#pragma unroll
                for (int v = 0; v < VEC; ++v) accX[k] = fmaxf(accX[k], x[k][v] * sw[v]);
          } else {
#pragma unroll
            for (int k = 0; k < MPW; ++k)
              if (q + k * G < N)
#pragma unroll
                for (int v = 0; v < VEC; ++v) accX[k] = fmaxf(accX[k], x[k][v]);
          }
        }
      }
      if (aborted) break;
    }
    if (aborted) break;

    // Chunk done: reduce lanes, write this chunk's partials.
#pragma unroll
    for (int k = 0; k < MPW; ++k) {
      const float m = warp_sum(accM[k]);
      const float a = warp_sum(accA[k]);
      const int i = q + k * G;
      if (lane == 0 && i < N) {
        d.part[static_cast<size_t>(c) * 2 * N + i] = static_cast<double>(m);
        d.part[static_cast<size_t>(c) * 2 * N + N + i] = static_cast<double>(a);
      }
    }
    if constexpr (MAXU) {
      unsigned int* const um = dp->umax;
      if (um != nullptr) {
#pragma unroll
        for (int k = 0; k < MPW; ++k) {
          float mx = accX[k];
#pragma unroll
          for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
          const int i = q + k * G;
          if (lane == 0 && i < N) atomicMax(um + i, fkey(mx));
        }
      }
    }
  }

  if (bad) atomicOr(p.err, bad);
  if (aborted && lane == 0 && q == 0) atomicOr(p.err, ERR_TIMEOUT);
  // On an early exit, let this group's copies in flight land before the CTA retires.
  if constexpr (!TMA) cp_async_wait_all();   // this thread's copies, before the CTA retires
  if ((TMA || CLS) && leader) {
    while (k_cons < P.n_issued) {
      const int slot = static_cast<int>(k_cons % depth);
      const uint32_t par = static_cast<uint32_t>((k_cons / depth) & 1);
      if (!mbar_wait_bounded(&my_bars[slot], par, kWaitTimeoutNs)) break;
      ++k_cons;
    }
  }
}

template <int VEC, int MPW, int G, int ISO, bool COEF, bool TMA, bool MAXU = false>
cudaError_t launch_stream_inst(const StreamParams& p, int grid, size_t smem, cudaStream_t s) {
  stream_kernel<VEC, MPW, G, ISO, COEF, TMA, MAXU><<<grid, kStreamThreads, smem, s>>>(p);
  return cudaGetLastError();
}

template <int VEC, int MPW, int G, int ISO, bool COEF, bool TMA, bool MAXU = false>
cudaError_t init_stream_inst(int smem) {
  return cudaFuncSetAttribute(stream_kernel<VEC, MPW, G, ISO, COEF, TMA, MAXU>,
                              cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
}

// All instantiations of one tile class (isovalue kind x coefficient pass x TMA).
template <int VEC, int MPW, int G>
struct StreamClass {
  static cudaError_t launch(const StreamParams& p, int iso, bool coef, int grid, size_t smem,
                            cudaStream_t s) {
    const bool tma = p.use_tma == 1;   // 2: unaligned rows through class maps (TMA = false)
    if (p.maxu && iso == ISOK_NONE && !coef)   // the first pass also reduces the maxima
      return tma ? launch_stream_inst<VEC, MPW, G, ISOK_NONE, false, true, true>(p, grid, smem, s)
                 : launch_stream_inst<VEC, MPW, G, ISOK_NONE, false, false, true>(p, grid, smem, s);
#define PIDK_STREAM_CASE(ISO)                                                           \
  if (iso == ISO) {                                                                     \
    if (tma) return coef ? launch_stream_inst<VEC, MPW, G, ISO, true, true>(p, grid, smem, s)  \
                         : launch_stream_inst<VEC, MPW, G, ISO, false, true>(p, grid, smem, s); \
    return coef ? launch_stream_inst<VEC, MPW, G, ISO, true, false>(p, grid, smem, s)          \
                : launch_stream_inst<VEC, MPW, G, ISO, false, false>(p, grid, smem, s);        \
  }
    PIDK_STREAM_CASE(ISOK_NONE)
    PIDK_STREAM_CASE(ISOK_NORMAL)
    PIDK_STREAM_CASE(ISOK_STEP)
#undef PIDK_STREAM_CASE
    return cudaErrorInvalidValue;
  }
  static cudaError_t init(int smem) {
    cudaError_t e = cudaSuccess;
#define PIDK_STREAM_INIT(ISO)                                                                \
  if (e == cudaSuccess) e = init_stream_inst<VEC, MPW, G, ISO, true, true>(smem);           \
  if (e == cudaSuccess) e = init_stream_inst<VEC, MPW, G, ISO, false, true>(smem);          \
  if (e == cudaSuccess) e = init_stream_inst<VEC, MPW, G, ISO, true, false>(smem);          \
  if (e == cudaSuccess) e = init_stream_inst<VEC, MPW, G, ISO, false, false>(smem);
    PIDK_STREAM_INIT(ISOK_NONE)
    PIDK_STREAM_INIT(ISOK_NORMAL)
    PIDK_STREAM_INIT(ISOK_STEP)
#undef PIDK_STREAM_INIT
    if (e == cudaSuccess) e = init_stream_inst<VEC, MPW, G, ISOK_NONE, false, true, true>(smem);
    if (e == cudaSuccess) e = init_stream_inst<VEC, MPW, G, ISOK_NONE, false, false, true>(smem);
    return e;
  }
};

}  // namespace pidk
