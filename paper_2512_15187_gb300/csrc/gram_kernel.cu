// Full PID on the 5th-generation tensor cores (sm_103a, tcgen05 + TMA + TMEM).
//
// Full PID needs every ordered pair's inclusion u_i subset_p u_j = G_ij / m_i with
// G_ij = sum_x w_x u_i(x) u_j(x) (Eq. 9, Eq. 10 with the weighted sums of Eq. 14): the N x N
// Gram of U' = U diag(sqrt w), a dense contraction over the M cells. One pass:
//
//   * 16 converter warps take each TMA-staged FP32 tile [N rows][TS cells], apply the
//     isovalue map (Sec. 3.5), run the exact PID-mean arithmetic of the streaming kernel
//     (mean contour, m_i, A_i) and write u sqrt(w) as tensor-core operands into a shared-
//     memory ring in the K-major 128-byte-swizzle layout: BF16, a hi + lo BF16 pair, or
//     E4M3 times a power-of-two scale;
//   * one thread issues tcgen05.mma with A = B = that operand tile (G = U' U'^T), M = 128
//     rows, N = N rounded up to 16, accumulating in FP32 in tensor memory (double-buffered
//     per cell chunk); split BF16 issues hi.hi + hi.lo + lo.hi;
//   * converter warps 0-3 (one per TMEM lane quarter) drain each chunk's accumulator with
//     tcgen05.ld into an FP32 partial Gram halfway through the next chunk, when its last
//     products have long landed; the finalisation reduces the partials over chunks in FP64
//     in a fixed order.
//
// Every wait is bounded; on a time-out the kernel raises the error word, lets its copies
// and tensor-core work drain (again bounded) and frees its tensor memory before returning.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_fp8.h>
#include <cuda_runtime.h>

#include "device.cuh"
#include "internal.h"
#include "stream_kernel.cuh"

namespace pidk {

namespace {

constexpr int VEC = 4;                  // cells per lane per register tile
constexpr int T = 32 * VEC;             // cells per register tile (= one TMA stage)
constexpr int MPW = 8;                  // members per warp: a group of G warps covers 8 G rows
constexpr uint32_t kTmemCols = 256;     // per CTA: each group's two accumulators of 8 G columns

__device__ __forceinline__ const EnsDesc& gdesc(const GramParams& p, int e) {
  return p.descs ? p.descs[e] : p.one;
}

__device__ __forceinline__ int gram_find_ens(const GramParams& p, int u) {
  if (p.descs == nullptr) return 0;
  int lo = 0, hi = p.n_ens - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (p.descs[mid].unit_begin <= u) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// Byte offset of (member row i, byte b of the 128-byte K-block row) in a swizzled plane.
__device__ __forceinline__ uint32_t sw128_offset(int i, int b) {
  return static_cast<uint32_t>((i >> 3) * 1024 + (i & 7) * 128 + ((((b >> 4) ^ (i & 7))) << 4) +
                               (b & 15));
}

}  // namespace

// PREC: 1 = BF16, 2 = split BF16 (hi + lo), 3 = E4M3. TMA: FP32 tiles staged by the tensor
// memory accelerator (rows 16-byte aligned) or read directly from global memory.
// A stage is 128 cells: two 64-element K-blocks of 16-bit operands or one 128-element
// K-block of E4M3, each K-block a [128 rows][128 bytes] swizzled plane.
//
// Schedule (16 warps, one CTA per SM): every warp converts its members' rows of a stage;
// after the first group barrier of stage k the leader thread issues the tensor-core work
// of stage k-1 (all its operands were written and fenced before that barrier) and commits
// it to the stage's "operand free" mbarrier and, at a chunk's end, to the accumulator's
// "ready" mbarrier; warps 0-3 drain the previous chunk's accumulator halfway through the
// next chunk.
template <int G, int ISO, int PREC, bool TMA>
__global__ void __launch_bounds__(kGramThreads, 1) gram_kernel(const __grid_constant__ GramParams p) {
  constexpr int NG = kGramConvWarps / G;             // independent groups per CTA
  constexpr int ROWS = MPW * G;                      // operand rows a group writes (>= N)
  constexpr uint32_t PLANE = ROWS * 128;             // one K-block: [ROWS][128 bytes]
  constexpr int PLANES = PREC == 2 ? 2 : 1;          // hi (+ lo)
  constexpr int KBLK = PREC == 3 ? 1 : 2;            // K-blocks per stage
  constexpr uint32_t OP_STAGE = PLANES * KBLK * PLANE;
  constexpr uint32_t FMT = PREC == 3 ? 0u : 1u;      // E4M3 : BF16
  constexpr int RB = G * T + T;                      // exchange buffer floats
  constexpr uint32_t BUFC = ROWS;                    // TMEM columns per accumulator
  extern __shared__ __align__(1024) unsigned char smem_raw[];

  const int warp = threadIdx.x >> 5;
  const int lane = threadIdx.x & 31;
  const int grp = warp / G;
  const int q = warp - grp * G;
  const bool leader = (q == 0) && (lane == 0);
  const int dF = p.dF, dO = p.dO, SF = p.stage_floats, TS = p.TS;

  // ---- shared memory carve-up: all operand rings first (1024-byte aligned) ----
  // An M = 128 MMA reads 128 rows from a plane's base; with 64-row planes the upper rows
  // come from the bytes that follow (garbage rows of D that are never read).
  const uint32_t raw = smem_u32(smem_raw);
  unsigned char* smem = smem_raw + ((1024u - (raw & 1023u)) & 1023u);
  float* f_all = reinterpret_cast<float*>(smem + static_cast<size_t>(NG) * dO * OP_STAGE);
  float* red_all = f_all + static_cast<size_t>(NG) * dF * SF;
  uint64_t* bars_all = reinterpret_cast<uint64_t*>(red_all + NG * 2 * RB);
  int* flags_all = reinterpret_cast<int*>(bars_all + NG * (dF + dO + 5));
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(flags_all + 2 * NG);

  unsigned char* op_ring = smem + static_cast<size_t>(grp) * dO * OP_STAGE;
  float* f_ring = f_all + static_cast<size_t>(grp) * dF * SF;
  float* red = red_all + grp * 2 * RB;
  uint64_t* bars = bars_all + grp * (dF + dO + 5);
  uint64_t* fF = bars;              // FP32 stage landed (TMA)
  uint64_t* opE = fF + dF;          // operand stage consumed (tcgen05.commit)
  uint64_t* accF = opE + dO;        // accumulator ready (tcgen05.commit)
  uint64_t* accE = accF + 2;        // accumulator drained (the group's warps 0-3)
  uint64_t* finB = accE + 2;        // all of the group's tensor-core work done
  // Abort flags, one per exchange-buffer parity: a warp that gives up on a wait sets the
  // flag of the group barrier it reaches next, and every warp of the group reads that flag
  // after that barrier, so all of them leave together.
  volatile int* cflag = flags_all + 2 * grp;

  if (leader) {
    for (int s = 0; s < dF; ++s) mbar_init(&fF[s], 1);
    for (int s = 0; s < dO; ++s) mbar_init(&opE[s], 1);
    for (int b = 0; b < 2; ++b) { mbar_init(&accF[b], 1); mbar_init(&accE[b], kGramEpiWarps); }
    mbar_init(finB, 1);
    cflag[0] = 0;
    cflag[1] = 0;
    fence_mbar_init();
  }
  // Operand rows past N must be finite on first use: clear every operand ring.
  for (uint32_t o = threadIdx.x * 16; o < static_cast<uint32_t>(NG) * dO * OP_STAGE; o += kGramThreads * 16)
    *reinterpret_cast<uint4*>(smem + o) = make_uint4(0, 0, 0, 0);
  fence_proxy_async_smem();
  if (warp == 0) {
    tmem_alloc(tmem_slot, kTmemCols);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem_base = *tmem_slot + static_cast<uint32_t>(grp) * 2 * BUFC;
  const int gid = blockIdx.x * NG + grp;
  const int total_groups = gridDim.x * NG;

  // ---- TMA producer cursor (leader) ----
  int iu = gid, ist = 0, ie = 0, icell0 = 0, in_st = 0;
  long n_issued = 0;
  auto set_unit = [&](int u) {
    ie = gram_find_ens(p, u);
    const EnsDesc& d = gdesc(p, ie);
    icell0 = (u - d.unit_begin) * d.chunk_cells;
    in_st = (min(d.chunk_cells, d.M - icell0) + TS - 1) / TS;
  };
  auto issue_next = [&]() {
    if (iu >= p.total_units) return;
    const EnsDesc& d = gdesc(p, ie);
    const int slot = static_cast<int>(n_issued % dF);
    float* dst = f_ring + static_cast<size_t>(slot) * SF;
    mbar_arrive_expect_tx(&fF[slot],
                          static_cast<uint32_t>(d.n_boxes * d.box_rows * TS + (d.w ? TS : 0)) * 4u);
    const int x0 = icell0 + ist * TS;
    for (int b = 0; b < d.n_boxes; ++b)
      tma_load_2d(dst + static_cast<size_t>(b) * d.box_rows * TS, &d.tmap, &fF[slot], x0,
                  b * d.box_rows);
    if (d.w) tma_load_1d(dst + SF - TS, &d.tmap_w, &fF[slot], x0);
    ++n_issued;
    if (++ist == in_st) {
      ist = 0;
      iu += total_groups;
      if (iu < p.total_units) set_unit(iu);
    }
  };
  if (TMA && leader) {
    if (iu < p.total_units) set_unit(iu);
    for (int s = 0; s < dF; ++s) issue_next();
  }

  // ---- tensor-core issue (leader): the stage written last, issued after the next barrier ----
  bool pend = false, pend_first = false, pend_last = false;
  int pend_slot = 0, pend_buf = 0;
  long pend_kc = 0;
  uint32_t pend_idesc = 0;
  auto issue_pending = [&]() -> bool {
    if (!pend) return true;
    pend = false;
    if (pend_first && pend_kc >= 2 &&
        !mbar_wait_bounded(&accE[pend_buf], static_cast<uint32_t>(((pend_kc >> 1) - 1) & 1),
                           kWaitTimeoutNs))
      return false;
    tc_fence_after();
    const uint32_t dt = tmem_base + static_cast<uint32_t>(pend_buf) * BUFC;
    // descriptor of the stage's first K-block; K steps advance its 16-byte address field
    const uint64_t d0 = umma_desc_sw128(smem_u32(op_ring) + static_cast<uint32_t>(pend_slot) * OP_STAGE);
#pragma unroll
    for (int kb = 0; kb < KBLK; ++kb) {
#pragma unroll
      for (int ks = 0; ks < 4; ++ks) {   // 4 x 32 bytes along K in the 128-byte row
        const uint64_t hi = d0 + static_cast<uint64_t>((kb * PLANE + ks * 32) >> 4);
        const uint32_t acc = (pend_first && kb == 0 && ks == 0) ? 0u : 1u;
        if constexpr (PREC == 3) {
          umma_f8(dt, hi, hi, pend_idesc, acc);
        } else {
          umma_f16(dt, hi, hi, pend_idesc, acc);
          if constexpr (PREC == 2) {
            const uint64_t lo = hi + static_cast<uint64_t>((KBLK * PLANE) >> 4);
            umma_f16(dt, hi, lo, pend_idesc, 1u);
            umma_f16(dt, lo, hi, pend_idesc, 1u);
          }
        }
      }
    }
    tc_commit(&opE[pend_slot]);
    if (pend_last) tc_commit(&accF[pend_buf]);
    return true;
  };

  // ---- accumulator drain of the CTA's kc-th unit u (warps 0-3, one TMEM lane quarter each) ----
  auto drain = [&](int u, long kc) -> bool {
    const EnsDesc& d = gdesc(p, gram_find_ens(p, u));
    const int N = d.N;
    const int c = u - d.unit_begin;
    const int nmma = (N + 15) & ~15;
    const int b = static_cast<int>(kc & 1);
    if (!mbar_wait_bounded(&accF[b], static_cast<uint32_t>((kc >> 1) & 1), kWaitTimeoutNs))
      return false;
    tc_fence_after();
    float unscale = 1.0f;
    if constexpr (PREC == 3) {
      const float sc = d.op_scale ? *d.op_scale : 256.0f;
      unscale = 1.0f / (sc * sc);
    }
    const int row = 32 * q + lane;
    float* gp = d.gpart + static_cast<size_t>(c) * N * N;
    for (int j0 = 0; j0 < nmma; j0 += 32) {
      float v[32];
      tmem_ld32(tmem_base + (static_cast<uint32_t>(32 * q) << 16) + b * BUFC + j0, v);
      if (row < N) {
#pragma unroll
        for (int jj = 0; jj < 32; ++jj)
          if (j0 + jj < N) gp[static_cast<size_t>(j0 + jj) * N + row] = v[jj] * unscale;
      }
    }
    tc_fence_before();
    __syncwarp();
    if (lane == 0) mbar_arrive(&accE[b]);
    return true;
  };

  // Swizzled byte offset of this lane's piece of row q; row q + m G adds m G 128 bytes
  // (G is a multiple of 8, so every owned row has the same row-in-atom q & 7).
  const uint32_t lane_off = PREC == 3 ? sw128_offset(q, lane * 4)
                                      : static_cast<uint32_t>(lane >> 4) * PLANE +
                                            sw128_offset(q, (lane & 15) * 8);
  long k = 0, kt = 0, kc = 0;
  int prev_u = -1;
  long prev_kc = -1;
  bool aborted = false;
  uint32_t bad = 0;
  for (int u = gid; u < p.total_units && !aborted; u += total_groups, ++kc) {
    const EnsDesc& d = gdesc(p, gram_find_ens(p, u));
    const int N = d.N;
    const int M = d.M;                       // descriptor fields kept in registers: the
    const bool validate = d.validate != 0;   // asm barriers below clobber memory
    const float* data = d.data;
    const float* wptr = d.w;
    const int64_t ld = d.ld;
    const int c = u - d.unit_begin;
    const int cell0 = c * d.chunk_cells;
    const int n_st = (min(d.chunk_cells, M - cell0) + TS - 1) / TS;
    const uint32_t idesc = umma_idesc(FMT, 128, static_cast<uint32_t>((N + 15) & ~15));
    const float iso_mu = d.iso_mu, iso_inv = d.iso_inv, iso_t = d.iso_t;
    const float dir = (d.iso_mode == ISO_STEP_ABOVE) ? -1.f : 1.f;
    const bool has_w = wptr != nullptr;
    const float inv_n = 1.0f / static_cast<float>(N);
    // Rows q, q+G, ... below N are this warp's members; rows past N are skipped
    // (warp-uniform guards), so their registers are never read.
    const int mlive = q < N ? (N - q + G - 1) / G : 0;
    float scale = 1.0f;
    if constexpr (PREC == 3) scale = d.op_scale ? *d.op_scale : 256.0f;
    float accM[MPW], accA[MPW];
#pragma unroll
    for (int m = 0; m < MPW; ++m) { accM[m] = 0.f; accA[m] = 0.f; }

    for (int st = 0; st < n_st; ++st, ++k, ++kt) {
      const int fslot = static_cast<int>(k % dF);
      const int oslot = static_cast<int>(k % dO);
      if (TMA && !mbar_wait_bounded(&fF[fslot], static_cast<uint32_t>((k / dF) & 1), kWaitTimeoutNs))
        cflag[kt & 1] = 1;
      const float* sb = f_ring + static_cast<size_t>(fslot) * SF;
      unsigned char* ob = op_ring + static_cast<size_t>(oslot) * OP_STAGE;

      const int x0 = cell0 + st * TS;
      const int xl = x0 + lane * VEC;
      const bool full = x0 + T <= M;
      float x[MPW][VEC];
      float wv[VEC] = {1.f, 1.f, 1.f, 1.f};
      if constexpr (TMA) {
#pragma unroll
        for (int m = 0; m < MPW; ++m) {
          if (m < mlive) {
            lds_vec<VEC>(x[m], sb + static_cast<size_t>(q + m * G) * TS + lane * VEC);
          } else {
#pragma unroll
            for (int v = 0; v < VEC; ++v) x[m][v] = 0.f;
          }
        }
        if (has_w) lds_vec<VEC>(wv, sb + SF - TS + lane * VEC);
      } else {
#pragma unroll
        for (int m = 0; m < MPW; ++m) {
          const int i = q + m * G;
#pragma unroll
          for (int v = 0; v < VEC; ++v)
            x[m][v] = m >= mlive ? 0.f
                                 : (xl + v < M ? __ldg(data + static_cast<int64_t>(i) * ld + xl + v) : 0.f);
        }
        if (has_w) {
#pragma unroll
          for (int v = 0; v < VEC; ++v) wv[v] = xl + v < M ? __ldg(wptr + xl + v) : 0.f;
        }
      }
      if (validate) {
#pragma unroll
        for (int v = 0; v < VEC; ++v) {
          if (xl + v < M) {
            if (has_w && (!(wv[v] > 0.f) || !(wv[v] < 3.0e38f))) bad |= ERR_DOMAIN;
#pragma unroll
            for (int m = 0; m < MPW; ++m) {
              if (m < mlive) {
                const float f = x[m][v];
                if (ISO != ISOK_NONE ? !(fabsf(f) < 3.0e38f) : !(f >= 0.f && f <= 1.f)) bad |= ERR_DOMAIN;
              }
            }
          }
        }
      }
      if constexpr (ISO != ISOK_NONE) {
#pragma unroll
        for (int m = 0; m < MPW; ++m)
          if (m < mlive) {
#pragma unroll
            for (int v = 0; v < VEC; ++v) x[m][v] = iso_map<ISO>(x[m][v], iso_mu, iso_inv, iso_t, dir);
          }
      }
      if (!full) {
#pragma unroll
        for (int v = 0; v < VEC; ++v) {
          if (xl + v >= M) {
            wv[v] = 0.f;
#pragma unroll
            for (int m = 0; m < MPW; ++m) x[m][v] = 0.f;
          }
        }
      }
      // ---- exact PID-mean arithmetic, as in the streaming kernel ----
      float s[VEC] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
      for (int m = 0; m < MPW; ++m)
        if (m < mlive) {
#pragma unroll
          for (int v = 0; v < VEC; ++v) s[v] += x[m][v];
        }
      float* rb = red + static_cast<int>(kt & 1) * RB;  // this group's exchange buffer
      *reinterpret_cast<float4*>(rb + q * T + lane * VEC) = make_float4(s[0], s[1], s[2], s[3]);
      named_barrier(1 + grp, G * 32);
      if (cflag[kt & 1]) { aborted = true; break; }
      if (leader) {
        if (!issue_pending()) cflag[(kt + 1) & 1] = 1;   // stage k-1 to the tensor cores
        if (TMA) issue_next();                          // every warp has read this FP32 stage
      }
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
#pragma unroll
        for (int v = 0; v < VEC; ++v) s[v] = 0.f;
#pragma unroll
        for (int r = 0; r < G; ++r) {
          float t[VEC];
          lds_vec<VEC>(t, rb + r * T + lane * VEC);
#pragma unroll
          for (int v = 0; v < VEC; ++v) s[v] += t[v];
        }
      }
#pragma unroll
      for (int v = 0; v < VEC; ++v) s[v] *= inv_n;
      float sw[VEC] = {1.f, 1.f, 1.f, 1.f};
      if (has_w) {
#pragma unroll
        for (int m = 0; m < MPW; ++m) {
          if (m < mlive) {
#pragma unroll
            for (int v = 0; v < VEC; ++v) {
              const float t = wv[v] * x[m][v];
              accM[m] += t;
              accA[m] = fmaf(t, s[v], accA[m]);
            }
          }
        }
#pragma unroll
        for (int v = 0; v < VEC; ++v) sw[v] = sqrtf(wv[v]);
      } else {
#pragma unroll
        for (int m = 0; m < MPW; ++m) {
          if (m < mlive) {
#pragma unroll
            for (int v = 0; v < VEC; ++v) {
              accM[m] += x[m][v];
              accA[m] = fmaf(x[m][v], s[v], accA[m]);
            }
          }
        }
      }
      // ---- operands: u sqrt(w) in the swizzled K-major layout, once the slot is free ----
      if (k >= dO &&
          !mbar_wait_bounded(&opE[oslot], static_cast<uint32_t>(((k / dO) - 1) & 1), kWaitTimeoutNs))
        cflag[(kt + 1) & 1] = 1;
      // 16-bit: lane l holds cells 4l..4l+3 = 8 bytes of K-block l / 16;
      // E4M3:   lane l holds bytes 4l..4l+3 of the single K-block.
#pragma unroll
      for (int m = 0; m < MPW; ++m) {
        if (m < mlive) {
          float a[VEC];
#pragma unroll
          for (int v = 0; v < VEC; ++v) a[v] = has_w ? x[m][v] * sw[v] : x[m][v];
          unsigned char* dst = ob + lane_off + static_cast<uint32_t>(m * G * 128);
          if constexpr (PREC == 3) {
            const uint32_t lo2 = __nv_cvt_float2_to_fp8x2(make_float2(a[0] * scale, a[1] * scale),
                                                          __NV_SATFINITE, __NV_E4M3);
            const uint32_t hi2 = __nv_cvt_float2_to_fp8x2(make_float2(a[2] * scale, a[3] * scale),
                                                          __NV_SATFINITE, __NV_E4M3);
            *reinterpret_cast<uint32_t*>(dst) = lo2 | (hi2 << 16);
          } else {
            const __nv_bfloat162 h01 = __floats2bfloat162_rn(a[0], a[1]);
            const __nv_bfloat162 h23 = __floats2bfloat162_rn(a[2], a[3]);
            uint2 hv;
            hv.x = *reinterpret_cast<const uint32_t*>(&h01);
            hv.y = *reinterpret_cast<const uint32_t*>(&h23);
            *reinterpret_cast<uint2*>(dst) = hv;
            if constexpr (PREC == 2) {
              const float2 f01 = __bfloat1622float2(h01), f23 = __bfloat1622float2(h23);
              const __nv_bfloat162 l01 = __floats2bfloat162_rn(a[0] - f01.x, a[1] - f01.y);
              const __nv_bfloat162 l23 = __floats2bfloat162_rn(a[2] - f23.x, a[3] - f23.y);
              uint2 lv;
              lv.x = *reinterpret_cast<const uint32_t*>(&l01);
              lv.y = *reinterpret_cast<const uint32_t*>(&l23);
              *reinterpret_cast<uint2*>(dst + KBLK * PLANE) = lv;
            }
          }
        }
      }
      fence_proxy_async_smem();
      if (leader) {   // this stage goes to the tensor cores after the next group barrier
        pend = true;
        pend_slot = oslot;
        pend_first = st == 0;
        pend_last = st == n_st - 1;
        pend_buf = static_cast<int>(kc & 1);
        pend_kc = kc;
        pend_idesc = idesc;
      }
      if (q < kGramEpiWarps && prev_u >= 0 && st == n_st / 2) {
        if (!drain(prev_u, prev_kc)) cflag[(kt + 1) & 1] = 1;
        prev_u = -1;
      }
    }
    if (aborted) break;
    prev_u = u;
    prev_kc = kc;
#pragma unroll
    for (int m = 0; m < MPW; ++m) {
      const float ms = warp_sum(accM[m]);
      const float as = warp_sum(accA[m]);
      const int i = q + m * G;
      if (lane == 0 && i < N) {
        d.part[static_cast<size_t>(c) * 2 * N + i] = static_cast<double>(ms);
        d.part[static_cast<size_t>(c) * 2 * N + N + i] = static_cast<double>(as);
      }
    }
  }
  if (!aborted) {
    // The last stage goes to the tensor cores after one more group barrier; then the last
    // chunk's accumulator is drained.
    named_barrier(1 + grp, G * 32);
    if (cflag[kt & 1]) aborted = true;
    if (!aborted && leader && !issue_pending()) aborted = true;
    if (!aborted && q < kGramEpiWarps && prev_u >= 0 && !drain(prev_u, prev_kc)) aborted = true;
  }
  if (bad) atomicOr(p.err, bad);
  if (aborted && lane == 0) atomicOr(p.err, ERR_TIMEOUT);
  if (leader) {
    // All tensor-core work issued so far must finish before the tensor memory is released,
    // and all TMA copies in flight must land before the CTA retires.
    tc_commit(finB);
    mbar_wait_bounded(finB, 0, kWaitTimeoutNs);
    if (TMA) {
      while (k < n_issued) {
        if (!mbar_wait_bounded(&fF[k % dF], static_cast<uint32_t>((k / dF) & 1), kWaitTimeoutNs)) break;
        ++k;
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 0) tmem_dealloc(*tmem_slot, kTmemCols);
}

size_t gram_smem_bytes(int G, int prec, int dF, int dO, int stage_floats) {
  const size_t NG = kGramConvWarps / G;
  const size_t plane = static_cast<size_t>(MPW) * G * 128;
  const size_t op_stage = (prec == 2 ? 2 : 1) * (prec == 3 ? 1 : 2) * plane;
  const size_t rb = static_cast<size_t>(G) * T + T;
  return 1024 + NG * (dO * op_stage + static_cast<size_t>(dF) * stage_floats * 4 + 2 * rb * 4 +
                      (static_cast<size_t>(dF) + dO + 5) * 8 + 8) + 16;
}

template <int G, int ISO, int PREC>
static cudaError_t gram_launch_t(const GramParams& p, int grid, size_t smem, cudaStream_t s) {
  if (p.use_tma)
    gram_kernel<G, ISO, PREC, true><<<grid, kGramThreads, smem, s>>>(p);
  else
    gram_kernel<G, ISO, PREC, false><<<grid, kGramThreads, smem, s>>>(p);
  return cudaGetLastError();
}

template <int G>
static cudaError_t launch_gram_g(const GramParams& p, int prec, int iso_kind, int grid,
                                 size_t smem, cudaStream_t s) {
#define PIDK_GRAM_CASE(ISO)                                                  \
  if (iso_kind == ISO) {                                                     \
    if (prec == 1) return gram_launch_t<G, ISO, 1>(p, grid, smem, s);        \
    if (prec == 2) return gram_launch_t<G, ISO, 2>(p, grid, smem, s);        \
    if (prec == 3) return gram_launch_t<G, ISO, 3>(p, grid, smem, s);        \
  }
  PIDK_GRAM_CASE(ISOK_NONE)
  PIDK_GRAM_CASE(ISOK_NORMAL)
  PIDK_GRAM_CASE(ISOK_STEP)
#undef PIDK_GRAM_CASE
  return cudaErrorInvalidValue;
}

cudaError_t launch_gram(const GramParams& p, int G, int prec, int iso_kind, int grid, size_t smem,
                        cudaStream_t s) {
  if (G == 8) return launch_gram_g<8>(p, prec, iso_kind, grid, smem, s);
  if (G == 16) return launch_gram_g<16>(p, prec, iso_kind, grid, smem, s);
  return cudaErrorInvalidValue;
}

template <int G>
static cudaError_t gram_init_g(int max_smem) {
  cudaError_t e = cudaSuccess;
#define PIDK_GRAM_INIT(ISO, PREC)                                                            \
  if (e == cudaSuccess)                                                                      \
    e = cudaFuncSetAttribute(gram_kernel<G, ISO, PREC, true>,                                \
                             cudaFuncAttributeMaxDynamicSharedMemorySize, max_smem);         \
  if (e == cudaSuccess)                                                                      \
    e = cudaFuncSetAttribute(gram_kernel<G, ISO, PREC, false>,                               \
                             cudaFuncAttributeMaxDynamicSharedMemorySize, max_smem);
  PIDK_GRAM_INIT(ISOK_NONE, 1) PIDK_GRAM_INIT(ISOK_NONE, 2) PIDK_GRAM_INIT(ISOK_NONE, 3)
  PIDK_GRAM_INIT(ISOK_NORMAL, 1) PIDK_GRAM_INIT(ISOK_NORMAL, 2) PIDK_GRAM_INIT(ISOK_NORMAL, 3)
  PIDK_GRAM_INIT(ISOK_STEP, 1) PIDK_GRAM_INIT(ISOK_STEP, 2) PIDK_GRAM_INIT(ISOK_STEP, 3)
#undef PIDK_GRAM_INIT
  return e;
}

cudaError_t gram_kernels_init(int max_smem) {
  cudaError_t e = gram_init_g<8>(max_smem);
  return e == cudaSuccess ? gram_init_g<16>(max_smem) : e;
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
