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
//     E4M3 times a power-of-two scale per member (see member_max_kernel);
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
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_fp8.h>
#include <cuda_runtime.h>

#include "device.cuh"
#include "internal.h"
#include "stream_kernel.cuh"

namespace pidk {

namespace {

// Tile shapes. Narrow (N <= 128): a group of G warps owns 8 G operand rows, a register
// tile (= one FP32 stage) is 128 cells, 4 per lane, and one 128-cell operand stage feeds
// one M = 128 MMA per K step into one of two accumulators (double-buffered per chunk).
// Wide (128 < N <= 256): 16 warps own 256 rows, 16 each; an FP32 stage is 64 cells, 2 per
// lane (the FP32 stage is then 64 KB), two FP32 stages fill one 128-cell operand stage,
// and every K step issues two M = 128 MMAs (row blocks 0-127 and 128-255 against all
// rows) into one 2 x 256-column accumulator that fills the tensor memory.
// Leader-only state of a group (TMA cursor and the operand stage waiting for its MMAs),
// kept in shared memory so that it takes no registers from the converter warps.
struct GramLeader {
  const EnsDesc* pd;   // descriptor of the ensemble being loaded
  long n_issued;       // FP32 stages issued so far
  long pend_kc;        // unit of the pending operand stage
  int iu, u_end, ist, in_st, icell0, slot;
  int e_begin, e_end, chunk, M, boxes, rows, has_w;
  int pend, pend_first, pend_last, pend_slot, pend_buf;
  uint32_t pend_idesc, pend_idesc1;
};

// NMPW: members per warp: 8 (narrow) or 16 (wide), or 6 / 12 for ensembles that fill at
// most three quarters of those tiles.
template <bool WIDE, int NMPW = (WIDE ? 16 : 8)>
struct GramShape {
  static constexpr int VEC = WIDE ? 2 : 4;             // cells per lane per register tile
  static constexpr int T = 32 * VEC;                   // cells per FP32 stage
  static constexpr int MPW = NMPW;                     // members per warp
  static constexpr int FPS = WIDE ? 2 : 1;             // FP32 stages per 128 cells
  static constexpr int MB = WIDE ? 2 : 1;              // M = 128 row blocks
  static constexpr int NBUF = WIDE ? 1 : 2;            // accumulator buffers
  static constexpr uint32_t TMEM_COLS = WIDE ? 512 : 256;
};

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
//
// EXACT = false (soft masks whose exact PID-mean sums m_i, A_i come from a streaming pass over
// the same data, e.g. the PID-mean item of the same ensemble in a batch): the converters
// skip the mean-contour arithmetic and its column-sum exchange; one group barrier per stage
// remains, after the stage's FP32 tile has been read, and the kernel writes no (m, A)
// partials.
//
// With one group of 16 converter warps and no exact sums (EXACT = false, G = 16), a 17th
// warp issues the tensor-core work: the converters mark each finished operand stage on an
// mbarrier and go on, so no converter waits at the group barrier while MMAs are being issued
// (the issue of a stage's 8 to 24 MMAs blocks while the tensor pipe's queue is full).
template <int G, bool EXACT>
constexpr bool gram_has_issuer() { return !EXACT && G == kGramConvWarps; }
template <int G, bool EXACT>
constexpr int gram_threads() { return kGramThreads + (gram_has_issuer<G, EXACT>() ? 32 : 0); }

template <int G, int ISO, int PREC, bool TMA, bool WIDE, int NMPW = (WIDE ? 16 : 8), bool EXACT = true>
__global__ void __launch_bounds__(gram_threads<G, EXACT>(), 1) gram_kernel(const __grid_constant__ GramParams p) {
  static_assert(EXACT || ISO == ISOK_NONE, "fields map in the Gram pass, with the exact sums");
  constexpr bool ISSUER = gram_has_issuer<G, EXACT>();
  using S = GramShape<WIDE, NMPW>;
  constexpr int VEC = S::VEC, T = S::T, MPW = S::MPW, FPS = S::FPS, MB = S::MB, NBUF = S::NBUF;
  // FP32 stages per operand stage: an E4M3 K-block is 128 cells (two wide FP32 stages); a
  // 16-bit K-block is 64 cells, so the wide tile's operand stage is one K-block (64 cells)
  // and the narrow tile's two (its 128-cell FP32 stage)
  constexpr int SPO = (WIDE && PREC == 3) ? 2 : 1;
  static_assert(!WIDE || G == 16, "the wide tile uses all 16 warps as one group");
  static_assert(SPO == 1 || SPO == 2, "FP32 stages per operand stage");
  static_assert(MPW <= kGramMaxMpw, "member scale slots per warp");
  constexpr int NG = kGramConvWarps / G;             // independent groups per CTA
  constexpr int ROWS = MPW * G;                      // operand rows a group writes (>= N)
  constexpr uint32_t PLANE = ROWS * 128;             // one K-block: [ROWS][128 bytes]
  constexpr int PLANES = PREC == 2 ? 2 : 1;          // hi (+ lo)
  constexpr int KBLK = (PREC == 3 || WIDE) ? 1 : 2;  // K-blocks per operand stage
  constexpr uint32_t OP_STAGE = PLANES * KBLK * PLANE;
  constexpr uint32_t FMT = PREC == 3 ? 0u : 1u;      // E4M3 : BF16
  constexpr int RB = G * T + T;                      // exchange buffer floats
  // TMEM columns per accumulator buffer: the group's rows rounded up to 64 or 128, so that
  // buffers and groups start at the same columns for 6 and 8 members per warp
  constexpr uint32_t BUFC = WIDE ? 512u : (ROWS <= 64 ? 64u : 128u);
  static_assert(WIDE || NBUF * BUFC * NG <= S::TMEM_COLS, "accumulators fit the allocation");
  extern __shared__ __align__(1024) unsigned char smem_raw[];

  const int warp = threadIdx.x >> 5;
  const int lane = threadIdx.x & 31;
  const bool issuer_warp = ISSUER && warp == kGramConvWarps;
  const int grp = issuer_warp ? 0 : warp / G;
  const int q = warp - grp * G;
  const bool leader = (q == 0) && (lane == 0);
  const int dF = p.dF, dO = p.dO, SF = p.stage_floats;
  constexpr int TS = T;   // cells per FP32 stage (the planner's TS)

  // ---- shared memory carve-up: all operand rings first (1024-byte aligned) ----
  // An M = 128 MMA reads 128 rows from a plane's base; with 64-row planes the upper rows
  // come from the bytes that follow (garbage rows of D that are never read).
  const uint32_t raw = smem_u32(smem_raw);
  unsigned char* smem = smem_raw + ((1024u - (raw & 1023u)) & 1023u);
  float* f_all = reinterpret_cast<float*>(smem + static_cast<size_t>(NG) * dO * OP_STAGE);
  float* red_all = f_all + static_cast<size_t>(NG) * dF * SF;
  uint64_t* bars_all = reinterpret_cast<uint64_t*>(red_all + NG * 2 * RB);
  int* flags_all = reinterpret_cast<int*>(bars_all + NG * (dF + 2 * dO + 5));
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(flags_all + 2 * NG);
  GramLeader* lead_all = reinterpret_cast<GramLeader*>(
      (reinterpret_cast<uintptr_t>(tmem_slot + 1) + 15) & ~static_cast<uintptr_t>(15));
  // E4M3: the per-member operand scales of each warp's members (written and read by that
  // warp alone)
  float* wsc = reinterpret_cast<float*>(lead_all + NG) + warp * kGramMaxMpw;

  unsigned char* op_ring = smem + static_cast<size_t>(grp) * dO * OP_STAGE;
  float* f_ring = f_all + static_cast<size_t>(grp) * dF * SF;
  float* red = red_all + grp * 2 * RB;
  uint64_t* bars = bars_all + grp * (dF + 2 * dO + 5);
  uint64_t* fF = bars;              // FP32 stage landed (TMA)
  uint64_t* opE = fF + dF;          // operand stage consumed (tcgen05.commit)
  uint64_t* accF = opE + dO;        // accumulator ready (tcgen05.commit)
  uint64_t* accE = accF + 2;        // accumulator drained (the group's warps 0-3)
  uint64_t* finB = accE + 2;        // all of the group's tensor-core work done
  uint64_t* opF = finB + 1;         // ISSUER: operand stage written (one arrival per warp)
  // Abort flags, one per exchange-buffer parity: a warp that gives up on a wait sets the
  // flag of the group barrier it reaches next, and every warp of the group reads that flag
  // after that barrier, so all of them leave together.
  volatile int* cflag = flags_all + 2 * grp;

  if (leader) {
    for (int s = 0; s < dF; ++s) mbar_init(&fF[s], 1);
    for (int s = 0; s < dO; ++s) mbar_init(&opE[s], 1);
    for (int b = 0; b < 2; ++b) { mbar_init(&accF[b], 1); mbar_init(&accE[b], kGramEpiWarps); }
    mbar_init(finB, 1);
    if constexpr (ISSUER)
      for (int s = 0; s < dO; ++s) mbar_init(&opF[s], static_cast<uint32_t>(G));
    cflag[0] = 0;
    cflag[1] = 0;
    fence_mbar_init();
  }
  // Operand rows past N must be finite on first use: clear every operand ring.
  for (uint32_t o = threadIdx.x * 16; o < static_cast<uint32_t>(NG) * dO * OP_STAGE; o += blockDim.x * 16)
    *reinterpret_cast<uint4*>(smem + o) = make_uint4(0, 0, 0, 0);
  fence_proxy_async_smem();
  if (warp == 0) {
    tmem_alloc(tmem_slot, S::TMEM_COLS);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem_base = *tmem_slot + static_cast<uint32_t>(grp) * NBUF * BUFC;
  // Each group takes a contiguous run of the flat unit list holding an equal share of the
  // work, so it looks an ensemble's descriptor up once per ensemble it meets.
  const int gid = blockIdx.x * NG + grp;
  const int total_groups = gridDim.x * NG;
  const int u_begin = unit_at_work(p, p.total_work * gid / total_groups);
  const int u_end = unit_at_work(p, p.total_work * (gid + 1) / total_groups);

  // ---- TMA producer cursor and pending MMA issue (leader only, in shared memory) ----
  GramLeader& L = lead_all[grp];
  auto set_unit = [&](int u) {
    if (u >= L.e_end) {
      const EnsDesc* pd = &gdesc(p, gram_find_ens(p, u));
      L.pd = pd;
      L.e_begin = pd->unit_begin;
      L.e_end = pd->unit_begin + pd->n_chunks;
      L.chunk = pd->chunk_cells;
      L.M = pd->M;
      L.boxes = pd->n_boxes;
      L.rows = pd->box_rows;
      L.has_w = pd->w != nullptr;
    }
    L.icell0 = (u - L.e_begin) * L.chunk;
    L.in_st = FPS * ((min(L.chunk, L.M - L.icell0) + 127) / 128);
  };
  auto issue_next = [&]() {
    if (L.iu >= L.u_end) return;
    const int slot = L.slot;
    L.slot = slot + 1 == dF ? 0 : slot + 1;
    float* dst = f_ring + static_cast<size_t>(slot) * SF;
    const int boxes = L.boxes, rows = L.rows;
    const bool hw = L.has_w != 0;
    const EnsDesc* pd = L.pd;
    mbar_arrive_expect_tx(&fF[slot], static_cast<uint32_t>(boxes * rows * TS + (hw ? TS : 0)) * 4u);
    const int x0 = L.icell0 + L.ist * TS;
    for (int b = 0; b < boxes; ++b)
      tma_load_2d(dst + static_cast<size_t>(b) * rows * TS, &pd->tmap, &fF[slot], x0, b * rows);
    if (hw) tma_load_1d(dst + SF - TS, &pd->tmap_w, &fF[slot], x0);
    ++L.n_issued;
    if (++L.ist == L.in_st) {
      L.ist = 0;
      if (++L.iu < L.u_end) set_unit(L.iu);
    }
  };
  if (leader) {
    L.pd = nullptr;
    L.n_issued = 0;
    L.pend_kc = 0;
    L.iu = u_begin;
    L.u_end = u_end;
    L.ist = 0;
    L.in_st = 0;
    L.icell0 = 0;
    L.slot = 0;
    L.e_begin = 0;
    L.e_end = 0;
    L.pend = 0;
    if (TMA) {
      if (L.iu < L.u_end) set_unit(L.iu);
      for (int s = 0; s < dF; ++s) issue_next();
    }
  }

  // ---- tensor-core issue of one operand stage (into accumulator buffer `buf`) ----
  auto issue_stage = [&](int slot, int buf, bool first, long pkc, uint32_t idsc, uint32_t idsc1,
                         bool last) -> bool {
    // The unit's first MMA overwrites its accumulator buffer: the unit that used that
    // buffer before must have been drained (two units back, or one with a single buffer).
    if (first && pkc >= NBUF &&
        !mbar_wait_bounded(&accE[buf], static_cast<uint32_t>((pkc / NBUF - 1) & 1), kWaitTimeoutNs))
      return false;
    tc_fence_after();
    const uint32_t dt = tmem_base + static_cast<uint32_t>(buf) * BUFC;
    // descriptor of the stage's first K-block; K steps advance its 16-byte address field,
    // row block b starts 128 rows (16 KB) into the plane
    const uint64_t d0 = umma_desc_sw128(smem_u32(op_ring) + static_cast<uint32_t>(slot) * OP_STAGE);
#pragma unroll
    for (int kb = 0; kb < KBLK; ++kb) {
#pragma unroll
      for (int ks = 0; ks < 4; ++ks) {   // 4 x 32 bytes along K in the 128-byte row
        const uint64_t hi = d0 + static_cast<uint64_t>((kb * PLANE + ks * 32) >> 4);
        const uint32_t acc = (first && kb == 0 && ks == 0) ? 0u : 1u;
        // Wide tile: row block 1 (members 128..) multiplies only the columns from 128 on;
        // its block left of the diagonal is the transpose of row block 0's right part, which
        // the drain mirrors.
#pragma unroll
        for (int mb = 0; mb < MB; ++mb) {
          const uint32_t dmb = dt + static_cast<uint32_t>(mb * 256);
          const uint64_t ha = hi + static_cast<uint64_t>((mb * 128 * 128) >> 4);
          const uint64_t hb = mb == 1 ? ha : hi;
          const uint32_t id = mb == 1 ? idsc1 : idsc;
          if constexpr (PREC == 3) {
            umma_f8(dmb, ha, hb, id, acc);
          } else {
            umma_f16(dmb, ha, hb, id, acc);
            if constexpr (PREC == 2) {
              const uint64_t lb = hb + static_cast<uint64_t>((KBLK * PLANE) >> 4);
              const uint64_t la = ha + static_cast<uint64_t>((KBLK * PLANE) >> 4);
              umma_f16(dmb, ha, lb, id, 1u);
              umma_f16(dmb, la, hb, id, 1u);
            }
          }
        }
      }
    }
    tc_commit(&opE[slot]);
    if (last) tc_commit(&accF[buf]);
    return true;
  };
  // The leader's form: the stage written last, issued after the next group barrier.
  auto issue_pending = [&]() -> bool {
    if (!L.pend) return true;
    L.pend = 0;
    return issue_stage(L.pend_slot, L.pend_buf, L.pend_first != 0, L.pend_kc, L.pend_idesc,
                       L.pend_idesc1, L.pend_last != 0);
  };

  // ---- accumulator drain of the group's kc-th unit (warps 0-3, one TMEM lane quarter each)
  // into that unit's partial Gram gp [N][N] ----
  // E4M3 operands carry the per-member scales osc[0..N) (nullptr: 256 for every member),
  // undone here exactly: G_ij = G'_ij / (s_i s_j), the inverses osc[N + i] being powers of two.
  auto drain = [&](float* gp, int N, const float* osc, long kc) -> bool {
    const int b = static_cast<int>(kc % NBUF);
    if (!mbar_wait_bounded(&accF[b], static_cast<uint32_t>((kc / NBUF) & 1), kWaitTimeoutNs))
      return false;
    tc_fence_after();
#pragma unroll
    for (int mb = 0; mb < MB; ++mb) {
      const int row = 128 * mb + 32 * q + lane;
      if (128 * mb >= N) break;
      // columns of this row block's accumulator: all N for block 0, those from 128 on for
      // block 1 (wide tile); block 0's columns past 127 also fill the mirrored entries
      const int jbase = 128 * mb;
      const int ncol = (N - jbase + 15) & ~15;
      const float ir = PREC == 3 ? (osc != nullptr ? osc[N + min(row, N - 1)] : 1.0f / 65536.0f) : 1.0f;
      for (int j0 = 0; j0 < ncol; j0 += 32) {
        float v[32];
        tmem_ld32(tmem_base + (static_cast<uint32_t>(32 * q) << 16) + b * BUFC + mb * 256 + j0, v);
        if (row < N) {
#pragma unroll
          for (int jj = 0; jj < 32; ++jj) {
            const int j = jbase + j0 + jj;
            if (j < N) {
              // E4M3: G_ij = G'_ij / (s_i s_j) with the inverse scales osc[N + .]
              const float g = PREC == 3 ? v[jj] * (osc != nullptr ? ir * osc[N + j] : ir) : v[jj];
              gp[static_cast<size_t>(j) * N + row] = g;
              if (WIDE && mb == 0 && j >= 128) gp[static_cast<size_t>(row) * N + j] = g;
            }
          }
        }
      }
    }
    tc_fence_before();
    __syncwarp();
    if (lane == 0) mbar_arrive(&accE[b]);
    return true;
  };

  // Swizzled byte offset of this lane's piece of row q; row q + m G adds m G 128 bytes
  // (G is a multiple of 8, so every owned row has the same row-in-atom q & 7).
  //   narrow, 16-bit: lane l holds cells 4l..4l+3 = 8 bytes of K-block l / 16;
  //   narrow, E4M3:   bytes 4l..4l+3 of the single K-block;
  //   wide, 16-bit:   cells 2l, 2l+1 = 4 bytes of K-block j (the FP32 stage's half);
  //   wide, E4M3:     bytes 64 j + 2l, 64 j + 2l + 1 of the single K-block.
  uint32_t lane_off0, lane_off1 = 0;
  if constexpr (WIDE) {
    lane_off0 = PREC == 3 ? sw128_offset(q, 2 * lane) : sw128_offset(q, 4 * lane);
    lane_off1 = PREC == 3 ? sw128_offset(q, 64 + 2 * lane) : PLANE + sw128_offset(q, 4 * lane);
  } else {
    lane_off0 = PREC == 3 ? sw128_offset(q, lane * 4)
                          : static_cast<uint32_t>(lane >> 4) * PLANE + sw128_offset(q, (lane & 15) * 8);
  }
  long k = 0, kt = 0, kc = 0;
  int f_slot = 0, o_slot = 0;
  uint32_t f_par = 0;
  long o_round = 0;
  float* prev_gp = nullptr;          // partial Gram of the previous unit, still to drain
  int prev_N = 0;
  const float* prev_osc = nullptr;   // its E4M3 member scales
  long prev_kc = -1;
  bool aborted = false;
  uint32_t bad = 0;
  // Descriptor fields of the current ensemble, kept in registers (the asm barriers below
  // clobber memory, so reading them through the descriptor would reload them every stage).
  const EnsDesc* dp = nullptr;
  int N = 0, M = 0, e_begin = 0, e_end = 0, e_chunk = 0;
  bool validate = false, has_w = false;
  const float* data = nullptr;
  const float* wptr = nullptr;
  int64_t ld = 0;
  uint32_t idesc = 0, idesc1 = 0;
  float iso_mu = 0.f, iso_inv = 0.f, iso_t = 0.f, dir = 1.f, pad = 0.f;
  const float* osc = nullptr;   // E4M3 member scales of the current ensemble
  int iso_md = 0;
  // ---- the issuer warp (lane 0): each finished operand stage to the tensor cores ----
  if (issuer_warp) {
    if (lane == 0) {
      bool ok = true;
      int os = 0, ie_begin = 0, ie_end = 0, ichunk = 0, iM = 0;
      long orr = 0, ikc = 0;
      uint32_t id0 = 0, id1 = 0;
      for (int u = u_begin; u < u_end && ok; ++u, ++ikc) {
        if (u >= ie_end) {
          const EnsDesc& de = gdesc(p, gram_find_ens(p, u));
          ie_begin = de.unit_begin;
          ie_end = ie_begin + de.n_chunks;
          ichunk = de.chunk_cells;
          iM = de.M;
          id0 = umma_idesc(FMT, 128, static_cast<uint32_t>((de.N + 15) & ~15));
          id1 = WIDE ? umma_idesc(FMT, 128, static_cast<uint32_t>(max(16, (de.N - 128 + 15) & ~15))) : id0;
        }
        const int cell0 = (u - ie_begin) * ichunk;
        const int n_ops = FPS * ((min(ichunk, iM - cell0) + 127) / 128) / SPO;
        for (int j = 0; j < n_ops; ++j) {
          // A converter that gives up stops arriving: this wait then ends the issue, and the
          // converters' own bounded waits on the operand slots end theirs.
          if (!mbar_wait_bounded(&opF[os], static_cast<uint32_t>(orr & 1), kWaitTimeoutNs) ||
              !issue_stage(os, static_cast<int>(ikc % NBUF), j == 0, ikc, id0, id1, j == n_ops - 1)) {
            ok = false;
            break;
          }
          if (++os == dO) { os = 0; ++orr; }
        }
      }
      if (!ok) atomicOr(p.err, ERR_TIMEOUT);
      tc_commit(finB);
      mbar_wait_bounded(finB, 0, kWaitTimeoutNs);
    }
    __syncwarp();
  }
  const int u_conv_end = issuer_warp ? u_begin : u_end;
  for (int u = u_begin; u < u_conv_end && !aborted; ++u, ++kc) {
    if (u >= e_end) {
      dp = &gdesc(p, gram_find_ens(p, u));
      N = dp->N;
      M = dp->M;
      e_begin = dp->unit_begin;
      e_end = e_begin + dp->n_chunks;
      e_chunk = dp->chunk_cells;
      validate = dp->validate != 0;
      data = dp->data;
      wptr = dp->w;
      ld = dp->ld;
      has_w = wptr != nullptr;
      idesc = umma_idesc(FMT, 128, static_cast<uint32_t>((N + 15) & ~15));
      idesc1 = WIDE ? umma_idesc(FMT, 128, static_cast<uint32_t>(max(16, (N - 128 + 15) & ~15))) : idesc;
      iso_mu = dp->iso_mu;
      iso_inv = dp->iso_inv;
      iso_t = dp->iso_t;
      iso_md = dp->iso_mode;
      dir = iso_pad_sign(iso_md);
      // Rows q, q+G, ... below N are this warp's members; rows past N read a padding value
      // that every isovalue kind maps to exactly 0 (and become zero operand rows, which only
      // feed accumulator rows that are never read).
      pad = ISO == ISOK_NONE ? 0.f
                             : (ISO == ISOK_NORMAL ? copysignf(__int_as_float(0x7f800000), iso_inv)
                                                   : dir * __int_as_float(0x7f800000));
      if constexpr (PREC == 3) {
        osc = dp->op_scale;
        if (lane < MPW) {
          const int i = q + lane * G;
          wsc[lane] = osc == nullptr ? 256.0f : (i < N ? osc[i] : 1.0f);
        }
        __syncwarp();
      }
    }
    const EnsDesc& d = *dp;
    const int c = u - e_begin;
    const int cell0 = c * e_chunk;
    const int n_st = FPS * ((min(e_chunk, M - cell0) + 127) / 128);   // FP32 stages
    float accM[EXACT ? MPW : 1], accA[EXACT ? MPW : 1];
#pragma unroll
    for (int m = 0; m < (EXACT ? MPW : 1); ++m) { accM[m] = 0.f; accA[m] = 0.f; }

    for (int st = 0; st < n_st; ++st, ++k, ++kt) {
      // Ring positions, kept incrementally (no 64-bit division per stage):
      // fslot = k % dF, f_par = (k / dF) & 1; operand stage ko = k / SPO, jh = k % SPO,
      // oslot = ko % dO, o_round = ko / dO.
      const int fslot = f_slot;
      const uint32_t fpar = f_par;
      const int jh = SPO == 1 ? 0 : static_cast<int>(k & (SPO - 1));
      const int oslot = o_slot;
      const long oround = o_round;
      if (++f_slot == dF) { f_slot = 0; f_par ^= 1u; }
      if (jh == SPO - 1 && ++o_slot == dO) { o_slot = 0; ++o_round; }
      if (TMA && !mbar_wait_bounded(&fF[fslot], fpar, kWaitTimeoutNs))
        cflag[kt & 1] = 1;
      const float* sb = f_ring + static_cast<size_t>(fslot) * SF;
      unsigned char* ob = op_ring + static_cast<size_t>(oslot) * OP_STAGE;

      const int x0 = cell0 + st * TS;
      const int xl = x0 + lane * VEC;
      const bool full = x0 + T <= M;
      float x[MPW][VEC];
      float wv[VEC];
#pragma unroll
      for (int v = 0; v < VEC; ++v) wv[v] = 1.f;
      if constexpr (TMA) {
#pragma unroll
        for (int m = 0; m < MPW; ++m) {
          if (q + m * G < N) {
            lds_vec<VEC>(x[m], sb + static_cast<size_t>(q + m * G) * TS + lane * VEC);
          } else {
#pragma unroll
            for (int v = 0; v < VEC; ++v) x[m][v] = pad;
          }
        }
        if (has_w) lds_vec<VEC>(wv, sb + SF - TS + lane * VEC);
      } else {
#pragma unroll
        for (int m = 0; m < MPW; ++m) {
          const int i = q + m * G;
#pragma unroll
          for (int v = 0; v < VEC; ++v)
            x[m][v] = i >= N ? pad
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
              if (q + m * G < N) {
                const float f = x[m][v];
                if (ISO != ISOK_NONE ? !(fabsf(f) < 3.0e38f) : !(f >= 0.f && f <= 1.f)) bad |= ERR_DOMAIN;
              }
            }
          }
        }
      }
      if constexpr (ISO != ISOK_NONE) iso_map_tile<ISO>(x, iso_mu, iso_inv, iso_t, dir, iso_md);
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
      if constexpr (EXACT) {
        // ---- exact PID-mean arithmetic, as in the streaming kernel ----
        float s[VEC];
        {
          float2 s2[VEC / 2];
#pragma unroll
          for (int v = 0; v < VEC / 2; ++v) s2[v] = f2(0.f);
#pragma unroll
          for (int m = 0; m < MPW; ++m)
#pragma unroll
            for (int v = 0; v < VEC / 2; ++v)
              s2[v] = f2_add(s2[v], make_float2(x[m][2 * v], x[m][2 * v + 1]));
#pragma unroll
          for (int v = 0; v < VEC / 2; ++v) { s[2 * v] = s2[v].x; s[2 * v + 1] = s2[v].y; }
        }
        float* rb = red + static_cast<int>(kt & 1) * RB;  // this group's exchange buffer
        sts_vec<VEC>(rb + q * T + lane * VEC, s);
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
          sum_partials<VEC, G>(s, rb + lane * VEC, T);
        }
        // uniform branches on the weights and on padding rows, as in the streaming kernel
        if (has_w) {
#pragma unroll
          for (int m = 0; m < MPW; ++m) {
            if (q + m * G < N) {
#pragma unroll
              for (int v = 0; v < VEC; ++v) {
                const float t = wv[v] * x[m][v];
                accM[m] += t;
                accA[m] = fmaf(t, s[v], accA[m]);
              }
            }
          }
        } else {
#pragma unroll
          for (int m = 0; m < MPW; ++m) {
            if (q + m * G < N) {
#pragma unroll
              for (int v = 0; v < VEC; ++v) {
                accM[m] += x[m][v];
                accA[m] = fmaf(x[m][v], s[v], accA[m]);
              }
            }
          }
        }
      } else {
        // every warp has read this FP32 stage, and written its operands of the previous one
        named_barrier(1 + grp, G * 32);
        if (cflag[kt & 1]) { aborted = true; break; }
        if (leader) {
          if (!ISSUER && !issue_pending()) cflag[(kt + 1) & 1] = 1;   // stage k-1 to the tensor cores
          if (TMA) issue_next();
        }
      }
      float sw[VEC];
#pragma unroll
      for (int v = 0; v < VEC; ++v) sw[v] = 1.f;
      if (has_w) {
#pragma unroll
        for (int v = 0; v < VEC; ++v) sw[v] = sqrtf(wv[v]);
      }
      // ---- operands: u sqrt(w) in the swizzled K-major layout, once the slot is free ----
      if (jh == 0 && oround >= 1 &&
          !mbar_wait_bounded(&opE[oslot], static_cast<uint32_t>((oround - 1) & 1), kWaitTimeoutNs))
        cflag[(kt + 1) & 1] = 1;
      const uint32_t loff = (SPO == 1 || jh == 0) ? lane_off0 : lane_off1;
#pragma unroll
      for (int m = 0; m < MPW; ++m) {
        uint32_t h[VEC / 2], l[VEC / 2];   // packed pairs of this lane's VEC operands
#pragma unroll
        for (int v = 0; v < VEC; v += 2) {
          float2 t = make_float2(x[m][v], x[m][v + 1]);
          if (has_w) t = f2_mul(t, make_float2(sw[v], sw[v + 1]));
          if constexpr (PREC == 3) {
            t = f2_mul(t, f2(wsc[m]));
            h[v / 2] = __nv_cvt_float2_to_fp8x2(t, __NV_SATFINITE, __NV_E4M3);
          } else {
            const __nv_bfloat162 hb = __floats2bfloat162_rn(t.x, t.y);
            h[v / 2] = *reinterpret_cast<const uint32_t*>(&hb);
            if constexpr (PREC == 2) {
              const float2 f = __bfloat1622float2(hb);
              const __nv_bfloat162 lb = __floats2bfloat162_rn(t.x - f.x, t.y - f.y);
              l[v / 2] = *reinterpret_cast<const uint32_t*>(&lb);
            }
          }
        }
        unsigned char* dst = ob + loff + static_cast<uint32_t>(m * G * 128);
        if constexpr (PREC == 3) {
          if constexpr (VEC == 4)
            *reinterpret_cast<uint32_t*>(dst) = (h[0] & 0xffffu) | (h[1] << 16);
          else
            *reinterpret_cast<uint16_t*>(dst) = static_cast<uint16_t>(h[0]);
        } else if constexpr (VEC == 4) {
          *reinterpret_cast<uint2*>(dst) = make_uint2(h[0], h[1]);
          if constexpr (PREC == 2) *reinterpret_cast<uint2*>(dst + KBLK * PLANE) = make_uint2(l[0], l[1]);
        } else {
          *reinterpret_cast<uint32_t*>(dst) = h[0];
          if constexpr (PREC == 2) *reinterpret_cast<uint32_t*>(dst + KBLK * PLANE) = l[0];
        }
      }
      fence_proxy_async_smem();
      if constexpr (ISSUER) {   // a full operand stage: every warp marks its rows written
        if (jh == SPO - 1) {
          __syncwarp();
          if (lane == 0) mbar_arrive(&opF[oslot]);
        }
      } else if (leader && jh == SPO - 1) {   // a full operand stage: to the tensor cores after the next barrier
        L.pend = 1;
        L.pend_slot = oslot;
        L.pend_first = st < SPO;
        L.pend_last = st == n_st - 1;
        L.pend_buf = static_cast<int>(kc % NBUF);
        L.pend_kc = kc;
        L.pend_idesc = idesc;
        L.pend_idesc1 = idesc1;
      }
      // Double-buffered accumulators are drained halfway through the next chunk, when the
      // last products have long landed; a single buffer must be drained before the next
      // chunk's first MMA, which is issued after the barrier of its second operand stage.
      if (q < kGramEpiWarps && prev_gp != nullptr && st == (NBUF == 2 ? n_st / 2 : 0)) {
        if (!drain(prev_gp, prev_N, prev_osc, prev_kc)) cflag[(kt + 1) & 1] = 1;
        prev_gp = nullptr;
      }
    }
    if (aborted) break;
    prev_gp = d.gpart + static_cast<size_t>(c) * N * N;
    prev_N = N;
    prev_osc = osc;
    prev_kc = kc;
    if constexpr (EXACT) {
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
  }
  if (!aborted) {
    // The last stage goes to the tensor cores after one more group barrier (the issuer warp
    // takes it without); then the last chunk's accumulator is drained.
    if constexpr (!ISSUER) {
      named_barrier(1 + grp, G * 32);
      if (cflag[kt & 1]) aborted = true;
      if (!aborted && leader && !issue_pending()) aborted = true;
    }
    if (!aborted && q < kGramEpiWarps && prev_gp != nullptr &&
        !drain(prev_gp, prev_N, prev_osc, prev_kc))
      aborted = true;
  }
  if (bad) atomicOr(p.err, bad);
  if (aborted && lane == 0) atomicOr(p.err, ERR_TIMEOUT);
  if (leader) {
    // All tensor-core work issued so far must finish before the tensor memory is released
    // (the issuer warp waits for its own), and all TMA copies in flight must land before
    // the CTA retires.
    if constexpr (!ISSUER) {
      tc_commit(finB);
      mbar_wait_bounded(finB, 0, kWaitTimeoutNs);
    }
    if (TMA) {
      while (k < L.n_issued) {
        if (!mbar_wait_bounded(&fF[k % dF], static_cast<uint32_t>((k / dF) & 1), kWaitTimeoutNs)) break;
        ++k;
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 0) tmem_dealloc(*tmem_slot, S::TMEM_COLS);
}

// Host-side launch and opt-in helpers of one tile (group size, members per warp, wide or
// narrow): gram_kernel.cu instantiates the narrow tiles with 8 members per warp,
// gram_narrow6.cu those with 6, gram_wide.cu the wide tile with 16 and gram_wide12.cu
// with 12.
template <int G, int ISO, int PREC, int NMPW, bool WIDE>
cudaError_t gram_tile_launch_t(const GramParams& p, int grid, size_t smem, cudaStream_t s) {
  if constexpr (ISO == ISOK_NONE) {
    if (!p.exact) {   // soft masks with the exact sums from a streaming pass
      constexpr int threads = gram_threads<G, false>();
      if (p.use_tma)
        gram_kernel<G, ISO, PREC, true, WIDE, NMPW, false><<<grid, threads, smem, s>>>(p);
      else
        gram_kernel<G, ISO, PREC, false, WIDE, NMPW, false><<<grid, threads, smem, s>>>(p);
      return cudaGetLastError();
    }
  }
  if (p.use_tma)
    gram_kernel<G, ISO, PREC, true, WIDE, NMPW><<<grid, kGramThreads, smem, s>>>(p);
  else
    gram_kernel<G, ISO, PREC, false, WIDE, NMPW><<<grid, kGramThreads, smem, s>>>(p);
  return cudaGetLastError();
}

template <int G, int NMPW, bool WIDE = false>
cudaError_t gram_tile_launch(const GramParams& p, int prec, int iso_kind, int grid,
                             size_t smem, cudaStream_t s) {
#define PIDK_GRAM_CASE(ISO)                                                             \
  if (iso_kind == ISO) {                                                                \
    if (prec == 1) return gram_tile_launch_t<G, ISO, 1, NMPW, WIDE>(p, grid, smem, s);  \
    if (prec == 2) return gram_tile_launch_t<G, ISO, 2, NMPW, WIDE>(p, grid, smem, s);  \
    if (prec == 3) return gram_tile_launch_t<G, ISO, 3, NMPW, WIDE>(p, grid, smem, s);  \
  }
  PIDK_GRAM_CASE(ISOK_NONE)
  PIDK_GRAM_CASE(ISOK_NORMAL)
  PIDK_GRAM_CASE(ISOK_STEP)
#undef PIDK_GRAM_CASE
  return cudaErrorInvalidValue;
}

template <int G, int NMPW, bool WIDE = false>
cudaError_t gram_tile_init(int max_smem) {
  cudaError_t e = cudaSuccess;
#define PIDK_GRAM_INIT(ISO, PREC)                                                            \
  if (e == cudaSuccess)                                                                      \
    e = cudaFuncSetAttribute(gram_kernel<G, ISO, PREC, true, WIDE, NMPW>,                    \
                             cudaFuncAttributeMaxDynamicSharedMemorySize, max_smem);         \
  if (e == cudaSuccess)                                                                      \
    e = cudaFuncSetAttribute(gram_kernel<G, ISO, PREC, false, WIDE, NMPW>,                   \
                             cudaFuncAttributeMaxDynamicSharedMemorySize, max_smem);
  PIDK_GRAM_INIT(ISOK_NONE, 1) PIDK_GRAM_INIT(ISOK_NONE, 2) PIDK_GRAM_INIT(ISOK_NONE, 3)
  PIDK_GRAM_INIT(ISOK_NORMAL, 1) PIDK_GRAM_INIT(ISOK_NORMAL, 2) PIDK_GRAM_INIT(ISOK_NORMAL, 3)
  PIDK_GRAM_INIT(ISOK_STEP, 1) PIDK_GRAM_INIT(ISOK_STEP, 2) PIDK_GRAM_INIT(ISOK_STEP, 3)
#undef PIDK_GRAM_INIT
#define PIDK_GRAM_INIT_LEAN(PREC)                                                                \
  if (e == cudaSuccess)                                                                          \
    e = cudaFuncSetAttribute(gram_kernel<G, ISOK_NONE, PREC, true, WIDE, NMPW, false>,           \
                             cudaFuncAttributeMaxDynamicSharedMemorySize, max_smem);             \
  if (e == cudaSuccess)                                                                          \
    e = cudaFuncSetAttribute(gram_kernel<G, ISOK_NONE, PREC, false, WIDE, NMPW, false>,          \
                             cudaFuncAttributeMaxDynamicSharedMemorySize, max_smem);
  PIDK_GRAM_INIT_LEAN(1) PIDK_GRAM_INIT_LEAN(2) PIDK_GRAM_INIT_LEAN(3)
#undef PIDK_GRAM_INIT_LEAN
  return e;
}

}  // namespace pidk
