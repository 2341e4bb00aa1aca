// Full PID on the tensor cores for 256 < N <= 512 members: the Gram G = U' U'^T of the
// weighted soft masks U' = U diag(sqrt w) (Eq. 9 and the weighted sums of Eq. 14), tiled
// over 128-row blocks.
//
// One CTA of the fused Gram kernel cannot hold this Gram in its 512 tensor-memory columns
// (the upper block triangle of a 512-member Gram is 10 blocks of 128 x 128 FP32), and
// converting every operand row in each CTA that needs it would repeat the isovalue map
// several times per cell. So the work is split in two kernels:
//
//   * gram_operand_kernel maps each input element once (isovalue map of Sec. 3.5, times
//     sqrt w) and stores the operand rows in HBM as BF16, as a BF16 hi + lo pair, or as
//     E4M3 times the member's power-of-two scale: [N][ldo] planes, cells contiguous;
//   * gram_tiled_kernel computes one tile of one cell chunk per CTA, from a table of the
//     upper block triangle's products (row block r of 128 members against column blocks
//     c >= r; the finalisation symmetrises). BF16 and E4M3 tiles take whole block rows,
//     the two shortest rows after the first paired, so every tile but one carries the
//     same work and each block is loaded by few CTAs of its chunk; split BF16, with two
//     planes per block, does so for three row blocks and otherwise takes at most two
//     column blocks per tile. The tensor memory
//     accelerator loads each 128-byte K-block of the operand rows in the 128-byte swizzle
//     layout the tensor cores read (rows past N and cells past M are zero-filled by the
//     copy), one thread issues tcgen05.mma into a 128 x 512 FP32 accumulator (at most 256
//     columns per instruction), and four warps drain it into the chunk's partial Gram,
//     writing both G_ij and its mirror G_ji for the off-diagonal blocks.
//
// The exact PID-mean sums (m_i, A_i) that calibrate the Gram come from the streaming
// kernel's pass over the same ensemble. Every wait is bounded; on a time-out the kernel
// raises the error word, lets its copies and tensor-core work drain (bounded) and frees its
// tensor memory before returning.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_fp8.h>
#include <cuda_runtime.h>

#include "device.cuh"
#include "internal.h"
#include "stream_kernel.cuh"

namespace pidk {

namespace {

constexpr int kOperandThreads = 256;          // 4 cells per thread: 1024 cells per CTA row
constexpr int kTiledThreads = 128;            // 4 warps: one per tensor-memory lane quarter
constexpr uint32_t kBlockBytes = 128 * 128;   // one 128-row block of a 128-byte K-block
constexpr uint32_t kTiledTmemCols = 512;      // 128 x 512 FP32 accumulator (all of it)

}  // namespace

// ISO: the isovalue map family (none, normal, step or piecewise), applied with the
// streaming kernel's own tile map, so the staged masks are bitwise those of its pass.
template <int PREC, int ISO>
__global__ void __launch_bounds__(kOperandThreads) gram_operand_kernel(const __grid_constant__ OperandParams p) {
  const int i = blockIdx.y;
  const int64_t x0 = (static_cast<int64_t>(blockIdx.x) * kOperandThreads + threadIdx.x) * 4;
  if (x0 >= p.M) return;
  const float* row = p.F + static_cast<int64_t>(i) * p.ld;
  const bool full = x0 + 4 <= p.M;
  float x[1][4], w[4] = {1.f, 1.f, 1.f, 1.f};
  if (p.vec_ok && full) {
    const float4 a = __ldcs(reinterpret_cast<const float4*>(row + x0));
    x[0][0] = a.x; x[0][1] = a.y; x[0][2] = a.z; x[0][3] = a.w;
    if (p.w) {
      const float4 b = __ldg(reinterpret_cast<const float4*>(p.w + x0));
      w[0] = b.x; w[1] = b.y; w[2] = b.z; w[3] = b.w;
    }
  } else {
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      x[0][v] = x0 + v < p.M ? __ldcs(row + x0 + v) : 0.f;
      if (p.w) w[v] = x0 + v < p.M ? __ldg(p.w + x0 + v) : 0.f;
    }
  }
  if constexpr (ISO != ISOK_NONE)
    iso_map_tile<ISO>(x, p.iso_mu, p.iso_inv, p.iso_t, iso_pad_sign(p.iso_mode), p.iso_mode);
  float t[4];
#pragma unroll
  for (int v = 0; v < 4; v += 2) {
    float2 u = make_float2(x[0][v], x[0][v + 1]);
    if (p.w) u = f2_mul(u, make_float2(sqrtf(w[v]), sqrtf(w[v + 1])));
    t[v] = u.x;
    t[v + 1] = u.y;
  }
  if (!full) {
#pragma unroll
    for (int v = 0; v < 4; ++v)
      if (x0 + v >= p.M) t[v] = 0.f;
  }
  // ldo is a multiple of 64 elements and x0 of 4: the 4 operands of a thread never cross
  // the end of the row's storage.
  if constexpr (PREC == 3) {
    const float sc = p.op_scale ? p.op_scale[i] : 256.0f;   // member i's power-of-two scale
    const uint32_t lo2 = __nv_cvt_float2_to_fp8x2(f2_mul(make_float2(t[0], t[1]), f2(sc)), __NV_SATFINITE, __NV_E4M3);
    const uint32_t hi2 = __nv_cvt_float2_to_fp8x2(f2_mul(make_float2(t[2], t[3]), f2(sc)), __NV_SATFINITE, __NV_E4M3);
    uint8_t* dst = static_cast<uint8_t*>(p.hi) + static_cast<int64_t>(i) * p.ldo + x0;
    *reinterpret_cast<uint32_t*>(dst) = (lo2 & 0xffffu) | (hi2 << 16);
  } else {
    uint32_t h[2], l[2];
#pragma unroll
    for (int v = 0; v < 2; ++v) {
      const __nv_bfloat162 hb = __floats2bfloat162_rn(t[2 * v], t[2 * v + 1]);
      h[v] = *reinterpret_cast<const uint32_t*>(&hb);
      if constexpr (PREC == 2) {
        const float2 g = __bfloat1622float2(hb);
        const __nv_bfloat162 lb = __floats2bfloat162_rn(t[2 * v] - g.x, t[2 * v + 1] - g.y);
        l[v] = *reinterpret_cast<const uint32_t*>(&lb);
      }
    }
    const int64_t off = static_cast<int64_t>(i) * p.ldo + x0;
    *reinterpret_cast<uint2*>(static_cast<uint16_t*>(p.hi) + off) = make_uint2(h[0], h[1]);
    if constexpr (PREC == 2)
      *reinterpret_cast<uint2*>(static_cast<uint16_t*>(p.lo) + off) = make_uint2(l[0], l[1]);
  }
}

// One CTA per (cell chunk, tile): the tile table (gram_tiles) lists, for every tile of a
// chunk, the 128-row blocks to load and the row-block x column-blocks products to form.
template <int PREC>
__global__ void __launch_bounds__(kTiledThreads, 1) gram_tiled_kernel(const __grid_constant__ TiledParams p) {
  constexpr int PLANES = PREC == 2 ? 2 : 1;
  constexpr uint32_t FMT = PREC == 3 ? 0u : 1u;   // E4M3 : BF16
  constexpr int KB = PREC == 3 ? 128 : 64;        // cells per 128-byte K-block
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  const uint32_t raw = smem_u32(smem_raw);
  unsigned char* smem = smem_raw + ((1024u - (raw & 1023u)) & 1023u);
  const int S = p.stages;
  const uint32_t PLANE = static_cast<uint32_t>(p.slots) * kBlockBytes;   // one plane of a stage
  const uint32_t STAGE = PLANES * PLANE;
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + static_cast<size_t>(S) * STAGE);
  uint64_t* empty = full + S;
  uint64_t* accF = empty + S;
  uint64_t* finB = accF + 1;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(finB + 1);
  int* issued = reinterpret_cast<int*>(tmem_slot + 1);

  const int c = static_cast<int>(blockIdx.x) / p.tiles_per_chunk;
  const TileDesc& td = p.tiles[static_cast<int>(blockIdx.x) - c * p.tiles_per_chunk];
  const int lb0 = td.lb0, nlb = td.nlb, xa = td.xa, nseg = td.nseg;
  // stage slot of row block b: the loaded range first, then the extra row block
  auto slot_of = [&](int b) { return (b >= lb0 && b < lb0 + nlb) ? b - lb0 : nlb; };
  const int N = p.N;
  const int cell0 = c * p.chunk_cells;
  const int cells = min(p.chunk_cells, p.M - cell0);
  const int nkb = (cells + KB - 1) / KB;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

  if (threadIdx.x == 0) {
    for (int s = 0; s < S; ++s) { mbar_init(&full[s], 1); mbar_init(&empty[s], 1); }
    mbar_init(accF, 1);
    mbar_init(finB, 1);
    *issued = 0;
    fence_mbar_init();
  }
  if (warp == 0) {
    tmem_alloc(tmem_slot, kTiledTmemCols);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  bool ok = true;

  // Stage layout, per plane (hi, then lo): [slot 0] .. [slot nlb - 1] [extra row block].
  if (warp == 0 && lane == 0) {
    const uint32_t bytes = static_cast<uint32_t>(PLANES * (nlb + (xa >= 0 ? 1 : 0))) * kBlockBytes;
    int kb = 0;
    for (; kb < nkb; ++kb) {
      const int slot = kb % S;
      if (kb >= S && !mbar_wait_bounded(&empty[slot], static_cast<uint32_t>((kb / S - 1) & 1), kWaitTimeoutNs)) {
        ok = false;
        break;
      }
      unsigned char* st = smem + static_cast<size_t>(slot) * STAGE;
      mbar_arrive_expect_tx(&full[slot], bytes);
      const int x = cell0 + kb * KB;
#pragma unroll
      for (int pl = 0; pl < PLANES; ++pl) {
        const CUtensorMap* map = pl ? &p.op_lo : &p.op_hi;
        unsigned char* base = st + pl * PLANE;
        for (int b = 0; b < nlb; ++b)
          tma_load_2d(base + b * kBlockBytes, map, &full[slot], x, 128 * (lb0 + b));
        if (xa >= 0) tma_load_2d(base + nlb * kBlockBytes, map, &full[slot], x, 128 * xa);
      }
    }
    *issued = kb;
  } else if (warp == 1 && lane == 0) {
    const uint32_t id256 = umma_idesc(FMT, 128, 256), id128 = umma_idesc(FMT, 128, 128);
    const uint64_t lo_off = PLANE >> 4;   // hi plane -> lo plane (descriptor units)
    for (int kb = 0; kb < nkb; ++kb) {
      const int slot = kb % S;
      if (!mbar_wait_bounded(&full[slot], static_cast<uint32_t>((kb / S) & 1), kWaitTimeoutNs)) {
        ok = false;
        break;
      }
      tc_fence_after();
      const uint32_t st = smem_u32(smem) + static_cast<uint32_t>(slot) * STAGE;
      for (int sg = 0; sg < nseg; ++sg) {
        const uint64_t ah = umma_desc_sw128(st + static_cast<uint32_t>(slot_of(td.ra[sg])) * kBlockBytes);
        const int width = 128 * td.nb[sg];
        // one MMA covers at most 256 columns: B rows n0 .. n0 + 255 start n0 x 128 bytes in
        for (int n0 = 0; n0 < width; n0 += 256) {
          const uint64_t bh = umma_desc_sw128(st + static_cast<uint32_t>(slot_of(td.cb[sg])) * kBlockBytes +
                                              static_cast<uint32_t>(n0) * 128u);
          const uint32_t idesc = width - n0 >= 256 ? id256 : id128;
          const uint32_t d = tmem + static_cast<uint32_t>(td.col[sg] + n0);
#pragma unroll
          for (int ks = 0; ks < 4; ++ks) {   // 4 x 32 bytes along K in the 128-byte row
            const uint64_t k16 = static_cast<uint64_t>((ks * 32) >> 4);
            const uint32_t acc = (kb == 0 && ks == 0) ? 0u : 1u;
            if constexpr (PREC == 3) {
              umma_f8(d, ah + k16, bh + k16, idesc, acc);
            } else {
              umma_f16(d, ah + k16, bh + k16, idesc, acc);
              if constexpr (PREC == 2) {
                umma_f16(d, ah + k16, bh + lo_off + k16, idesc, 1u);
                umma_f16(d, ah + lo_off + k16, bh + k16, idesc, 1u);
              }
            }
          }
        }
      }
      tc_commit(&empty[slot]);
    }
    tc_commit(accF);
  }
  __syncwarp();

  // Drain: warp w holds accumulator rows 32 w .. 32 w + 31 of every segment (member
  // 128 ra + 32 w + lane).
  if (!mbar_wait_bounded(accF, 0u, kWaitTimeoutNs)) ok = false;
  __syncwarp();
  tc_fence_after();
  {
    float* gp = p.gpart + static_cast<size_t>(c) * N * N;
    // E4M3: G_ij = G'_ij / (s_i s_j) with the members' power-of-two scales (inverses at
    // op_scale[N + i]); the product of two inverses is exact
    const float* inv = PREC == 3 && p.op_scale ? p.op_scale + N : nullptr;
    for (int sg = 0; sg < nseg; ++sg) {
      const int ra = td.ra[sg], cb = td.cb[sg], width = 128 * td.nb[sg];
      const int i = 128 * ra + 32 * warp + lane;
      for (int j0 = 0; j0 < width; j0 += 32) {
        const int jb = 128 * cb + j0;                 // first member of these columns
        if (jb >= N) break;                           // the same for the whole warp
        float v[32];
        tmem_ld32(tmem + (static_cast<uint32_t>(32 * warp) << 16) + static_cast<uint32_t>(td.col[sg] + j0), v);
        const bool mirror = jb / 128 != ra;           // off the diagonal block
        if (i < N) {
          const float ir = PREC != 3 ? 1.0f : (inv ? inv[i] : 1.0f / 65536.0f);
#pragma unroll
          for (int jj = 0; jj < 32; ++jj) {
            const int j = jb + jj;
            if (j < N) {
              const float g = PREC != 3 ? v[jj] : v[jj] * (inv ? ir * inv[j] : ir);
              gp[static_cast<size_t>(j) * N + i] = g;
              if (mirror) gp[static_cast<size_t>(i) * N + j] = g;
            }
          }
        }
      }
    }
  }
  if (!ok) atomicOr(p.err, ERR_TIMEOUT);
  // All tensor-core work must finish before the tensor memory is released, and all copies
  // in flight must land before the CTA retires.
  if (warp == 1 && lane == 0) {
    tc_commit(finB);
    mbar_wait_bounded(finB, 0u, kWaitTimeoutNs);
  }
  if (warp == 0 && lane == 0) {
    const int n = *issued;
    for (int kb = n > S ? n - S : 0; kb < n; ++kb)
      if (!mbar_wait_bounded(&full[kb % S], static_cast<uint32_t>((kb / S) & 1), kWaitTimeoutNs)) break;
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 0) tmem_dealloc(tmem, kTiledTmemCols);
}

int gram_tiles(int R, bool wide, TileDesc* out) {
  int n = 0;
  auto add = [&](int lb0, int nlb, int xa, int nseg, const int* ra, const int* cb, const int* nb) {
    TileDesc t{};
    t.lb0 = static_cast<int8_t>(lb0);
    t.nlb = static_cast<int8_t>(nlb);
    t.xa = static_cast<int8_t>(xa);
    t.nseg = static_cast<int8_t>(nseg);
    int col = 0;
    for (int s = 0; s < nseg; ++s) {
      t.ra[s] = static_cast<int8_t>(ra[s]);
      t.cb[s] = static_cast<int8_t>(cb[s]);
      t.nb[s] = static_cast<int8_t>(nb[s]);
      t.col[s] = static_cast<int16_t>(col);
      col += 128 * nb[s];
    }
    out[n++] = t;
  };
  if (wide && (R == 3 || R == 4)) {
    // whole rows of the upper block triangle, the two shortest rows after the first paired:
    // R = 3: {0: 0-2}, {1: 1-2, 2: 2}; R = 4: {0: 0-3}, {1: 1-3, 3: 3}, {2: 2-3}
    {
      const int ra[1] = {0}, cb[1] = {0}, nb[1] = {R};
      add(0, R, -1, 1, ra, cb, nb);
    }
    {
      const int ra[2] = {1, R - 1}, cb[2] = {1, R - 1}, nb[2] = {R - 1, 1};
      add(1, R - 1, -1, 2, ra, cb, nb);
    }
    if (R == 4) {
      const int ra[1] = {2}, cb[1] = {2}, nb[1] = {2};
      add(2, 2, -1, 1, ra, cb, nb);
    }
    return n;
  }
  // row block r against the column blocks r, r+1, ... in pairs; the row block is loaded
  // apart unless it is the pair's first block
  for (int r = 0; r < R; ++r) {
    for (int c0 = r; c0 < R; c0 += 2) {
      const int ra[1] = {r}, cb[1] = {c0}, nb[1] = {c0 + 1 < R ? 2 : 1};
      add(c0, nb[0], c0 == r ? -1 : r, 1, ra, cb, nb);
    }
  }
  return n;
}

size_t gram_tiled_smem_bytes(int prec, int slots, int stages) {
  return 1024 + static_cast<size_t>(stages) * (prec == 2 ? 2u : 1u) * slots * kBlockBytes +
         (2 * stages + 2) * 8 + 16;
}

template <int PREC>
static void operand_launch(const OperandParams& p, dim3 grid, cudaStream_t s) {
  const int kind = iso_kind(p.iso_mode);
  if (kind == ISOK_NONE) gram_operand_kernel<PREC, ISOK_NONE><<<grid, kOperandThreads, 0, s>>>(p);
  else if (kind == ISOK_NORMAL) gram_operand_kernel<PREC, ISOK_NORMAL><<<grid, kOperandThreads, 0, s>>>(p);
  else gram_operand_kernel<PREC, ISOK_STEP><<<grid, kOperandThreads, 0, s>>>(p);
}

cudaError_t launch_gram_operands(const OperandParams& p, int prec, cudaStream_t s) {
  const dim3 grid(static_cast<unsigned>((p.M + 4 * kOperandThreads - 1) / (4 * kOperandThreads)),
                  static_cast<unsigned>(p.N));
  if (prec == 1) operand_launch<1>(p, grid, s);
  else if (prec == 2) operand_launch<2>(p, grid, s);
  else if (prec == 3) operand_launch<3>(p, grid, s);
  else return cudaErrorInvalidValue;
  return cudaGetLastError();
}

cudaError_t launch_gram_tiled(const TiledParams& p, int prec, int grid, size_t smem, cudaStream_t s) {
  if (prec == 1) gram_tiled_kernel<1><<<grid, kTiledThreads, smem, s>>>(p);
  else if (prec == 2) gram_tiled_kernel<2><<<grid, kTiledThreads, smem, s>>>(p);
  else if (prec == 3) gram_tiled_kernel<3><<<grid, kTiledThreads, smem, s>>>(p);
  else return cudaErrorInvalidValue;
  return cudaGetLastError();
}

cudaError_t gram_tiled_init(int max_smem) {
  cudaError_t e = cudaFuncSetAttribute(gram_tiled_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, max_smem);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(gram_tiled_kernel<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, max_smem);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(gram_tiled_kernel<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, max_smem);
  return e;
}

}  // namespace pidk
