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
//     E4M3 times the ensemble's power-of-two scale: [N][ldo] planes, cells contiguous;
//   * gram_tiled_kernel computes one tile of one cell chunk per CTA: row block r (128
//     members) against one or two column blocks c >= r (the upper block triangle; the
//     finalisation symmetrises). The tensor memory accelerator loads each 128-byte K-block
//     of the operand rows in the 128-byte swizzle layout the tensor cores read (rows past
//     N and cells past M are zero-filled by the copy), one thread issues tcgen05.mma into
//     a 128 x 256 FP32 accumulator, and four warps drain it into the chunk's partial Gram,
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
constexpr uint32_t kTiledTmemCols = 256;      // 128 x 256 FP32 accumulator

// Operand bytes per stage and plane: the row block and up to two column blocks.
__host__ __device__ constexpr uint32_t tiled_stage_bytes(int prec) { return (prec == 2 ? 2u : 1u) * 3u * kBlockBytes; }

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
    const float sc = p.op_scale ? *p.op_scale : 256.0f;
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

// One CTA per (cell chunk, row block r, column tile): the tiles of a chunk run r = 0..R-1,
// each over the column blocks r, r+1, ... in pairs, so a chunk has
// tiles_per_chunk = sum_r ceil((R - r) / 2) of them (4 for R = 3, 6 for R = 4).
template <int PREC>
__global__ void __launch_bounds__(kTiledThreads, 1) gram_tiled_kernel(const __grid_constant__ TiledParams p) {
  constexpr int PLANES = PREC == 2 ? 2 : 1;
  constexpr uint32_t FMT = PREC == 3 ? 0u : 1u;   // E4M3 : BF16
  constexpr int KB = PREC == 3 ? 128 : 64;        // cells per 128-byte K-block
  constexpr uint32_t STAGE = tiled_stage_bytes(PREC);
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  const uint32_t raw = smem_u32(smem_raw);
  unsigned char* smem = smem_raw + ((1024u - (raw & 1023u)) & 1023u);
  const int S = p.stages;
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + static_cast<size_t>(S) * STAGE);
  uint64_t* empty = full + S;
  uint64_t* accF = empty + S;
  uint64_t* finB = accF + 1;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(finB + 1);
  int* issued = reinterpret_cast<int*>(tmem_slot + 1);

  const int c = static_cast<int>(blockIdx.x) / p.tiles_per_chunk;
  int t = static_cast<int>(blockIdx.x) - c * p.tiles_per_chunk;
  int r = 0;
  for (; r < p.R - 1; ++r) {
    const int nt = (p.R - r + 1) / 2;
    if (t < nt) break;
    t -= nt;
  }
  const int cb0 = r + 2 * t;                   // first column block of the tile
  const int nb = min(2, p.R - cb0);            // column blocks: 1 or 2
  const bool a_in_b = cb0 == r;                // the row block is the first column block
  const uint32_t width = static_cast<uint32_t>(nb) * 128u;
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

  // Stage layout, per plane (hi, then lo): [row block][column block 0][column block 1].
  if (warp == 0 && lane == 0) {
    const uint32_t bytes = static_cast<uint32_t>(PLANES * ((a_in_b ? 0 : 1) + nb)) * kBlockBytes;
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
        unsigned char* base = st + pl * 3 * kBlockBytes;
        if (!a_in_b) tma_load_2d(base, map, &full[slot], x, 128 * r);
        for (int b = 0; b < nb; ++b)
          tma_load_2d(base + (1 + b) * kBlockBytes, map, &full[slot], x, 128 * (cb0 + b));
      }
    }
    *issued = kb;
  } else if (warp == 1 && lane == 0) {
    const uint32_t idesc = umma_idesc(FMT, 128, width);
    for (int kb = 0; kb < nkb; ++kb) {
      const int slot = kb % S;
      if (!mbar_wait_bounded(&full[slot], static_cast<uint32_t>((kb / S) & 1), kWaitTimeoutNs)) {
        ok = false;
        break;
      }
      tc_fence_after();
      const uint32_t st = smem_u32(smem) + static_cast<uint32_t>(slot) * STAGE;
      const uint64_t bh = umma_desc_sw128(st + kBlockBytes);
      const uint64_t ah = a_in_b ? bh : umma_desc_sw128(st);
      constexpr uint64_t lo_off = (3 * kBlockBytes) >> 4;   // hi plane -> lo plane
#pragma unroll
      for (int ks = 0; ks < 4; ++ks) {   // 4 x 32 bytes along K in the 128-byte row
        const uint64_t k16 = static_cast<uint64_t>((ks * 32) >> 4);
        const uint32_t acc = (kb == 0 && ks == 0) ? 0u : 1u;
        if constexpr (PREC == 3) {
          umma_f8(tmem, ah + k16, bh + k16, idesc, acc);
        } else {
          umma_f16(tmem, ah + k16, bh + k16, idesc, acc);
          if constexpr (PREC == 2) {
            umma_f16(tmem, ah + k16, bh + lo_off + k16, idesc, 1u);
            umma_f16(tmem, ah + lo_off + k16, bh + k16, idesc, 1u);
          }
        }
      }
      tc_commit(&empty[slot]);
    }
    tc_commit(accF);
  }
  __syncwarp();

  // Drain: warp w holds accumulator rows 32 w .. 32 w + 31 (member 128 r + 32 w + lane).
  if (!mbar_wait_bounded(accF, 0u, kWaitTimeoutNs)) ok = false;
  __syncwarp();
  tc_fence_after();
  {
    const int i = 128 * r + 32 * warp + lane;
    float* gp = p.gpart + static_cast<size_t>(c) * N * N;
    float unscale = 1.0f;
    if constexpr (PREC == 3) {
      const float sc = p.op_scale ? *p.op_scale : 256.0f;
      unscale = 1.0f / (sc * sc);
    }
    for (uint32_t j0 = 0; j0 < width; j0 += 32) {
      const int jb = 128 * cb0 + static_cast<int>(j0);   // first member of these columns
      if (jb >= N) break;                                 // the same for the whole warp
      float v[32];
      tmem_ld32(tmem + (static_cast<uint32_t>(32 * warp) << 16) + j0, v);
      const bool mirror = !(a_in_b && j0 < 128);          // off the diagonal block
      if (i < N) {
#pragma unroll
        for (int jj = 0; jj < 32; ++jj) {
          const int j = jb + jj;
          if (j < N) {
            const float g = v[jj] * unscale;
            gp[static_cast<size_t>(j) * N + i] = g;
            if (mirror) gp[static_cast<size_t>(i) * N + j] = g;
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

size_t gram_tiled_smem_bytes(int prec, int stages) {
  return 1024 + static_cast<size_t>(stages) * tiled_stage_bytes(prec) + (2 * stages + 2) * 8 + 16;
}

int gram_tiled_threads() { return kTiledThreads; }

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
