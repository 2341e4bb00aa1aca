// Host-side dispatch of the streaming pass (kernel in stream_kernel.cuh, instantiated per
// tile class in stream_c*.cu) and the two small kernels of the library:
//   * finalize_kernel — fixed-order FP64 reduction of the per-chunk partials, then the
//                      inclusion fractions, depths and ranks of Eq. 10 / Eq. 16.
//   * iso_kernel      — the isovalue map alone (pid_soft_masks, Sec. 3.5).
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "device.cuh"
#include "internal.h"

namespace pidk {

// ---------------------------------------------------------------------------------------
// Streaming pass: dispatch to the per-class instantiations (stream_c*.cu)
// ---------------------------------------------------------------------------------------

#define PIDK_CLASS(V, M, G)                                                                  \
  cudaError_t launch_stream_c##V##_##M##_##G(const StreamParams&, int, bool, int, size_t,  \
                                             cudaStream_t);                                \
  cudaError_t init_stream_c##V##_##M##_##G(int);
PIDK_CLASS(4, 8, 1)
PIDK_CLASS(4, 8, 2)
PIDK_CLASS(4, 6, 4)
PIDK_CLASS(4, 8, 4)
PIDK_CLASS(4, 6, 8)
PIDK_CLASS(4, 8, 8)
PIDK_CLASS(4, 6, 16)
PIDK_CLASS(4, 8, 16)
PIDK_CLASS(2, 12, 16)
PIDK_CLASS(2, 13, 16)
PIDK_CLASS(2, 16, 16)
PIDK_CLASS(1, 20, 16)
PIDK_CLASS(1, 24, 16)
PIDK_CLASS(1, 28, 16)
PIDK_CLASS(1, 32, 16)
#undef PIDK_CLASS

cudaError_t launch_stream(const StreamParams& p, int vec, int mpw, int G, int iso_kind, bool coef,
                          int grid, size_t smem, cudaStream_t s) {
#define PIDK_CASE(V, M, GG)                                                                   \
  if (vec == V && mpw == M && G == GG)                                                       \
    return launch_stream_c##V##_##M##_##GG(p, iso_kind, coef, grid, smem, s);
  PIDK_CASE(4, 8, 1)
  PIDK_CASE(4, 8, 2)
  PIDK_CASE(4, 6, 4)
  PIDK_CASE(4, 8, 4)
  PIDK_CASE(4, 6, 8)
  PIDK_CASE(4, 8, 8)
  PIDK_CASE(4, 6, 16)
  PIDK_CASE(4, 8, 16)
  PIDK_CASE(2, 12, 16)
  PIDK_CASE(2, 13, 16)
  PIDK_CASE(2, 16, 16)
  PIDK_CASE(1, 20, 16)
  PIDK_CASE(1, 24, 16)
  PIDK_CASE(1, 28, 16)
  PIDK_CASE(1, 32, 16)
#undef PIDK_CASE
  return cudaErrorInvalidValue;
}

cudaError_t finalize_kernel_init();

// Opt every streaming instantiation in to the largest dynamic shared memory once per
// device (before any launch, so that launches can be captured into graphs).
cudaError_t stream_kernels_init(int max_smem) {
  cudaError_t e = finalize_kernel_init();
  if (e == cudaSuccess) e = init_stream_c4_8_1(max_smem);
  if (e == cudaSuccess) e = init_stream_c4_8_2(max_smem);
  if (e == cudaSuccess) e = init_stream_c4_6_4(max_smem);
  if (e == cudaSuccess) e = init_stream_c4_8_4(max_smem);
  if (e == cudaSuccess) e = init_stream_c4_6_8(max_smem);
  if (e == cudaSuccess) e = init_stream_c4_8_8(max_smem);
  if (e == cudaSuccess) e = init_stream_c4_6_16(max_smem);
  if (e == cudaSuccess) e = init_stream_c4_8_16(max_smem);
  if (e == cudaSuccess) e = init_stream_c2_12_16(max_smem);
  if (e == cudaSuccess) e = init_stream_c2_13_16(max_smem);
  if (e == cudaSuccess) e = init_stream_c2_16_16(max_smem);
  if (e == cudaSuccess) e = init_stream_c1_20_16(max_smem);
  if (e == cudaSuccess) e = init_stream_c1_24_16(max_smem);
  if (e == cudaSuccess) e = init_stream_c1_28_16(max_smem);
  if (e == cudaSuccess) e = init_stream_c1_32_16(max_smem);
  return e;
}

size_t stream_smem_bytes(int vec, int G, int depth, int stage_floats) {
  const int T = 32 * vec;
  const int n_groups = kStreamWarps / G;
  return static_cast<size_t>(n_groups) * depth * stage_floats * 4 +
         static_cast<size_t>(n_groups) * 2 * (G * T + T) * 4 +
         static_cast<size_t>(n_groups) * depth * 8 + static_cast<size_t>(n_groups) * 8 + 64 +
         static_cast<size_t>(n_groups) * kStreamProducerBytes + 16;
}

// ---------------------------------------------------------------------------------------
// Finalisation
// ---------------------------------------------------------------------------------------

constexpr int kFinThreads = 1024;

__device__ __forceinline__ const FinDesc& fin_desc(const FinParams& p, int e) {
  return p.descs ? p.descs[e] : p.one;
}

// Column block `cb` of a [rows][cols] array: 32 columns (lanes) x 32 warps over rows;
// the 32 warp sums are then combined in warp order. Deterministic.
template <typename Src>
__device__ void reduce_columns(const Src* src, int rows, int cols, int cb, double* dst,
                               double (*scratch)[33]) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int col = cb * 32 + lane;
  double acc = 0.0;
  if (col < cols) {
#pragma unroll 4
    for (int r = warp; r < rows; r += 32) acc += static_cast<double>(src[static_cast<size_t>(r) * cols + col]);
  }
  scratch[warp][lane] = acc;
  __syncthreads();
  if (warp == 0) {
    double t = 0.0;
    for (int w = 0; w < 32; ++w) t += scratch[w][lane];
    if (col < cols) dst[col] = t;
  }
  __syncthreads();
}

// acc + comp carries the running sum; comp holds the low-order part lost by acc (Kahan).
__device__ __forceinline__ void kahan_add(float& acc, float& comp, float v) {
  const float y = v - comp;
  const float t = acc + y;
  comp = (t - acc) - y;
  acc = t;
}

// Row r of an [N][N] FP32 matrix, dotted with the shared vector v (v == nullptr: summed),
// by one warp: lane l takes the columns l, l + 32, ... in order, then a fixed xor tree. A
// lane loads 8 columns (a 256-column block) before it adds them, so a block costs one
// memory round trip instead of one per column. SHARED: the row is in this CTA's shared
// memory; else it was written by this kernel's grid and is read through L2.
template <bool SHARED = false>
__device__ __forceinline__ float row_dot_warp(const float* row, const float* v, int N, int ln) {
  float acc = 0.f;
  for (int b = 0; b < N; b += 256) {
    float x[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      const int j = b + ln + 32 * k;
      x[k] = j < N ? (SHARED ? row[j] : __ldcg(row + j)) : 0.f;
    }
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      const int j = b + ln + 32 * k;
      if (j < N) acc = v ? fmaf(x[k], v[j], acc) : acc + x[k];
    }
  }
  return warp_sum(acc);
}

// The calibrated Gram C0 of an ensemble of up to 128 members stays in the finishing CTA's
// shared memory: the Sinkhorn sweeps then read it at shared-memory latency instead of one
// L2 round trip per sweep (the cost that dominated small ensembles).
constexpr int kFinC0Floats = 128 * 128;

__global__ void __launch_bounds__(kFinThreads, 1) finalize_kernel(const __grid_constant__ FinParams p) {
  extern __shared__ float fin_c0[];
  const FinDesc& d = fin_desc(p, blockIdx.y);
  if (static_cast<int>(blockIdx.x) >= d.slices) return;
  __shared__ double scratch[32][33];
  __shared__ unsigned long long skey[1024];   // order keys of the depths (ranks)
  __shared__ double sred[1024];
  __shared__ float sd[kGramTiledMaxN], sdn[kGramTiledMaxN];   // Gram calibration scales
  __shared__ float sdm[kGramTiledMaxN];                       // d_j / m_j (0 for zero mass)
  __shared__ int is_last;

  const int N = d.N;
  const int nb_stream = (2 * N + 31) / 32;
  const int nb_gram = d.kind == FIN_GRAM ? fin_gram_items(N) : 0;
  const int nb = nb_stream + nb_gram;
  const int dst_off = d.kind == FIN_LIN2 ? 2 * N : 0;

  // Phase 1: this CTA's share of the work items: 32-column blocks of the (m, A) partials
  // (all warps on one block, rows split across warps), then 1024-column items of the Gram
  // partials (each warp sums one 32-column block over every chunk, in chunk order).
  for (int cb = blockIdx.x; cb < nb; cb += d.slices) {
    if (cb < nb_stream) {
      reduce_columns<double>(d.part, d.n_chunks, 2 * N, cb, d.sums + dst_off, scratch);
    } else {
      const int col = (cb - nb_stream) * 1024 + static_cast<int>(threadIdx.x);
      const int NN = N * N;
      if (col < NN) {
        // Compensated (Kahan) FP32 sum in chunk order: close to an FP64 sum, at the FP32
        // rate (GB300 issues FP64 adds at a small fraction of it, and this sum has
        // n_gchunks * N^2 terms per ensemble). 8 chunks' values are loaded before they are
        // added, so the loop is not one memory round trip per chunk.
        float acc = 0.f, comp = 0.f;
        const float* src = d.gpart + col;
        int r = 0;
        for (; r + 8 <= d.n_gchunks; r += 8) {
          float v[8];
#pragma unroll
          for (int k = 0; k < 8; ++k) v[k] = __ldcs(src + static_cast<size_t>(r + k) * NN);
#pragma unroll
          for (int k = 0; k < 8; ++k) kahan_add(acc, comp, v[k]);
        }
        for (; r < d.n_gchunks; ++r) kahan_add(acc, comp, __ldcs(src + static_cast<size_t>(r) * NN));
        reinterpret_cast<float*>(d.sums + 4 * N)[col] = acc;
      }
    }
  }
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) is_last = (atomicAdd(d.ticket, 1u) == static_cast<unsigned>(d.slices - 1));
  __syncthreads();
  if (!is_last) return;
  __threadfence();

  // Phase 2 for ensembles larger than the CTA (member-blocked path, no Gram): the same
  // per-member outputs over a strided loop; ranks come from a separate kernel.
  if (N > kFinThreads) {
    const double* S = d.sums;
    const bool wm = d.kind == FIN_WMEAN;
    double acc = 0.0;
    for (int j = threadIdx.x; j < N; j += kFinThreads)
      acc += wm ? __ldcg(S + j) * static_cast<double>(__ldg(d.coef + j)) : __ldcg(S + j);
    sred[threadIdx.x] = acc;
    __syncthreads();
    for (int o = kFinThreads / 2; o > 0; o >>= 1) {
      if (static_cast<int>(threadIdx.x) < o) sred[threadIdx.x] += sred[threadIdx.x + o];
      __syncthreads();
    }
    const double mbar = wm ? sred[0] : sred[0] / N;
    for (int j = threadIdx.x; j < N; j += kFinThreads) {
      const double m = __ldcg(S + j), A = wm ? __ldcg(S + N + j) : __ldcg(S + N + j) / N;
      const double in_in = m > 0.0 ? A / m : 0.0;
      const double mean_out = mbar > 0.0 ? A / mbar : 0.0;
      if (d.mass) d.mass[j] = m;
      if (d.mean_depth) d.mean_depth[j] = fmin(in_in, mean_out);
      if (d.kind == FIN_LIN1) {
        d.coef[j] = m > 0.0 ? static_cast<float>(1.0 / (static_cast<double>(N) * m)) : 0.0f;
        continue;
      }
      const double in_out = d.kind == FIN_LIN2 ? __ldcg(S + 3 * N + j) : mean_out;
      if (d.depth) d.depth[j] = fmin(in_in, in_out);
      if (d.in_in) d.in_in[j] = in_in;
      if (d.in_out) d.in_out[j] = in_out;
    }
    __syncthreads();
    if (threadIdx.x == 0) *d.ticket = 0u;
    return;
  }

  // Phase 2 (last CTA of this ensemble): per-member outputs and ranks.
  const int i = threadIdx.x;
  const double* S = d.sums;
  double m = 0.0, A = 0.0;
  // The kernels sum A_i against the column sum N u_bar: the 1/N of Eq. 15 is applied here.
  // Against a weighted mean contour sum_j c_j u_j (sum_j c_j = 1) A_i needs no scaling and
  // the mean contour's mass is sum_j c_j m_j.
  const bool wm = d.kind == FIN_WMEAN;
  if (i < N) { m = __ldcg(S + i); A = wm ? __ldcg(S + N + i) : __ldcg(S + N + i) / N; }
  // m_bar = (1/N) sum_i m_i, a fixed-order tree over the thread index.
  sred[i] = (i < N) ? (wm ? m * static_cast<double>(__ldg(d.coef + i)) : m) : 0.0;
  __syncthreads();
  for (int o = kFinThreads / 2; o > 0; o >>= 1) {
    if (i < o) sred[i] += sred[i + o];
    __syncthreads();
  }
  const double mbar = wm ? sred[0] : sred[0] / N;
  __syncthreads();

  double depth = 0.0, in_in = 0.0, in_out = 0.0, err = 0.0;
  if (i < N) {
    const double in_in_exact = m > 0.0 ? A / m : 0.0;        // u_i subset_p u_bar (Eq. 17)
    const double mean_out = mbar > 0.0 ? A / mbar : 0.0;     // u_bar subset_p u_i (Eq. 16)
    const double mean_depth = fmin(in_in_exact, mean_out);
    if (d.mass) d.mass[i] = m;
    if (d.mean_depth) d.mean_depth[i] = mean_depth;
    if (d.kind == FIN_MEAN || wm) {
      in_in = in_in_exact; in_out = mean_out;
    } else if (d.kind == FIN_LIN1) {
      d.coef[i] = m > 0.0 ? static_cast<float>(1.0 / (static_cast<double>(N) * m)) : 0.0f;
    } else if (d.kind == FIN_LIN2) {
      in_in = in_in_exact;
      in_out = __ldcg(S + 3 * N + i);
    } else {  // FIN_GRAM: see the calibration below
      in_in = in_in_exact;
    }
    depth = fmin(in_in, in_out);
  }
  if (d.kind == FIN_LIN1) {
    __syncthreads();
    if (threadIdx.x == 0) *d.ticket = 0u;
    return;
  }
  if (d.kind == FIN_GRAM) {
    // The tensor-core Gram G' (G'[i + j N] ~ G_ij = sum_x w u_i u_j) carries each member's
    // rounding bias in its row and column. Its row sums are known exactly from the same pass:
    // sum_j G_ij = N A_i (the recall identity, Eq. 17). Calibrate by a symmetric diagonal
    // scaling C_ij = d_i d_j (G'_ij + G'_ji) / 2 with d_i sum_j C... = N A_i (symmetric
    // Sinkhorn iteration, FP64), then P_ij = C_ij / m_i, IN_in = mean_j P_ij (= A_i / m_i),
    // IN_out = mean_j P_ji. err_est reports the uncalibrated |mean_j G'_ij / m_i - A_i / m_i|.
    // GB300's FP64 rate is a small fraction of its FP32 rate, so the O(N^2) calibration
    // runs in FP32 (the scales converge to FP32 precision, ~1e-7, far inside the Gram
    // bound); only the per-member scalars stay in FP64.
    const float* Cg = reinterpret_cast<const float*>(d.sums + 4 * N);   // G' (phase 1)
    const bool c0s = N * N <= kFinC0Floats;                             // C0 in shared memory
    float* C0 = c0s ? fin_c0 : reinterpret_cast<float*>(d.sums + 4 * N) + N * N;   // (G' + G'^T) / 2
    const int wi = threadIdx.x >> 5, ln = threadIdx.x & 31;
    // Every row loop below runs one warp per row with the lanes on contiguous columns.
    // Raw sums: row r of the stored array is G'_{., r}, which equals row r of G' up to
    // the rounding of the tensor-core sums.
    for (int r = wi; r < N; r += kFinThreads / 32) {
      const float acc = row_dot_warp(Cg + r * N, nullptr, N, ln);
      if (ln == 0) sdn[r] = acc;
    }
    // C0 = (G' + G'^T) / 2, one warp per row, each lane's 8 columns of a 256-column block
    // loaded together
    for (int r = wi; r < N; r += kFinThreads / 32) {
      for (int c0 = 0; c0 < N; c0 += 256) {
        float a[8], b[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) {
          const int c = c0 + ln + 32 * k;
          a[k] = c < N ? __ldcg(Cg + r + c * N) : 0.f;
          b[k] = c < N ? __ldcg(Cg + r * N + c) : 0.f;
        }
#pragma unroll
        for (int k = 0; k < 8; ++k) {
          const int c = c0 + ln + 32 * k;
          if (c < N) C0[r * N + c] = 0.5f * (a[k] + b[k]);
        }
      }
    }
    __syncthreads();
    if (i < N) {
      const double raw = sdn[i];
      err = m > 0.0 ? fabs(raw / (m * N) - A / m) : 0.0;
      sd[i] = (A > 0.0 && raw > 0.0) ? 1.0f : 0.0f;
      sdm[i] = static_cast<float>(N * A);   // row-sum targets N A_i, kept here until IN_out
    }
    __syncthreads();
    // Symmetric Sinkhorn: d_r <- sqrt(d_r N A_r / sum_j C0_rj d_j), until no scale moves by
    // more than 2^-22 relative (at most 24 sweeps).
    for (int it = 0; it < 24; ++it) {
      for (int r = wi; r < N; r += kFinThreads / 32) {
        const float acc = c0s ? row_dot_warp<true>(C0 + r * N, sd, N, ln) : row_dot_warp(C0 + r * N, sd, N, ln);
        if (ln == 0) sdn[r] = (sd[r] > 0.f && acc > 0.f) ? sqrtf(sd[r] * sdm[r] / acc) : 0.f;
      }
      __syncthreads();
      bool moved = false;
      if (i < N) {
        moved = fabsf(sdn[i] - sd[i]) > 2.4e-7f * sd[i];
        sd[i] = sdn[i];
      }
      if (!__syncthreads_or(moved)) break;
    }
    // IN_out(i) = (1/N) sum_j C_ji / m_j = (d_i / N) sum_j (d_j / m_j) C0_ij (C0 symmetric).
    if (i < N) sdm[i] = m > 0.0 ? static_cast<float>(sd[i] / m) : 0.f;
    __syncthreads();
    for (int r = wi; r < N; r += kFinThreads / 32) {
      const float acc = c0s ? row_dot_warp<true>(C0 + r * N, sdm, N, ln) : row_dot_warp(C0 + r * N, sdm, N, ln);
      if (ln == 0) sdn[r] = sd[r] * acc;
    }
    __syncthreads();
    if (i < N) {
      in_out = static_cast<double>(sdn[i]) / N;
      depth = fmin(in_in, in_out);
    }
  }
  skey[i] = order_key((i < N) ? depth : 0.0);
  sred[i] = err;
  __syncthreads();
  if (i < N) {
    if (d.depth) d.depth[i] = depth;
    if (d.in_in) d.in_in[i] = in_in;
    if (d.in_out) d.in_out[i] = in_out;
    if (d.rank) {
      const unsigned long long ki = skey[i];
      int r = 0;
      for (int j = 0; j < N; ++j) {
        const unsigned long long kj = skey[j];
        r += (kj > ki) || (kj == ki && j < i);
      }
      d.rank[i] = r;
    }
  }
  if (d.kind == FIN_GRAM) {
    for (int o = kFinThreads / 2; o > 0; o >>= 1) {
      if (i < o) sred[i] = fmax(sred[i], sred[i + o]);
      __syncthreads();
    }
    if (i == 0 && d.err_est) d.err_est[0] = sred[0];
    if (d.P) {
      const float* C0 = N * N <= kFinC0Floats ? fin_c0 : reinterpret_cast<const float*>(S + 4 * N) + N * N;
      // P[r][cc] = C_{r,cc} / m_r: one warp per row, one FP64 division per row
      const int wi = threadIdx.x >> 5, ln = threadIdx.x & 31;
      for (int r = wi; r < N; r += kFinThreads / 32) {
        const double mr = __ldcg(S + r);
        const double inv = mr > 0.0 ? 1.0 / mr : 0.0;
        for (int c0 = 0; c0 < N; c0 += 256) {
          float x[8];
#pragma unroll
          for (int k = 0; k < 8; ++k) {
            const int cc = c0 + ln + 32 * k;
            x[k] = cc < N ? C0[r * N + cc] : 0.f;   // written by this CTA (shared or global)
          }
#pragma unroll
          for (int k = 0; k < 8; ++k) {
            const int cc = c0 + ln + 32 * k;
            if (cc < N) d.P[static_cast<size_t>(r) * N + cc] = static_cast<double>(sd[r] * sd[cc] * x[k]) * inv;
          }
        }
      }
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) *d.ticket = 0u;
}

cudaError_t finalize_kernel_init() {
  return cudaFuncSetAttribute(finalize_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              static_cast<int>(kFinC0Floats * sizeof(float)));
}

cudaError_t launch_finalize(const FinParams& p, int grid_x, int grid_y, cudaStream_t s) {
  finalize_kernel<<<dim3(grid_x, grid_y), kFinThreads, kFinC0Floats * sizeof(float), s>>>(p);
  return cudaGetLastError();
}

// Coefficients of a weighted mean contour (Sec. 4.1): c_j = r_j / sum_k r_k from member
// weights r_j >= 0, summed in FP64 in a fixed order (strided per thread, then a tree).
// Weights that are negative, not finite, or all zero set the domain bit and give c = 0.
__global__ void __launch_bounds__(kFinThreads, 1) member_coef_kernel(const double* r, int64_t N,
                                                                     float* coef, uint32_t* err) {
  __shared__ double sred[kFinThreads];
  double acc = 0.0;
  int bad = 0;
  for (int64_t j = threadIdx.x; j < N; j += kFinThreads) {
    const double v = r[j];
    if (v >= 0.0 && v <= 1.7976931348623157e308) acc += v; else bad = 1;
  }
  sred[threadIdx.x] = acc;
  __syncthreads();
  for (int o = kFinThreads / 2; o > 0; o >>= 1) {
    if (static_cast<int>(threadIdx.x) < o) sred[threadIdx.x] += sred[threadIdx.x + o];
    __syncthreads();
  }
  const double R = sred[0];
  bad = __syncthreads_or(bad || !(R > 0.0 && R <= 1.7976931348623157e308));
  if (bad && threadIdx.x == 0) atomicOr(err, ERR_DOMAIN);
  for (int64_t j = threadIdx.x; j < N; j += kFinThreads)
    coef[j] = bad ? 0.0f : static_cast<float>(r[j] / R);
}

cudaError_t launch_member_coef(const double* r, int64_t N, float* coef, uint32_t* err,
                               cudaStream_t s) {
  member_coef_kernel<<<1, kFinThreads, 0, s>>>(r, N, coef, err);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------------------
// Isovalue map alone (pid_soft_masks)
// ---------------------------------------------------------------------------------------

// Stores VEC soft masks, as float32 or rounded to nearest-even bfloat16.
template <bool BF16>
__device__ __forceinline__ void iso_store4(void* base, int64_t off, const float4& u) {
  if constexpr (BF16) {
    const __nv_bfloat162 a = __floats2bfloat162_rn(u.x, u.y), b = __floats2bfloat162_rn(u.z, u.w);
    uint2 v;
    v.x = *reinterpret_cast<const uint32_t*>(&a);
    v.y = *reinterpret_cast<const uint32_t*>(&b);
    *reinterpret_cast<uint2*>(static_cast<__nv_bfloat16*>(base) + off) = v;
  } else {
    *reinterpret_cast<float4*>(static_cast<float*>(base) + off) = u;
  }
}

template <bool BF16>
__device__ __forceinline__ void iso_store1(void* base, int64_t off, float u) {
  if constexpr (BF16) static_cast<__nv_bfloat16*>(base)[off] = __float2bfloat16_rn(u);
  else static_cast<float*>(base)[off] = u;
}

template <bool BF16>
__global__ void __launch_bounds__(256) iso_kernel(const __grid_constant__ IsoParams p) {
  // vector path: 16-byte aligned input rows, output rows aligned to 4 elements
  const bool vec = ((p.ld & 3) == 0) && ((p.ld_out & 3) == 0) &&
                   ((reinterpret_cast<uintptr_t>(p.F) & 15) == 0) &&
                   ((reinterpret_cast<uintptr_t>(p.U) & (BF16 ? 7 : 15)) == 0);
  const int64_t per_row = vec ? (p.M + 3) / 4 : p.M;
  const int64_t total = per_row * p.N;
  const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
  for (int64_t t = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; t < total; t += stride) {
    const int64_t i = t / per_row;
    const int64_t j = t - i * per_row;
    const float* src = p.F + i * p.ld;
    const int64_t row = i * p.ld_out;
    if (vec) {
      const int64_t x = j * 4;
      if (x + 4 <= p.M) {
        const float4 f = __ldg(reinterpret_cast<const float4*>(src + x));
        float4 u;
        u.x = iso_value(f.x, p.iso_mode, p.iso_mu, p.iso_inv, p.iso_t);
        u.y = iso_value(f.y, p.iso_mode, p.iso_mu, p.iso_inv, p.iso_t);
        u.z = iso_value(f.z, p.iso_mode, p.iso_mu, p.iso_inv, p.iso_t);
        u.w = iso_value(f.w, p.iso_mode, p.iso_mu, p.iso_inv, p.iso_t);
        iso_store4<BF16>(p.U, row + x, u);
      } else {
        for (int64_t xx = x; xx < p.M; ++xx)
          iso_store1<BF16>(p.U, row + xx,
                           iso_value(__ldg(src + xx), p.iso_mode, p.iso_mu, p.iso_inv, p.iso_t));
      }
    } else {
      iso_store1<BF16>(p.U, row + j,
                       iso_value(__ldg(src + j), p.iso_mode, p.iso_mu, p.iso_inv, p.iso_t));
    }
  }
}

cudaError_t launch_iso(const IsoParams& p, cudaStream_t s) {
  int dev = 0, sms = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int64_t work = p.N * ((p.M + 3) / 4);
  int64_t blocks = (work + 255) / 256;
  const int64_t cap = static_cast<int64_t>(sms) * 8;
  if (blocks > cap) blocks = cap;
  if (blocks < 1) blocks = 1;
  if (p.out_bf16)
    iso_kernel<true><<<static_cast<int>(blocks), 256, 0, s>>>(p);
  else
    iso_kernel<false><<<static_cast<int>(blocks), 256, 0, s>>>(p);
  return cudaGetLastError();
}

}  // namespace pidk
