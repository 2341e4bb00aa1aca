// Streaming kernels of the PID library (sm_103a):
//   * stream_kernel  — one pass over an ensemble [N][M]: per cell tile the column sum
//                      s(x) = sum_j c_j u_j(x) is formed on chip, then every member's
//                      m_i = sum_x w u_i and A_i = sum_x w u_i s are accumulated.
//                      With c_j = 1/N this is PID-mean (Eq. 15-16): s = u_bar and
//                      IN_in = A_i / m_i, IN_out = A_i / m_bar. With c_j = 1/(N m_j) it is
//                      the second pass of the exact O(NM) full PID: A_i = IN_out(i).
//                      The isovalue map of Sec. 3.5 is optionally applied to each element
//                      as it is read. Tiles arrive by TMA into a per-group shared-memory ring.
//   * finalize_kernel — fixed-order FP64 reduction of the per-chunk partials, then the
//                      inclusion fractions, depths and ranks of Eq. 10 / Eq. 16.
//   * iso_kernel      — the isovalue map alone (pid_soft_masks).
#include <cuda.h>
#include <cuda_runtime.h>

#include "device.cuh"
#include "internal.h"

namespace pidk {

// ---------------------------------------------------------------------------------------
// Streaming pass
// ---------------------------------------------------------------------------------------

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

template <int VEC>
struct VecT;
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

// Layout of the dynamic shared memory (per CTA):
//   ring  [n_groups][depth][stage_floats]   TMA destinations [rows][SUB*T]; the last SUB*T
//                                           floats of a stage hold the cell measures
//   red   [n_groups][2][G*T + T]            partial column sums and their total, double-buffered
//   bars  [n_groups][depth]                 "stage full" mbarriers
//   flags [n_groups]                        abort flags (bounded wait ran out)
template <int VEC, int MPW, bool TMA, bool COEF>
__global__ void __launch_bounds__(kStreamThreads, 1)
stream_kernel(const __grid_constant__ StreamParams p) {
  static_assert(MPW <= 32, "member coefficients are broadcast from one lane each");
  constexpr int T = 32 * VEC;
  extern __shared__ __align__(1024) unsigned char smem[];

  const int warp = threadIdx.x >> 5;
  const int lane = threadIdx.x & 31;
  const int G = p.G;
  const int n_groups = kStreamWarps / G;
  const int grp = warp / G;
  const int q = warp - grp * G;
  const int depth = p.depth;
  const int SF = p.stage_floats;
  const int SUB = p.sub;        // register tiles of T cells per TMA stage
  const int TS = SUB * T;       // cells per stage (TMA box width)

  float* ring = reinterpret_cast<float*>(smem);
  float* red = ring + static_cast<size_t>(n_groups) * depth * SF;
  const int RB = G * T + T;  // floats per exchange buffer
  uint64_t* bars = reinterpret_cast<uint64_t*>(red + n_groups * 2 * RB);
  volatile int* flags = reinterpret_cast<volatile int*>(bars + n_groups * depth);

  float* my_ring = ring + static_cast<size_t>(grp) * depth * SF;
  float* my_red = red + grp * 2 * RB;
  uint64_t* my_bars = bars + grp * depth;
  const bool leader = (q == 0) && (lane == 0);

  if (TMA && leader) {
    for (int s = 0; s < depth; ++s) mbar_init(&my_bars[s], 1);
    fence_mbar_init();
  }
  if (threadIdx.x < n_groups) flags[threadIdx.x] = 0;
  __syncthreads();

  const int gid = blockIdx.x * n_groups + grp;
  const int total_groups = gridDim.x * n_groups;

  // ---- producer cursor (leader lane of the group only) ----
  int iu = gid, ist = 0, ie = 0, icell0 = 0, in_st = 0;
  long n_issued = 0;
  auto set_unit = [&](int u) {
    ie = stream_find_ens(p, u);
    const EnsDesc& d = stream_desc(p, ie);
    const int c = u - d.unit_begin;
    icell0 = c * d.chunk_cells;
    const int cells = min(d.chunk_cells, d.M - icell0);
    in_st = (cells + TS - 1) / TS;
  };
  auto issue_next = [&]() {
    if (iu >= p.total_units) return;
    const EnsDesc& d = stream_desc(p, ie);
    const int slot = static_cast<int>(n_issued % depth);
    float* dst = my_ring + static_cast<size_t>(slot) * SF;
    const uint32_t bytes =
        static_cast<uint32_t>(d.n_boxes * d.box_rows * TS + (d.w ? TS : 0)) * 4u;
    mbar_arrive_expect_tx(&my_bars[slot], bytes);
    const int x0 = icell0 + ist * TS;
    for (int b = 0; b < d.n_boxes; ++b)
      tma_load_2d(dst + static_cast<size_t>(b) * d.box_rows * TS, &d.tmap, &my_bars[slot], x0,
                  b * d.box_rows);
    if (d.w) tma_load_1d(dst + SF - TS, &d.tmap_w, &my_bars[slot], x0);
    ++n_issued;
    if (++ist == in_st) {
      ist = 0;
      iu += total_groups;
      if (iu < p.total_units) set_unit(iu);
    }
  };
  if (TMA && leader) {
    if (iu < p.total_units) set_unit(iu);
    for (int s = 0; s < depth; ++s) issue_next();
  }

  // ---- consumers: every warp of the group ----
  long k_cons = 0;
  long k_sub = 0;   // register tiles processed (parity of the exchange buffer)
  bool aborted = false;
  uint32_t bad = 0;

  for (int u = gid; u < p.total_units && !aborted; u += total_groups) {
    const int e = stream_find_ens(p, u);
    const EnsDesc& d = stream_desc(p, e);
    const int N = d.N;
    const int c = u - d.unit_begin;
    const int cell0 = c * d.chunk_cells;
    const int cells = min(d.chunk_cells, d.M - cell0);
    const int n_st = (cells + TS - 1) / TS;
    const int iso = d.iso_mode;
    const float iso_mu = d.iso_mu, iso_inv = d.iso_inv, iso_t = d.iso_t;
    const bool has_w = d.w != nullptr;

    // Column-sum coefficients: lane k holds c_j of this warp's k-th member (pass 2), or
    // every member weighs 1/N, applied once per cell (pass 1).
    float my_cf = 0.f;
    if constexpr (COEF) {
      const int i = q + lane * G;
      if (lane < MPW && i < N) my_cf = d.coef[i];
    }
    const float inv_n = 1.0f / static_cast<float>(N);
    float accM[MPW], accA[MPW];
#pragma unroll
    for (int k = 0; k < MPW; ++k) { accM[k] = 0.f; accA[k] = 0.f; }

    for (int st = 0; st < n_st && !aborted; ++st, ++k_cons) {
      const int slot = static_cast<int>(k_cons % depth);
      const uint32_t par = static_cast<uint32_t>((k_cons / depth) & 1);
      const float* sb = my_ring + static_cast<size_t>(slot) * SF;
      if constexpr (TMA) {
        if (!mbar_wait_bounded(&my_bars[slot], par, kWaitTimeoutNs)) flags[grp] = 1;
      }
      for (int j = 0; j < SUB; ++j, ++k_sub) {
        const int xl = cell0 + st * TS + j * T + lane * VEC;  // first cell of this lane
        float x[MPW][VEC];
        float wv[VEC];

        if constexpr (TMA) {
#pragma unroll
          for (int k = 0; k < MPW; ++k) {
            const int i = q + k * G;
            if (i < N) {
              lds_vec<VEC>(x[k], sb + static_cast<size_t>(i) * TS + j * T + lane * VEC);
            } else {
#pragma unroll
              for (int v = 0; v < VEC; ++v) x[k][v] = 0.f;
            }
          }
          if (has_w) {
            lds_vec<VEC>(wv, sb + SF - TS + j * T + lane * VEC);
          } else {
#pragma unroll
            for (int v = 0; v < VEC; ++v) wv[v] = 1.f;
          }
        } else {
#pragma unroll
          for (int k = 0; k < MPW; ++k) {
            const int i = q + k * G;
#pragma unroll
            for (int v = 0; v < VEC; ++v) {
              const int xc = xl + v;
              x[k][v] = (i < N && xc < d.M) ? __ldg(d.data + static_cast<int64_t>(i) * d.ld + xc)
                                            : 0.f;
            }
          }
#pragma unroll
          for (int v = 0; v < VEC; ++v) {
            const int xc = xl + v;
            wv[v] = has_w ? ((xc < d.M) ? __ldg(d.w + xc) : 0.f) : 1.f;
          }
        }
        // Cells past the end of the ensemble carry no measure.
#pragma unroll
        for (int v = 0; v < VEC; ++v)
          if (xl + v >= d.M) wv[v] = 0.f;

        if (d.validate) {
#pragma unroll
          for (int v = 0; v < VEC; ++v) {
            if (xl + v < d.M) {
              if (!(wv[v] > 0.f) || !(wv[v] < 3.0e38f)) bad |= ERR_DOMAIN;
#pragma unroll
              for (int k = 0; k < MPW; ++k) {
                if (q + k * G < N) {
                  const float f = x[k][v];
                  if (iso != ISO_NONE ? !(fabsf(f) < 3.0e38f) : !(f >= 0.f && f <= 1.f))
                    bad |= ERR_DOMAIN;
                }
              }
            }
          }
        }
        if (iso != ISO_NONE) {
#pragma unroll
          for (int k = 0; k < MPW; ++k)
#pragma unroll
            for (int v = 0; v < VEC; ++v) x[k][v] = iso_value(x[k][v], iso, iso_mu, iso_inv, iso_t);
        }

        // Column sum over this warp's members (rows past N are dropped) ...
        float s[VEC];
#pragma unroll
        for (int v = 0; v < VEC; ++v) s[v] = 0.f;
#pragma unroll
        for (int k = 0; k < MPW; ++k) {
          if constexpr (COEF) {
            const float cfk = __shfl_sync(0xffffffffu, my_cf, k);
#pragma unroll
            for (int v = 0; v < VEC; ++v) s[v] = fmaf(cfk, x[k][v], s[v]);
          } else {
            if (q + k * G < N) {  // iso-mapped padding rows are not zero
#pragma unroll
              for (int v = 0; v < VEC; ++v) s[v] += x[k][v];
            }
          }
        }
        // ... then across the G warps of the group: every warp posts its partial; for G <= 2
        // each warp adds the others' directly, for larger G warp r first totals the cells
        // [r T/G, (r+1) T/G) (reduce-scatter) and every warp then reads the totals.
        float* rb = my_red + static_cast<int>(k_sub & 1) * RB;
        if (G > 1) {
#pragma unroll
          for (int v = 0; v < VEC; ++v) rb[q * T + lane * VEC + v] = s[v];
          named_barrier(1 + grp, G * 32);
        } else {
          __syncwarp();
        }
        if (flags[grp]) { aborted = true; break; }
        if constexpr (TMA) {
          if (leader && j == SUB - 1) issue_next();  // every warp has read this slot: refill it
        }
        if (G > 2 && p.xchg == 1) {
          const int cpw = T / G;
          if (lane < cpw) {
            const int cc = q * cpw + lane;
            float acc = 0.f;
            for (int r = 0; r < G; ++r) acc += rb[r * T + cc];
            rb[G * T + cc] = acc;
          }
          named_barrier(1 + grp, G * 32);
          lds_vec<VEC>(s, rb + G * T + lane * VEC);
        } else if (G > 1) {
          // every warp adds the G partials in warp order (the same order as above)
#pragma unroll
          for (int v = 0; v < VEC; ++v) s[v] = 0.f;
          for (int r = 0; r < G; ++r) {
            float t[VEC];
            lds_vec<VEC>(t, rb + r * T + lane * VEC);
#pragma unroll
            for (int v = 0; v < VEC; ++v) s[v] += t[v];
          }
        }
        if constexpr (!COEF) {
#pragma unroll
          for (int v = 0; v < VEC; ++v) s[v] *= inv_n;
        }
        // Per-member accumulation: m_i += w u_i, A_i += w u_i s.
#pragma unroll
        for (int k = 0; k < MPW; ++k) {
#pragma unroll
          for (int v = 0; v < VEC; ++v) {
            const float t = wv[v] * x[k][v];
            accM[k] += t;
            accA[k] = fmaf(t, s[v], accA[k]);
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
  }

  if (bad) atomicOr(p.err, bad);
  if (aborted && lane == 0 && q == 0) atomicOr(p.err, ERR_TIMEOUT);
  // On an early exit, let this group's copies in flight land before the CTA retires.
  if (TMA && leader) {
    while (k_cons < n_issued) {
      const int slot = static_cast<int>(k_cons % depth);
      const uint32_t par = static_cast<uint32_t>((k_cons / depth) & 1);
      if (!mbar_wait_bounded(&my_bars[slot], par, kWaitTimeoutNs)) break;
      ++k_cons;
    }
  }
}

size_t stream_smem_bytes(int vec, int G, int depth, int stage_floats) {
  const int T = 32 * vec;
  const int n_groups = kStreamWarps / G;
  return static_cast<size_t>(n_groups) * depth * stage_floats * 4 +
         static_cast<size_t>(n_groups) * 2 * (G * T + T) * 4 +
         static_cast<size_t>(n_groups) * depth * 8 + static_cast<size_t>(n_groups) * 4 + 64;
}

template <int VEC, int MPW, bool TMA, bool COEF>
static cudaError_t launch_one(const StreamParams& p, int grid, size_t smem, cudaStream_t s) {
  auto k = stream_kernel<VEC, MPW, TMA, COEF>;
  k<<<grid, kStreamThreads, smem, s>>>(p);
  return cudaGetLastError();
}

template <int VEC, int MPW>
static cudaError_t set_smem_attrs(int bytes) {
  cudaError_t e;
  if ((e = cudaFuncSetAttribute(stream_kernel<VEC, MPW, true, true>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize, bytes)) != cudaSuccess)
    return e;
  if ((e = cudaFuncSetAttribute(stream_kernel<VEC, MPW, true, false>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize, bytes)) != cudaSuccess)
    return e;
  if ((e = cudaFuncSetAttribute(stream_kernel<VEC, MPW, false, true>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize, bytes)) != cudaSuccess)
    return e;
  return cudaFuncSetAttribute(stream_kernel<VEC, MPW, false, false>,
                              cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
}

// Opt every streaming instantiation in to the largest dynamic shared memory once per
// device (before any launch, so that launches can be captured into graphs).
cudaError_t stream_kernels_init(int max_smem) {
  cudaError_t e;
  if ((e = set_smem_attrs<4, 8>(max_smem)) != cudaSuccess) return e;
  if ((e = set_smem_attrs<2, 16>(max_smem)) != cudaSuccess) return e;
  return set_smem_attrs<1, 32>(max_smem);
}

template <int VEC, int MPW>
static cudaError_t launch_stream_t(const StreamParams& p, bool coef, int grid, size_t smem,
                                   cudaStream_t s) {
  if (p.use_tma)
    return coef ? launch_one<VEC, MPW, true, true>(p, grid, smem, s)
                : launch_one<VEC, MPW, true, false>(p, grid, smem, s);
  return coef ? launch_one<VEC, MPW, false, true>(p, grid, smem, s)
              : launch_one<VEC, MPW, false, false>(p, grid, smem, s);
}

// Tile classes (cells per lane VEC, members per warp MPW): see stream_cfg on the host.
cudaError_t launch_stream(const StreamParams& p, int vec, bool coef, int grid, size_t smem,
                          cudaStream_t s) {
  switch (vec) {
    case 4: return launch_stream_t<4, 8>(p, coef, grid, smem, s);
    case 2: return launch_stream_t<2, 16>(p, coef, grid, smem, s);
    case 1: return launch_stream_t<1, 32>(p, coef, grid, smem, s);
    default: return cudaErrorInvalidValue;
  }
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

__global__ void __launch_bounds__(kFinThreads, 1) finalize_kernel(const __grid_constant__ FinParams p) {
  const FinDesc& d = fin_desc(p, blockIdx.y);
  if (static_cast<int>(blockIdx.x) >= d.slices) return;
  __shared__ double scratch[32][33];
  __shared__ double sdepth[1024];
  __shared__ double sred[1024];
  __shared__ int is_last;

  const int N = d.N;
  const int nb_stream = (2 * N + 31) / 32;
  const int nb_gram = d.kind == FIN_GRAM ? (N * N + 31) / 32 : 0;
  const int nb = nb_stream + nb_gram;
  const int dst_off = d.kind == FIN_LIN2 ? 2 * N : 0;

  // Phase 1: this CTA's share of the column blocks.
  for (int cb = blockIdx.x; cb < nb; cb += d.slices) {
    if (cb < nb_stream)
      reduce_columns<double>(d.part, d.n_chunks, 2 * N, cb, d.sums + dst_off, scratch);
    else
      reduce_columns<float>(d.gpart, d.n_gchunks, N * N, cb - nb_stream, d.sums + 4 * N, scratch);
  }
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) is_last = (atomicAdd(d.ticket, 1u) == static_cast<unsigned>(d.slices - 1));
  __syncthreads();
  if (!is_last) return;
  __threadfence();

  // Phase 2 (last CTA of this ensemble): per-member outputs and ranks.
  const int i = threadIdx.x;
  const double* S = d.sums;
  double m = 0.0, A = 0.0;
  if (i < N) { m = __ldcg(S + i); A = __ldcg(S + N + i); }
  // m_bar = (1/N) sum_i m_i, a fixed-order tree over the thread index.
  sred[i] = (i < N) ? m : 0.0;
  __syncthreads();
  for (int o = kFinThreads / 2; o > 0; o >>= 1) {
    if (i < o) sred[i] += sred[i + o];
    __syncthreads();
  }
  const double mbar = sred[0] / N;
  __syncthreads();

  double depth = 0.0, in_in = 0.0, in_out = 0.0, err = 0.0;
  if (i < N) {
    const double in_in_exact = m > 0.0 ? A / m : 0.0;        // u_i subset_p u_bar (Eq. 17)
    const double mean_out = mbar > 0.0 ? A / mbar : 0.0;     // u_bar subset_p u_i (Eq. 16)
    const double mean_depth = fmin(in_in_exact, mean_out);
    if (d.mass) d.mass[i] = m;
    if (d.mean_depth) d.mean_depth[i] = mean_depth;
    if (d.kind == FIN_MEAN) {
      in_in = in_in_exact; in_out = mean_out;
    } else if (d.kind == FIN_LIN1) {
      d.coef[i] = m > 0.0 ? static_cast<float>(1.0 / (static_cast<double>(N) * m)) : 0.0f;
    } else if (d.kind == FIN_LIN2) {
      in_in = in_in_exact;
      in_out = __ldcg(S + 3 * N + i);
    } else {  // FIN_GRAM: G[i + j N] = sum_x w u_i u_j
      const double* Gm = S + 4 * N;
      double si = 0.0, so = 0.0;
      for (int j = 0; j < N; ++j) {
        const double gij = __ldcg(Gm + i + static_cast<size_t>(j) * N);
        const double mj = __ldcg(S + j);
        si += gij;
        if (mj > 0.0) so += __ldcg(Gm + j + static_cast<size_t>(i) * N) / mj;
      }
      in_in = m > 0.0 ? si / (m * N) : 0.0;
      in_out = so / N;
      err = fabs(in_in - in_in_exact);
    }
    depth = fmin(in_in, in_out);
  }
  if (d.kind == FIN_LIN1) {
    __syncthreads();
    if (threadIdx.x == 0) *d.ticket = 0u;
    return;
  }
  sdepth[i] = (i < N) ? depth : 0.0;
  sred[i] = err;
  __syncthreads();
  if (i < N) {
    if (d.depth) d.depth[i] = depth;
    if (d.in_in) d.in_in[i] = in_in;
    if (d.in_out) d.in_out[i] = in_out;
    if (d.rank) {
      int r = 0;
      for (int j = 0; j < N; ++j) {
        const double dj = sdepth[j];
        r += (dj > depth) || (dj == depth && j < i);
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
      const double* Gm = S + 4 * N;
      for (int k = threadIdx.x; k < N * N; k += kFinThreads) {
        const int r = k / N, cc = k - r * N;   // P[r][cc] = G_{r,cc} / m_r
        const double mr = __ldcg(S + r);
        d.P[k] = mr > 0.0 ? __ldcg(Gm + r + static_cast<size_t>(cc) * N) / mr : 0.0;
      }
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) *d.ticket = 0u;
}

cudaError_t launch_finalize(const FinParams& p, int grid_x, int grid_y, cudaStream_t s) {
  finalize_kernel<<<dim3(grid_x, grid_y), kFinThreads, 0, s>>>(p);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------------------
// Isovalue map alone (pid_soft_masks)
// ---------------------------------------------------------------------------------------

__global__ void __launch_bounds__(256) iso_kernel(const __grid_constant__ IsoParams p) {
  const bool vec = ((p.ld & 3) == 0) && ((p.ld_out & 3) == 0) &&
                   ((reinterpret_cast<uintptr_t>(p.F) & 15) == 0) &&
                   ((reinterpret_cast<uintptr_t>(p.U) & 15) == 0);
  const int64_t per_row = vec ? (p.M + 3) / 4 : p.M;
  const int64_t total = per_row * p.N;
  const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
  for (int64_t t = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; t < total; t += stride) {
    const int64_t i = t / per_row;
    const int64_t j = t - i * per_row;
    const float* src = p.F + i * p.ld;
    float* dst = p.U + i * p.ld_out;
    if (vec) {
      const int64_t x = j * 4;
      if (x + 4 <= p.M) {
        const float4 f = __ldg(reinterpret_cast<const float4*>(src + x));
        float4 u;
        u.x = iso_value(f.x, p.iso_mode, p.iso_mu, p.iso_inv, p.iso_t);
        u.y = iso_value(f.y, p.iso_mode, p.iso_mu, p.iso_inv, p.iso_t);
        u.z = iso_value(f.z, p.iso_mode, p.iso_mu, p.iso_inv, p.iso_t);
        u.w = iso_value(f.w, p.iso_mode, p.iso_mu, p.iso_inv, p.iso_t);
        *reinterpret_cast<float4*>(dst + x) = u;
      } else {
        for (int64_t xx = x; xx < p.M; ++xx)
          dst[xx] = iso_value(__ldg(src + xx), p.iso_mode, p.iso_mu, p.iso_inv, p.iso_t);
      }
    } else {
      dst[j] = iso_value(__ldg(src + j), p.iso_mode, p.iso_mu, p.iso_inv, p.iso_t);
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
  iso_kernel<<<static_cast<int>(blocks), 256, 0, s>>>(p);
  return cudaGetLastError();
}

}  // namespace pidk
