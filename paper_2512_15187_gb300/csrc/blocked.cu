// PID-mean and exact full PID for ensembles beyond one CTA's tile (N > 512 members).
//
// The fused streaming kernel holds every member of a cell tile on chip, which bounds N by
// the rows one CTA group can own. Larger ensembles go through three simpler passes per
// streaming pass, all over the member-major data [N][ld]:
//   1. colsum_kernel  per block of kBlockRows members, the column sum
//                     s_b(x) = sum_{j in b} c_j u_j(x) (compensated FP32), one row per block;
//   2. combine_kernel s(x) = sum_b s_b(x) in block order, in FP64, stored as FP32;
//   3. accum_kernel   per member i and chunk of cells, m_i = sum_x w u_i and
//                     A_i = sum_x w u_i s (FP32 per lane, one warp per (member, chunk)),
//                     written as the same per-chunk partials the fused kernel writes.
// With c_j = 1 this is PID-mean's pass (A_i = N x the sum against u_bar, Eq. 15-16); with
// c_j = 1/(N m_j) it is the second pass of the exact full PID (IN_out of Eq. 10 with the
// sums of Eq. 14). The isovalue map of Sec. 3.5 is applied to each element as it is read.
// rank_kernel ranks more members than the finalisation's single CTA holds.
#include <cuda.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>

#include "capi_internal.h"
#include "device.cuh"
#include "internal.h"

namespace pidk {

constexpr int kBlockRows = 512;      // members per column-sum block
constexpr int kAccChunk = 8192;      // cells per accumulation chunk (one partial per member)

struct BlockedParams {
  const float* data;     // [N][ld]
  const float* w;        // [M] or nullptr
  const float* coef;     // [N] column-sum coefficients, or nullptr (every c_j = 1)
  float* S;              // [n_blocks][ldS] per-block column sums
  float* s;              // [ldS] combined column sum
  double* part;          // [n_chunks][2N]
  int64_t N, M, ld, ldS;
  int32_t n_blocks, n_chunks;
  int32_t iso_mode;
  float iso_mu, iso_inv, iso_t;
};

__device__ __forceinline__ float blocked_u(const BlockedParams& p, float f) {
  return p.iso_mode == ISO_NONE ? f : iso_value(f, p.iso_mode, p.iso_mu, p.iso_inv, p.iso_t);
}

// Grid: x over 4-cell groups, y over member blocks. Kahan-compensated FP32 sums.
__global__ void __launch_bounds__(256) colsum_kernel(const __grid_constant__ BlockedParams p) {
  const int64_t x = (static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x) * 4;
  if (x >= p.M) return;
  const int64_t r0 = static_cast<int64_t>(blockIdx.y) * kBlockRows;
  const int64_t r1 = min(r0 + kBlockRows, p.N);
  const bool vec = (p.ld & 3) == 0 && (reinterpret_cast<uintptr_t>(p.data) & 15) == 0 &&
                   x + 4 <= p.M;
  float sum[4] = {0.f, 0.f, 0.f, 0.f}, comp[4] = {0.f, 0.f, 0.f, 0.f};
  for (int64_t i = r0; i < r1; ++i) {
    const float* row = p.data + i * p.ld + x;
    float v[4];
    if (vec) {
      const float4 q = __ldg(reinterpret_cast<const float4*>(row));
      v[0] = q.x; v[1] = q.y; v[2] = q.z; v[3] = q.w;
    } else {
#pragma unroll
      for (int k = 0; k < 4; ++k) v[k] = x + k < p.M ? __ldg(row + k) : 0.f;
    }
    const float c = p.coef ? __ldg(p.coef + i) : 1.0f;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const float term = c * blocked_u(p, v[k]) - comp[k];
      const float t = sum[k] + term;
      comp[k] = (t - sum[k]) - term;
      sum[k] = t;
    }
  }
  float* out = p.S + static_cast<int64_t>(blockIdx.y) * p.ldS + x;
#pragma unroll
  for (int k = 0; k < 4; ++k)
    if (x + k < p.M) out[k] = sum[k];
}

__global__ void __launch_bounds__(256) combine_kernel(const __grid_constant__ BlockedParams p) {
  const int64_t x = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (x >= p.M) return;
  double acc = 0.0;
  for (int b = 0; b < p.n_blocks; ++b) acc += static_cast<double>(p.S[b * p.ldS + x]);
  p.s[x] = static_cast<float>(acc);
}

// One warp per (member, chunk): lanes stride the chunk's cells 4 at a time.
__global__ void __launch_bounds__(256) accum_kernel(const __grid_constant__ BlockedParams p) {
  const int64_t wid = (static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (wid >= p.N * p.n_chunks) return;
  const int64_t i = wid % p.N;
  const int64_t c = wid / p.N;
  const int64_t x0 = c * kAccChunk;
  const int64_t x1 = min(x0 + kAccChunk, p.M);
  const bool vec = (p.ld & 3) == 0 && (reinterpret_cast<uintptr_t>(p.data) & 15) == 0 &&
                   (p.w == nullptr || (reinterpret_cast<uintptr_t>(p.w) & 15) == 0);
  const float* row = p.data + i * p.ld;
  float m = 0.f, a = 0.f;
  for (int64_t x = x0 + lane * 4; x < x1; x += 32 * 4) {
    float v[4], sv[4], wv[4] = {1.f, 1.f, 1.f, 1.f};
    if (vec && x + 4 <= x1) {
      const float4 q = __ldg(reinterpret_cast<const float4*>(row + x));
      const float4 qs = __ldg(reinterpret_cast<const float4*>(p.s + x));
      v[0] = q.x; v[1] = q.y; v[2] = q.z; v[3] = q.w;
      sv[0] = qs.x; sv[1] = qs.y; sv[2] = qs.z; sv[3] = qs.w;
      if (p.w) {
        const float4 qw = __ldg(reinterpret_cast<const float4*>(p.w + x));
        wv[0] = qw.x; wv[1] = qw.y; wv[2] = qw.z; wv[3] = qw.w;
      }
    } else {
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const bool in = x + k < x1;
        v[k] = in ? __ldg(row + x + k) : 0.f;
        sv[k] = in ? __ldg(p.s + x + k) : 0.f;
        if (p.w) wv[k] = in ? __ldg(p.w + x + k) : 0.f;
      }
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      if (x + k < x1) {
        const float t = wv[k] * blocked_u(p, v[k]);
        m += t;
        a = fmaf(t, sv[k], a);
      }
    }
  }
  m = warp_sum(m);
  a = warp_sum(a);
  if (lane == 0) {
    p.part[c * 2 * p.N + i] = static_cast<double>(m);
    p.part[c * 2 * p.N + p.N + i] = static_cast<double>(a);
  }
}

// rank[i] = #{j : d_j > d_i or (d_j == d_i and j < i)}; depths staged through shared memory.
// rank[i] += number of members j in this block's slice of [0, N) (blockIdx.y of gridDim.y
// equal slices) that are deeper than i, or as deep with a lower index. The slices run as
// separate blocks for occupancy; the counts are integers, so adding them with atomics
// gives the same ranks in any order. rank must be zero before the launch.
__global__ void __launch_bounds__(256) rank_kernel(const double* depth, int64_t N, int32_t* rank) {
  __shared__ unsigned long long tile[2048];   // order keys of the depths
  const int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  const unsigned long long di = order_key(i < N ? depth[i] : 0.0);
  const int64_t lo = N * blockIdx.y / gridDim.y, hi = N * (blockIdx.y + 1) / gridDim.y;
  int64_t r = 0;
  for (int64_t j0 = lo; j0 < hi; j0 += 2048) {
    const int64_t n = hi - j0 < 2048 ? hi - j0 : 2048;
    __syncthreads();
    for (int64_t k = threadIdx.x; k < n; k += blockDim.x) tile[k] = order_key(depth[j0 + k]);
    __syncthreads();
    if (i < N) {
      for (int64_t k = 0; k < n; ++k) {
        const unsigned long long dj = tile[k];
        r += (dj > di) || (dj == di && j0 + k < i);
      }
    }
  }
  if (i < N && r > 0) atomicAdd(rank + i, static_cast<int32_t>(r));
}

}  // namespace pidk

namespace pidh {

using namespace pidk;

static int64_t rup(int64_t a, int64_t b) { return (a + b - 1) / b * b; }

static pid_status blocked_pass(pid_handle h, const BlockedParams& p, double bytes, cudaStream_t s) {
  ProfScope ps(h, PID_KERNEL_STREAM, bytes, 0.0, s);
  const dim3 gc(static_cast<unsigned>((p.M + 4 * 256 - 1) / (4 * 256)), static_cast<unsigned>(p.n_blocks));
  colsum_kernel<<<gc, 256, 0, s>>>(p);
  combine_kernel<<<static_cast<unsigned>((p.M + 255) / 256), 256, 0, s>>>(p);
  const int64_t warps = p.N * p.n_chunks;
  accum_kernel<<<static_cast<unsigned>((warps * 32 + 255) / 256), 256, 0, s>>>(p);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(h, e, "member-blocked pass launch");
  return PID_OK;
}

pid_status run_blocked(pid_handle h, const EnsInput& in, const EnsOutputs& out, cudaStream_t s) {
  if (in.mode == PID_MODE_FULL && in.precision != PID_FP32)
    return fail(h, PID_ERR_UNSUPPORTED,
                "the tensor-core Gram takes N <= 512; use PID_MODE_FULL_LINEAR");
  if (in.validate)
    return fail(h, PID_ERR_UNSUPPORTED, "validation is not available for N > 512");
  const bool linear = in.mode != PID_MODE_MEAN;
  const int64_t N = in.N, M = in.M;
  const int64_t ldS = rup(M, 4);
  const int n_blocks = static_cast<int>((N + kBlockRows - 1) / kBlockRows);
  const int n_chunks = static_cast<int>((M + kAccChunk - 1) / kAccChunk);
  const bool big = N > 1024;                      // ranks beyond the finalisation's CTA
  const size_t S_bytes = rup(static_cast<int64_t>(n_blocks) * ldS * 4, 256);
  const size_t s_bytes = rup(ldS * 4, 256);
  const size_t part_bytes = rup(static_cast<int64_t>(n_chunks) * 2 * N * 8, 256);
  const size_t sums_bytes = rup(4 * N * 8, 256);
  const size_t coef_bytes = rup(N * 4, 256);
  const size_t dtmp_bytes = (big && out.rank && !out.depth) ? rup(N * 8, 256) : 0;
  pid_status st = ensure_workspace(h, S_bytes + s_bytes + part_bytes + sums_bytes + coef_bytes +
                                          dtmp_bytes, s);
  if (st != PID_OK) return st;
  char* ws = static_cast<char*>(h->ws);
  BlockedParams p;
  std::memset(&p, 0, sizeof(p));
  p.S = reinterpret_cast<float*>(ws);
  p.s = reinterpret_cast<float*>(ws + S_bytes);
  p.part = reinterpret_cast<double*>(ws + S_bytes + s_bytes);
  double* sums = reinterpret_cast<double*>(ws + S_bytes + s_bytes + part_bytes);
  float* coef = reinterpret_cast<float*>(ws + S_bytes + s_bytes + part_bytes + sums_bytes);
  double* dtmp = dtmp_bytes ? reinterpret_cast<double*>(ws + S_bytes + s_bytes + part_bytes +
                                                        sums_bytes + coef_bytes)
                            : nullptr;
  p.data = in.data; p.w = in.w; p.N = N; p.M = M; p.ld = in.ld; p.ldS = ldS;
  p.n_blocks = n_blocks; p.n_chunks = n_chunks;
  iso_fill(in.is_field ? &in.iso : nullptr, &p.iso_mode, &p.iso_mu, &p.iso_inv, &p.iso_t);
  const double bytes = 4.0 * N * M + (in.w ? 4.0 * M : 0.0);

  FinDesc fd;
  std::memset(&fd, 0, sizeof(fd));
  fd.part = p.part;
  fd.N = static_cast<int32_t>(N);
  fd.n_chunks = n_chunks;
  fd.sums = sums;
  fd.coef = coef;
  fd.ticket = h->tickets;
  fd.depth = out.depth ? out.depth : dtmp;
  fd.in_in = out.in_in;
  fd.in_out = out.in_out;
  fd.rank = big ? nullptr : out.rank;
  fd.mass = out.mass;
  fd.mean_depth = out.mean_depth;

  if (in.member_weights) {   // PID-mean against the weighted mean contour: one pass
    if ((st = launch_member_coef_one(h, in.member_weights, N, coef, s)) != PID_OK) return st;
    p.coef = coef;
    if ((st = blocked_pass(h, p, bytes, s)) != PID_OK) return st;
    fd.kind = FIN_WMEAN;
    if ((st = launch_fin_one(h, fd, s)) != PID_OK) return st;
  } else if ((st = blocked_pass(h, p, bytes, s)) != PID_OK) {
    return st;
  } else if (!linear) {
    fd.kind = FIN_MEAN;
    if ((st = launch_fin_one(h, fd, s)) != PID_OK) return st;
  } else {
    FinDesc f1 = fd;
    f1.kind = FIN_LIN1;
    f1.depth = nullptr; f1.in_in = nullptr; f1.in_out = nullptr; f1.rank = nullptr;
    if ((st = launch_fin_one(h, f1, s)) != PID_OK) return st;
    p.coef = coef;
    if ((st = blocked_pass(h, p, bytes, s)) != PID_OK) return st;
    FinDesc f2 = fd;
    f2.kind = FIN_LIN2;
    f2.mass = nullptr; f2.mean_depth = nullptr;
    if ((st = launch_fin_one(h, f2, s)) != PID_OK) return st;
  }
  if (big && out.rank) {
    const unsigned slices = static_cast<unsigned>(N / 4096 < 1 ? 1 : (N / 4096 > 16 ? 16 : N / 4096));
    cudaError_t e = cudaMemsetAsync(out.rank, 0, static_cast<size_t>(N) * sizeof(int32_t), s);
    if (e != cudaSuccess) return cuda_fail(h, e, "rank reset");
    rank_kernel<<<dim3(static_cast<unsigned>((N + 255) / 256), slices), 256, 0, s>>>(fd.depth, N,
                                                                                    out.rank);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(h, e, "rank kernel launch");
  }
  return PID_OK;
}

}  // namespace pidh
