// PID from an inclusion matrix, optionally within groups of members (pid_depth_from_matrix).
//
// With the matrix P[i][j] = u_i subset_p u_j (Eq. 9) that the Gram modes of pid_full
// return, the inclusion fractions of Eq. 10 are row and column means of P. Restricting
// both means to the members of i's own group C(i) gives the depth of i within its mode of a
// multimodal ensemble (Sec. 2.2 cites depth for multimodal contour ensembles as an
// extension of inclusion depth):
//   IN_in(i)  = (1/|C(i)|) sum_{j in C(i)} P[i][j]
//   IN_out(i) = (1/|C(i)|) sum_{j in C(i)} P[j][i],   depth = min, rank within C(i).
// Two small FP64 kernels, O(N^2) each: one block of 256 threads per 256 members forms the
// column means with coalesced loads (thread = column) and the row means with one warp per
// row; a second kernel ranks each member within its group.
#include <cuda_runtime.h>

#include <cstring>

#include "capi_internal.h"
#include "device.cuh"
#include "internal.h"

namespace pidk {

struct MatrixParams {
  const double* P;       // [N][ldp]
  const int32_t* labels; // [N] or nullptr (one group)
  int64_t N, ldp;
  double* depth;         // [N] (required: the ranks read it)
  double* in_in;         // [N] or nullptr
  double* in_out;        // [N] or nullptr
};

constexpr int kMatThreads = 256;

__global__ void __launch_bounds__(kMatThreads)
matrix_depth_kernel(const __grid_constant__ MatrixParams p) {
  __shared__ double s_out[kMatThreads];
  __shared__ int64_t s_cnt[kMatThreads];
  const int64_t i0 = static_cast<int64_t>(blockIdx.x) * kMatThreads;
  const int64_t ic = i0 + threadIdx.x;
  // Column means: thread t owns column i0 + t and walks the rows (coalesced across threads).
  {
    double acc = 0.0;
    int64_t cnt = 0;
    if (ic < p.N) {
      const int32_t li = p.labels ? __ldg(p.labels + ic) : 0;
      for (int64_t j = 0; j < p.N; ++j) {
        if (p.labels == nullptr || __ldg(p.labels + j) == li) {
          acc += __ldg(p.P + j * p.ldp + ic);
          ++cnt;
        }
      }
    }
    s_out[threadIdx.x] = acc;
    s_cnt[threadIdx.x] = cnt;
  }
  __syncthreads();
  // Row means: warp w takes rows i0 + w, i0 + w + 8, ...; lanes stride over the columns,
  // then a fixed-order shuffle tree.
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int r = warp; r < kMatThreads; r += kMatThreads / 32) {
    const int64_t i = i0 + r;
    if (i >= p.N) break;
    const int32_t li = p.labels ? __ldg(p.labels + i) : 0;
    double acc = 0.0;
    for (int64_t j = lane; j < p.N; j += 32)
      if (p.labels == nullptr || __ldg(p.labels + j) == li) acc += __ldg(p.P + i * p.ldp + j);
    acc = warp_sum(acc);
    if (lane == 0) {
      const double n = static_cast<double>(s_cnt[r]);
      const double a = acc / n, b = s_out[r] / n;
      if (p.in_in) p.in_in[i] = a;
      if (p.in_out) p.in_out[i] = b;
      p.depth[i] = fmin(a, b);
    }
  }
}

// rank[i] = number of members of i's group that are deeper, or as deep with a lower index.
__global__ void __launch_bounds__(kMatThreads) group_rank_kernel(const double* depth,
                                                                 const int32_t* labels, int64_t N,
                                                                 int32_t* rank) {
  __shared__ unsigned long long td[kMatThreads];   // order keys of the depths
  __shared__ int32_t tl[kMatThreads];
  const int64_t i = static_cast<int64_t>(blockIdx.x) * kMatThreads + threadIdx.x;
  const unsigned long long di = order_key(i < N ? depth[i] : 0.0);
  const int32_t li = (i < N && labels) ? labels[i] : 0;
  int64_t r = 0;
  for (int64_t j0 = 0; j0 < N; j0 += kMatThreads) {
    const int64_t n = N - j0 < kMatThreads ? N - j0 : kMatThreads;
    __syncthreads();
    if (threadIdx.x < n) {
      td[threadIdx.x] = order_key(depth[j0 + threadIdx.x]);
      tl[threadIdx.x] = labels ? labels[j0 + threadIdx.x] : 0;
    }
    __syncthreads();
    if (i < N) {
      for (int64_t k = 0; k < n; ++k)
        r += tl[k] == li && ((td[k] > di) || (td[k] == di && j0 + k < i));
    }
  }
  if (i < N) rank[i] = static_cast<int32_t>(r);
}

}  // namespace pidk

using namespace pidk;
using namespace pidh;

extern "C" pid_status pid_depth_from_matrix(pid_handle h, const double* P, int64_t N, int64_t ldp,
                                            const int32_t* labels, double* depth, double* in_in,
                                            double* in_out, int32_t* rank, void* stream) {
  if (!h) return PID_ERR_INVALID_ARG;
  if (!P) return fail(h, PID_ERR_INVALID_ARG, "P must be non-NULL");
  if (N < 1 || ldp < N) return fail(h, PID_ERR_INVALID_ARG, "need N >= 1 and ldp >= N");
  if (N > kMaxMatrixMembers)
    return fail(h, PID_ERR_UNSUPPORTED, "N above the supported maximum (65536) of a matrix call");
  if (!depth && !in_in && !in_out && !rank) return PID_OK;
  DeviceGuard g(h->device);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  double* dd = depth;
  if (!dd) {   // the kernel writes depths (the ranks read them): keep them in the workspace
    const pid_status st = ensure_workspace(h, static_cast<size_t>(N) * 8, s);
    if (st != PID_OK) return st;
    dd = static_cast<double*>(h->ws);
  }
  MatrixParams mp;
  std::memset(&mp, 0, sizeof(mp));
  mp.P = P; mp.labels = labels; mp.N = N; mp.ldp = ldp;
  mp.depth = dd; mp.in_in = in_in; mp.in_out = in_out;
  const unsigned grid = static_cast<unsigned>((N + kMatThreads - 1) / kMatThreads);
  {
    ProfScope ps(h, PID_KERNEL_FINALIZE, 16.0 * N * N, 0.0, s);
    matrix_depth_kernel<<<grid, kMatThreads, 0, s>>>(mp);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(h, e, "matrix depth launch");
  }
  if (rank) {
    ProfScope ps(h, PID_KERNEL_FINALIZE, 12.0 * N * N / kMatThreads, 0.0, s);
    group_rank_kernel<<<grid, kMatThreads, 0, s>>>(dd, labels, N, rank);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(h, e, "group rank launch");
  }
  return PID_OK;
}
