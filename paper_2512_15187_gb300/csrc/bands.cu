// Contour boxplot bands (Sec. 6): binarise every member at a probability threshold and
// collect, per cell, the unions and intersections over the deepest members and over all
// members, and the median member. One HBM-bound pass over the ensemble: 4 B read per
// member-cell, 1 B written per cell.
#include <cuda.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>

#include "capi_internal.h"
#include "internal.h"

namespace pidk {

struct BandParams {
  const float* data;     // [N][ld]
  const int32_t* rank;   // [N], 0 = deepest
  uint8_t* out;          // [M]
  int64_t N, M, ld;
  int32_t n_inner;       // members with rank < n_inner form the inner population
  int32_t cmp;           // 0: value > thr, 1: value < thr, 2: value > thr (field, super-level),
                         // 3: thr < value < thr2 (field, level map)
  float thr, thr2;
};

// Band bits of 4 cells as 4-bit masks, one bit per cell.
__device__ __forceinline__ uint32_t bin4(float a, float b, float c, float d, int cmp, float t,
                                         float t2) {
  if (cmp == 1)
    return (a < t ? 1u : 0u) | (b < t ? 2u : 0u) | (c < t ? 4u : 0u) | (d < t ? 8u : 0u);
  if (cmp == 3)
    return (a > t && a < t2 ? 1u : 0u) | (b > t && b < t2 ? 2u : 0u) |
           (c > t && c < t2 ? 4u : 0u) | (d > t && d < t2 ? 8u : 0u);
  return (a > t ? 1u : 0u) | (b > t ? 2u : 0u) | (c > t ? 4u : 0u) | (d > t ? 8u : 0u);
}

__global__ void __launch_bounds__(256) bands_kernel(const __grid_constant__ BandParams p) {
  const bool vec = (p.ld & 3) == 0 && (reinterpret_cast<uintptr_t>(p.data) & 15) == 0;
  const int64_t groups = (p.M + 3) / 4;
  const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
  for (int64_t g = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; g < groups;
       g += stride) {
    const int64_t x = g * 4;
    const bool full = vec && x + 4 <= p.M;
    uint32_t iu = 0, ii = 15, au = 0, ai = 15, med = 0;
    bool any_inner = false;
#pragma unroll 8
    for (int64_t i = 0; i < p.N; ++i) {
      const float* row = p.data + i * p.ld + x;
      float4 v;
      if (full) {
        v = __ldg(reinterpret_cast<const float4*>(row));
      } else {
        v.x = x < p.M ? __ldg(row) : 0.f;
        v.y = x + 1 < p.M ? __ldg(row + 1) : 0.f;
        v.z = x + 2 < p.M ? __ldg(row + 2) : 0.f;
        v.w = x + 3 < p.M ? __ldg(row + 3) : 0.f;
      }
      const uint32_t b = bin4(v.x, v.y, v.z, v.w, p.cmp, p.thr, p.thr2);
      const int32_t r = __ldg(p.rank + i);
      au |= b;
      ai &= b;
      if (r < p.n_inner) {
        iu |= b;
        ii &= b;
        any_inner = true;
      }
      if (r == 0) med = b;
    }
    if (!any_inner) ii = 0;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      if (x + k < p.M) {
        const uint32_t s = 1u << k;
        p.out[x + k] = static_cast<uint8_t>(((iu & s) ? 1u : 0u) | ((ii & s) ? 2u : 0u) |
                                            ((au & s) ? 4u : 0u) | ((ai & s) ? 8u : 0u) |
                                            ((med & s) ? 16u : 0u));
      }
    }
  }
}

cudaError_t launch_bands(const BandParams& p, int sms, cudaStream_t s) {
  const int64_t groups = (p.M + 3) / 4;
  int64_t grid = (groups + 255) / 256;
  if (grid > int64_t(sms) * 8) grid = int64_t(sms) * 8;
  if (grid < 1) grid = 1;
  bands_kernel<<<static_cast<unsigned>(grid), 256, 0, s>>>(p);
  return cudaGetLastError();
}

}  // namespace pidk

using namespace pidk;
using namespace pidh;

namespace {

// z with Phi(z) = p (0 < p < 1), by bisection on the FP64 complementary error function.
double normal_quantile(double pr) {
  double lo = -40.0, hi = 40.0;
  for (int it = 0; it < 200 && hi - lo > 0.0; ++it) {
    const double mid = 0.5 * (lo + hi);
    if (mid == lo || mid == hi) break;
    if (0.5 * std::erfc(-mid / std::sqrt(2.0)) < pr) lo = mid; else hi = mid;
  }
  return 0.5 * (lo + hi);
}

float float_at_or_above(double v) {
  float f = static_cast<float>(v);
  if (static_cast<double>(f) < v) f = std::nextafter(f, INFINITY);
  return f;
}

float float_at_or_below(double v) {
  float f = static_cast<float>(v);
  if (static_cast<double>(f) > v) f = std::nextafter(f, -INFINITY);
  return f;
}

}  // namespace

extern "C" pid_status pid_contour_bands(pid_handle h, const float* data, int64_t N, int64_t M,
                                        int64_t ld, const pid_iso* iso, const int32_t* rank,
                                        double tau, double inner_fraction, uint8_t* bands,
                                        void* stream) {
  pid_status st = check_shape(h, data, N, M, ld);
  if (st == PID_ERR_UNSUPPORTED && N > kMaxMembers) st = PID_OK;  // elementwise: any N
  if (st != PID_OK) return st;
  if (iso && (st = check_iso(h, iso)) != PID_OK) return st;
  if (!rank || !bands) return fail(h, PID_ERR_INVALID_ARG, "rank and bands must be non-NULL");
  if (!(tau > 0.0 && tau < 1.0)) return fail(h, PID_ERR_INVALID_ARG, "tau must be in (0, 1)");
  if (!(inner_fraction > 0.0 && inner_fraction <= 1.0))
    return fail(h, PID_ERR_INVALID_ARG, "inner_fraction must be in (0, 1]");
  BandParams p;
  std::memset(&p, 0, sizeof(p));
  p.data = data; p.rank = rank; p.out = bands; p.N = N; p.M = M; p.ld = ld;
  p.n_inner = static_cast<int32_t>(std::ceil(inner_fraction * static_cast<double>(N)));
  // The binarisation u > tau, decided exactly: for soft masks u > tau <=> u > (largest float
  // <= tau); for fields u is monotone in F, so u(F) > tau <=> F beyond F_tau with
  // u(F_tau) = tau, i.e. F compared with the float nearest F_tau on the correct side.
  if (!iso) {
    p.cmp = 0;
    p.thr = float_at_or_below(tau);
  } else if (iso->kind == PID_ISO_UNIFORM) {
    const double h = iso->sigma;
    if (!iso->superlevel) {            // u = (mu + h - F) / 2h > tau <=> F < mu + h (1 - 2 tau)
      p.cmp = 1;
      p.thr = float_at_or_above(iso->mu + h * (1.0 - 2.0 * tau));
    } else {                           // u = (F - mu + h) / 2h > tau <=> F > mu + h (2 tau - 1)
      p.cmp = 2;
      p.thr = float_at_or_below(iso->mu + h * (2.0 * tau - 1.0));
    }
  } else if (iso->kind == PID_ISO_LEVEL) {  // 1 - |F - mu| / h > tau <=> |F - mu| < h (1 - tau)
    const double r = iso->sigma * (1.0 - tau);
    p.cmp = 3;
    p.thr = float_at_or_below(iso->mu - r);
    p.thr2 = float_at_or_above(iso->mu + r);
  } else if (iso->sigma > 0.0) {
    const double z = normal_quantile(tau);
    if (!iso->superlevel) {            // u = Phi((mu - F) / sigma) > tau <=> F < mu - sigma z
      p.cmp = 1;
      p.thr = float_at_or_above(iso->mu - iso->sigma * z);
    } else {                           // u = Phi((F - mu) / sigma) > tau <=> F > mu + sigma z
      p.cmp = 2;
      p.thr = float_at_or_below(iso->mu + iso->sigma * z);
    }
  } else {                             // u in {0, 1}: u > tau <=> u = 1
    p.cmp = iso->superlevel ? 2 : 1;
    p.thr = iso->superlevel ? float_at_or_below(iso->mu) : float_at_or_above(iso->mu);
  }
  DeviceGuard g(h->device);
  ProfScope ps(h, PID_KERNEL_BANDS, 4.0 * N * M + M, 0.0, static_cast<cudaStream_t>(stream));
  cudaError_t e = launch_bands(p, h->sms, static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return cuda_fail(h, e, "bands kernel launch");
  return PID_OK;
}
