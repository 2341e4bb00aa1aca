// pid_mean_noalloc: PID-mean without any device allocation.
//
// Some callers cannot allocate device memory when they need a depth: real-time loops where
// a cudaMalloc would synchronise the device, and host applications that hand out all
// device memory through their own allocator. The regular entry points allocate workspace through
// a handle; this one keeps its scratch (the per-chunk partial sums, the FP64 totals, the
// finalisation ticket and the device error word) in a fixed array compiled into the
// library, and otherwise runs the same streaming and finalisation kernels as pid_mean.
#include <cuda_runtime.h>

#include <cstring>
#include <mutex>

#include "capi_internal.h"
#include "internal.h"

using namespace pidk;

namespace {

// 4 MiB per device, held by every GPU that loads the library until the process exits.
constexpr size_t kScratchBytes = size_t(4) << 20;
constexpr size_t kHeaderBytes = 256;  // [0] error word, [1] finalisation ticket (uint32)

__device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
struct DeviceState {
  bool ready = false;
  char* scratch = nullptr;  // device address of g_noalloc_scratch on this device
  int sms = 0;
};
DeviceState g_dev[kMaxDevices];
std::mutex g_mu;

// Once per device, with that device current: look up the array's device address (the
// array's name in host code is only a host-side stand-in) and opt the kernels in to their
// shared memory. Nothing here allocates.
pid_status setup_current_device(DeviceState** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return PID_ERR_CUDA;
  std::lock_guard<std::mutex> lock(g_mu);
  DeviceState& st = g_dev[dev];
  if (!st.ready) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || p == nullptr) {
      cudaGetLastError();
      return PID_ERR_CUDA;
    }
    int max_smem = 0, sms = 0;
    if (cudaDeviceGetAttribute(&max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        stream_kernels_init(max_smem) != cudaSuccess) {
      cudaGetLastError();
      return PID_ERR_CUDA;
    }
    st.scratch = static_cast<char*>(p);
    st.sms = sms;
    st.ready = true;
  }
  *out = &st;
  return PID_OK;
}

}  // namespace

extern "C" pid_status pid_mean_noalloc(const float* U, int64_t N, int64_t M, int64_t ld,
                                       const float* w, double* depth, double* in_in,
                                       double* in_out, int32_t* rank, uint32_t* device_status,
                                       void* stream) {
  DeviceState* ds = nullptr;
  pid_status st = setup_current_device(&ds);
  if (st != PID_OK) return st;

  // A handle-shaped planning context on the stack (no allocation) for the shared planner.
  pid_handle_s ctx;
  ctx.sms = ds->sms;
  if ((st = pidh::check_shape(&ctx, U, N, M, ld)) != PID_OK) return st;
  pidh::EnsInput in;
  in.data = U; in.N = N; in.M = M; in.ld = ld; in.w = w;
  pidh::EnsPlan pl;
  if ((st = pidh::plan_stream(&ctx, in, &pl)) != PID_OK) return st;

  // Scratch layout: header | FP64 totals [4N] | per-chunk partials [n_chunks][2N].
  const size_t sums_bytes = (static_cast<size_t>(4 * N) * 8 + 255) / 256 * 256;
  const size_t part_bytes = static_cast<size_t>(pl.desc.n_chunks) * 2 * N * 8;
  if (kHeaderBytes + sums_bytes + part_bytes > kScratchBytes) return PID_ERR_UNSUPPORTED;
  char* base = ds->scratch;
  uint32_t* err_word = reinterpret_cast<uint32_t*>(base);
  unsigned int* ticket = reinterpret_cast<unsigned int*>(base) + 1;
  double* sums = reinterpret_cast<double*>(base + kHeaderBytes);
  double* part = reinterpret_cast<double*>(base + kHeaderBytes + sums_bytes);

  cudaStream_t s = static_cast<cudaStream_t>(stream);
  // The array keeps the previous call's contents: the error word and ticket must start at 0.
  if (cudaMemsetAsync(base, 0, kHeaderBytes, s) != cudaSuccess) return PID_ERR_CUDA;

  StreamParams sp;
  std::memset(&sp, 0, sizeof(sp));
  sp.one = pl.desc;
  sp.one.part = part;
  sp.one.coef = nullptr;
  sp.one.unit_begin = 0;
  sp.n_ens = 1;
  sp.total_units = pl.desc.n_chunks;
  sp.one.work_begin = 0;
  sp.total_work = static_cast<int64_t>(pl.desc.N) * pl.desc.M;
  sp.G = pl.cfg.G;
  sp.sub = pl.cfg.sub;
  sp.use_tma = pl.use_tma ? 1 : (pl.cls ? 2 : 0);
  sp.err = err_word;
  sp.stage_floats = pl.stage_floats;
  int ring_depth;
  size_t smem;
  pidh::stream_launch_geometry(pl.cfg, pl.stage_floats, &ring_depth, &smem);
  sp.depth = ring_depth;
  sp.xchg = pidh::default_xchg(pl.cfg);
  const int n_groups = kStreamWarps / pl.cfg.G;
  int grid = (sp.total_units + n_groups - 1) / n_groups;
  grid = grid < 1 ? 1 : (grid > ds->sms ? ds->sms : grid);
  if (launch_stream(sp, pl.cfg.vec, pl.cfg.mpw, pl.cfg.G, iso_kind(sp.one.iso_mode), false, grid,
                    smem, s) !=
      cudaSuccess)
    return PID_ERR_CUDA;

  FinParams fp;
  std::memset(&fp, 0, sizeof(fp));
  FinDesc& fd = fp.one;
  fd.part = part;
  fd.N = pl.desc.N;
  fd.n_chunks = pl.desc.n_chunks;
  fd.kind = FIN_MEAN;
  fd.sums = sums;
  fd.ticket = ticket;
  fd.depth = depth;
  fd.in_in = in_in;
  fd.in_out = in_out;
  fd.rank = rank;
  const int nb = (2 * fd.N + 31) / 32;
  fd.slices = nb < 1 ? 1 : (nb > 2 * ds->sms ? 2 * ds->sms : nb);
  fp.n_ens = 1;
  fp.err = err_word;
  if (launch_finalize(fp, fd.slices, 1, s) != cudaSuccess) return PID_ERR_CUDA;
  if (device_status &&
      cudaMemcpyAsync(device_status, err_word, sizeof(uint32_t), cudaMemcpyDeviceToDevice, s) !=
          cudaSuccess)
    return PID_ERR_CUDA;
  return PID_OK;
}
