// C ABI of the PID library: handle, argument checks, planning and launch sequences.
// The computation itself lives in stream.cu (PID-mean, exact full PID, isovalue map,
// finalisation) and gram.cu (tensor-core Gram for full PID).
#include <cuda.h>
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/pid.h"
#include "capi_internal.h"
#include "internal.h"
#include "device.cuh"

using namespace pidk;

namespace pidh {

// ---------------------------------------------------------------------------------------
// Status helpers
// ---------------------------------------------------------------------------------------

pid_status fail(pid_handle h, pid_status s, const std::string& msg) {
  if (h) h->last_error = msg;
  return s;
}

pid_status cuda_fail(pid_handle h, cudaError_t e, const char* where) {
  if (h) h->last_error = std::string(where) + ": " + cudaGetErrorString(e);
  return PID_ERR_CUDA;
}

DeviceGuard::DeviceGuard(int dev) {
  cudaGetDevice(&prev_);
  if (prev_ != dev) cudaSetDevice(dev);
  dev_ = dev;
}
DeviceGuard::~DeviceGuard() {
  if (prev_ != dev_) cudaSetDevice(prev_);
}

// ---------------------------------------------------------------------------------------
// Kernel timing
// ---------------------------------------------------------------------------------------

cudaEvent_t prof_event(pid_handle h) {
  if (!h->event_pool.empty()) {
    cudaEvent_t e = h->event_pool.back();
    h->event_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

// NVTX range names of the kernel kinds (pid_kernel_kind order): every launch the library
// makes is bracketed by a host range, so external profilers attribute kernels to the calls.
static const char* const kNvtxNames[PID_KERNEL_KINDS] = {
    "pid: streaming pass", "pid: tensor-core Gram (BF16)", "pid: finalisation",
    "pid: isovalue map", "pid: contour bands", "pid: tensor-core Gram (split BF16)",
    "pid: tensor-core Gram (E4M3)", "pid: Gram operand staging", "pid: E4M3 member scales"};

ProfScope::ProfScope(pid_handle h, int kind, double bytes, double flops, cudaStream_t s)
    : h_(h), s_(s) {
  nvtxRangePushA(kind >= 0 && kind < PID_KERNEL_KINDS ? kNvtxNames[kind] : "pid");
  if (!h_ || !h_->profiling) return;
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  cudaStreamIsCapturing(s_, &cs);
  ProfRecord r{kind, nullptr, nullptr, bytes, flops};
  if (cs != cudaStreamCaptureStatusNone) {
    // only the library's own profiled batch graphs are timed (a caller's capture is not)
    if (!h_->prof_graph) return;
    r.start = prof_event(h_);
    r.stop = prof_event(h_);
    cudaEventRecordWithFlags(r.start, s_, cudaEventRecordExternal);
    h_->prof_captured.push_back(r);
    idx_ = static_cast<int>(h_->prof_captured.size()) - 1;
    captured_ = true;
    return;
  }
  r.start = prof_event(h_);
  r.stop = prof_event(h_);
  cudaEventRecord(r.start, s_);
  h_->prof_pending.push_back(r);
  idx_ = static_cast<int>(h_->prof_pending.size()) - 1;
}

ProfScope::~ProfScope() {
  if (idx_ >= 0) {
    if (captured_)
      cudaEventRecordWithFlags(h_->prof_captured[idx_].stop, s_, cudaEventRecordExternal);
    else
      cudaEventRecord(h_->prof_pending[idx_].stop, s_);
  }
  nvtxRangePop();
}

static void prof_drain(pid_handle h) {
  for (ProfRecord& r : h->prof_pending) {
    float ms = 0.f;
    cudaEventSynchronize(r.stop);
    cudaEventElapsedTime(&ms, r.start, r.stop);
    pid_kernel_stats& t = h->prof_total[r.kind];
    t.launches += 1;
    t.total_ms += ms;
    t.bytes += r.bytes;
    t.flops += r.flops;
    h->event_pool.push_back(r.start);
    h->event_pool.push_back(r.stop);
  }
  h->prof_pending.clear();
}

// ---------------------------------------------------------------------------------------
// TMA descriptor encoding through the runtime's driver entry point (no libcuda link).
// ---------------------------------------------------------------------------------------

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                  const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                  const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiledFn get_encode_fn() {
  static EncodeTiledFn fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(p);
  });
  return fn;
}

bool encode_2d(CUtensorMap* m, const void* base, uint64_t inner, uint64_t outer,
               uint64_t row_bytes, uint32_t box_inner, uint32_t box_outer) {
  EncodeTiledFn fn = get_encode_fn();
  if (!fn) return false;
  cuuint64_t dims[2] = {inner, outer};
  cuuint64_t strides[1] = {row_bytes};
  cuuint32_t box[2] = {box_inner, box_outer};
  cuuint32_t es[2] = {1, 1};
  return fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<void*>(base), dims, strides, box, es,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
            CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// Operand plane [outer rows][inner elements] of 2-byte (BF16) or 1-byte (E4M3) elements,
// read in boxes of 128 bytes x 128 rows in the 128-byte swizzle layout of the tensor cores;
// elements past the extents read as zero.
bool encode_2d_sw128(CUtensorMap* m, const void* base, int elem_bytes, uint64_t inner,
                     uint64_t outer, uint64_t row_bytes) {
  EncodeTiledFn fn = get_encode_fn();
  if (!fn || (elem_bytes != 1 && elem_bytes != 2)) return false;
  cuuint64_t dims[2] = {inner, outer};
  cuuint64_t strides[1] = {row_bytes};
  cuuint32_t box[2] = {static_cast<cuuint32_t>(128 / elem_bytes), 128};
  cuuint32_t es[2] = {1, 1};
  return fn(m, elem_bytes == 2 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_UINT8, 2,
            const_cast<void*>(base), dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
            CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

bool encode_1d(CUtensorMap* m, const void* base, uint64_t n, uint32_t box) {
  EncodeTiledFn fn = get_encode_fn();
  if (!fn) return false;
  cuuint64_t dims[1] = {n};
  cuuint64_t strides[1] = {0};
  cuuint32_t bx[1] = {box};
  cuuint32_t es[1] = {1};
  return fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 1, const_cast<void*>(base), dims, strides, bx, es,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
            CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// ---------------------------------------------------------------------------------------
// Planning
// ---------------------------------------------------------------------------------------

// Tile class of the streaming kernel as a function of N alone, so that an ensemble is
// always processed with the same arithmetic order, alone or inside a batch.
// Each warp holds MPW = ceil(N / G) members x VEC cells in registers (MPW x VEC <= 32);
// a TMA stage moves sub x T cells of every member (sub = 1 keeps three stages in flight
// for N up to 512).
// The streaming tile classes {VEC, G, T, sub, members per warp}, in order of the member rows
// they hold (G x members per warp). Every member slot of a class costs arithmetic whether
// or not a member fills it, so the classes above 16 members come in steps that keep the
// empty slots to about a fifth; an ensemble's default class is the first that holds it.
static const StreamCfg kStreamClasses[] = {
    {4, 1, 128, 1, 8},  {4, 2, 128, 1, 8},   {4, 4, 128, 1, 6},  {4, 4, 128, 1, 8},
    {4, 8, 128, 1, 6},  {4, 8, 128, 1, 8},   {4, 16, 128, 1, 6}, {4, 16, 128, 1, 8},
    {2, 16, 64, 1, 12}, {2, 16, 64, 1, 13},  {2, 16, 64, 1, 16}, {1, 16, 32, 1, 20},
    {1, 16, 32, 1, 24}, {1, 16, 32, 1, 28},  {1, 16, 32, 1, 32}};
constexpr int kNumStreamClasses = sizeof(kStreamClasses) / sizeof(kStreamClasses[0]);

static int default_stream_class(int64_t N) {
  for (int c = 0; c < kNumStreamClasses; ++c)
    if (static_cast<int64_t>(kStreamClasses[c].G) * kStreamClasses[c].mpw >= N) return c;
  return kNumStreamClasses - 1;
}

StreamCfg stream_cfg(int64_t N) { return kStreamClasses[default_stream_class(N)]; }

static int log2_floor(int64_t v) {
  int lg = 0;
  while ((int64_t(1) << (lg + 1)) <= v) ++lg;
  return lg;
}

// Shape keys of the tile choices: member count, cell-count octave, isovalue kind, weights.
static std::string stream_shape_key(const EnsInput& in) {
  char buf[96];
  std::snprintf(buf, sizeof(buf), "stream n%lld m%d iso%d w%d", static_cast<long long>(in.N),
                log2_floor(in.M), in.is_field ? (in.iso.sigma > 0 ? 1 : 2) : 0, in.w != nullptr);
  return buf;
}

std::string gram_shape_key(const EnsInput& in) {
  char buf[96];
  std::snprintf(buf, sizeof(buf), "gram n%lld m%d p%d iso%d w%d", static_cast<long long>(in.N),
                log2_floor(in.M), in.precision, in.is_field ? (in.iso.sigma > 0 ? 1 : 2) : 0,
                in.w != nullptr);
  return buf;
}

StreamCfg stream_cfg_for(pid_handle h, const EnsInput& in) {
  const int def = default_stream_class(in.N);
  if (h && !h->shapes.empty()) {
    auto it = h->shapes.find(stream_shape_key(in));
    if (it != h->shapes.end() && it->second >= def && it->second < kNumStreamClasses)
      return kStreamClasses[it->second];
  }
  return kStreamClasses[def];
}

static int64_t round_up(int64_t a, int64_t b) { return (a + b - 1) / b * b; }

void iso_fill(const pid_iso* iso, int32_t* mode, float* mu, float* inv, float* t) {
  if (!iso) { *mode = ISO_NONE; *mu = 0.f; *inv = 0.f; *t = 0.f; return; }
  if (iso->kind == PID_ISO_UNIFORM) {    // q ~ U[mu - h, mu + h]
    const double h = iso->sigma;
    *mode = iso->superlevel ? ISO_UNIFORM_ABOVE : ISO_UNIFORM_BELOW;
    *mu = static_cast<float>(iso->superlevel ? iso->mu - h : iso->mu + h);
    *inv = static_cast<float>(1.0 / (2.0 * h));
    *t = 0.f;
    return;
  }
  if (iso->kind == PID_ISO_LEVEL) {
    *mode = ISO_LEVEL;
    *mu = static_cast<float>(iso->mu);
    *inv = static_cast<float>(1.0 / iso->sigma);
    *t = 0.f;
    return;
  }
  *mu = static_cast<float>(iso->mu);
  if (iso->sigma > 0.0) {
    *mode = ISO_NORMAL;
    const double inv_d = kSqrtLog2e / (iso->sigma * std::sqrt(2.0));
    *inv = static_cast<float>(iso->superlevel ? -inv_d : inv_d);
    *t = 0.f;
  } else {
    // F < mu (exact, in double) <=> F < t with t the smallest float >= mu;
    // F > mu <=> F > t with t the largest float <= mu.
    float t32 = static_cast<float>(iso->mu);
    if (!iso->superlevel) {
      if (static_cast<double>(t32) < iso->mu) t32 = std::nextafter(t32, INFINITY);
      *mode = ISO_STEP_BELOW;
    } else {
      if (static_cast<double>(t32) > iso->mu) t32 = std::nextafter(t32, -INFINITY);
      *mode = ISO_STEP_ABOVE;
    }
    *t = t32;
    *inv = 0.f;
  }
}

pid_status check_iso(pid_handle h, const pid_iso* iso) {
  if (!iso) return fail(h, PID_ERR_INVALID_ARG, "iso must not be NULL");
  if (iso->kind != PID_ISO_NORMAL && iso->kind != PID_ISO_UNIFORM && iso->kind != PID_ISO_LEVEL)
    return fail(h, PID_ERR_UNSUPPORTED, "unknown iso kind");
  if (!std::isfinite(iso->mu) || !std::isfinite(iso->sigma) || iso->sigma < 0.0)
    return fail(h, PID_ERR_INVALID_ARG, "iso needs finite mu and sigma >= 0");
  if (iso->superlevel != 0 && iso->superlevel != 1)
    return fail(h, PID_ERR_INVALID_ARG, "iso.superlevel must be 0 or 1");
  if (iso->kind != PID_ISO_NORMAL && !(iso->sigma > 0.0))
    return fail(h, PID_ERR_INVALID_ARG, "uniform and level maps need a half-width sigma > 0");
  if (iso->kind != PID_ISO_NORMAL &&
      !(std::fabs(iso->mu) + iso->sigma < 1e38 && 1.0 / (2.0 * iso->sigma) < 1e38))
    return fail(h, PID_ERR_INVALID_ARG, "uniform and level maps need mu +- sigma and 1/(2 sigma) "
                                        "inside the float range");
  if (iso->kind == PID_ISO_LEVEL && iso->superlevel)
    return fail(h, PID_ERR_INVALID_ARG, "the level map has no super-level form");
  return PID_OK;
}

pid_status check_shape(pid_handle h, const void* data, int64_t N, int64_t M, int64_t ld,
                       int64_t max_n) {
  if (!h) return PID_ERR_INVALID_ARG;
  if (!data) return fail(h, PID_ERR_INVALID_ARG, "data pointer is NULL");
  if (N < 1 || M < 1) return fail(h, PID_ERR_INVALID_ARG, "N and M must be >= 1");
  if (ld < M) return fail(h, PID_ERR_INVALID_ARG, "ld must be >= M");
  if (M > (int64_t(1) << 31) - 4096) return fail(h, PID_ERR_UNSUPPORTED, "M must be < 2^31 - 4096");
  if (ld > (int64_t(1) << 37)) return fail(h, PID_ERR_UNSUPPORTED, "ld too large");
  if (N > max_n)
    return fail(h, PID_ERR_UNSUPPORTED,
                max_n == kMaxMembers ? "N above the supported maximum (512) of batches and serving"
                                     : "N above the supported maximum (2^22)");
  return PID_OK;
}

pid_status check_opt(pid_handle h, const pid_options* o) {
  if (!o) return PID_OK;
  if (o->mode < PID_MODE_MEAN || o->mode > PID_MODE_FULL_LINEAR)
    return fail(h, PID_ERR_INVALID_ARG, "unknown mode");
  if (o->precision < PID_FP32 || o->precision > PID_FP8)
    return fail(h, PID_ERR_INVALID_ARG, "unknown precision");
  if (o->validate != 0 && o->validate != 1)
    return fail(h, PID_ERR_INVALID_ARG, "validate must be 0 or 1");
  if (o->reserved != 0) return fail(h, PID_ERR_INVALID_ARG, "reserved must be 0");
  return PID_OK;
}

// Plan one ensemble for the streaming kernel. Pointers into the workspace are filled later.
pid_status plan_stream(pid_handle h, const EnsInput& in, EnsPlan* pl) {
  std::memset(pl, 0, sizeof(*pl));
  const StreamCfg cfg = stream_cfg_for(h, in);
  pl->cfg = cfg;
  EnsDesc& d = pl->desc;
  d.data = in.data;
  d.w = in.w;
  d.ld = in.ld;
  d.N = static_cast<int32_t>(in.N);
  d.M = static_cast<int32_t>(in.M);
  const int n_groups = kStreamWarps / cfg.G;
  const int64_t total_groups = static_cast<int64_t>(h->sms) * n_groups;
  const int64_t TS = static_cast<int64_t>(cfg.T) * cfg.sub;
  int64_t chunk = round_up((in.M + total_groups - 1) / total_groups, TS);
  chunk = std::max<int64_t>(TS, std::min<int64_t>(chunk, 256 * cfg.T));
  d.chunk_cells = static_cast<int32_t>(chunk);
  d.n_chunks = static_cast<int32_t>((in.M + chunk - 1) / chunk);
  d.n_boxes = static_cast<int32_t>((in.N + 255) / 256);
  d.box_rows = static_cast<int32_t>((in.N + d.n_boxes - 1) / d.n_boxes);
  iso_fill(in.is_field ? &in.iso : nullptr, &d.iso_mode, &d.iso_mu, &d.iso_inv, &d.iso_t);
  d.validate = in.validate;
  const uintptr_t a = reinterpret_cast<uintptr_t>(in.data);
  const bool tma_ok = (in.ld % 4 == 0) && (a % 16 == 0) &&
                      (in.w == nullptr || reinterpret_cast<uintptr_t>(in.w) % 16 == 0);
  pl->use_tma = false;
  pl->cls = false;
  if (tma_ok && get_encode_fn()) {
    bool ok = encode_2d(&d.tmap, in.data, static_cast<uint64_t>(in.M), static_cast<uint64_t>(in.N),
                        static_cast<uint64_t>(in.ld) * 4, static_cast<uint32_t>(TS),
                        static_cast<uint32_t>(d.box_rows));
    if (ok && in.w) ok = encode_1d(&d.tmap_w, in.w, static_cast<uint64_t>(in.M), static_cast<uint32_t>(TS));
    pl->use_tma = ok;
  }
  if (!pl->use_tma && get_encode_fn()) {
    // Rows that are not 16-byte aligned: members of one residue class (i mod n_cls) share
    // their offset from the 16-byte boundary and lie n_cls ld floats apart, so each class is
    // a 2D tensor of its own (base rounded down, cells shifted by the offset) and TMA boxes
    // of TS + 4 cells stage each row's aligned span. A warp's members must share a class
    // (G a multiple of n_cls) and the cell measures be aligned for their 1D map; otherwise
    // the rows are staged by cp.async, as they are in the one-cell-per-lane classes (N > 256),
    // where a span of TS + 4 = 36 cells per row and stage costs more L2 traffic than the
    // copies it saves.
    const int ncls = in.ld % 2 != 0 ? 4 : (in.ld % 4 != 0 ? 2 : 1);
    const bool w_ok = in.w == nullptr || reinterpret_cast<uintptr_t>(in.w) % 16 == 0;
    if (cfg.vec > 1 && w_ok && cfg.G % ncls == 0 && in.N >= ncls) {
      const int64_t crows = (in.N + ncls - 1) / ncls;   // rows of the largest class
      const int32_t nb = static_cast<int32_t>((crows + 255) / 256);
      // boxes of a multiple of 8 rows: every box lands on a 128-byte boundary of the stage
      const int32_t br = static_cast<int32_t>(round_up((crows + nb - 1) / nb, 8));
      bool ok = br <= 256;
      for (int c = 0; c < ncls && ok; ++c) {
        const uintptr_t row_c = a + static_cast<uintptr_t>(c) * static_cast<uintptr_t>(in.ld) * 4;
        const uintptr_t base_c = row_c & ~static_cast<uintptr_t>(15);
        const uint64_t r_c = (row_c - base_c) / 4;
        const uint64_t rows_c = static_cast<uint64_t>((in.N - c + ncls - 1) / ncls);
        CUtensorMap* m = c == 0 ? &d.tmap : &d.tmap_cls[c - 1];
        ok = encode_2d(m, reinterpret_cast<const void*>(base_c), static_cast<uint64_t>(in.M) + r_c,
                       rows_c, static_cast<uint64_t>(ncls) * in.ld * 4,
                       static_cast<uint32_t>(TS + 4), static_cast<uint32_t>(br));
      }
      if (ok && in.w) ok = encode_1d(&d.tmap_w, in.w, static_cast<uint64_t>(in.M), static_cast<uint32_t>(TS));
      if (ok) {
        pl->cls = true;
        d.n_cls = ncls;
        d.n_boxes = nb;
        d.box_rows = br;
      }
    }
  }
  // rows of TS cells (TMA), or of TS + 4: the 16-byte-aligned spans of unaligned rows; with
  // class maps, ncls class slots of n_boxes x box_rows rows each
  const int64_t row_floats = pl->use_tma ? TS : TS + 4;
  const int64_t stage_rows = pl->cls ? int64_t(d.n_cls) * d.n_boxes * d.box_rows
                                     : int64_t(d.n_boxes) * d.box_rows;
  pl->stage_floats = static_cast<int32_t>(round_up(stage_rows * row_floats + TS, 32));
  pl->part_bytes = round_up(static_cast<int64_t>(d.n_chunks) * 2 * in.N * 8, 256);
  pl->sums_bytes = round_up((4 * in.N + in.N * in.N) * 8, 256);
  pl->coef_bytes = round_up(in.N * 4, 256);
  return PID_OK;
}

// Exchange scheme of the column sums: 0 = every warp adds the G partials, 1 = reduce-scatter
// then gather (two barriers). Both add the partials in the same order.
int default_xchg(const StreamCfg& cfg) { return cfg.G >= 16 ? 1 : 0; }

// Choose ring depth and smem size for a launch whose largest stage has `stage_floats`.
void stream_launch_geometry(const StreamCfg& cfg, int32_t stage_floats, int* depth, size_t* smem) {
  const int n_groups = kStreamWarps / cfg.G;
  const size_t red = static_cast<size_t>(n_groups) * 2 * (cfg.G * cfg.T + cfg.T) * 4;
  const size_t budget = 220 * 1024 - red;
  const size_t per_stage = static_cast<size_t>(n_groups) * stage_floats * 4;
  int dpt = static_cast<int>(budget / per_stage);
  dpt = std::max(1, std::min(dpt, 8));
  *depth = dpt;
  *smem = stream_smem_bytes(cfg.vec, cfg.G, dpt, stage_floats);
}

// ---------------------------------------------------------------------------------------
// Streaming launches and their autotuning
// ---------------------------------------------------------------------------------------

static std::string stream_tune_key(const StreamCfg& cfg, bool coef, const pidk::StreamParams& sp,
                                   int32_t max_n, int64_t cells) {
  const int lg = log2_floor(cells);
  const pidk::EnsDesc& d = sp.one;   // iso and weight flags: those of the class's first ensemble
  char buf[160];
  std::snprintf(buf, sizeof(buf), "stream v%d k%d g%d s%d c%d iso%d w%d tma%d n%d m%d", cfg.vec,
                cfg.mpw, cfg.G,
                cfg.sub, coef ? 1 : 0, d.iso_mode != 0, d.w != nullptr, sp.use_tma,
                (max_n + 7) / 8 * 8, lg);
  return buf;
}

void load_tune_cache(pid_handle h) {
  const char* f = std::getenv("PID_AUTOTUNE_CACHE");
  if (!f || !*f) return;
  h->tune_file = f;
  FILE* fp = std::fopen(f, "r");
  if (!fp) return;
  char line[256];
  while (std::fgets(line, sizeof(line), fp)) {
    std::string l(line);
    const size_t bar = l.find('|');
    if (bar == std::string::npos) continue;
    int x = 0, d = 0;
    if (l.compare(0, 6, "shape ") == 0) {   // "shape <key>|<choice>"
      if (std::sscanf(l.c_str() + bar + 1, "%d", &x) == 1) h->shapes[l.substr(6, bar - 6)] = x;
      continue;
    }
    if (std::sscanf(l.c_str() + bar + 1, "%d %d", &x, &d) == 2) h->tuned[l.substr(0, bar)] = {x, d};
  }
  std::fclose(fp);
}

pid_status stream_launch(pid_handle h, StreamParams sp, const StreamCfg& cfg, bool coef, int grid,
                         int32_t max_n, int64_t cells, double bytes, cudaStream_t s) {
  int dmax;
  size_t smem;
  stream_launch_geometry(cfg, sp.stage_floats, &dmax, &smem);
  sp.depth = dmax;
  sp.xchg = default_xchg(cfg);
  const int ik = iso_kind(sp.one.iso_mode);
  const std::string key = stream_tune_key(cfg, coef, sp, max_n, cells);
  auto it = h->tuned.find(key);
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  cudaStreamIsCapturing(s, &cs);
  if (it == h->tuned.end() && h->autotune && cs == cudaStreamCaptureStatusNone) {
    // Candidates that leave the results unchanged: exchange scheme x ring depth.
    std::vector<std::pair<int, int>> cand;
    for (int x = 0; x <= (cfg.G > 2 ? 1 : 0); ++x)
      for (int d = dmax; d >= std::max(1, dmax - 1); --d) cand.push_back({x, d});
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    float best = 1e30f;
    std::pair<int, int> pick{sp.xchg, dmax};
    for (auto c : cand) {
      StreamParams t = sp;
      t.xchg = c.first;
      t.depth = c.second;
      const size_t sm = stream_smem_bytes(cfg.vec, cfg.G, c.second, sp.stage_floats);
      cudaError_t e = launch_stream(t, cfg.vec, cfg.mpw, cfg.G, ik, coef, grid, sm, s);  // warm-up
      if (e != cudaSuccess) { cudaEventDestroy(e0); cudaEventDestroy(e1); return cuda_fail(h, e, "tune"); }
      cudaEventRecord(e0, s);
      for (int r = 0; r < 3; ++r) launch_stream(t, cfg.vec, cfg.mpw, cfg.G, ik, coef, grid, sm, s);
      cudaEventRecord(e1, s);
      cudaEventSynchronize(e1);
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      if (ms < best) { best = ms; pick = c; }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    h->tuned[key] = pick;
    if (!h->tune_file.empty()) {
      if (FILE* fp = std::fopen(h->tune_file.c_str(), "a")) {
        std::fprintf(fp, "%s|%d %d\n", key.c_str(), pick.first, pick.second);
        std::fclose(fp);
      }
    }
    it = h->tuned.find(key);
  }
  if (it != h->tuned.end()) {
    sp.xchg = it->second.first;
    sp.depth = std::min(it->second.second, dmax);
    smem = stream_smem_bytes(cfg.vec, cfg.G, sp.depth, sp.stage_floats);
  }
  ProfScope ps(h, PID_KERNEL_STREAM, bytes, 0.0, s);
  cudaError_t e = launch_stream(sp, cfg.vec, cfg.mpw, cfg.G, ik, coef, grid, smem, s);
  if (e != cudaSuccess) return cuda_fail(h, e, "stream kernel launch");
  return PID_OK;
}

// ---------------------------------------------------------------------------------------
// Workspace
// ---------------------------------------------------------------------------------------

pid_status ensure_workspace(pid_handle h, size_t bytes, cudaStream_t s) {
  if (bytes <= h->ws_bytes) return PID_OK;
  if (h->budget && bytes + h->fixed_bytes > h->budget)
    return fail(h, PID_ERR_OOM, "workspace would exceed the handle's HBM budget");
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  cudaStreamIsCapturing(s, &cs);
  if (cs != cudaStreamCaptureStatusNone)
    return fail(h, PID_ERR_OOM, "workspace must grow, but the stream is being captured");
  if (h->ws) {
    cudaStreamSynchronize(s);
    cudaFree(h->ws);
    h->ws = nullptr;
    h->ws_bytes = 0;
  }
  const size_t alloc = round_up(static_cast<int64_t>(bytes), 1 << 20);
  cudaError_t e = cudaMalloc(&h->ws, alloc);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(h, PID_ERR_OOM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
  }
  h->ws_bytes = alloc;
  return PID_OK;
}

// ---------------------------------------------------------------------------------------
// Launch sequences for one ensemble (single calls)
// ---------------------------------------------------------------------------------------

static pid_status launch_stream_one(pid_handle h, EnsPlan& pl, const float* coef, cudaStream_t s) {
  StreamParams sp;
  std::memset(&sp, 0, sizeof(sp));
  sp.one = pl.desc;
  sp.one.coef = coef;
  sp.one.unit_begin = 0;
  sp.descs = nullptr;
  sp.n_ens = 1;
  sp.total_units = pl.desc.n_chunks;
  sp.one.work_begin = 0;
  sp.total_work = static_cast<int64_t>(pl.desc.N) * pl.desc.M;
  sp.G = pl.cfg.G;
  sp.sub = pl.cfg.sub;
  sp.use_tma = pl.use_tma ? 1 : (pl.cls ? 2 : 0);
  sp.err = h->err_word;
  sp.stage_floats = pl.stage_floats;
  if (coef) sp.one.umax = nullptr;
  sp.maxu = sp.one.umax != nullptr ? 1 : 0;
  const int n_groups = kStreamWarps / pl.cfg.G;
  int grid = std::min<int>(h->sms, (sp.total_units + n_groups - 1) / n_groups);
  grid = std::max(grid, 1);
  const double bytes = 4.0 * pl.desc.N * pl.desc.M + (pl.desc.w ? 4.0 * pl.desc.M : 0.0);
  return stream_launch(h, sp, pl.cfg, coef != nullptr, grid, pl.desc.N,
                       static_cast<int64_t>(pl.desc.N) * pl.desc.M, bytes, s);
}

pid_status launch_fin_one(pid_handle h, FinDesc fd, cudaStream_t s) {
  const int nb_stream = (2 * fd.N + 31) / 32;
  const int nb_gram = fd.kind == FIN_GRAM ? fin_gram_items(fd.N) : 0;
  fd.slices = std::max(1, std::min(nb_stream + nb_gram, 2 * h->sms));
  FinParams fp;
  std::memset(&fp, 0, sizeof(fp));
  fp.one = fd;
  fp.descs = nullptr;
  fp.n_ens = 1;
  fp.err = h->err_word;
  ProfScope ps(h, PID_KERNEL_FINALIZE, 0.0, 0.0, s);
  cudaError_t e = launch_finalize(fp, fd.slices, 1, s);
  if (e != cudaSuccess) return cuda_fail(h, e, "finalize launch");
  return PID_OK;
}

pid_status launch_member_coef_one(pid_handle h, const double* r, int64_t N, float* coef,
                                  cudaStream_t s) {
  ProfScope ps(h, PID_KERNEL_FINALIZE, 8.0 * N + 4.0 * N, 0.0, s);
  cudaError_t e = launch_member_coef(r, N, coef, h->err_word, s);
  if (e != cudaSuccess) return cuda_fail(h, e, "member coefficient launch");
  return PID_OK;
}

// Full PID on the tensor cores for 256 < N <= 512: the streaming pass gives the exact
// PID-mean sums (m_i, N A_i) that calibrate the Gram, the operand rows are staged in HBM,
// the tiled kernel forms the chunk partial Grams, and the finalisation does the rest.
static pid_status run_gram_tiled(pid_handle h, const EnsInput& in, EnsPlan& pl,
                                 const EnsOutputs& out, cudaStream_t s) {
  TiledPlan tp;
  pid_status st = plan_gram_tiled(h, in, &tp);
  if (st != PID_OK) return st;
  const size_t off_sums = pl.part_bytes;
  const size_t off_coef = off_sums + pl.sums_bytes;
  const size_t off_scale = off_coef + pl.coef_bytes;
  const size_t off_gpart = off_scale + kScaleBytes;
  const size_t off_op = off_gpart + tp.gpart_bytes;
  st = ensure_workspace(h, off_op + tp.op_bytes, s);
  if (st != PID_OK) return st;
  char* ws = static_cast<char*>(h->ws);
  double* part = reinterpret_cast<double*>(ws);
  float* gpart = reinterpret_cast<float*>(ws + off_gpart);
  pl.desc.part = part;
  // BF16 operands come straight from the streaming pass (its one-cell-per-lane classes,
  // which every N > 256 uses); split BF16 and E4M3 are staged by their own kernel.
  const bool fused = tp.prec == PID_BF16 && pl.cfg.vec == 1;
  if (fused) {
    pl.desc.op_out = reinterpret_cast<uint16_t*>(ws + off_op);
    pl.desc.op_ld = tp.ldo;
  }
  // E4M3 of soft masks: the streaming pass also reduces the per-member maxima of the scales
  float* scale = reinterpret_cast<float*>(ws + off_scale);
  const bool keys_from_stream = tp.prec == PID_FP8 && !in.is_field;
  if (keys_from_stream) {
    pl.desc.umax = scale_keys(scale);
    const cudaError_t e = cudaMemsetAsync(pl.desc.umax, 0, static_cast<size_t>(in.N) * 4, s);
    if (e != cudaSuccess) return cuda_fail(h, e, "scale key reset");
  }
  if ((st = launch_stream_one(h, pl, nullptr, s)) != PID_OK) return st;
  if (keys_from_stream && (st = launch_scales_from_keys(h, in.N, scale, s)) != PID_OK) return st;
  st = launch_gram_tiled_one(h, in, tp, ws + off_op, gpart, scale, !fused, s, keys_from_stream);
  if (st != PID_OK) return st;
  FinDesc fd;
  std::memset(&fd, 0, sizeof(fd));
  fd.kind = FIN_GRAM;
  fd.part = part;
  fd.N = pl.desc.N;
  fd.n_chunks = pl.desc.n_chunks;
  fd.gpart = gpart;
  fd.n_gchunks = tp.n_gchunks;
  fd.sums = reinterpret_cast<double*>(ws + off_sums);
  fd.coef = reinterpret_cast<float*>(ws + off_coef);
  fd.ticket = h->tickets;
  fd.depth = out.depth;
  fd.in_in = out.in_in;
  fd.in_out = out.in_out;
  fd.rank = out.rank;
  fd.mass = out.mass;
  fd.mean_depth = out.mean_depth;
  fd.P = out.P;
  fd.err_est = out.err_est;
  return launch_fin_one(h, fd, s);
}

pid_status run_single(pid_handle h, const EnsInput& in, const EnsOutputs& out, cudaStream_t s) {
  if (in.N > kMaxMembers) return run_blocked(h, in, out, s);
  EnsPlan pl;
  pid_status st = plan_stream(h, in, &pl);
  if (st != PID_OK) return st;
  const bool gram = in.mode == PID_MODE_FULL && in.precision != PID_FP32;
  const bool linear = in.mode == PID_MODE_FULL_LINEAR || (in.mode == PID_MODE_FULL && !gram);
  if (gram && in.N > kGramMaxN) return run_gram_tiled(h, in, pl, out, s);
  GramPlan gp;
  size_t part_bytes = pl.part_bytes, gram_bytes = 0;
  if (gram) {
    if ((st = plan_gram(h, in, &gp)) != PID_OK) return st;
    part_bytes = std::max(part_bytes, gp.part_bytes);
    gram_bytes = gp.gpart_bytes + kScaleBytes;  // partial Grams + the E4M3 member scales
  }
  const size_t need = part_bytes + pl.sums_bytes + pl.coef_bytes + gram_bytes;
  st = ensure_workspace(h, need, s);
  if (st != PID_OK) return st;
  char* ws = static_cast<char*>(h->ws);
  double* part = reinterpret_cast<double*>(ws);
  double* sums = reinterpret_cast<double*>(ws + part_bytes);
  float* coef = reinterpret_cast<float*>(ws + part_bytes + pl.sums_bytes);
  char* gbase = ws + part_bytes + pl.sums_bytes + pl.coef_bytes;
  pl.desc.part = part;

  FinDesc fd;
  std::memset(&fd, 0, sizeof(fd));
  fd.part = part;
  fd.N = pl.desc.N;
  fd.n_chunks = pl.desc.n_chunks;
  fd.sums = sums;
  fd.coef = coef;
  fd.ticket = h->tickets;
  fd.depth = out.depth;
  fd.in_in = out.in_in;
  fd.in_out = out.in_out;
  fd.rank = out.rank;
  fd.mass = out.mass;
  fd.mean_depth = out.mean_depth;

  if (gram) {
    float* gpart = reinterpret_cast<float*>(gbase + kScaleBytes);
    float* scale = reinterpret_cast<float*>(gbase);
    // E4M3 of soft masks needs a pass over the data for its member scales anyway: that pass
    // is the streaming kernel, which also forms the exact (m, A) partials, and the Gram pass
    // then skips them
    const bool own_pass = gp.prec == PID_FP8 && !in.is_field;
    if (own_pass) {
      pl.desc.umax = scale_keys(scale);
      const cudaError_t e = cudaMemsetAsync(pl.desc.umax, 0, static_cast<size_t>(in.N) * 4, s);
      if (e != cudaSuccess) return cuda_fail(h, e, "scale key reset");
      if ((st = launch_stream_one(h, pl, nullptr, s)) != PID_OK) return st;
      if ((st = launch_scales_from_keys(h, in.N, scale, s)) != PID_OK) return st;
      gp.exact = false;
    }
    st = launch_gram_one(h, in, gp, part, gpart, scale, s, own_pass);
    if (st != PID_OK) return st;
    fd.kind = FIN_GRAM;
    fd.n_chunks = own_pass ? pl.desc.n_chunks : gp.n_gchunks;
    fd.gpart = gpart;
    fd.n_gchunks = gp.n_gchunks;
    fd.P = out.P;
    fd.err_est = out.err_est;
    return launch_fin_one(h, fd, s);
  }
  if (in.member_weights) {   // PID-mean against the weighted mean contour: one pass
    if ((st = launch_member_coef_one(h, in.member_weights, in.N, coef, s)) != PID_OK) return st;
    if ((st = launch_stream_one(h, pl, coef, s)) != PID_OK) return st;
    fd.kind = FIN_WMEAN;
    return launch_fin_one(h, fd, s);
  }
  st = launch_stream_one(h, pl, nullptr, s);
  if (st != PID_OK) return st;
  if (!linear) {
    fd.kind = FIN_MEAN;
    return launch_fin_one(h, fd, s);
  }
  FinDesc f1 = fd;
  f1.kind = FIN_LIN1;
  f1.depth = nullptr; f1.in_in = nullptr; f1.in_out = nullptr; f1.rank = nullptr;
  st = launch_fin_one(h, f1, s);
  if (st != PID_OK) return st;
  st = launch_stream_one(h, pl, coef, s);
  if (st != PID_OK) return st;
  FinDesc f2 = fd;
  f2.kind = FIN_LIN2;
  f2.mass = nullptr; f2.mean_depth = nullptr;
  return launch_fin_one(h, f2, s);
}

}  // namespace pidh

using namespace pidh;

// =======================================================================================
// Exported C ABI
// =======================================================================================

namespace {

// Time `reps` runs of `fn` on `s` with CUDA events, after one untimed run.
template <typename Fn>
static float time_runs(cudaStream_t s, int reps, Fn&& fn, pid_status* st) {
  *st = fn();
  if (*st != PID_OK) return 0.f;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  cudaEventRecord(e0, s);
  for (int r = 0; r < reps && *st == PID_OK; ++r) *st = fn();
  cudaEventRecord(e1, s);
  cudaEventSynchronize(e1);
  float ms = 0.f;
  cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return ms;
}

static void record_shape(pid_handle h, const std::string& key, int choice) {
  h->shapes[key] = choice;
  if (h->tune_file.empty()) return;
  if (FILE* fp = std::fopen(h->tune_file.c_str(), "a")) {
    std::fprintf(fp, "shape %s|%d\n", key.c_str(), choice);
    std::fclose(fp);
  }
}

}  // namespace

extern "C" {

pid_status pid_gram_operands(int32_t precision, int64_t cells, int32_t want_matrix,
                             int32_t* operands) {
  if (!operands || precision < PID_FP32 || precision > PID_FP8 || cells < 0)
    return PID_ERR_INVALID_ARG;
  *operands = gram_operand_precision(precision, cells, want_matrix != 0);
  return PID_OK;
}

const char* pid_status_string(pid_status s) {
  switch (s) {
    case PID_OK: return "ok";
    case PID_ERR_INVALID_ARG: return "invalid argument";
    case PID_ERR_DOMAIN: return "input outside the domain (u not in [0,1], NaN, or w <= 0)";
    case PID_ERR_OOM: return "out of device memory or over the HBM budget";
    case PID_ERR_CUDA: return "CUDA error";
    case PID_ERR_TIMEOUT: return "bounded device wait timed out";
    case PID_ERR_BUSY: return "busy";
    case PID_ERR_CANCELLED: return "cancelled";
    case PID_ERR_UNSUPPORTED: return "unsupported size or option";
  }
  return "unknown status";
}

pid_status pid_create(pid_handle* out, int device, size_t hbm_budget_bytes) {
  if (!out) return PID_ERR_INVALID_ARG;
  *out = nullptr;
  int n = 0;
  cudaError_t e = cudaGetDeviceCount(&n);
  if (e != cudaSuccess || device < 0 || device >= n) {
    cudaGetLastError();
    return e != cudaSuccess ? PID_ERR_CUDA : PID_ERR_INVALID_ARG;
  }
  pid_handle h = new pid_handle_s();
  h->device = device;
  h->budget = hbm_budget_bytes;
  DeviceGuard g(device);
  cudaDeviceGetAttribute(&h->sms, cudaDevAttrMultiProcessorCount, device);
  int major = 0, minor = 0;
  cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, device);
  cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, device);
  h->cc = major * 10 + minor;
  int max_smem = 0;
  cudaDeviceGetAttribute(&max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, device);
  h->max_smem = max_smem;
  e = stream_kernels_init(max_smem);
  if (e == cudaSuccess && h->cc >= 100) e = gram_kernels_init(max_smem);
  if (e != cudaSuccess) {
    cudaGetLastError();
    delete h;
    return PID_ERR_CUDA;
  }
  h->fixed_bytes = sizeof(uint32_t) * (1 + kMaxTickets) + 256;
  e = cudaMalloc(&h->fixed, h->fixed_bytes);
  if (e != cudaSuccess) {
    delete h;
    return PID_ERR_OOM;
  }
  cudaMemset(h->fixed, 0, h->fixed_bytes);
  h->err_word = static_cast<uint32_t*>(h->fixed);
  load_tune_cache(h);
  h->tickets = reinterpret_cast<unsigned int*>(static_cast<char*>(h->fixed) + 256);
  e = cudaDeviceSynchronize();
  if (e != cudaSuccess) {
    cudaFree(h->fixed);
    delete h;
    return PID_ERR_CUDA;
  }
  *out = h;
  return PID_OK;
}

pid_status pid_destroy(pid_handle h) {
  if (!h) return PID_OK;
  {
    DeviceGuard g(h->device);
    destroy_batch_cache(h);
    prof_drain(h);
    for (cudaEvent_t e : h->event_pool) cudaEventDestroy(e);
    if (h->ws) cudaFree(h->ws);
    if (h->fixed) cudaFree(h->fixed);
    if (h->desc_dev) cudaFree(h->desc_dev);
    if (h->desc_host) cudaFreeHost(h->desc_host);
  }
  delete h;
  return PID_OK;
}

pid_status pid_sync(pid_handle h, void* stream) {
  if (!h) return PID_ERR_INVALID_ARG;
  DeviceGuard g(h->device);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaError_t e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(h, e, "cudaStreamSynchronize");
  uint32_t word = 0;
  e = cudaMemcpy(&word, h->err_word, sizeof(word), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(h, e, "reading the device error word");
  if (word == 0) return PID_OK;
  cudaMemset(h->fixed, 0, h->fixed_bytes);  // clear the word and any ticket left by an early exit
  cudaDeviceSynchronize();
  if (word & ERR_TIMEOUT) return fail(h, PID_ERR_TIMEOUT, "a bounded device wait ran out");
  if (word & ERR_DOMAIN) return fail(h, PID_ERR_DOMAIN, "validation: u outside [0,1], NaN, or w <= 0");
  return fail(h, PID_ERR_CUDA, "internal device error");
}

const char* pid_last_error(pid_handle h) { return h ? h->last_error.c_str() : "no handle"; }

pid_status pid_profile_enable(pid_handle h, int enable) {
  if (!h) return PID_ERR_INVALID_ARG;
  DeviceGuard g(h->device);
  prof_drain(h);
  for (auto& t : h->prof_total) t = pid_kernel_stats{};
  h->profiling = enable != 0;
  return PID_OK;
}

pid_status pid_autotune_enable(pid_handle h, int enable, int32_t* n_entries) {
  if (!h) return PID_ERR_INVALID_ARG;
  h->autotune = enable != 0;
  if (n_entries) *n_entries = static_cast<int32_t>(h->tuned.size());
  return PID_OK;
}

pid_status pid_autotune_shapes(pid_handle h, const pid_ensemble* ens, int32_t count, void* stream) {
  if (!h) return PID_ERR_INVALID_ARG;
  if (count < 0 || (count > 0 && !ens)) return fail(h, PID_ERR_INVALID_ARG, "bad ensemble array");
  DeviceGuard g(h->device);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  cudaStreamIsCapturing(s, &cs);
  if (cs != cudaStreamCaptureStatusNone)
    return fail(h, PID_ERR_INVALID_ARG, "tile shapes are tuned outside stream capture");
  for (int32_t k = 0; k < count; ++k) {
    const pid_ensemble& e = ens[k];
    pid_status st = check_shape(h, e.data, e.N, e.M, e.ld);
    if (st != PID_OK) return st;
    if (e.is_field && (st = check_iso(h, &e.iso)) != PID_OK) return st;
    if ((st = check_opt(h, &e.opt)) != PID_OK) return st;
    EnsInput in;
    in.data = e.data; in.N = e.N; in.M = e.M; in.ld = e.ld; in.w = e.w;
    in.is_field = e.is_field;
    if (e.is_field) in.iso = e.iso;
    in.mode = e.opt.mode;
    in.precision = e.opt.mode == PID_MODE_FULL ? gram_operand_precision(e.opt.precision, e.M, e.P != nullptr)
                                               : PID_FP32;
    // Streaming tile: the default class and the next two larger ones (more member slots per
    // warp, other cell widths), each timed over 3 runs of the PID-mean pass on this data.
    const std::string skey = stream_shape_key(in);
    if (!h->shapes.count(skey)) {
      const int def = default_stream_class(in.N);
      float best = 1e30f;
      int pick = def;
      for (int c = def; c < std::min(def + 3, kNumStreamClasses); ++c) {
        h->shapes[skey] = c;
        EnsPlan pl;
        if ((st = plan_stream(h, in, &pl)) != PID_OK) break;
        if ((st = ensure_workspace(h, pl.part_bytes, s)) != PID_OK) break;
        pl.desc.part = static_cast<double*>(h->ws);
        const float ms = time_runs(s, 3, [&] { return launch_stream_one(h, pl, nullptr, s); }, &st);
        if (st != PID_OK) break;
        if (ms < best) { best = ms; pick = c; }
      }
      if (st != PID_OK) { h->shapes.erase(skey); return st; }
      record_shape(h, skey, pick);
    }
    // Tensor-core Gram (fused tile, up to 256 members): the chunk of cells per partial Gram,
    // as planned, halved or doubled.
    if (in.mode == PID_MODE_FULL && in.precision != PID_FP32 && in.N <= kGramMaxN) {
      const std::string gkey = gram_shape_key(in);
      if (!h->shapes.count(gkey)) {
        float best = 1e30f;
        int pick = 0;
        for (int c : {0, 1, -1}) {
          h->shapes[gkey] = c;
          GramPlan gp;
          if ((st = plan_gram(h, in, &gp)) != PID_OK) break;
          const size_t need = gp.part_bytes + kScaleBytes + gp.gpart_bytes;
          if ((st = ensure_workspace(h, need, s)) != PID_OK) break;
          char* ws = static_cast<char*>(h->ws);
          double* part = reinterpret_cast<double*>(ws);
          float* scale = reinterpret_cast<float*>(ws + gp.part_bytes);
          float* gpart = reinterpret_cast<float*>(ws + gp.part_bytes + kScaleBytes);
          const float ms =
              time_runs(s, 3, [&] { return launch_gram_one(h, in, gp, part, gpart, scale, s); }, &st);
          if (st != PID_OK) break;
          if (ms < best) { best = ms; pick = c; }
        }
        if (st != PID_OK) { h->shapes.erase(gkey); return st; }
        record_shape(h, gkey, pick);
      }
    }
  }
  return pid_sync(h, stream);
}

int32_t pid_autotune_describe(pid_handle h, char* buf, int32_t cap) {
  if (!h) return -1;
  std::string out;
  for (const auto& kv : h->shapes) out += "shape " + kv.first + " -> " + std::to_string(kv.second) + "\n";
  for (const auto& kv : h->tuned)
    out += kv.first + " -> xchg " + std::to_string(kv.second.first) + " depth " +
           std::to_string(kv.second.second) + "\n";
  if (buf && cap > 0) {
    const size_t n = std::min<size_t>(out.size(), static_cast<size_t>(cap) - 1);
    std::memcpy(buf, out.data(), n);
    buf[n] = 0;
  }
  return static_cast<int32_t>(out.size());
}

pid_status pid_profile_read(pid_handle h, int kind, pid_kernel_stats* out) {
  if (!h || !out || kind < 0 || kind >= PID_KERNEL_KINDS) return PID_ERR_INVALID_ARG;
  DeviceGuard g(h->device);
  prof_drain(h);
  *out = h->prof_total[kind];
  return PID_OK;
}

size_t pid_workspace_bytes(pid_handle h) { return h ? h->ws_bytes : 0; }

static pid_status soft_masks_common(pid_handle h, const float* F, int64_t N, int64_t M, int64_t ld,
                                    const pid_iso* iso, void* U_out, int64_t ld_out, bool bf16,
                                    void* stream) {
  pid_status st = check_shape(h, F, N, M, ld);
  if (st == PID_ERR_UNSUPPORTED && N > kMaxMembers) st = PID_OK;  // elementwise: any N
  if (st != PID_OK) return st;
  if ((st = check_iso(h, iso)) != PID_OK) return st;
  if (!U_out || ld_out < M) return fail(h, PID_ERR_INVALID_ARG, "U_out must be non-NULL with ld_out >= M");
  DeviceGuard g(h->device);
  IsoParams p;
  std::memset(&p, 0, sizeof(p));
  p.F = F; p.U = U_out; p.N = N; p.M = M; p.ld = ld; p.ld_out = ld_out;
  p.out_bf16 = bf16 ? 1 : 0;
  iso_fill(iso, &p.iso_mode, &p.iso_mu, &p.iso_inv, &p.iso_t);
  ProfScope ps(h, PID_KERNEL_ISO, (bf16 ? 6.0 : 8.0) * N * M, 0.0, static_cast<cudaStream_t>(stream));
  cudaError_t e = launch_iso(p, static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return cuda_fail(h, e, "iso kernel launch");
  return PID_OK;
}

pid_status pid_soft_masks(pid_handle h, const float* F, int64_t N, int64_t M, int64_t ld,
                          const pid_iso* iso, float* U_out, int64_t ld_out, void* stream) {
  return soft_masks_common(h, F, N, M, ld, iso, U_out, ld_out, false, stream);
}

pid_status pid_soft_masks_bf16(pid_handle h, const float* F, int64_t N, int64_t M, int64_t ld,
                               const pid_iso* iso, uint16_t* U_out, int64_t ld_out, void* stream) {
  return soft_masks_common(h, F, N, M, ld, iso, U_out, ld_out, true, stream);
}

static pid_status common_call(pid_handle h, const float* data, int64_t N, int64_t M, int64_t ld,
                              const float* w, const pid_iso* iso, int mode, int prec, int validate,
                              const EnsOutputs& out, void* stream,
                              const double* member_weights = nullptr) {
  EnsInput in;
  in.member_weights = member_weights;
  in.data = data; in.N = N; in.M = M; in.ld = ld; in.w = w;
  in.is_field = iso != nullptr;
  if (iso) in.iso = *iso;
  in.mode = mode; in.precision = prec; in.validate = validate;
  DeviceGuard g(h->device);
  return run_single(h, in, out, static_cast<cudaStream_t>(stream));
}

pid_status pid_mean(pid_handle h, const float* U, int64_t N, int64_t M, int64_t ld,
                    const float* w, double* depth, double* in_in, double* in_out, int32_t* rank,
                    void* stream) {
  pid_status st = check_shape(h, U, N, M, ld, kMaxBlockedMembers);
  if (st != PID_OK) return st;
  EnsOutputs out{};
  out.depth = depth; out.in_in = in_in; out.in_out = in_out; out.rank = rank;
  return common_call(h, U, N, M, ld, w, nullptr, PID_MODE_MEAN, PID_FP32, 0, out, stream);
}

pid_status pid_full(pid_handle h, const float* U, int64_t N, int64_t M, int64_t ld,
                    const float* w, const pid_options* opt, double* depth, double* in_in,
                    double* in_out, int32_t* rank, double* P, double* err_est, void* stream) {
  pid_status st = check_shape(h, U, N, M, ld, kMaxBlockedMembers);
  if (st != PID_OK) return st;
  if ((st = check_opt(h, opt)) != PID_OK) return st;
  pid_options o{PID_MODE_FULL_LINEAR, PID_FP32, 0, 0};
  if (opt) o = *opt;
  if (o.mode == PID_MODE_MEAN) return fail(h, PID_ERR_INVALID_ARG, "pid_full needs a full-PID mode");
  EnsOutputs out{};
  out.depth = depth; out.in_in = in_in; out.in_out = in_out; out.rank = rank;
  out.P = P; out.err_est = err_est;
  const int prec = o.mode == PID_MODE_FULL ? gram_operand_precision(o.precision, M, P != nullptr) : o.precision;
  return common_call(h, U, N, M, ld, w, nullptr, o.mode, prec, o.validate, out, stream);
}

pid_status pid_from_fields(pid_handle h, const float* F, int64_t N, int64_t M, int64_t ld,
                           const float* w, const pid_iso* iso, const pid_options* opt,
                           double* depth, double* in_in, double* in_out, int32_t* rank,
                           void* stream) {
  pid_status st = check_shape(h, F, N, M, ld, kMaxBlockedMembers);
  if (st != PID_OK) return st;
  if ((st = check_iso(h, iso)) != PID_OK) return st;
  if ((st = check_opt(h, opt)) != PID_OK) return st;
  pid_options o{PID_MODE_MEAN, PID_FP32, 0, 0};
  if (opt) o = *opt;
  EnsOutputs out{};
  out.depth = depth; out.in_in = in_in; out.in_out = in_out; out.rank = rank;
  const int prec = o.mode == PID_MODE_FULL ? gram_operand_precision(o.precision, M, false) : o.precision;
  return common_call(h, F, N, M, ld, w, iso, o.mode, prec, o.validate, out, stream);
}

pid_status pid_mean_weighted(pid_handle h, const float* data, int64_t N, int64_t M, int64_t ld,
                             const float* w, const pid_iso* iso, const double* member_weights,
                             double* depth, double* in_in, double* in_out, int32_t* rank,
                             void* stream) {
  pid_status st = check_shape(h, data, N, M, ld, kMaxBlockedMembers);
  if (st != PID_OK) return st;
  if (iso && (st = check_iso(h, iso)) != PID_OK) return st;
  if (!member_weights) return fail(h, PID_ERR_INVALID_ARG, "member_weights must be non-NULL");
  EnsOutputs out{};
  out.depth = depth; out.in_in = in_in; out.in_out = in_out; out.rank = rank;
  return common_call(h, data, N, M, ld, w, iso, PID_MODE_MEAN, PID_FP32, 0, out, stream,
                     member_weights);
}

}  // extern "C"
