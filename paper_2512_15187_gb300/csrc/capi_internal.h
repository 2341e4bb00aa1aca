// Host-side internals of the C ABI (handle, plans). Not part of the public interface.
#pragma once

#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>
#include <map>
#include <string>
#include <vector>

#include "../../include/pid.h"
#include "internal.h"

namespace pidh {

constexpr int64_t kMaxMembers = 512;   // largest N of the fused single-pass kernels
constexpr int64_t kMaxBlockedMembers = int64_t(1) << 22;   // single calls, member-blocked path
constexpr int kMaxTickets = 8192;      // ensembles per batch (one finalisation ticket each)
constexpr int64_t kMaxMatrixMembers = 65536;   // members of pid_depth_from_matrix
constexpr int kMaxSpacetimeSteps = 65536;   // time steps of one space-time ensemble

struct BatchCache;  // batch.cu

struct ProfRecord {
  int kind;
  cudaEvent_t start, stop;
  double bytes, flops;
};

// Brackets one kernel launch with events when profiling is on (RAII on the host side).
// While the library records a batch into a CUDA graph with profiling on, the events become
// event-record nodes of the graph (re-armed with fresh events at every replay).
class ProfScope {
 public:
  ProfScope(pid_handle h, int kind, double bytes, double flops, cudaStream_t s);
  ~ProfScope();
 private:
  pid_handle h_;
  int idx_ = -1;
  bool captured_ = false;
  cudaStream_t s_;
};
cudaEvent_t prof_event(pid_handle h);   // a timing event from the handle's pool

}  // namespace pidh

struct pid_handle_s {
  int device = 0;
  int sms = 148;
  int cc = 0;
  int max_smem = 0;
  size_t budget = 0;
  void* ws = nullptr;          // growable workspace
  size_t ws_bytes = 0;
  void* fixed = nullptr;       // error word + tickets (zeroed at creation)
  size_t fixed_bytes = 0;
  uint32_t* err_word = nullptr;
  unsigned int* tickets = nullptr;
  void* desc_dev = nullptr;    // batch descriptor arrays (device)
  void* desc_host = nullptr;   // pinned mirror
  size_t desc_bytes = 0;
  pidh::BatchCache* batch = nullptr;
  std::string last_error;
  bool profiling = false;
  std::vector<pidh::ProfRecord> prof_pending;
  std::vector<cudaEvent_t> event_pool;
  pid_kernel_stats prof_total[PID_KERNEL_KINDS] = {};
  bool prof_graph = false;     // recording a profiled batch graph: time captured launches
  std::vector<pidh::ProfRecord> prof_captured;   // their events, turned into graph nodes
  bool autotune = false;
  std::map<std::string, std::pair<int, int>> tuned;  // key -> (exchange scheme, ring depth)
  std::map<std::string, int> shapes;   // shape key -> tile choice (pid_autotune_shapes)
  std::string tune_file;
};

namespace pidh {

struct StreamCfg {
  int vec;  // cells per lane per register tile (4, 2, 1)
  int G;    // warps per group
  int T;    // cells per register tile (32 * vec)
  int sub;  // register tiles per TMA stage (1: a stage is one register tile)
  int mpw;  // members per warp: the class holds G * mpw member rows
};

struct EnsInput {
  const float* data = nullptr;
  int64_t N = 0, M = 0, ld = 0;
  const float* w = nullptr;
  int is_field = 0;
  pid_iso iso{};
  int mode = PID_MODE_MEAN;
  int precision = PID_FP32;
  int validate = 0;
  const double* member_weights = nullptr;  // weighted mean contour (PID_MODE_MEAN only)
};

struct EnsOutputs {
  double* depth = nullptr;
  double* in_in = nullptr;
  double* in_out = nullptr;
  int32_t* rank = nullptr;
  double* mass = nullptr;
  double* mean_depth = nullptr;
  double* P = nullptr;
  double* err_est = nullptr;
};

struct EnsPlan {
  pidk::EnsDesc desc;
  StreamCfg cfg;
  bool use_tma;            // rows 16-byte aligned: TMA boxes of the rows
  bool cls;                // rows not aligned, staged by TMA through residue-class maps
  int32_t stage_floats;
  size_t part_bytes, sums_bytes, coef_bytes;
};

struct GramPlan {
  pidk::EnsDesc desc;      // tensor maps and chunking of the Gram pass
  int prec = 0;            // PID_BF16, PID_SPLIT_BF16 or PID_FP8
  bool tma = true;         // rows 16-byte aligned: FP32 tiles staged by TMA
  int G = 16;              // warps per group (8: two groups per CTA for N <= 64)
  int mpw = 8;             // members per warp: narrow 8 (6 for N <= 48, 64 < N <= 96),
                           // wide 16 (12 for N <= 192)
  bool wide = false;       // 128 < N <= 256: 16 warps on 256 rows, two M = 128 row blocks
  int TS = 128;            // cells per FP32 stage (64 for the wide tile)
  int n_gchunks = 0;
  int64_t chunk_cells = 0;
  int32_t stage_floats = 0;
  int dF = 2, dO = 2;
  size_t smem = 0;
  bool exact = true;       // false: soft masks whose (m, A) come from a streaming pass
  size_t gpart_bytes = 0;  // [n_gchunks][N][N] float32
  size_t part_bytes = 0;   // [n_gchunks][2N] float64 (exact PID-mean partials)
  double bytes = 0, flops = 0;
};

// Row-block-tiled Gram for 256 < N <= 512 (gram.cu, kernels in gram_tiled.cu): the
// operand rows are staged in HBM and each CTA computes one tile of one cell chunk.
struct TiledPlan {
  int prec = 0;            // PID_BF16, PID_SPLIT_BF16 or PID_FP8
  int R = 0;               // 128-row blocks
  int tiles = 0;           // tiles per chunk (gram_tiles)
  pidk::TileDesc tile[pidk::kMaxTiles];
  int slots = 0;           // 128-row blocks per stage and plane
  int64_t ldo = 0;         // operand row stride in elements (a multiple of 64)
  int elem_bytes = 2;      // 2 (BF16) or 1 (E4M3)
  int planes = 1;          // 2 for split BF16
  int64_t chunk_cells = 0;
  int n_gchunks = 0;
  int stages = 2;
  size_t smem = 0;
  size_t op_bytes = 0;     // operand planes
  size_t gpart_bytes = 0;  // [n_gchunks][N][N] float32
  double op_rw_bytes = 0, gemm_bytes = 0, flops = 0;
};

class DeviceGuard {
 public:
  explicit DeviceGuard(int dev);
  ~DeviceGuard();
 private:
  int prev_ = 0, dev_ = 0;
};

pid_status fail(pid_handle h, pid_status s, const std::string& msg);
pid_status cuda_fail(pid_handle h, cudaError_t e, const char* where);
StreamCfg stream_cfg(int64_t N);
// The streaming tile class of an ensemble: the tuned choice of its shape, else the default.
StreamCfg stream_cfg_for(pid_handle h, const EnsInput& in);
std::string gram_shape_key(const EnsInput& in);
void iso_fill(const pid_iso* iso, int32_t* mode, float* mu, float* inv, float* t);
pid_status check_iso(pid_handle h, const pid_iso* iso);
pid_status check_shape(pid_handle h, const void* data, int64_t N, int64_t M, int64_t ld,
                       int64_t max_n = kMaxMembers);
pid_status launch_member_coef_one(pid_handle h, const double* r, int64_t N, float* coef,
                                  cudaStream_t s);
pid_status launch_fin_one(pid_handle h, pidk::FinDesc fd, cudaStream_t s);
pid_status run_blocked(pid_handle h, const EnsInput& in, const EnsOutputs& out, cudaStream_t s);
pid_status check_opt(pid_handle h, const pid_options* o);
pid_status plan_stream(pid_handle h, const EnsInput& in, EnsPlan* pl);
void stream_launch_geometry(const StreamCfg& cfg, int32_t stage_floats, int* depth, size_t* smem);
int default_xchg(const StreamCfg& cfg);
// Launch the streaming kernel with tuned (or default) exchange scheme and ring depth.
pid_status stream_launch(pid_handle h, pidk::StreamParams sp, const StreamCfg& cfg, bool coef,
                         int grid, int32_t max_n, int64_t cells, double bytes, cudaStream_t s);
void load_tune_cache(pid_handle h);
pid_status ensure_workspace(pid_handle h, size_t bytes, cudaStream_t s);
pid_status run_single(pid_handle h, const EnsInput& in, const EnsOutputs& out, cudaStream_t s);
bool encode_2d(CUtensorMap* m, const void* base, uint64_t inner, uint64_t outer, uint64_t row_bytes,
               uint32_t box_inner, uint32_t box_outer);
bool encode_1d(CUtensorMap* m, const void* base, uint64_t n, uint32_t box);
bool encode_2d_sw128(CUtensorMap* m, const void* base, int elem_bytes, uint64_t inner,
                     uint64_t outer, uint64_t row_bytes);

// E4M3 operands carry 3 mantissa bits: per-element rounding up to 2^-4 of the value, noise
// that averages over the cells of a member (~0.04 / sqrt(cells)). Depths and IN_out meet the
// 1e-3 bar from kFp8MinCells cells on; single inclusions P_ij are not averaged over
// members. A PID_FP8 request with fewer cells, or one that asks for P, therefore computes
// the Gram from BF16 operands.
constexpr int64_t kFp8MinCells = 4096;
inline int gram_operand_precision(int prec, int64_t cells, bool want_matrix) {
  return (prec == PID_FP8 && (want_matrix || cells < kFp8MinCells)) ? PID_BF16 : prec;
}

// gram.cu
// Per-member E4M3 operand scales of one ensemble into `region` (pidk::kScaleBytes of
// workspace: [2N] scales and inverses, then reduction keys or CTA maxima).
pid_status launch_member_scales_one(pid_handle h, const EnsInput& in, float* region, cudaStream_t s);
// The scales of several ensembles, up to pidk::kScaleBatch per pair of launches; from_keys:
// a streaming pass already reduced the maxima into the region's keys.
struct ScaleJob {
  EnsInput in;
  float* region;
  bool from_keys;
};
pid_status launch_member_scales_many(pid_handle h, const std::vector<ScaleJob>& jobs, cudaStream_t s);
// The reduction keys inside a scale region, and the scales from keys a streaming pass filled.
inline unsigned int* scale_keys(float* region) {
  return reinterpret_cast<unsigned int*>(region + 2 * pidk::kGramTiledMaxN);
}
pid_status launch_scales_from_keys(pid_handle h, int64_t N, float* region, cudaStream_t s);
pid_status plan_gram(pid_handle h, const EnsInput& in, GramPlan* gp);
void gram_geometry(pid_handle h, int G, int mpw, bool wide, int prec, int32_t stage_floats,
                   int* dF, int* dO, size_t* smem);
pid_status launch_gram_one(pid_handle h, const EnsInput& in, GramPlan& gp, double* part,
                           float* gpart, float* scale, cudaStream_t s, bool scales_ready = false);
// Gram launch over `count` device descriptors (part / gpart / op_scale already set).
pid_status launch_gram_batch(pid_handle h, const GramPlan& gp, const pidk::EnsDesc* descs,
                             int count, int total_units, int64_t total_work, int iso_mode,
                             double bytes, double flops,
                             cudaStream_t s);

pid_status plan_gram_tiled(pid_handle h, const EnsInput& in, TiledPlan* tp);
// Operand staging (unless the streaming pass already wrote the BF16 operands) and the
// tiled Gram launch; `op` holds tp.op_bytes, `gpart` tp.gpart_bytes, `scale`
// pidk::kScaleBytes (E4M3 member scales).
// scales_ready: the E4M3 scales in `scale` were already computed (from streaming-pass keys).
pid_status launch_gram_tiled_one(pid_handle h, const EnsInput& in, const TiledPlan& tp, void* op,
                                 float* gpart, float* scale, bool stage_operands, cudaStream_t s,
                                 bool scales_ready = false);

// batch.cu
void destroy_batch_cache(pid_handle h);
// Record batches into CUDA graphs and replay them while the layout repeats (default on).
void batch_use_graphs(pid_handle h, bool on);
// Let BF16 / split-BF16 Gram items take the exact (m, A) partials of a first-pass sibling
// over the same soft masks (default on); off keeps every item bitwise equal to its single
// call whatever it is batched with.
void batch_share_sums(pid_handle h, bool on);

}  // namespace pidh
