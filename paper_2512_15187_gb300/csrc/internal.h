// Internal descriptors shared by the host planner and the kernels (not part of the ABI).
#pragma once

#include <cuda.h>
#include <cstddef>
#include <cstdint>

namespace pidk {

// How a kernel turns an input element into a soft-mask value (Sec. 3.5).
enum IsoMode : int32_t {
  ISO_NONE = 0,        // data are soft masks already
  ISO_NORMAL = 1,      // u = erfc((F - mu) * inv) / 2, inv = +-1 / (sigma sqrt 2)
  ISO_STEP_BELOW = 2,  // sigma = 0, sub-level:   u = 1[F < t]
  ISO_STEP_ABOVE = 3,  // sigma = 0, super-level: u = 1[F > t]
  ISO_UNIFORM_BELOW = 4,  // u = clamp((mu - F) inv, 0, 1): q ~ U[mu - 1/inv, mu], P(F < q)
  ISO_UNIFORM_ABOVE = 5,  // u = clamp((F - mu) inv, 0, 1): q ~ U[mu, mu + 1/inv], P(F > q)
  ISO_LEVEL = 6           // u = max(0, 1 - |F - mu| inv)
};

// Padding rows read this sign of infinity so that the piecewise maps give exactly 0.
inline constexpr float iso_pad_sign(int32_t mode) {
  return (mode == ISO_STEP_ABOVE || mode == ISO_UNIFORM_ABOVE) ? -1.f : 1.f;
}

// Bits of the device error word.
enum ErrBits : uint32_t { ERR_DOMAIN = 1u, ERR_TIMEOUT = 2u, ERR_INTERNAL = 4u };

// Bounded device waits give up after this many nanoseconds of %globaltimer.
constexpr uint64_t kWaitTimeoutNs = 1000000000ull;

// Streaming pass: 16 consumer warps per CTA, grouped G warps per cell tile.
constexpr int kStreamWarps = 16;
constexpr int kStreamThreads = kStreamWarps * 32;
constexpr int kStreamProducerBytes = 96;   // shared-memory TMA cursor per group

// One ensemble as seen by the streaming kernel.
struct EnsDesc {  // 64-byte aligned through its CUtensorMap members
  CUtensorMap tmap;     // data [N][ld] float32; box {T cells, box_rows members}
                        // (n_cls > 0: residue class 0, see tmap_cls)
  CUtensorMap tmap_w;   // weights [M] float32; box {T}
  // Rows that are not 16-byte aligned, staged by TMA (n_cls > 0): members c, c + n_cls,
  // c + 2 n_cls, ... start at the same offset r_c = (data + c ld) mod 16 bytes and lie
  // n_cls ld floats apart (a multiple of 16 bytes; n_cls = 4 for odd ld, 2 for ld = 2 mod 4,
  // 1 for a base alone off the boundary). Class c's map has its base rounded down to
  // 16 bytes, cells x' = x + r_c / 4 (extent M + r_c / 4) and its members as rows; a box of
  // T + 4 cells at x' = x0 holds the aligned span around cells [x0, x0 + T) of each row.
  // tmap is class 0's map, tmap_cls[c - 1] class c's.
  CUtensorMap tmap_cls[3];
  const float* data;    // [N][ld]
  const float* w;       // [M] or nullptr (unit cell measure)
  const float* coef;    // [N] column-sum coefficients c_j; nullptr = 1/N for every member
  double* part;         // [n_chunks][2N] partial sums: m_i, then N A_i (pass 1) or B_i (pass 2)
  int64_t ld;
  int32_t N, M;
  int32_t chunk_cells;  // multiple of the stage width sub*T
  int32_t n_chunks;
  int32_t unit_begin;   // index of chunk 0 in the launch's flat unit list
  int32_t box_rows;     // members per TMA box (<= 256)
  int32_t n_boxes;      // boxes per stage along the member axis
  int32_t iso_mode;     // IsoMode
  float iso_mu, iso_inv, iso_t;
  int32_t validate;
  int32_t n_cls;        // 0: TMA rows (tmap) or cp.async spans; 1, 2, 4: class maps (above),
                        // each class taking n_boxes boxes of box_rows rows in a stage
  float* gpart;         // Gram launches: [n_chunks][N][N] float32 partial Gram (G_ij at j*N + i)
  const float* op_scale;  // Gram E4M3: [2N] per-member scales s_i, then 1/s_i (nullptr = 256)
  int64_t work_begin;   // member-cells of the launch's earlier ensembles (0 for the first)
  float* u_out;         // streaming pass 1 of a field: also store the soft masks here,
                        // [N][round_up(M, 4)] float32, for pass 2 to read (nullptr = no)
  uint16_t* op_out;     // first streaming pass: also store u sqrt(w) as BF16 tensor-core
                        // operands of the row-block-tiled Gram, [N][op_ld] (nullptr = no)
  int64_t op_ld;        // a multiple of 64
  unsigned int* umax;   // first streaming pass of soft masks: per-member maxima of u sqrt(w)
                        // as order-preserving keys (atomicMax; zeroed before), the E4M3
                        // scales of a Gram over the same data (nullptr = no)
};

struct StreamParams {
  EnsDesc one;             // used when descs == nullptr (single ensemble)
  const EnsDesc* descs;    // device array of n_ens descriptors (batch)
  int32_t n_ens;
  int32_t total_units;     // chunks over all ensembles
  int64_t total_work;      // sum of N * M over all ensembles (groups split it evenly)
  int32_t G;               // warps per group (1, 2, 4, 8, 16)
  int32_t depth;           // stages in each group's ring
  int32_t stage_floats;    // floats per stage; the last sub*T floats hold the weights
  int32_t use_tma;
  int32_t sub;             // register tiles of T cells per TMA stage
  int32_t xchg;            // column-sum exchange: 0 direct, 1 reduce-scatter (G > 2)
  uint32_t* err;           // device error word
  int32_t maxu;            // some descriptor has umax: the instantiation that tracks maxima
  int32_t pad;
};

// Tensor-core Gram pass: 16 warps convert tiles (the streaming arithmetic plus operand
// conversion); thread 0 also issues the tensor-core work and warps 0-3 drain it.
constexpr int kGramConvWarps = 16;
constexpr int kGramEpiWarps = 4;      // converter warps 0..3, one per TMEM lane quarter
constexpr int kGramThreads = kGramConvWarps * 32;
constexpr int kGramMaxN = 256;        // two M = 128 tensor-core row blocks (the wide tile)
constexpr int kGramNarrowMaxN = 128;  // one M = 128 row block
constexpr int kGramTiledMaxN = 512;   // row-block-tiled Gram over operands staged in HBM
constexpr int kGramMaxMpw = 16;       // members per converter warp (the 256-row wide tile)

struct GramParams {
  EnsDesc one;
  const EnsDesc* descs;
  int32_t n_ens;
  int32_t total_units;
  int64_t total_work;    // sum of N * M over all ensembles (groups split it evenly)
  int32_t dF;            // FP32 stages in the TMA ring
  int32_t dO;            // operand stages
  int32_t stage_floats;  // floats per FP32 stage (rows x TS + TS)
  int32_t TS;            // cells per FP32 stage: 128, or 64 for the wide tile (N > 128)
  int32_t xchg;
  int32_t use_tma;       // 0: converters read FP32 directly (rows not 16-byte aligned)
  uint32_t* err;
  int32_t exact;         // 1: the converters also form the exact PID-mean sums (m, A);
                         // 0: soft masks whose sums come from a streaming pass
  int32_t pad;
};

// Row-block-tiled Gram (256 < N <= 512): operand rows staged in HBM, then one CTA per
// (cell chunk, 128-row block, column tile).
struct OperandParams {
  const float* F;          // [N][ld] soft masks, or fields mapped by iso_mode
  const float* w;          // [M] cell measures or nullptr
  void* hi;                // [N][ldo] BF16 bit patterns, or E4M3 bytes
  void* lo;                // split BF16: [N][ldo] low parts; else nullptr
  const float* op_scale;   // E4M3: [2N] per-member scales s_i, then 1/s_i (nullptr = 256)
  int64_t ld, ldo;         // ldo: a multiple of 64 elements
  int32_t N, M;
  int32_t iso_mode;
  float iso_mu, iso_inv, iso_t;
  int32_t vec_ok;          // rows and weights 16-byte aligned: 4-cell vector loads
  int32_t pad;
};

// One tile of a cell chunk: the 128-row blocks lb0 .. lb0 + nlb - 1 are loaded per K-block
// (plus block xa when xa >= 0), and each segment multiplies row block ra[s] against the nb[s]
// column blocks from cb[s] on, into accumulator columns from col[s] on (at most 512 in all).
struct TileDesc {
  int8_t lb0, nlb, xa, nseg;
  int8_t ra[2], cb[2], nb[2];
  int16_t col[2];
};
constexpr int kMaxTiles = 8;

struct TiledParams {
  CUtensorMap op_hi;       // [N][ldo] operands; box {128 bytes of cells, 128 rows}, 128-byte swizzle
  CUtensorMap op_lo;       // split BF16: the low parts
  float* gpart;            // [n_chunks][N][N] FP32 partial Grams (G_ij at j*N + i)
  const float* op_scale;   // E4M3: [2N] per-member scales s_i, then 1/s_i (nullptr = 256)
  int32_t N, M, R;         // members, cells, 128-row blocks
  int32_t chunk_cells;     // multiple of 128
  int32_t n_chunks, tiles_per_chunk;
  int32_t stages;          // operand stages in the ring
  int32_t slots;           // 128-row blocks per stage and plane
  TileDesc tiles[kMaxTiles];
  uint32_t* err;
};

// Finalisation of one ensemble: fixed-order FP64 reduction of the chunk partials, then
// inclusion fractions, depth and rank.
enum FinKind : int32_t {
  FIN_MEAN = 0,   // PID-mean outputs from (m, A)
  FIN_LIN1 = 1,   // first pass of exact full PID: keep (m, A), emit coefficients 1/(N m_j)
  FIN_LIN2 = 2,   // second pass: B_i = IN_out(i); full-PID outputs
  FIN_GRAM = 3,   // full PID from the Gram partials plus (m, A)
  FIN_WMEAN = 4   // PID-mean against the weighted mean contour sum_j c_j u_j (coef = c)
};

struct FinDesc {
  const double* part;      // [n_chunks][2N]
  const float* gpart;      // FIN_GRAM: [n_gchunks][N][N] float32 Gram partials (col-major)
  int32_t N, n_chunks;
  int32_t n_gchunks, kind;
  int32_t slices;          // CTAs working on this ensemble
  int32_t pad0;
  double* sums;            // workspace [4N] FP64 m, A, (second-pass m), B; then FP32 G [N*N], C0 [N*N]
  float* coef;             // FIN_LIN1 writes [N] coefficients here; FIN_WMEAN reads c_j
  unsigned int* ticket;    // zero before the launch; the last CTA resets it
  double* depth;
  double* in_in;
  double* in_out;
  int32_t* rank;
  double* mass;
  double* mean_depth;
  double* P;               // FIN_GRAM: [N][N] inclusion matrix
  double* err_est;         // FIN_GRAM: max |IN_in(Gram) - A_i/m_i|
};

struct FinParams {
  FinDesc one;
  const FinDesc* descs;
  int32_t n_ens;
  int32_t pad;
  uint32_t* err;
};

struct IsoParams {
  const float* F;
  void* U;                 // float32 [N][ld_out], or bfloat16 bit patterns when out_bf16
  int64_t N, M, ld, ld_out;
  int32_t iso_mode;
  float iso_mu, iso_inv, iso_t;
  int32_t out_bf16;
};

// Work items of the finalisation's Gram reduction: 32 warps each sum one 32-column block
// of the [n_gchunks][N*N] partials, so an item covers 1024 columns.
constexpr int fin_gram_items(int N) { return (N * N + 1023) / 1024; }

// Launchers (stream.cu).
// Kernel family of an isovalue mode: 0 none, 1 normal, 2 step (either direction) and the
// piecewise-linear maps (uniform isovalue, level map), chosen at run time inside the kernel.
inline int iso_kind(int32_t iso_mode) { return iso_mode == ISO_NONE ? 0 : (iso_mode == ISO_NORMAL ? 1 : 2); }

cudaError_t launch_stream(const StreamParams& p, int vec, int mpw, int G, int iso_kind, bool coef,
                          int grid, size_t smem, cudaStream_t s);
cudaError_t launch_finalize(const FinParams& p, int grid_x, int grid_y, cudaStream_t s);
cudaError_t launch_iso(const IsoParams& p, cudaStream_t s);
cudaError_t launch_member_coef(const double* r, int64_t N, float* coef, uint32_t* err,
                               cudaStream_t s);
size_t stream_smem_bytes(int vec, int G, int depth, int stage_floats);
size_t gram_smem_bytes(int G, int mpw, bool wide, int prec, int dF, int dO, int stage_floats);
cudaError_t launch_gram(const GramParams& p, int G, int mpw, bool wide, int prec, int iso_kind,
                        int grid, size_t smem, cudaStream_t s);
cudaError_t gram_kernels_init(int max_smem);
// Per-member E4M3 operand scales (gram_kernel.cu): s_i is the largest power of two with
// max_x u_i(x) sqrt(w_x) s_i <= 448, the largest finite E4M3 value.
struct ScaleDesc {
  const float* data;       // [N][ld] soft masks, or fields mapped by iso_mode
  const float* w;          // [M] cell measures or nullptr
  int64_t ld;
  int32_t N, M;
  int32_t iso_mode;
  float iso_mu, iso_inv, iso_t;
  int32_t vec_ok;          // rows and weights 16-byte aligned: 4-cell vector loads
  int32_t proxy;           // unweighted fields: reduce the proxy of F (see iso_proxy)
  int32_t from_keys;       // the maxima are already reduced into the region's keys
  int32_t segs;            // CTAs per member of the max pass (segs * N <= kScaleMaxSlots)
  int32_t seg_cells;       // cells per CTA (a multiple of 1024)
  int32_t block_begin;     // the ensemble's first CTA in the max pass
  float* scale;            // scale region: [2N] out (s_i, then 1/s_i), then keys or CTA maxima
};
// Ensembles per scale launch (the descriptors travel as kernel parameters).
constexpr int kScaleBatch = 32;
struct ScaleBatchParams {
  int32_t n;               // descriptors
  int32_t total_blocks;    // CTAs of the max pass (descriptors with from_keys = 0)
  ScaleDesc d[kScaleBatch];
};
// The per-member maxima of every descriptor that has no keys yet (one launch, each CTA
// writing the maximum of its segment), then every descriptor's scales (one launch).
cudaError_t launch_member_scales(const ScaleBatchParams& p, cudaStream_t s);
// Workspace of one ensemble's scales: [2N] floats, then from float 2 * 512 on either [N]
// reduction keys (maxima reduced by a streaming pass) or [N][segs] CTA maxima.
constexpr size_t kScaleBytes = 8192;
constexpr int kScaleMaxSlots = static_cast<int>(kScaleBytes / 4) - 2 * kGramTiledMaxN;
// Row-block-tiled Gram (gram_tiled.cu).
cudaError_t launch_gram_operands(const OperandParams& p, int prec, cudaStream_t s);
cudaError_t launch_gram_tiled(const TiledParams& p, int prec, int grid, size_t smem, cudaStream_t s);
cudaError_t gram_tiled_init(int max_smem);
size_t gram_tiled_smem_bytes(int prec, int slots, int stages);
// The tiles of one cell chunk for R row blocks: whole rows of the upper block triangle
// (short rows paired) when `wide`, else at most two column blocks per tile.
int gram_tiles(int R, bool wide, TileDesc* out);
cudaError_t stream_kernels_init(int max_smem);

}  // namespace pidk
