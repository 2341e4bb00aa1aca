// Host side of the tensor-core Gram path (kernel in gram_kernel.cu): planning, workspace
// sizing and launches, for single calls and for batches.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>

#include "capi_internal.h"
#include "internal.h"

using namespace pidk;

namespace pidh {

static int64_t rup(int64_t a, int64_t b) { return (a + b - 1) / b * b; }

pid_status plan_gram(pid_handle h, const EnsInput& in, GramPlan* gp) {
  *gp = GramPlan{};
  if (in.N > kGramMaxN)
    return fail(h, PID_ERR_UNSUPPORTED, "the fused tensor-core Gram takes N <= 256");
  const uintptr_t a = reinterpret_cast<uintptr_t>(in.data);
  gp->tma = in.ld % 4 == 0 && a % 16 == 0 && (!in.w || reinterpret_cast<uintptr_t>(in.w) % 16 == 0);
  gp->prec = in.precision;
  gp->G = in.N <= 64 ? 8 : 16;        // two independent 8-warp groups when N <= 64
  gp->wide = in.N > kGramNarrowMaxN;   // two M = 128 row blocks, 64-cell FP32 stages
  // 6 members per warp when they hold the ensemble (48 or 96 rows): the converters then
  // skip the rows a tile of 8 per warp would leave empty
  gp->mpw = gp->wide ? (in.N <= 192 ? 12 : (in.N <= 208 ? 13 : 16))
                     : ((in.N <= 48 || (in.N > 64 && in.N <= 96)) ? 6 : 8);
  gp->TS = gp->wide ? 64 : 128;
  // Chunks (one FP32 partial Gram each) of 32 to 256 operand stages: every chunk costs a
  // TMEM drain, an N x N partial written and read back, and the MMA pipeline's ramp, so a
  // few large chunks per ensemble beat one per group (batches supply the parallelism); the
  // upper bound keeps the exact FP32 PID-mean sums of a chunk short enough for 1e-6.
  // Small ensembles (up to 2^16 cells) take chunks from 4 stages (512 cells) on: their few
  // long chunks would otherwise run as a latency-bound chain on a handful of SMs.
  const int64_t groups = static_cast<int64_t>(h->sms) * (kGramConvWarps / gp->G);
  const int64_t min_chunk = in.M <= 65536 ? 4 * 128 : 32 * 128;
  int64_t chunk = rup((in.M + groups - 1) / groups, 128);
  chunk = std::max<int64_t>(chunk, std::min<int64_t>(rup(in.M, 128), min_chunk));
  chunk = std::min<int64_t>(chunk, 256 * 128);
  // A tuned shape may halve or double the chunk (pid_autotune_shapes), within the same bounds.
  if (!h->shapes.empty()) {
    auto it = h->shapes.find(gram_shape_key(in));
    if (it != h->shapes.end() && it->second != 0) {
      chunk = it->second > 0 ? 2 * chunk : rup(chunk / 2, 128);
      chunk = std::min<int64_t>(std::max<int64_t>(chunk, std::min<int64_t>(rup(in.M, 128), min_chunk)),
                                256 * 128);
    }
  }
  gp->chunk_cells = chunk;
  gp->n_gchunks = static_cast<int>((in.M + chunk - 1) / chunk);

  EnsDesc& d = gp->desc;
  std::memset(&d, 0, sizeof(d));
  d.data = in.data;
  d.w = in.w;
  d.ld = in.ld;
  d.N = static_cast<int32_t>(in.N);
  d.M = static_cast<int32_t>(in.M);
  d.chunk_cells = static_cast<int32_t>(chunk);
  d.n_chunks = gp->n_gchunks;
  d.n_boxes = 1;
  d.box_rows = static_cast<int32_t>(in.N);
  iso_fill(in.is_field ? &in.iso : nullptr, &d.iso_mode, &d.iso_mu, &d.iso_inv, &d.iso_t);
  d.validate = in.validate;
  if (gp->tma &&
      (!encode_2d(&d.tmap, in.data, static_cast<uint64_t>(in.M), static_cast<uint64_t>(in.N),
                  static_cast<uint64_t>(in.ld) * 4, static_cast<uint32_t>(gp->TS),
                  static_cast<uint32_t>(in.N)) ||
       (in.w && !encode_1d(&d.tmap_w, in.w, static_cast<uint64_t>(in.M), static_cast<uint32_t>(gp->TS)))))
    return fail(h, PID_ERR_CUDA, "tensor map encoding failed");

  // Without TMA the FP32 ring is unused: keep one minimal stage.
  gp->stage_floats = gp->tma ? static_cast<int32_t>(rup(in.N * gp->TS + gp->TS, 32)) : 32;
  gp->gpart_bytes = rup(static_cast<int64_t>(gp->n_gchunks) * in.N * in.N * 4, 256);
  gp->part_bytes = rup(static_cast<int64_t>(gp->n_gchunks) * 2 * in.N * 8, 256);
  gram_geometry(h, gp->G, gp->mpw, gp->wide, gp->prec, gp->stage_floats, &gp->dF, &gp->dO,
                &gp->smem);
  gp->flops = (in.precision == PID_SPLIT_BF16 ? 3.0 : 1.0) * 2.0 * static_cast<double>(in.N) *
              in.N * in.M;
  gp->bytes = 4.0 * in.N * in.M + (in.w ? 4.0 * in.M : 0.0);
  return PID_OK;
}

// Ring depths that fit the shared memory: at least two FP32 stages, then as many operand
// stages as fit (at most four), then the FP32 ring deepened to at most six stages.
void gram_geometry(pid_handle h, int G, int mpw, bool wide, int prec, int32_t stage_floats,
                   int* dF, int* dO, size_t* smem) {
  const size_t cap = static_cast<size_t>(h->max_smem > 0 ? h->max_smem : 232448);
  int f = 2, o = 4;
  while (o > 1 && gram_smem_bytes(G, mpw, wide, prec, f, o, stage_floats) > cap) --o;
  while (f > 1 && gram_smem_bytes(G, mpw, wide, prec, f, o, stage_floats) > cap) --f;
  while (f < 6 && gram_smem_bytes(G, mpw, wide, prec, f + 1, o, stage_floats) <= cap) ++f;
  *dF = f;
  *dO = o;
  *smem = gram_smem_bytes(G, mpw, wide, prec, f, o, stage_floats);
}

pid_status launch_member_scales_many(pid_handle h, const std::vector<ScaleJob>& jobs, cudaStream_t s) {
  for (size_t j0 = 0; j0 < jobs.size(); j0 += kScaleBatch) {
    ScaleBatchParams sb;
    std::memset(&sb, 0, sizeof(sb));
    double bytes = 0.0;
    const size_t j1 = std::min(jobs.size(), j0 + kScaleBatch);
    // member rows of this launch that need a max pass: about four CTAs per SM over all of
    // them (the maxima are exact whatever the segments, so the scales do not depend on it)
    int64_t rows = 0;
    for (size_t j = j0; j < j1; ++j)
      if (!jobs[j].from_keys) rows += jobs[j].in.N;
    const int64_t want = std::max<int64_t>(1, (4LL * h->sms + rows - 1) / std::max<int64_t>(1, rows));
    for (size_t j = j0; j < j1; ++j) {
      const EnsInput& in = jobs[j].in;
      ScaleDesc& d = sb.d[sb.n++];
      d.data = in.data;
      d.w = in.w;
      d.ld = in.ld;
      d.N = static_cast<int32_t>(in.N);
      d.M = static_cast<int32_t>(in.M);
      iso_fill(in.is_field ? &in.iso : nullptr, &d.iso_mode, &d.iso_mu, &d.iso_inv, &d.iso_t);
      d.vec_ok = in.ld % 4 == 0 && reinterpret_cast<uintptr_t>(in.data) % 16 == 0 &&
                 (!in.w || reinterpret_cast<uintptr_t>(in.w) % 16 == 0);
      d.proxy = in.is_field && in.w == nullptr;
      d.scale = jobs[j].region;
      d.from_keys = jobs[j].from_keys ? 1 : 0;
      if (d.from_keys) {
        bytes += 4.0 * in.N;
        continue;
      }
      // segments of at least 4096 cells, the CTA maxima within the region
      int64_t segs = std::max<int64_t>(
          1, std::min({want, (in.M + 4095) / 4096, static_cast<int64_t>(kScaleMaxSlots) / in.N}));
      d.seg_cells = static_cast<int32_t>(((in.M + segs - 1) / segs + 1023) / 1024 * 1024);
      segs = (in.M + d.seg_cells - 1) / d.seg_cells;
      d.segs = static_cast<int32_t>(segs);
      d.block_begin = sb.total_blocks;
      sb.total_blocks += static_cast<int32_t>(segs * in.N);
      bytes += 4.0 * in.N * in.M + (in.w ? 4.0 * in.M : 0.0);
    }
    ProfScope ps(h, PID_KERNEL_SCALE, bytes, 0.0, s);
    const cudaError_t e = launch_member_scales(sb, s);
    if (e != cudaSuccess) return cuda_fail(h, e, "E4M3 member scale launch");
  }
  return PID_OK;
}

pid_status launch_member_scales_one(pid_handle h, const EnsInput& in, float* region, cudaStream_t s) {
  return launch_member_scales_many(h, {ScaleJob{in, region, false}}, s);
}

pid_status launch_scales_from_keys(pid_handle h, int64_t N, float* region, cudaStream_t s) {
  EnsInput in;
  in.N = N;
  return launch_member_scales_many(h, {ScaleJob{in, region, true}}, s);
}

static int gram_kind(int prec) {
  return prec == PID_SPLIT_BF16 ? PID_KERNEL_GRAM_SPLIT : (prec == PID_FP8 ? PID_KERNEL_GRAM_FP8 : PID_KERNEL_GRAM);
}

static pid_status gram_launch(pid_handle h, const GramParams& gpar, int G, int mpw, bool wide,
                              int prec, int iso_mode, int grid, size_t smem, double bytes,
                              double flops, cudaStream_t s) {
  ProfScope ps(h, gram_kind(prec), bytes, flops, s);
  cudaError_t e = launch_gram(gpar, G, mpw, wide, prec, iso_kind(iso_mode), grid, smem, s);
  if (e != cudaSuccess) return cuda_fail(h, e, "Gram kernel launch");
  return PID_OK;
}

pid_status launch_gram_one(pid_handle h, const EnsInput& in, GramPlan& gp, double* part,
                           float* gpart, float* scale, cudaStream_t s, bool scales_ready) {
  GramParams gpar;
  std::memset(&gpar, 0, sizeof(gpar));
  gpar.one = gp.desc;
  gpar.one.part = part;
  gpar.one.gpart = gpart;
  gpar.one.op_scale = nullptr;
  if (gp.prec == PID_FP8) {
    if (!scales_ready) {
      const pid_status st = launch_member_scales_one(h, in, scale, s);
      if (st != PID_OK) return st;
    }
    gpar.one.op_scale = scale;
  }
  gpar.n_ens = 1;
  gpar.total_units = gp.n_gchunks;
  gpar.one.work_begin = 0;
  gpar.total_work = static_cast<int64_t>(in.N) * in.M;
  gpar.dF = gp.dF;
  gpar.dO = gp.dO;
  gpar.stage_floats = gp.stage_floats;
  gpar.TS = gp.TS;
  gpar.xchg = gp.G >= 16 ? 1 : 0;   // one group barrier per stage for 8-warp groups
  gpar.use_tma = gp.tma ? 1 : 0;
  gpar.err = h->err_word;
  gpar.exact = gp.exact ? 1 : 0;
  const int ng = kGramConvWarps / gp.G;
  const int grid = std::max(1, std::min(h->sms, (gp.n_gchunks + ng - 1) / ng));
  return gram_launch(h, gpar, gp.G, gp.mpw, gp.wide, gp.prec, gp.desc.iso_mode, grid, gp.smem,
                     gp.bytes, gp.flops, s);
}

pid_status launch_gram_batch(pid_handle h, const GramPlan& gp, const EnsDesc* descs, int count,
                             int total_units, int64_t total_work, int iso_mode, double bytes,
                             double flops, cudaStream_t s) {
  GramParams gpar;
  std::memset(&gpar, 0, sizeof(gpar));
  gpar.descs = descs;
  gpar.n_ens = count;
  gpar.total_units = total_units;
  gpar.total_work = total_work;
  gpar.dF = gp.dF;
  gpar.dO = gp.dO;
  gpar.stage_floats = gp.stage_floats;
  gpar.TS = gp.TS;
  gpar.xchg = gp.G >= 16 ? 1 : 0;
  gpar.use_tma = gp.tma ? 1 : 0;
  gpar.err = h->err_word;
  gpar.exact = gp.exact ? 1 : 0;
  const int ng = kGramConvWarps / gp.G;
  const int grid = std::max(1, std::min(h->sms, (total_units + ng - 1) / ng));
  return gram_launch(h, gpar, gp.G, gp.mpw, gp.wide, gp.prec, iso_mode, grid, gp.smem, bytes,
                     flops, s);
}

// ---------------------------------------------------------------------------------------
// Row-block-tiled Gram (256 < N <= 512)
// ---------------------------------------------------------------------------------------

pid_status plan_gram_tiled(pid_handle h, const EnsInput& in, TiledPlan* tp) {
  *tp = TiledPlan{};
  if (in.N > kGramTiledMaxN)
    return fail(h, PID_ERR_UNSUPPORTED,
                "the tensor-core Gram takes N <= 512; use PID_MODE_FULL_LINEAR");
  tp->prec = in.precision;
  tp->R = static_cast<int>((in.N + 127) / 128);
  // BF16 and E4M3: whole rows of the block triangle per tile (up to 4 blocks per stage);
  // split BF16 carries two planes per block: whole rows for 3 row blocks (two stages of
  // 96 KB), else tiles of at most two column blocks
  tp->tiles = gram_tiles(tp->R, in.precision != PID_SPLIT_BF16 || tp->R == 3, tp->tile);
  tp->slots = 0;
  for (int t = 0; t < tp->tiles; ++t)
    tp->slots = std::max(tp->slots, tp->tile[t].nlb + (tp->tile[t].xa >= 0 ? 1 : 0));
  tp->elem_bytes = in.precision == PID_FP8 ? 1 : 2;
  tp->planes = in.precision == PID_SPLIT_BF16 ? 2 : 1;
  tp->ldo = rup(in.M, 64);
  // Chunks: about two waves of CTAs over the SMs; every chunk adds an N x N FP32 partial
  // (written by the tiles, read by the finalisation), so chunks stay at 4096 cells or more.
  const int64_t target = std::max<int64_t>(1, 2 * static_cast<int64_t>(h->sms) / tp->tiles);
  int64_t chunk = rup((in.M + target - 1) / target, 256);
  chunk = std::min<int64_t>(std::max<int64_t>(chunk, 4096), 65536);
  tp->chunk_cells = chunk;
  tp->n_gchunks = static_cast<int>((in.M + chunk - 1) / chunk);
  const size_t cap = static_cast<size_t>(h->max_smem > 0 ? h->max_smem : 232448);
  tp->stages = 6;
  while (tp->stages > 2 && gram_tiled_smem_bytes(tp->prec, tp->slots, tp->stages) > cap) --tp->stages;
  tp->smem = gram_tiled_smem_bytes(tp->prec, tp->slots, tp->stages);
  if (tp->smem > cap) return fail(h, PID_ERR_UNSUPPORTED, "tiled Gram stages do not fit shared memory");
  const int64_t plane = rup(static_cast<int64_t>(in.N) * tp->ldo * tp->elem_bytes, 1024);
  tp->op_bytes = static_cast<size_t>(tp->planes * plane);
  tp->gpart_bytes = rup(static_cast<int64_t>(tp->n_gchunks) * in.N * in.N * 4, 256);
  const double nm = static_cast<double>(in.N) * in.M;
  tp->op_rw_bytes = 4.0 * nm + (in.w ? 4.0 * in.M : 0.0) + nm * tp->elem_bytes * tp->planes;
  tp->gemm_bytes = nm * tp->elem_bytes * tp->planes;
  // useful products: the upper block triangle of 128-row blocks, as issued
  double blocks = 0;
  for (int r = 0; r < tp->R; ++r) blocks += tp->R - r;
  tp->flops = (in.precision == PID_SPLIT_BF16 ? 3.0 : 1.0) * 2.0 * blocks * 128.0 * 128.0 * in.M;
  return PID_OK;
}

pid_status launch_gram_tiled_one(pid_handle h, const EnsInput& in, const TiledPlan& tp, void* op,
                                 float* gpart, float* scale, bool stage_operands, cudaStream_t s,
                                 bool scales_ready) {
  const float* op_scale = nullptr;
  if (tp.prec == PID_FP8) {
    if (!scales_ready) {
      const pid_status st = launch_member_scales_one(h, in, scale, s);
      if (st != PID_OK) return st;
    }
    op_scale = scale;
  }
  const int64_t plane = rup(static_cast<int64_t>(in.N) * tp.ldo * tp.elem_bytes, 1024);
  char* hi = static_cast<char*>(op);
  char* lo = tp.planes == 2 ? hi + plane : nullptr;

  OperandParams op_p;
  std::memset(&op_p, 0, sizeof(op_p));
  op_p.F = in.data;
  op_p.w = in.w;
  op_p.hi = hi;
  op_p.lo = lo;
  op_p.op_scale = op_scale;
  op_p.ld = in.ld;
  op_p.ldo = tp.ldo;
  op_p.N = static_cast<int32_t>(in.N);
  op_p.M = static_cast<int32_t>(in.M);
  iso_fill(in.is_field ? &in.iso : nullptr, &op_p.iso_mode, &op_p.iso_mu, &op_p.iso_inv, &op_p.iso_t);
  op_p.vec_ok = in.ld % 4 == 0 && reinterpret_cast<uintptr_t>(in.data) % 16 == 0 &&
                (!in.w || reinterpret_cast<uintptr_t>(in.w) % 16 == 0);
  if (stage_operands) {
    ProfScope ps(h, PID_KERNEL_OPERANDS, tp.op_rw_bytes, 0.0, s);
    cudaError_t e = launch_gram_operands(op_p, tp.prec, s);
    if (e != cudaSuccess) return cuda_fail(h, e, "Gram operand launch");
  }

  TiledParams tpar;
  std::memset(&tpar, 0, sizeof(tpar));
  const uint64_t row_bytes = static_cast<uint64_t>(tp.ldo) * tp.elem_bytes;
  if (!encode_2d_sw128(&tpar.op_hi, hi, tp.elem_bytes, static_cast<uint64_t>(in.M),
                       static_cast<uint64_t>(in.N), row_bytes) ||
      (lo && !encode_2d_sw128(&tpar.op_lo, lo, tp.elem_bytes, static_cast<uint64_t>(in.M),
                              static_cast<uint64_t>(in.N), row_bytes)))
    return fail(h, PID_ERR_CUDA, "tensor map encoding failed");
  if (!lo) tpar.op_lo = tpar.op_hi;
  tpar.gpart = gpart;
  tpar.op_scale = op_scale;
  tpar.N = static_cast<int32_t>(in.N);
  tpar.M = static_cast<int32_t>(in.M);
  tpar.R = tp.R;
  tpar.chunk_cells = static_cast<int32_t>(tp.chunk_cells);
  tpar.n_chunks = tp.n_gchunks;
  tpar.tiles_per_chunk = tp.tiles;
  tpar.stages = tp.stages;
  tpar.slots = tp.slots;
  for (int t = 0; t < tp.tiles; ++t) tpar.tiles[t] = tp.tile[t];
  tpar.err = h->err_word;
  ProfScope ps(h, gram_kind(tp.prec), tp.gemm_bytes, tp.flops, s);
  cudaError_t e = launch_gram_tiled(tpar, tp.prec, tp.n_gchunks * tp.tiles, tp.smem, s);
  if (e != cudaSuccess) return cuda_fail(h, e, "tiled Gram launch");
  return PID_OK;
}

}  // namespace pidh
