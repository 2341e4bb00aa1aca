// Batched execution: many ensembles of uneven N and M per call.
//
// Ensembles are grouped by tile class (a function of N alone, so each ensemble keeps the
// arithmetic order of a single call and its results are bitwise identical to it). Each
// class runs as one persistent launch of the streaming kernel over the flat list of all its
// (ensemble, chunk) units; one finalisation launch then serves every ensemble. The exact
// full PID adds a second streaming launch per class and a second finalisation. Full PID on
// tensor cores runs one Gram launch per class instead of the first streaming pass; above 256
// members the Gram is row-block-tiled (operands staged in HBM, one launch pair per ensemble)
// and the ensemble's exact PID-mean sums come from the first streaming pass of its class.
// Items over the same data share first passes: a Gram item of soft masks takes the (m, A)
// of a PID-mean or exact item's pass, and a PID-mean item those of an exact item's pass.
//
// The whole sequence (descriptor upload + launches) is recorded once into a CUDA graph and
// replayed while the caller submits the same batch layout (same pointers and shapes).
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <map>
#include <vector>

#include "capi_internal.h"
#include "internal.h"

using namespace pidk;

namespace pidh {

struct BatchCache {
  std::vector<unsigned char> key;     // serialized batch layout of the cached graph
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  void* host_desc = nullptr;          // pinned descriptor image read by the graph's memcpy
  size_t host_bytes = 0;
  bool use_graphs = true;
  bool share_sums = true;             // BF16 / split Gram items may take a sibling's (m, A)
  int64_t replays = 0;
  // A graph recorded with profiling on brackets every kernel with two event-record nodes;
  // each replay sets fresh events on them, so every replay's launches are timed.
  struct ProfNodes { cudaGraphNode_t start, stop; int kind; double bytes, flops; };
  std::vector<ProfNodes> prof;
  // Side streams on which the independent launches of one phase (the streaming classes of a
  // pass, the Gram classes) run side by side, forked from and joined back to the caller's
  // stream by events (in a recorded graph: parallel branches).
  static constexpr int kSide = 4;
  cudaStream_t side[kSide] = {};
  cudaEvent_t fork_ev = nullptr;
  cudaEvent_t join_ev[kSide] = {};
};

static pid_status ensure_side_streams(pid_handle h, BatchCache* c) {
  if (c->fork_ev) return PID_OK;
  for (int k = 0; k < BatchCache::kSide; ++k) {
    if (cudaStreamCreateWithFlags(&c->side[k], cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->join_ev[k], cudaEventDisableTiming) != cudaSuccess) {
      cudaGetLastError();
      return fail(h, PID_ERR_CUDA, "batch side streams");
    }
  }
  if (cudaEventCreateWithFlags(&c->fork_ev, cudaEventDisableTiming) != cudaSuccess) {
    cudaGetLastError();
    return fail(h, PID_ERR_CUDA, "batch side streams");
  }
  return PID_OK;
}

// Fresh events on the graph's timing nodes, queued for the profiler, before a replay.
static pid_status arm_graph_profiling(pid_handle h, BatchCache* c) {
  for (const auto& pn : c->prof) {
    ProfRecord r{pn.kind, prof_event(h), prof_event(h), pn.bytes, pn.flops};
    if (cudaGraphExecEventRecordNodeSetEvent(c->exec, pn.start, r.start) != cudaSuccess ||
        cudaGraphExecEventRecordNodeSetEvent(c->exec, pn.stop, r.stop) != cudaSuccess) {
      cudaGetLastError();
      return fail(h, PID_ERR_CUDA, "re-arming the timing nodes of the batch graph");
    }
    h->prof_pending.push_back(r);
  }
  return PID_OK;
}

// The event-record nodes that the captured ProfScopes left in `graph`.
static pid_status collect_graph_profiling(pid_handle h, cudaGraph_t graph, BatchCache* c) {
  c->prof.clear();
  size_t n = 0;
  if (cudaGraphGetNodes(graph, nullptr, &n) != cudaSuccess) return fail(h, PID_ERR_CUDA, "graph nodes");
  std::vector<cudaGraphNode_t> nodes(n);
  if (n && cudaGraphGetNodes(graph, nodes.data(), &n) != cudaSuccess)
    return fail(h, PID_ERR_CUDA, "graph nodes");
  std::map<cudaEvent_t, cudaGraphNode_t> by_event;
  for (cudaGraphNode_t nd : nodes) {
    cudaGraphNodeType t;
    cudaEvent_t e = nullptr;
    if (cudaGraphNodeGetType(nd, &t) == cudaSuccess && t == cudaGraphNodeTypeEventRecord &&
        cudaGraphEventRecordNodeGetEvent(nd, &e) == cudaSuccess)
      by_event[e] = nd;
  }
  for (const ProfRecord& r : h->prof_captured) {
    auto a = by_event.find(r.start), b = by_event.find(r.stop);
    if (a == by_event.end() || b == by_event.end())
      return fail(h, PID_ERR_CUDA, "a timing node of the batch graph is missing");
    c->prof.push_back({a->second, b->second, r.kind, r.bytes, r.flops});
    h->event_pool.push_back(r.start);   // the graph's nodes get fresh events at every replay
    h->event_pool.push_back(r.stop);
  }
  h->prof_captured.clear();
  return PID_OK;
}

void batch_use_graphs(pid_handle h, bool on) {
  if (!h->batch) h->batch = new BatchCache();
  h->batch->use_graphs = on;
}

void batch_share_sums(pid_handle h, bool on) {
  if (!h->batch) h->batch = new BatchCache();
  h->batch->share_sums = on;
}

void destroy_batch_cache(pid_handle h) {
  if (!h->batch) return;
  BatchCache* c = h->batch;
  if (c->exec) cudaGraphExecDestroy(c->exec);
  if (c->graph) cudaGraphDestroy(c->graph);
  if (c->host_desc) cudaFreeHost(c->host_desc);
  for (int k = 0; k < BatchCache::kSide; ++k) {
    if (c->side[k]) cudaStreamDestroy(c->side[k]);
    if (c->join_ev[k]) cudaEventDestroy(c->join_ev[k]);
  }
  if (c->fork_ev) cudaEventDestroy(c->fork_ev);
  delete c;
  h->batch = nullptr;
}

static int64_t align_up(int64_t a, int64_t b) { return (a + b - 1) / b * b; }

// How a streaming plan stages its rows: 1 = TMA boxes of aligned rows, 2 = TMA boxes through
// residue-class maps (rows not 16-byte aligned), 0 = cp.async spans. Each mode launches
// apart.
static int stage_mode(const EnsPlan& p) { return p.use_tma ? 1 : (p.cls ? 2 : 0); }

// One persistent launch per key. Ensembles staged in different ways (stage_mode) launch
// apart, so that one unaligned ensemble does not slow down its whole class.
struct ClassKey {
  int vec, G, coef, iso, tma, mpw;
  bool operator<(const ClassKey& o) const {
    if (tma != o.tma) return tma < o.tma;
    if (mpw != o.mpw) return mpw < o.mpw;
    if (vec != o.vec) return vec < o.vec;
    if (G != o.G) return G < o.G;
    if (coef != o.coef) return coef < o.coef;
    return iso < o.iso;
  }
};

struct Launch {
  enum Kind { STREAM, GRAM, FIN, TILED } kind;
  int first, count;        // descriptor range (stream/gram: EnsDesc index; fin: FinDesc index)
  StreamCfg cfg;
  bool coef = false;
  bool tma = true;
  bool cls = true;         // STREAM: every row staged through residue-class maps
  int32_t stage_floats = 0;
  int32_t total_units = 0;
  int32_t max_n = 0;
  int64_t cells = 0;     // sum of N * M over the launch (tuning bucket)
  int grid_x = 1;
  double bytes = 0, flops = 0;
  GramPlan gp;             // GRAM launches
  int iso_mode = 0;
  // E4M3 member scales to compute before the Gram launch: by a pass of their own, or from
  // the keys that a first streaming pass over the same soft masks reduced (from_keys)
  struct Scale { EnsInput in; float* out; bool from_keys; };
  std::vector<Scale> scales;
  bool maxu = false;       // STREAM: some descriptor reduces E4M3 maxima (umax)
  // TILED launches (one ensemble or time step): operand staging + tiled Gram
  EnsInput in;
  TiledPlan tp;
  void* op = nullptr;
  bool stage = true;       // stage the operands (else the streaming pass wrote them)
  float* gpart = nullptr;
  float* scale = nullptr;
  bool scale_from_keys = false;   // E4M3: the streaming pass reduced the maxima
};

struct BatchPlan {
  std::vector<EnsDesc> sdesc;   // streaming descriptors (pass 1 then pass 2), grouped by class
  std::vector<FinDesc> fdesc;   // finalisation descriptors (phase 1 then phase 2)
  std::vector<Launch> launches;
  std::vector<std::pair<unsigned int*, int64_t>> key_resets;   // E4M3 keys zeroed first
  size_t desc_bytes = 0;
  size_t work_bytes = 0;
};

static pid_status to_input(pid_handle h, const pid_ensemble& e, EnsInput* in) {
  pid_status st = check_shape(h, e.data, e.N, e.M, e.ld);
  if (st != PID_OK) return st;
  if (e.is_field != 0 && e.is_field != 1) return fail(h, PID_ERR_INVALID_ARG, "is_field must be 0 or 1");
  if (e.is_field && (st = check_iso(h, &e.iso)) != PID_OK) return st;
  if ((st = check_opt(h, &e.opt)) != PID_OK) return st;
  if (e.reserved != 0) return fail(h, PID_ERR_INVALID_ARG, "reserved must be 0");
  in->data = e.data; in->N = e.N; in->M = e.M; in->ld = e.ld; in->w = e.w;
  in->is_field = e.is_field;
  if (e.is_field) in->iso = e.iso;
  in->mode = e.opt.mode;
  in->precision = e.opt.precision;
  in->validate = e.opt.validate;
  return PID_OK;
}

// Lay out descriptors and workspace for the batch. Pointers are offsets from `base`.
// store_u: for exact full PID of a field, pass 1 also writes the soft masks into the
// workspace and pass 2 streams them (instead of repeating the isovalue map); and the
// streaming pass of a BF16 tiled-Gram ensemble writes its operands into a buffer of its own
// (instead of a staging pass into one shared buffer).
// steps > 1: the `count` == `steps` records are the time steps of ONE space-time ensemble
// (4D PID: the cells (x, t) of all steps concatenated). Step t writes its chunk partials
// right after those of step t - 1, and one finalisation reduces all of them.
static pid_status plan_batch(pid_handle h, const pid_ensemble* ens, int count, char* base,
                             bool store_u, BatchPlan* bp, int steps = 1) {
  const bool st4 = steps > 1;
  auto owner = [&](int e) { return st4 ? 0 : e; };
  std::vector<EnsInput> in(count);
  std::vector<EnsPlan> pl(count);
  std::vector<GramPlan> gp(count);
  std::vector<TiledPlan> tp(count);
  std::vector<int> is_gram(count, 0), is_lin(count, 0), stored(count, 0), tiled(count, 0);
  std::vector<EnsPlan> pl2(count);   // pass 2 over the stored soft masks
  for (int e = 0; e < count; ++e) {
    pid_status st = to_input(h, ens[e], &in[e]);
    if (st != PID_OK) return st;
    // E4M3 requests below its cell floor, or asking for P, take BF16 operands (the Gram of
    // a space-time ensemble sums over the cells of all its steps)
    if (in[e].mode == PID_MODE_FULL)
      in[e].precision = gram_operand_precision(in[e].precision, in[e].M * steps,
                                               ens[owner(e)].P != nullptr);
    if ((st = plan_stream(h, in[e], &pl[e])) != PID_OK) return st;
    is_gram[e] = in[e].mode == PID_MODE_FULL && in[e].precision != PID_FP32;
    is_lin[e] = in[e].mode == PID_MODE_FULL_LINEAR || (in[e].mode == PID_MODE_FULL && !is_gram[e]);
    tiled[e] = is_gram[e] && in[e].N > kGramMaxN;
    if (tiled[e]) {
      if ((st = plan_gram_tiled(h, in[e], &tp[e])) != PID_OK) return st;
    } else if (is_gram[e] && (st = plan_gram(h, in[e], &gp[e])) != PID_OK) {
      return st;
    }
    stored[e] = store_u && is_lin[e] && in[e].is_field;
  }
  if (st4) {
    for (int e = 1; e < count; ++e) {
      if (in[e].N != in[0].N || in[e].M != in[0].M || in[e].w != in[0].w ||
          in[e].is_field != in[0].is_field || in[e].mode != in[0].mode ||
          in[e].precision != in[0].precision || pl[e].desc.n_chunks != pl[0].desc.n_chunks ||
          (is_gram[e] && gp[e].n_gchunks != gp[0].n_gchunks) ||
          (tiled[e] && tp[e].n_gchunks != tp[0].n_gchunks))
        return fail(h, PID_ERR_INVALID_ARG, "the time steps of a space-time ensemble differ");
    }
  }
  // A fused-Gram ensemble of soft masks takes its exact PID-mean partials (m, A) from a
  // first streaming pass over the same data where the batch has one (a PID-mean or exact
  // full-PID item of the same masks: same pointer, shape, stride and cell measures), and its
  // converters then skip that arithmetic. An E4M3 ensemble without such a sibling runs a
  // streaming pass of its own, as a single call does, which also reduces its member scales.
  // E4M3 items always take a first pass (their own, or an identical sibling's: the same
  // plan, hence bitwise the same partials); BF16 and split-BF16 items take a sibling's
  // partials unless the handle keeps every item bitwise equal to its single call (serving).
  const bool share = !h->batch || h->batch->share_sums;
  // A PID-mean item whose masks (or fields) the batch also streams for an exact full PID
  // takes that item's first-pass partials instead of a pass of its own: both passes sum
  // m_i and N A_i (Eq. 6, 16; the exact full PID's IN_in is the same A_i / m_i, Eq. 17), and
  // with the same data, cell measures, isovalue map and tile plan they sum them in the same
  // order, so the shared partials are bitwise those the item's own pass would give.
  std::vector<int> mshare(count, -1);
  if (!st4 && share) {
    auto same_iso = [&](const EnsInput& a, const EnsInput& b) {
      return !a.is_field || (a.iso.kind == b.iso.kind && a.iso.superlevel == b.iso.superlevel &&
                             a.iso.mu == b.iso.mu && a.iso.sigma == b.iso.sigma);
    };
    for (int e = 0; e < count; ++e) {
      if (is_gram[e] || is_lin[e]) continue;
      for (int f = 0; f < count && mshare[e] < 0; ++f) {
        if (!is_lin[f] || in[f].data != in[e].data || in[f].N != in[e].N || in[f].M != in[e].M ||
            in[f].ld != in[e].ld || in[f].w != in[e].w || in[f].is_field != in[e].is_field ||
            !same_iso(in[f], in[e]) || in[f].validate < in[e].validate)
          continue;
        const EnsPlan &a = pl[e], &b = pl[f];
        if (a.cfg.vec == b.cfg.vec && a.cfg.G == b.cfg.G && a.cfg.mpw == b.cfg.mpw &&
            a.cfg.sub == b.cfg.sub && a.use_tma == b.use_tma && a.cls == b.cls &&
            a.desc.n_chunks == b.desc.n_chunks && a.desc.chunk_cells == b.desc.chunk_cells &&
            a.desc.iso_mode == b.desc.iso_mode && a.desc.iso_mu == b.desc.iso_mu &&
            a.desc.iso_inv == b.desc.iso_inv && a.desc.iso_t == b.desc.iso_t)
          mshare[e] = f;
      }
    }
  }
  std::vector<int> sib(count, -1), own_pass(count, 0);
  if (!st4) {
    for (int e = 0; e < count; ++e) {
      if (!is_gram[e] || tiled[e] || in[e].is_field) continue;
      if (!share && in[e].precision != PID_FP8) continue;
      for (int f = 0; f < count && sib[e] < 0; ++f) {
        // (a PID-mean item that shares an exact item's pass runs none of its own)
        if (f != e && !(is_gram[f] && !tiled[f]) && !in[f].is_field && mshare[f] < 0 &&
            in[f].data == in[e].data &&
            in[f].N == in[e].N && in[f].M == in[e].M && in[f].ld == in[e].ld && in[f].w == in[e].w)
          sib[e] = f;
      }
      if (sib[e] < 0 && in[e].precision == PID_FP8) {
        sib[e] = e;
        own_pass[e] = 1;
      }
      gp[e].exact = sib[e] < 0;
    }
  }
  // Workspace: descriptors first (64-byte aligned tensor maps), then per-ensemble buffers.
  std::map<ClassKey, std::vector<int>> pass1, pass2;
  // ((((precision x 2 + TMA) x 2 + wide) x 32 + group size) x 32 + members per warp,
  //  isovalue kind)
  std::map<std::pair<int, int>, std::vector<int>> gram_cls;
  for (int e = 0; e < count; ++e) {
    if (is_gram[e] && !tiled[e]) {
      gram_cls[{((((gp[e].prec * 2 + (gp[e].tma ? 1 : 0)) * 2 + (gp[e].wide ? 1 : 0)) * 32 +
                  gp[e].G) * 32 + gp[e].mpw) * 2 + (gp[e].exact ? 1 : 0),
                iso_kind(gp[e].desc.iso_mode)}]
          .push_back(e);
      if (own_pass[e])
        pass1[{pl[e].cfg.vec, pl[e].cfg.G, 0, iso_kind(pl[e].desc.iso_mode), stage_mode(pl[e]),
               pl[e].cfg.mpw}].push_back(e);
    } else {
      const int ik = iso_kind(pl[e].desc.iso_mode);
      if (mshare[e] < 0)
        pass1[{pl[e].cfg.vec, pl[e].cfg.G, 0, ik, stage_mode(pl[e]), pl[e].cfg.mpw}].push_back(e);
      if (is_lin[e]) {
        // stored soft masks are 16-byte aligned rows, read through TMA in pass 2
        const int tma2 = stored[e] ? 1 : stage_mode(pl[e]);
        pass2[{pl[e].cfg.vec, pl[e].cfg.G, 1, stored[e] ? 0 : ik, tma2, pl[e].cfg.mpw}].push_back(e);
      }
    }
  }
  int n_s = 0;
  for (auto& kv : pass1) n_s += static_cast<int>(kv.second.size());
  for (auto& kv : pass2) n_s += static_cast<int>(kv.second.size());
  for (auto& kv : gram_cls) n_s += static_cast<int>(kv.second.size());
  int n_lin = 0, n_logical = 0;
  for (int e = 0; e < count; ++e) {
    if (owner(e) != e) continue;
    n_lin += is_lin[e];
    ++n_logical;
  }
  const int n_f = n_logical + n_lin;
  const size_t sdesc_bytes = align_up(static_cast<int64_t>(n_s) * sizeof(EnsDesc), 256);
  const size_t fdesc_bytes = align_up(static_cast<int64_t>(n_f) * sizeof(FinDesc), 256);
  bp->desc_bytes = sdesc_bytes + fdesc_bytes;
  size_t off = bp->desc_bytes;
  std::vector<double*> part(count), sums(count);
  std::vector<float*> coef(count), gpart(count, nullptr);
  std::vector<float*> scale(count, nullptr);
  // Operand planes of the tiled Gram: written by the streaming pass into one buffer per
  // ensemble (BF16, store_u), else staged into one buffer reused by the launches in turn.
  std::vector<int> fused(count, 0);
  std::vector<void*> op_own(count, nullptr);
  size_t op_bytes = 0;
  for (int e = 0; e < count; ++e) {
    if (!tiled[e]) continue;
    fused[e] = store_u && tp[e].prec == PID_BF16 && pl[e].cfg.vec == 1;
    if (fused[e]) {
      op_own[e] = base + off;
      off += align_up(static_cast<int64_t>(tp[e].op_bytes), 1024);
      pl[e].desc.op_out = static_cast<uint16_t*>(op_own[e]);
      pl[e].desc.op_ld = tp[e].ldo;
    } else {
      op_bytes = std::max(op_bytes, tp[e].op_bytes);
    }
  }
  void* op_buf = nullptr;
  if (op_bytes) { op_buf = base + off; off += align_up(static_cast<int64_t>(op_bytes), 1024); }
  // chunks of an ensemble's (m, A) partials and of its Gram partials
  auto part_chunks = [&](int e) { return is_gram[e] && !tiled[e] ? gp[e].n_gchunks : pl[e].desc.n_chunks; };
  auto gram_chunks = [&](int e) { return tiled[e] ? tp[e].n_gchunks : gp[e].n_gchunks; };
  for (int e = 0; e < count; ++e) {
    const int o = owner(e);
    if (o == e) {
      const size_t pb = is_gram[e] && !tiled[e] ? std::max(pl[e].part_bytes, gp[e].part_bytes) : pl[e].part_bytes;
      part[e] = reinterpret_cast<double*>(base + off); off += pb * steps;
      sums[e] = reinterpret_cast<double*>(base + off); off += pl[e].sums_bytes;
      coef[e] = reinterpret_cast<float*>(base + off); off += pl[e].coef_bytes;
      if (is_gram[e]) {
        gpart[e] = reinterpret_cast<float*>(base + off);
        off += (tiled[e] ? tp[e].gpart_bytes : gp[e].gpart_bytes) * steps;
      }
    } else {   // a later time step: its partials follow those of the steps before it
      part[e] = part[o] + static_cast<int64_t>(e) * part_chunks(e) * 2 * in[e].N;
      sums[e] = sums[o];
      coef[e] = coef[o];
      if (is_gram[e]) gpart[e] = gpart[o] + static_cast<int64_t>(e) * gram_chunks(e) * in[e].N * in[e].N;
    }
    // E4M3 member scales: every ensemble (and every time step) has its own, undone before
    // its partial Grams are summed
    if (is_gram[e] && in[e].precision == PID_FP8) {
      scale[e] = reinterpret_cast<float*>(base + off);
      off += kScaleBytes;
    }
    pl[e].desc.part = part[e];
    if (stored[e]) {
      const int64_t ldu = (in[e].M + 3) / 4 * 4;
      float* ub = reinterpret_cast<float*>(base + off);
      off += align_up(in[e].N * ldu * 4, 256);
      pl[e].desc.u_out = ub;
      EnsInput u = in[e];
      u.data = ub;
      u.ld = ldu;
      u.is_field = 0;
      u.validate = 0;    // checked on the fields in pass 1
      const pid_status st2 = plan_stream(h, u, &pl2[e]);
      if (st2 != PID_OK) return st2;
      pl2[e].desc.part = part[e];
    }
  }
  bp->work_bytes = off;
  if (n_logical > kMaxTickets) return fail(h, PID_ERR_UNSUPPORTED, "too many ensembles in one batch");
  // E4M3 scales of soft masks from a first streaming pass over the same data, where the
  // batch has one: a tiled Gram's own exact-sums pass, or a PID-mean / exact full PID item of
  // the same masks (same pointer, shape, stride and cell measures); otherwise a pass of
  // their own before the Gram.
  std::vector<int> keys_src(count, -1);
  auto claim = [&](int e, int f) {
    pl[f].desc.umax = scale_keys(scale[e]);
    keys_src[e] = f;
    bp->key_resets.push_back({pl[f].desc.umax, in[e].N});
  };
  for (int e = 0; e < count; ++e)
    if (tiled[e] && in[e].precision == PID_FP8 && !in[e].is_field) claim(e, e);
  for (int e = 0; e < count; ++e)   // a second E4M3 item on the same masks runs its own max pass
    if (is_gram[e] && !tiled[e] && in[e].precision == PID_FP8 && sib[e] >= 0 &&
        pl[sib[e]].desc.umax == nullptr)
      claim(e, sib[e]);

  auto add_stream_class = [&](const std::vector<int>& members, bool coef_pass) {
    Launch L;
    L.kind = Launch::STREAM;
    L.first = static_cast<int>(bp->sdesc.size());
    L.count = static_cast<int>(members.size());
    L.cfg = pl[members[0]].cfg;
    L.coef = coef_pass;
    L.tma = true;
    int32_t units = 0;
    for (int e : members) {
      const EnsPlan& p = (coef_pass && stored[e]) ? pl2[e] : pl[e];
      EnsDesc d = p.desc;
      if (coef_pass) { d.u_out = nullptr; d.op_out = nullptr; d.umax = nullptr; }
      L.maxu = L.maxu || d.umax != nullptr;
      d.unit_begin = units;
      d.work_begin = L.cells;
      d.coef = coef_pass ? coef[e] : nullptr;
      units += d.n_chunks;
      L.stage_floats = std::max(L.stage_floats, p.stage_floats);
      L.tma = L.tma && p.use_tma;
      L.cls = L.cls && p.cls;
      L.bytes += 4.0 * d.N * d.M + (d.w ? 4.0 * d.M : 0.0);
      L.max_n = std::max(L.max_n, d.N);
      L.cells += static_cast<int64_t>(d.N) * d.M;
      bp->sdesc.push_back(d);
    }
    L.total_units = units;
    bp->launches.push_back(L);
  };
  auto fin_for = [&](int e, int kind) {
    FinDesc f;
    std::memset(&f, 0, sizeof(f));
    f.part = part[e];
    f.N = static_cast<int32_t>(in[e].N);
    f.n_chunks = steps * part_chunks(e);
    f.kind = kind;
    f.sums = sums[e];
    f.coef = coef[e];
    f.ticket = h->tickets + e;
    const pid_ensemble& o = ens[e];
    if (kind != FIN_LIN1) {
      f.depth = o.depth; f.in_in = o.in_in; f.in_out = o.in_out; f.rank = o.rank;
    }
    if (kind != FIN_LIN2) { f.mass = o.mass; f.mean_depth = o.mean_depth; }
    if (kind == FIN_MEAN && mshare[e] >= 0) {   // (m, A) from the exact item's first pass
      f.part = part[mshare[e]];
      f.n_chunks = pl[mshare[e]].desc.n_chunks;
    }
    if (kind == FIN_GRAM) {
      f.gpart = gpart[e];
      f.n_gchunks = steps * gram_chunks(e);
      f.P = o.P;
      f.err_est = o.err_est;
      if (sib[e] >= 0) {   // (m, A) from the first streaming pass over the same masks
        f.part = part[sib[e]];
        f.n_chunks = pl[sib[e]].desc.n_chunks;
      }
    }
    const int nb = (2 * f.N + 31) / 32 + (kind == FIN_GRAM ? fin_gram_items(f.N) : 0);
    f.slices = std::max(1, std::min(nb, 2 * h->sms));
    return f;
  };

  // Phase 1: first streaming passes (which may also reduce E4M3 maxima), then the Gram
  // launches.
  for (auto& kv : pass1) add_stream_class(kv.second, false);
  for (auto& kv : gram_cls) {
    Launch L;
    L.kind = Launch::GRAM;
    L.first = static_cast<int>(bp->sdesc.size());
    L.count = static_cast<int>(kv.second.size());
    L.gp = gp[kv.second[0]];
    int32_t units = 0;
    for (int e : kv.second) {
      EnsDesc d = gp[e].desc;
      d.unit_begin = units;
      d.work_begin = L.cells;
      L.cells += static_cast<int64_t>(d.N) * d.M;
      d.part = part[e];
      d.gpart = gpart[e];
      d.op_scale = nullptr;
      if (gp[e].prec == PID_FP8) {
        d.op_scale = scale[e];
        L.scales.push_back({in[e], scale[e], keys_src[e] >= 0});
      }
      units += gp[e].n_gchunks;
      L.bytes += gp[e].bytes;
      L.flops += gp[e].flops;
      L.gp.stage_floats = std::max(L.gp.stage_floats, gp[e].stage_floats);
      bp->sdesc.push_back(d);
    }
    gram_geometry(h, L.gp.G, L.gp.mpw, L.gp.wide, L.gp.prec, L.gp.stage_floats, &L.gp.dF, &L.gp.dO,
                  &L.gp.smem);
    L.iso_mode = gp[kv.second[0]].desc.iso_mode;
    L.total_units = units;
    bp->launches.push_back(L);
  }
  for (int e = 0; e < count; ++e) {
    if (!tiled[e]) continue;
    Launch L;
    L.kind = Launch::TILED;
    L.first = e;
    L.count = 1;
    L.in = in[e];
    L.tp = tp[e];
    L.op = fused[e] ? op_own[e] : op_buf;
    L.stage = !fused[e];
    L.gpart = gpart[e];
    L.scale = scale[e];
    L.scale_from_keys = keys_src[e] >= 0;
    bp->launches.push_back(L);
  }
  {
    Launch L;
    L.kind = Launch::FIN;
    L.first = static_cast<int>(bp->fdesc.size());
    for (int e = 0; e < count; ++e) {
      if (owner(e) != e) continue;
      const int kind = is_gram[e] ? FIN_GRAM : (is_lin[e] ? FIN_LIN1 : FIN_MEAN);
      bp->fdesc.push_back(fin_for(e, kind));
      L.grid_x = std::max(L.grid_x, bp->fdesc.back().slices);
    }
    L.count = static_cast<int>(bp->fdesc.size()) - L.first;
    bp->launches.push_back(L);
  }
  // Phase 2: exact full PID, second streaming pass and its finalisation.
  if (n_lin) {
    for (auto& kv : pass2) add_stream_class(kv.second, true);
    Launch L;
    L.kind = Launch::FIN;
    L.first = static_cast<int>(bp->fdesc.size());
    for (int e = 0; e < count; ++e) {
      if (!is_lin[e] || owner(e) != e) continue;
      bp->fdesc.push_back(fin_for(e, FIN_LIN2));
      L.grid_x = std::max(L.grid_x, bp->fdesc.back().slices);
    }
    L.count = static_cast<int>(bp->fdesc.size()) - L.first;
    bp->launches.push_back(L);
  }
  return PID_OK;
}

static pid_status enqueue(pid_handle h, const BatchPlan& bp, char* base, const void* host_image,
                          cudaStream_t s) {
  cudaError_t e = cudaMemcpyAsync(base, host_image, bp.desc_bytes, cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) return cuda_fail(h, e, "batch descriptor upload");
  for (const auto& kr : bp.key_resets) {
    e = cudaMemsetAsync(kr.first, 0, static_cast<size_t>(kr.second) * sizeof(unsigned int), s);
    if (e != cudaSuccess) return cuda_fail(h, e, "scale key reset");
  }
  const EnsDesc* sdev = reinterpret_cast<const EnsDesc*>(base);
  const size_t sdesc_bytes = align_up(static_cast<int64_t>(bp.sdesc.size()) * sizeof(EnsDesc), 256);
  const FinDesc* fdev = reinterpret_cast<const FinDesc*>(base + sdesc_bytes);
  auto launch_one = [&](const Launch& L, cudaStream_t s) -> pid_status {
    cudaError_t e = cudaSuccess;
    if (L.kind == Launch::STREAM) {
      StreamParams sp;
      std::memset(&sp, 0, sizeof(sp));
      sp.one = bp.sdesc[L.first];  // host copy: tuning key (iso / weights of the class)
      sp.descs = sdev + L.first;
      sp.n_ens = L.count;
      sp.total_units = L.total_units;
      sp.total_work = L.cells;
      sp.G = L.cfg.G;
      sp.sub = L.cfg.sub;
      sp.use_tma = L.tma ? 1 : (L.cls ? 2 : 0);
      sp.err = h->err_word;
      sp.stage_floats = L.stage_floats;
      sp.maxu = L.maxu ? 1 : 0;
      const int n_groups = kStreamWarps / L.cfg.G;
      const int grid = std::max(1, std::min<int>(h->sms, (L.total_units + n_groups - 1) / n_groups));
      pid_status st = stream_launch(h, sp, L.cfg, L.coef, grid, L.max_n, L.cells, L.bytes, s);
      if (st != PID_OK) return st;
    } else if (L.kind == Launch::GRAM) {
      if (!L.scales.empty()) {
        std::vector<ScaleJob> jobs;
        jobs.reserve(L.scales.size());
        for (const auto& sc : L.scales) jobs.push_back(ScaleJob{sc.in, sc.out, sc.from_keys});
        const pid_status st = launch_member_scales_many(h, jobs, s);
        if (st != PID_OK) return st;
      }
      pid_status st = launch_gram_batch(h, L.gp, sdev + L.first, L.count, L.total_units,
                                        L.cells, L.iso_mode, L.bytes, L.flops, s);
      if (st != PID_OK) return st;
    } else if (L.kind == Launch::TILED) {
      pid_status st = PID_OK;
      if (L.scale_from_keys && (st = launch_scales_from_keys(h, L.in.N, L.scale, s)) != PID_OK)
        return st;
      st = launch_gram_tiled_one(h, L.in, L.tp, L.op, L.gpart, L.scale, L.stage, s,
                                 L.scale_from_keys);
      if (st != PID_OK) return st;
    } else {
      FinParams fp;
      std::memset(&fp, 0, sizeof(fp));
      fp.descs = fdev + L.first;
      fp.n_ens = L.count;
      fp.err = h->err_word;
      ProfScope ps(h, PID_KERNEL_FINALIZE, 0.0, 0.0, s);
      e = launch_finalize(fp, L.grid_x, L.count, s);
      if (e != cudaSuccess) return cuda_fail(h, e, "batch finalize launch");
    }
    return PID_OK;
  };
  // Consecutive streaming launches (one pass's classes) are independent: they run on the
  // side streams, forked from `s` and joined back before the next phase, so that classes
  // whose grids leave SMs idle (a few small ensembles) fill them. Gram launches fill the
  // GPU on their own and run in order on `s`.
  BatchCache* c = h->batch;
  const size_t n = bp.launches.size();
  for (size_t i = 0; i < n;) {
    const Launch::Kind kind = bp.launches[i].kind;
    size_t j = i + 1;
    if (kind == Launch::STREAM)
      while (j < n && bp.launches[j].kind == kind) ++j;
    if (j - i == 1 || !c || !c->fork_ev) {
      for (size_t k = i; k < j; ++k) {
        const pid_status st = launch_one(bp.launches[k], s);
        if (st != PID_OK) return st;
      }
    } else {
      if ((e = cudaEventRecord(c->fork_ev, s)) != cudaSuccess) return cuda_fail(h, e, "fork");
      const int used = static_cast<int>(std::min<size_t>(j - i, BatchCache::kSide));
      for (int k = 0; k < used; ++k)
        if ((e = cudaStreamWaitEvent(c->side[k], c->fork_ev, 0)) != cudaSuccess)
          return cuda_fail(h, e, "fork");
      for (size_t k = i; k < j; ++k) {
        const pid_status st = launch_one(bp.launches[k], c->side[(k - i) % BatchCache::kSide]);
        if (st != PID_OK) return st;
      }
      for (int k = 0; k < used; ++k) {
        if ((e = cudaEventRecord(c->join_ev[k], c->side[k])) != cudaSuccess ||
            (e = cudaStreamWaitEvent(s, c->join_ev[k], 0)) != cudaSuccess)
          return cuda_fail(h, e, "join");
      }
    }
    i = j;
  }
  return PID_OK;
}

}  // namespace pidh

using namespace pidh;

namespace {

pid_status run_batch(pid_handle h, const pid_ensemble* ens, int32_t count, int steps,
                     void* stream) {
  DeviceGuard g(h->device);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (!h->batch) h->batch = new BatchCache();
  BatchCache* c = h->batch;

  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  cudaStreamIsCapturing(s, &cs);
  const bool capturing = cs != cudaStreamCaptureStatusNone;
  const bool profiled = h->profiling;
  // Replay the cached graph when the batch is the one it was recorded for (same ensemble
  // records, same workspace): no planning, no tensor-map encoding, one graph launch.
  // key: the records, the workspace address, the steps and whether the graph is profiled
  std::vector<unsigned char> key(sizeof(pid_ensemble) * count + sizeof(void*) + sizeof(int) + 1);
  std::memcpy(key.data(), ens, sizeof(pid_ensemble) * count);
  std::memcpy(key.data() + sizeof(pid_ensemble) * count, &h->ws, sizeof(void*));
  std::memcpy(key.data() + sizeof(pid_ensemble) * count + sizeof(void*), &steps, sizeof(int));
  key.back() = profiled ? 1 : 0;
  if (c->use_graphs && !capturing && c->exec && key == c->key) {
    if (profiled) {
      const pid_status ps = arm_graph_profiling(h, c);
      if (ps != PID_OK) return ps;
    }
    cudaError_t e = cudaGraphLaunch(c->exec, s);
    if (e != cudaSuccess) return cuda_fail(h, e, "batch graph replay");
    ++c->replays;
    return PID_OK;
  }
  // Plan against a null base to size the workspace, then for real. Soft masks of fields in
  // exact full PID are stored for the second pass when the extra workspace fits the
  // handle's budget (or, without one, half of the free device memory).
  BatchPlan sizing;
  bool store_u = true;
  pid_status st = plan_batch(h, ens, count, nullptr, store_u, &sizing, steps);
  if (st != PID_OK) return st;
  {
    BatchPlan lean;
    if ((st = plan_batch(h, ens, count, nullptr, false, &lean, steps)) != PID_OK) return st;
    const size_t extra = sizing.work_bytes - lean.work_bytes;
    size_t free_b = 0, total_b = 0;
    if (extra > 0) cudaMemGetInfo(&free_b, &total_b);
    const size_t have = h->ws_bytes;
    const size_t grow = sizing.work_bytes > have ? sizing.work_bytes - have : 0;
    if (extra > 0 && ((h->budget && sizing.work_bytes + h->fixed_bytes > h->budget) ||
                      (!h->budget && grow > free_b / 2))) {
      store_u = false;
      sizing = lean;
    }
  }
  if ((st = ensure_workspace(h, sizing.work_bytes, s)) != PID_OK) return st;
  if ((st = ensure_side_streams(h, c)) != PID_OK) return st;
  std::memcpy(key.data() + sizeof(pid_ensemble) * count, &h->ws, sizeof(void*));
  BatchPlan bp;
  char* base = static_cast<char*>(h->ws);
  if ((st = plan_batch(h, ens, count, base, store_u, &bp, steps)) != PID_OK) return st;
  // Host image of the descriptors (pinned, so the upload is asynchronous and graph-safe).
  if (c->host_bytes < bp.desc_bytes) {
    if (c->exec) { cudaStreamSynchronize(s); }
    if (c->host_desc) cudaFreeHost(c->host_desc);
    c->host_desc = nullptr;
    c->host_bytes = 0;
    if (cudaMallocHost(&c->host_desc, bp.desc_bytes) != cudaSuccess) {
      cudaGetLastError();
      return fail(h, PID_ERR_OOM, "pinned descriptor staging");
    }
    c->host_bytes = bp.desc_bytes;
  } else {
    cudaStreamSynchronize(s);  // a previous upload may still read the staging image
  }
  std::memset(c->host_desc, 0, bp.desc_bytes);
  std::memcpy(c->host_desc, bp.sdesc.data(), bp.sdesc.size() * sizeof(EnsDesc));
  const size_t sdesc_bytes = align_up(static_cast<int64_t>(bp.sdesc.size()) * sizeof(EnsDesc), 256);
  std::memcpy(static_cast<char*>(c->host_desc) + sdesc_bytes, bp.fdesc.data(),
              bp.fdesc.size() * sizeof(FinDesc));

  if (!c->use_graphs || capturing) {
    return enqueue(h, bp, base, c->host_desc, s);
  }
  if (h->autotune) {
    // Tune on the caller's stream before recording: captured launches are never tuned.
    st = enqueue(h, bp, base, c->host_desc, s);
    if (st != PID_OK) return st;
  }
  // Record the sequence into a graph on a private stream, then launch it on the caller's.
  if (c->exec) { cudaGraphExecDestroy(c->exec); c->exec = nullptr; }
  if (c->graph) { cudaGraphDestroy(c->graph); c->graph = nullptr; }
  cudaStream_t cap;
  cudaError_t e = cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking);
  if (e != cudaSuccess) return cuda_fail(h, e, "capture stream");
  e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) { cudaStreamDestroy(cap); return cuda_fail(h, e, "begin capture"); }
  h->prof_graph = profiled;
  h->prof_captured.clear();
  st = enqueue(h, bp, base, c->host_desc, cap);
  h->prof_graph = false;
  cudaGraph_t graph = nullptr;
  e = cudaStreamEndCapture(cap, &graph);
  cudaStreamDestroy(cap);
  c->prof.clear();
  if (st == PID_OK && e == cudaSuccess && profiled) st = collect_graph_profiling(h, graph, c);
  for (const ProfRecord& r : h->prof_captured) {   // left over after a failed capture
    h->event_pool.push_back(r.start);
    h->event_pool.push_back(r.stop);
  }
  h->prof_captured.clear();
  if (st != PID_OK) { if (graph) cudaGraphDestroy(graph); return st; }
  if (e != cudaSuccess) return cuda_fail(h, e, "end capture");
  cudaGraphExec_t exec = nullptr;
  e = cudaGraphInstantiate(&exec, graph, 0);
  if (e != cudaSuccess) { cudaGraphDestroy(graph); return cuda_fail(h, e, "graph instantiate"); }
  c->graph = graph;
  c->exec = exec;
  c->key = key;
  if (profiled && (st = arm_graph_profiling(h, c)) != PID_OK) return st;
  e = cudaGraphLaunch(exec, s);
  if (e != cudaSuccess) return cuda_fail(h, e, "batch graph launch");
  return PID_OK;
}

}  // namespace

extern "C" pid_status pid_batch(pid_handle h, const pid_ensemble* ens, int32_t count, void* stream) {
  if (!h) return PID_ERR_INVALID_ARG;
  if (count < 0 || (count > 0 && !ens)) return fail(h, PID_ERR_INVALID_ARG, "bad ensemble array");
  if (count == 0) return PID_OK;
  return run_batch(h, ens, count, 1, stream);
}

extern "C" pid_status pid_spacetime(pid_handle h, const float* const* steps_host, int32_t T, int64_t N,
                                    int64_t M, int64_t ld, const float* w, const pid_iso* iso,
                                    const pid_options* opt, double* depth, double* in_in,
                                    double* in_out, int32_t* rank, double* P, double* err_est,
                                    void* stream) {
  if (!h) return PID_ERR_INVALID_ARG;
  if (!steps_host || T < 1) return fail(h, PID_ERR_INVALID_ARG, "need T >= 1 time-step pointers");
  if (T > kMaxSpacetimeSteps)
    return fail(h, PID_ERR_UNSUPPORTED, "too many time steps (at most 65536)");
  if (M > 0 && static_cast<int64_t>(T) * ((M + 4095) / 4096) > (int64_t(1) << 26))
    return fail(h, PID_ERR_UNSUPPORTED, "T x M too large for one space-time ensemble");
  pid_options o{PID_MODE_MEAN, PID_FP32, 0, 0};
  if (opt) o = *opt;
  std::vector<pid_ensemble> rec(T);
  for (int32_t t = 0; t < T; ++t) {
    pid_ensemble& e = rec[t];
    std::memset(&e, 0, sizeof(e));
    e.data = steps_host[t];
    e.N = N; e.M = M; e.ld = ld; e.w = w;
    e.is_field = iso != nullptr;
    if (iso) e.iso = *iso;
    e.opt = o;
  }
  rec[0].depth = depth; rec[0].in_in = in_in; rec[0].in_out = in_out; rec[0].rank = rank;
  rec[0].P = P; rec[0].err_est = err_est;
  return run_batch(h, rec.data(), T, T, stream);
}
