// Serving: continuous batching of depth requests over device-resident ensembles.
//
// Host threads submit requests (ensemble id + options) into a queue. One scheduler thread
// owns `max_inflight` slots, each with its own stream, handle (workspace) and output
// arena. Whenever a slot is free and requests are waiting, it takes up to `max_batch` of
// them (and at most `max_step_member_cells` of work), launches them as one pid_batch on
// that slot's stream and copies the results to pinned host memory behind it; a completed
// step hands its results to the waiting callers. Requests that arrive while steps are on
// the GPU therefore join the next step, and up to `max_inflight` steps overlap on the
// device. Ensembles stay resident between requests (and time steps) and are admitted
// against an HBM budget.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "../../include/pid.h"
#include "capi_internal.h"

namespace {

using Clock = std::chrono::steady_clock;

struct Ensemble {
  int64_t id = 0;
  float* data = nullptr;
  float* w = nullptr;
  bool owned = false;
  int64_t N = 0, M = 0, ld = 0;
  int32_t is_field = 0;
  pid_iso iso{};
  size_t bytes = 0;
  int inflight = 0;   // steps currently reading it
};

struct Request {
  uint64_t ticket = 0;
  int64_t ens_id = 0;
  pid_options opt{};
  int64_t N = 0, M = 0;
  Clock::time_point t_submit, t_done;
  pid_status status = PID_OK;
  bool done = false;
  std::vector<double> depth, in_in, in_out, mean_depth;
  std::vector<int32_t> rank;
};

struct Slot {
  pid_handle h = nullptr;
  cudaStream_t stream = nullptr;
  cudaEvent_t ev = nullptr;
  bool busy = false;
  std::vector<std::shared_ptr<Request>> reqs;
  std::vector<size_t> offsets;
  void* dev_out = nullptr;
  size_t dev_bytes = 0;
  void* host_out = nullptr;
  size_t host_bytes = 0;
};

size_t out_block_bytes(int64_t N) {  // depth, in_in, in_out, mean_depth (f64) + rank (i32)
  return (static_cast<size_t>(N) * (4 * 8 + 4) + 255) / 256 * 256;
}

}  // namespace

struct pid_server_s {
  pid_serve_cfg cfg{};
  std::mutex mu;
  std::condition_variable cv_sched, cv_done, cv_idle;
  int active = 0;              // threads inside a pid_serve_* call (counted under mu)
  std::once_flag join_once;    // the scheduler is joined by the first pid_serve_cancel
  std::deque<std::shared_ptr<Request>> queue;
  std::unordered_map<uint64_t, std::shared_ptr<Request>> reqs;
  std::map<int64_t, std::unique_ptr<Ensemble>> ens;
  std::vector<Slot> slots;
  std::thread sched;
  bool stopping = false;
  uint64_t next_ticket = 1;
  int64_t next_ens = 1;
  size_t resident = 0;
  int64_t submitted = 0, completed = 0, failed = 0, steps = 0, batched = 0;
  double member_cells = 0;
  std::vector<double> lat_ms;
  Clock::time_point t_first, t_last;
  bool have_first = false;
};

namespace {

// Counts the calling thread as inside the server for the scope's lifetime; s->mu must be
// held when the scope begins and when it ends (declare it after the lock).
class CallScope {
 public:
  explicit CallScope(pid_server s) : s_(s) { ++s_->active; }
  ~CallScope() {
    if (--s_->active == 0) s_->cv_idle.notify_all();
  }
 private:
  pid_server s_;
};

void finish(pid_server s, const std::shared_ptr<Request>& r, pid_status st) {
  r->status = st;
  r->done = true;
  r->t_done = Clock::now();
  if (st == PID_OK) {
    ++s->completed;
    s->member_cells += static_cast<double>(r->N) * r->M;
    s->lat_ms.push_back(std::chrono::duration<double, std::milli>(r->t_done - r->t_submit).count());
    s->t_last = r->t_done;
  } else {
    ++s->failed;
  }
}

Ensemble* find_ens(pid_server s, int64_t id) {
  auto it = s->ens.find(id);
  return it == s->ens.end() ? nullptr : it->second.get();
}

// Completion of a step: results are in the slot's pinned arena.
void complete_slot(pid_server s, Slot& sl, pid_status st) {
  if (st == PID_OK) st = pid_sync(sl.h, sl.stream);  // device error word of the step
  for (size_t k = 0; k < sl.reqs.size(); ++k) {
    auto& r = sl.reqs[k];
    if (Ensemble* e = find_ens(s, r->ens_id)) --e->inflight;
    if (st == PID_OK) {
      const char* base = static_cast<const char*>(sl.host_out) + sl.offsets[k];
      const size_t n = static_cast<size_t>(r->N);
      r->depth.assign(reinterpret_cast<const double*>(base), reinterpret_cast<const double*>(base) + n);
      r->in_in.assign(reinterpret_cast<const double*>(base) + n, reinterpret_cast<const double*>(base) + 2 * n);
      r->in_out.assign(reinterpret_cast<const double*>(base) + 2 * n, reinterpret_cast<const double*>(base) + 3 * n);
      r->mean_depth.assign(reinterpret_cast<const double*>(base) + 3 * n, reinterpret_cast<const double*>(base) + 4 * n);
      const int32_t* rk = reinterpret_cast<const int32_t*>(base + 4 * 8 * n);
      r->rank.assign(rk, rk + n);
    }
    finish(s, r, st);
  }
  sl.reqs.clear();
  sl.busy = false;
  s->cv_done.notify_all();
}

// Form one step from the queue and launch it on a free slot (called with the lock held).
void launch_step(pid_server s, Slot& sl) {
  std::vector<std::shared_ptr<Request>> take;
  std::vector<Ensemble*> used;
  int64_t cells = 0;
  while (!s->queue.empty() && static_cast<int32_t>(take.size()) < s->cfg.max_batch) {
    auto r = s->queue.front();
    Ensemble* e = find_ens(s, r->ens_id);
    if (!e) {  // unregistered after submission
      s->queue.pop_front();
      finish(s, r, PID_ERR_INVALID_ARG);
      s->cv_done.notify_all();
      continue;
    }
    const int64_t mc = e->N * e->M;
    if (!take.empty() && s->cfg.max_step_member_cells > 0 && cells + mc > s->cfg.max_step_member_cells)
      break;
    s->queue.pop_front();
    take.push_back(r);
    used.push_back(e);
    cells += mc;
  }
  if (take.empty()) return;
  size_t total = 0;
  sl.offsets.clear();
  for (size_t k = 0; k < take.size(); ++k) {
    take[k]->N = used[k]->N;
    take[k]->M = used[k]->M;
    sl.offsets.push_back(total);
    total += out_block_bytes(used[k]->N);
  }
  pid_status st = total > 0 ? PID_OK : PID_ERR_INVALID_ARG;
  if (total > sl.dev_bytes) {
    if (sl.dev_out) cudaFree(sl.dev_out);
    sl.dev_out = nullptr;
    sl.dev_bytes = 0;
    if (cudaMalloc(&sl.dev_out, total * 2) == cudaSuccess) sl.dev_bytes = total * 2;
    else { cudaGetLastError(); st = PID_ERR_OOM; }
  }
  if (st == PID_OK && total > sl.host_bytes) {
    if (sl.host_out) cudaFreeHost(sl.host_out);
    sl.host_out = nullptr;
    sl.host_bytes = 0;
    if (cudaMallocHost(&sl.host_out, total * 2) == cudaSuccess) sl.host_bytes = total * 2;
    else { cudaGetLastError(); st = PID_ERR_OOM; }
  }
  std::vector<pid_ensemble> arr(take.size());
  if (st == PID_OK && (sl.dev_out == nullptr || sl.host_out == nullptr || total > sl.dev_bytes ||
                       total > sl.host_bytes))
    st = PID_ERR_OOM;
  if (st == PID_OK) {
    for (size_t k = 0; k < take.size(); ++k) {
      const Ensemble* e = used[k];
      pid_ensemble& pe = arr[k];
      std::memset(&pe, 0, sizeof(pe));
      pe.data = e->data;
      pe.N = e->N;
      pe.M = e->M;
      pe.ld = e->ld;
      pe.w = e->w;
      pe.is_field = e->is_field;
      pe.iso = e->iso;
      pe.opt = take[k]->opt;
      char* base = static_cast<char*>(sl.dev_out) + sl.offsets[k];
      const size_t n = static_cast<size_t>(e->N);
      pe.depth = reinterpret_cast<double*>(base);
      pe.in_in = reinterpret_cast<double*>(base) + n;
      pe.in_out = reinterpret_cast<double*>(base) + 2 * n;
      pe.mean_depth = reinterpret_cast<double*>(base) + 3 * n;
      pe.rank = reinterpret_cast<int32_t*>(base + 4 * 8 * n);
    }
    st = pid_batch(sl.h, arr.data(), static_cast<int32_t>(arr.size()), sl.stream);
  }
  if (st == PID_OK &&
      (cudaMemcpyAsync(sl.host_out, sl.dev_out, total, cudaMemcpyDeviceToHost, sl.stream) != cudaSuccess ||
       cudaEventRecord(sl.ev, sl.stream) != cudaSuccess)) {
    cudaGetLastError();
    st = PID_ERR_CUDA;
  }
  ++s->steps;
  s->batched += static_cast<int64_t>(take.size());
  if (st != PID_OK) {
    for (auto& r : take) finish(s, r, st);
    s->cv_done.notify_all();
    return;
  }
  for (Ensemble* e : used) ++e->inflight;
  sl.reqs = std::move(take);
  sl.busy = true;
}

void scheduler(pid_server s) {
  cudaSetDevice(s->cfg.device);
  std::unique_lock<std::mutex> lk(s->mu);
  while (true) {
    bool any_busy = false;
    for (Slot& sl : s->slots) {
      if (!sl.busy) continue;
      const cudaError_t q = cudaEventQuery(sl.ev);
      if (q == cudaSuccess) {
        complete_slot(s, sl, PID_OK);
      } else if (q != cudaErrorNotReady) {
        cudaGetLastError();
        complete_slot(s, sl, PID_ERR_CUDA);
      } else {
        any_busy = true;
      }
    }
    if (s->stopping) {
      while (!s->queue.empty()) {
        finish(s, s->queue.front(), PID_ERR_CANCELLED);
        s->queue.pop_front();
      }
      s->cv_done.notify_all();
      if (!any_busy) break;
    } else {
      for (Slot& sl : s->slots) {
        if (s->queue.empty()) break;
        if (!sl.busy) {
          launch_step(s, sl);
          any_busy = any_busy || sl.busy;
        }
      }
    }
    if (any_busy)
      s->cv_sched.wait_for(lk, std::chrono::microseconds(20));
    else
      s->cv_sched.wait(lk, [&] { return s->stopping || !s->queue.empty(); });
  }
}

}  // namespace

using namespace pidh;

extern "C" {

pid_status pid_serve_start(pid_server* out, const pid_serve_cfg* cfg) {
  if (!out || !cfg) return PID_ERR_INVALID_ARG;
  *out = nullptr;
  if (cfg->max_inflight < 1 || cfg->max_batch < 1 || cfg->max_queue < 1 || cfg->max_step_member_cells < 0)
    return PID_ERR_INVALID_ARG;
  auto s = std::make_unique<pid_server_s>();
  s->cfg = *cfg;
  s->slots.resize(cfg->max_inflight);
  DeviceGuard g(cfg->device);
  for (Slot& sl : s->slots) {
    pid_status st = pid_create(&sl.h, cfg->device, 0);
    if (st != PID_OK) return st;
    batch_use_graphs(sl.h, false);  // a new batch layout every step: launch directly
    batch_share_sums(sl.h, false);  // a request's results do not depend on its step-mates
    if (cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&sl.ev, cudaEventDisableTiming) != cudaSuccess) {
      cudaGetLastError();
      return PID_ERR_CUDA;
    }
  }
  pid_server raw = s.release();
  raw->sched = std::thread(scheduler, raw);
  *out = raw;
  return PID_OK;
}

pid_status pid_serve_cancel(pid_server s) {
  if (!s) return PID_ERR_INVALID_ARG;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stopping = true;
  }
  s->cv_sched.notify_all();
  // The scheduler cancels the queue, lets the running steps finish and exits; every
  // request is then done and every waiter has been woken.
  std::call_once(s->join_once, [s] {
    if (s->sched.joinable()) s->sched.join();
  });
  return PID_OK;
}

pid_status pid_serve_stop(pid_server s) {
  if (!s) return PID_OK;
  pid_serve_cancel(s);
  {
    // threads still inside a call (a wait that has just been woken) leave before the
    // server is freed
    std::unique_lock<std::mutex> lk(s->mu);
    s->cv_idle.wait(lk, [s] { return s->active == 0; });
  }
  DeviceGuard g(s->cfg.device);
  for (Slot& sl : s->slots) {
    if (sl.stream) cudaStreamSynchronize(sl.stream);
    if (sl.dev_out) cudaFree(sl.dev_out);
    if (sl.host_out) cudaFreeHost(sl.host_out);
    if (sl.ev) cudaEventDestroy(sl.ev);
    if (sl.stream) cudaStreamDestroy(sl.stream);
    pid_destroy(sl.h);
  }
  for (auto& kv : s->ens) {
    if (kv.second->owned) {
      cudaFree(kv.second->data);
      if (kv.second->w) cudaFree(kv.second->w);
    }
  }
  delete s;
  return PID_OK;
}

pid_status pid_serve_register(pid_server s, const float* data, int64_t N, int64_t M, int64_t ld,
                              const float* w, int32_t is_field, const pid_iso* iso, int32_t copy,
                              int64_t* ensemble_id) {
  if (!s || !ensemble_id) return PID_ERR_INVALID_ARG;
  pid_status st = check_shape(s->slots[0].h, data, N, M, ld);
  if (st != PID_OK) return st;
  if (is_field && (st = check_iso(s->slots[0].h, iso)) != PID_OK) return st;
  if (copy != 0 && copy != 1) return PID_ERR_INVALID_ARG;
  auto e = std::make_unique<Ensemble>();
  e->N = N; e->M = M; e->ld = ld; e->is_field = is_field;
  if (is_field) e->iso = *iso;
  e->owned = copy != 0;
  // HBM footprint of the resident ensemble, owned or adopted
  e->bytes = static_cast<size_t>(N) * ld * 4 + (w ? static_cast<size_t>(M) * 4 : 0);
  DeviceGuard g(s->cfg.device);
  std::lock_guard<std::mutex> lk(s->mu);
  CallScope cs(s);
  if (s->stopping) return PID_ERR_CANCELLED;
  const size_t reserve = static_cast<size_t>(s->cfg.max_inflight) * s->cfg.workspace_reserve_bytes;
  if (s->cfg.hbm_budget_bytes && s->resident + e->bytes + reserve > s->cfg.hbm_budget_bytes)
    return PID_ERR_OOM;
  if (e->owned) {
    void* p = nullptr;
    if (cudaMalloc(&p, static_cast<size_t>(N) * ld * 4) != cudaSuccess) { cudaGetLastError(); return PID_ERR_OOM; }
    e->data = static_cast<float*>(p);
    if (cudaMemcpy(e->data, data, static_cast<size_t>(N) * ld * 4, cudaMemcpyHostToDevice) != cudaSuccess) {
      cudaGetLastError();
      cudaFree(p);
      return PID_ERR_CUDA;
    }
    if (w) {
      if (cudaMalloc(&p, static_cast<size_t>(M) * 4) != cudaSuccess) {
        cudaGetLastError();
        cudaFree(e->data);
        return PID_ERR_OOM;
      }
      e->w = static_cast<float*>(p);
      if (cudaMemcpy(e->w, w, static_cast<size_t>(M) * 4, cudaMemcpyHostToDevice) != cudaSuccess) {
        cudaGetLastError();
        cudaFree(e->data);
        cudaFree(e->w);
        return PID_ERR_CUDA;
      }
    }
  } else {
    e->data = const_cast<float*>(data);
    e->w = const_cast<float*>(w);
  }
  e->id = s->next_ens++;
  s->resident += e->bytes;
  *ensemble_id = e->id;
  s->ens[e->id] = std::move(e);
  return PID_OK;
}

pid_status pid_serve_update(pid_server s, int64_t ensemble_id, const float* data_host) {
  if (!s || !data_host) return PID_ERR_INVALID_ARG;
  DeviceGuard g(s->cfg.device);
  std::unique_lock<std::mutex> lk(s->mu);
  CallScope cs(s);
  Ensemble* e = find_ens(s, ensemble_id);
  if (!e || !e->owned) return PID_ERR_INVALID_ARG;
  s->cv_done.wait(lk, [&] { return e->inflight == 0; });
  if (cudaMemcpy(e->data, data_host, static_cast<size_t>(e->N) * e->ld * 4, cudaMemcpyHostToDevice) !=
      cudaSuccess) {
    cudaGetLastError();
    return PID_ERR_CUDA;
  }
  return PID_OK;
}

pid_status pid_serve_unregister(pid_server s, int64_t ensemble_id) {
  if (!s) return PID_ERR_INVALID_ARG;
  DeviceGuard g(s->cfg.device);
  std::unique_lock<std::mutex> lk(s->mu);
  CallScope cs(s);
  Ensemble* e = find_ens(s, ensemble_id);
  if (!e) return PID_ERR_INVALID_ARG;
  s->cv_done.wait(lk, [&] { return e->inflight == 0; });
  if (e->owned) {
    cudaFree(e->data);
    if (e->w) cudaFree(e->w);
  }
  s->resident -= e->bytes;
  s->ens.erase(ensemble_id);
  return PID_OK;
}

pid_status pid_serve_submit(pid_server s, int64_t ensemble_id, const pid_options* opt,
                            uint64_t* ticket) {
  if (!s || !ticket) return PID_ERR_INVALID_ARG;
  pid_status st = check_opt(s->slots[0].h, opt);
  if (st != PID_OK) return st;
  auto r = std::make_shared<Request>();
  r->ens_id = ensemble_id;
  r->opt = opt ? *opt : pid_options{PID_MODE_MEAN, PID_FP32, 0, 0};
  {
    std::lock_guard<std::mutex> lk(s->mu);
    CallScope cs(s);
    if (s->stopping) return PID_ERR_CANCELLED;
    if (!find_ens(s, ensemble_id)) return PID_ERR_INVALID_ARG;
    if (static_cast<int32_t>(s->queue.size()) >= s->cfg.max_queue) return PID_ERR_BUSY;
    r->ticket = s->next_ticket++;
    r->t_submit = Clock::now();
    if (!s->have_first) { s->t_first = r->t_submit; s->have_first = true; }
    ++s->submitted;
    s->reqs[r->ticket] = r;
    s->queue.push_back(r);
    *ticket = r->ticket;
  }
  s->cv_sched.notify_one();
  return PID_OK;
}

pid_status pid_serve_wait(pid_server s, uint64_t ticket, int64_t timeout_ms, double* depth_host,
                          double* in_in_host, double* in_out_host, int32_t* rank_host,
                          double* mean_depth_host) {
  if (!s) return PID_ERR_INVALID_ARG;
  std::unique_lock<std::mutex> lk(s->mu);
  CallScope cs(s);
  auto it = s->reqs.find(ticket);
  if (it == s->reqs.end()) return PID_ERR_INVALID_ARG;
  std::shared_ptr<Request> r = it->second;
  if (timeout_ms < 0) {
    s->cv_done.wait(lk, [&] { return r->done; });
  } else if (!s->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), [&] { return r->done; })) {
    return PID_ERR_TIMEOUT;
  }
  s->reqs.erase(r->ticket);   // `it` may be stale: other tickets were erased while we waited
  if (r->status == PID_OK) {
    const size_t n = r->depth.size();
    if (depth_host) std::memcpy(depth_host, r->depth.data(), n * 8);
    if (in_in_host) std::memcpy(in_in_host, r->in_in.data(), n * 8);
    if (in_out_host) std::memcpy(in_out_host, r->in_out.data(), n * 8);
    if (rank_host) std::memcpy(rank_host, r->rank.data(), n * 4);
    if (mean_depth_host) std::memcpy(mean_depth_host, r->mean_depth.data(), n * 8);
  }
  return r->status;
}

pid_status pid_serve_stats_get(pid_server s, pid_serve_stats* out) {
  if (!s || !out) return PID_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(s->mu);
  CallScope cs(s);
  std::memset(out, 0, sizeof(*out));
  out->submitted = s->submitted;
  out->completed = s->completed;
  out->failed = s->failed;
  out->steps = s->steps;
  out->mean_batch = s->steps ? static_cast<double>(s->batched) / s->steps : 0.0;
  out->resident_bytes = s->resident;
  if (!s->lat_ms.empty()) {
    std::vector<double> v = s->lat_ms;
    std::sort(v.begin(), v.end());
    auto pct = [&](double p) {
      const size_t k = std::min(v.size() - 1, static_cast<size_t>(p * (v.size() - 1) + 0.5));
      return v[k];
    };
    out->p50_ms = pct(0.50);
    out->p99_ms = pct(0.99);
    out->max_ms = v.back();
    const double span = std::chrono::duration<double>(s->t_last - s->t_first).count();
    if (span > 0) {
      out->requests_per_s = s->completed / span;
      out->member_cells_per_s = s->member_cells / span;
    }
  }
  return PID_OK;
}

pid_status pid_serve_stats_reset(pid_server s) {
  if (!s) return PID_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(s->mu);
  CallScope cs(s);
  s->submitted = s->completed = s->failed = s->steps = s->batched = 0;
  s->member_cells = 0;
  s->lat_ms.clear();
  s->have_first = false;
  return PID_OK;
}

}  // extern "C"
