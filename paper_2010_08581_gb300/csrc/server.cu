// Serving layer of libtrals.so: continuous batching of independent TR-ALS-Sampled requests
// (Alg. 2 per request, stopped when the relative fit changes by less than a tolerance between
// sweeps, one of the criteria of Sec. 4.1) over the batched stages of batched.cu.
//
// Host side only: admission (FIFO, HBM budget, first-fit arena), the slot table, one CUDA
// graph per slot-count bucket, the tick loop and a worker thread. Each tick replays the graph
// of the occupied slots; the kernels read every slot's own step counter, so a request admitted
// between two ticks simply joins the next one.
#include <algorithm>
#include <chrono>
#include <climits>
#include <cmath>
#include <condition_variable>
#include <cstdarg>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "fit_tc.cuh"
#include "host_util.h"

namespace trk {
cudaError_t init_kernel_attributes(const char** which);
}

namespace {

using namespace trk;

int64_t now_ns() {
  return std::chrono::duration_cast<std::chrono::nanoseconds>(
             std::chrono::steady_clock::now().time_since_epoch())
      .count();
}

size_t round256(size_t b) { return (b + 255) & ~size_t(255); }

// First-fit allocator over [0, size) with coalescing of adjacent free ranges.
class ArenaAlloc {
 public:
  void reset(size_t size) {
    free_.clear();
    if (size) free_[0] = size;
  }
  size_t alloc(size_t bytes) {
    bytes = round256(bytes);
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second < bytes) continue;
      const size_t off = it->first, len = it->second;
      free_.erase(it);
      if (len > bytes) free_[off + bytes] = len - bytes;
      return off;
    }
    return SIZE_MAX;
  }
  void release(size_t off, size_t bytes) {
    bytes = round256(bytes);
    auto it = free_.emplace(off, bytes).first;
    auto nx = std::next(it);
    if (nx != free_.end() && it->first + it->second == nx->first) {
      it->second += nx->second;
      free_.erase(nx);
    }
    if (it != free_.begin()) {
      auto pv = std::prev(it);
      if (pv->first + pv->second == it->first) {
        pv->second += it->second;
        free_.erase(it);
      }
    }
  }

 private:
  std::map<size_t, size_t> free_;
};

struct Slot {
  bool used = false;
  int64_t ticket = -1;
  size_t ws_off = 0, ws_bytes = 0, charge = 0;
};

struct Pending {
  int64_t ticket;
  tr_request req;
  size_t ws_bytes, charge;
};

std::string g_server_error;   // message of the last failed tr_server_create

}  // namespace

struct tr_server {
  tr_server_config cfg{};
  bool f64 = false, xf64 = false;
  BLaunch geo{};                    // launch geometry (all but tab / count)
  // device memory
  char* arena = nullptr;
  BInst* dtab = nullptr;
  SlotState* dstate = nullptr;
  double* dfitp = nullptr;          // [max_slots][2 * kFitParts]
  double* dhist = nullptr;          // [max_slots][kMaxServedSweeps]
  unsigned* dcounter = nullptr;     // [max_slots]
  unsigned* derr = nullptr;
  // pinned host mirrors
  BInst* htab = nullptr;
  SlotState* hstate = nullptr;
  double* hhist = nullptr;          // [max_slots][kMaxServedSweeps]
  unsigned* herr = nullptr;
  cudaStream_t st = nullptr, side = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_info = nullptr, ev_join = nullptr;
  std::vector<int> buckets;
  std::vector<cudaGraphExec_t> graphs;
  // bookkeeping (guarded by mu)
  std::vector<Slot> slots;
  int hi = 0;                       // 1 + highest occupied slot
  int active = 0;
  ArenaAlloc alloc;
  std::deque<Pending> queue;
  std::unordered_map<int64_t, tr_result> results;
  size_t charged = 0;
  int64_t next_ticket = 1;
  tr_server_stats stats{};
  bool failed = false;
  std::string last_error;
  std::mutex mu;                    // queue, results, slots, stats, last_error
  std::mutex tick_mu;               // one tick at a time
  std::condition_variable cv_work, cv_done;
  std::thread worker;
  bool worker_on = false, stopping = false;
};

namespace {

tr_status sfail(tr_server* s, tr_status code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  if (s) {
    std::lock_guard<std::mutex> lk(s->mu);
    s->last_error = buf;
  } else {
    g_server_error = buf;
  }
  return code;
}

void free_all(tr_server* s) {
  for (cudaGraphExec_t g : s->graphs)
    if (g) cudaGraphExecDestroy(g);
  s->graphs.clear();
  if (s->arena) cudaFree(s->arena);
  if (s->dtab) cudaFree(s->dtab);
  if (s->dstate) cudaFree(s->dstate);
  if (s->dfitp) cudaFree(s->dfitp);
  if (s->dhist) cudaFree(s->dhist);
  if (s->dcounter) cudaFree(s->dcounter);
  if (s->derr) cudaFree(s->derr);
  if (s->htab) cudaFreeHost(s->htab);
  if (s->hstate) cudaFreeHost(s->hstate);
  if (s->hhist) cudaFreeHost(s->hhist);
  if (s->herr) cudaFreeHost(s->herr);
  if (s->st) cudaStreamDestroy(s->st);
  if (s->side) cudaStreamDestroy(s->side);
  if (s->ev_fork) cudaEventDestroy(s->ev_fork);
  if (s->ev_info) cudaEventDestroy(s->ev_info);
  if (s->ev_join) cudaEventDestroy(s->ev_join);
}

// Workspace of one request: distributions, per-update scratch, and the right factors of
// the fit's mode split (in X's precision).
void carve_request(Carver& c, const tr_request& r, bool f64, bool xf64, BInst& d) {
  carve_instance(c, r.N, r.dims, r.ranks, r.J, f64, d);
  const FitSplit f = fit_split(r.N, r.dims, r.ranks);
  const size_t simt = static_cast<size_t>(f.cols) * f.K * (xf64 ? 8 : 4);
  const size_t tcb = fit_use_tc(f, xf64) ? fit_tc_right_bytes(f) : 0;
  d.fitw = c.take<char>(simt > tcb ? simt : tcb);
}

size_t request_ws(const tr_request& r, bool f64, bool xf64) {
  Carver c(nullptr);
  BInst d{};
  carve_request(c, r, f64, xf64, d);
  return round256(c.off);
}

size_t request_charge(const tr_request& r, bool xf64, size_t ws) {
  size_t xb = xf64 ? 8 : 4, cb = 0;
  for (int k = 0; k < r.N; ++k) {
    xb *= static_cast<size_t>(r.dims[k]);
    cb += static_cast<size_t>(r.dims[k]) * r.ranks[(k - 1 + r.N) % r.N] * r.ranks[k] * 8;
  }
  return xb + cb + ws;
}

int bucket_of(const tr_server* s, int hi) {
  for (size_t i = 0; i < s->buckets.size(); ++i)
    if (s->buckets[i] >= hi) return static_cast<int>(i);
  return static_cast<int>(s->buckets.size()) - 1;
}

// The launches of one tick for the first `count` table entries.
cudaError_t issue_tick(tr_server* s, int count, cudaStream_t st) {
  BLaunch bl = s->geo;
  bl.tab = s->dtab;
  bl.count = count;
  cudaError_t e = bl_init_cores(bl, st);
  if (e != cudaSuccess) return e;
  const StepStreams ss{st, s->side, s->ev_fork, s->ev_info, s->ev_join};
  if ((e = issue_step(bl, 0, s->derr, ss)) != cudaSuccess) return e;
  if ((e = bl_fit(bl, s->derr, st)) != cudaSuccess) return e;
  return bl_advance(bl, st);
}

// Fills the table entry and initial state of a newly admitted request.
void setup_slot(tr_server* s, int id, const tr_request& r) {
  BInst& d = s->htab[id];
  d = BInst{};
  Carver c(s->arena + s->slots[id].ws_off);
  carve_request(c, r, s->f64, s->xf64, d);
  d.X = r.X;
  d.N = r.N;
  d.xf64 = s->xf64 ? 1 : 0;
  const int max_sw = r.max_sweeps > 0 ? r.max_sweeps : s->cfg.max_sweeps;
  d.nupd = max_sw * r.N;
  d.draw_init = r.init_given ? 0 : 1;
  d.J = r.J;
  d.seed = r.seed;
  row_major_strides(r.N, r.dims, d.stride);
  for (int k = 0; k < r.N; ++k) {
    d.dims[k] = r.dims[k];
    d.ranks[k] = r.ranks[k];
    d.cores[k] = r.cores[k];
  }
  d.counter = s->dcounter + id;
  d.slot = s->dstate + id;
  d.fitp = s->dfitp + static_cast<size_t>(id) * 2 * kFitParts;
  d.hist = s->dhist + static_cast<size_t>(id) * kMaxServedSweeps;
  SlotState& ss = s->hstate[id];
  ss = SlotState{};
  ss.step = 1 - r.N;
  ss.status = kSlotRunning;
  ss.max_sweeps = max_sw;
  ss.tol = r.fit_tol >= 0.0 ? r.fit_tol : s->cfg.fit_tol;
  ss.fit = 0.0;
  ss.fit_prev = 0.0;
}

tr_status status_of(int slot_status) {
  switch (slot_status) {
    case kSlotConverged: return TR_OK;
    case kSlotCapped: return TR_ERR_NOT_CONVERGED;
    case kSlotFailed: return TR_ERR_SINGULAR;
    default: return TR_ERR_CUDA;
  }
}

// Ends every occupied slot and queued request with `code` (after a failed tick).
void abandon_all(tr_server* s, tr_status code) {
  std::lock_guard<std::mutex> lk(s->mu);
  const int64_t t = now_ns();
  for (Slot& sl : s->slots) {
    if (!sl.used) continue;
    tr_result& res = s->results[sl.ticket];
    res.done = 1;
    res.status = code;
    res.t_done_ns = t;
    sl = Slot{};
  }
  for (const Pending& p : s->queue) {
    tr_result& res = s->results[p.ticket];
    res.done = 1;
    res.status = code;
    res.t_done_ns = t;
  }
  s->queue.clear();
  s->active = 0;
  s->hi = 0;
  s->charged = 0;
  s->failed = true;
  s->cv_done.notify_all();
}

tr_status run_tick(tr_server* s, int* active_out) {
  std::lock_guard<std::mutex> tl(s->tick_mu);
  if (s->failed) return sfail(s, TR_ERR_CUDA, "the server failed earlier");
  DeviceGuard g(s->cfg.device);
  const int64_t t0 = now_ns();
  std::vector<int> admitted;
  int hi;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    while (!s->queue.empty()) {
      const Pending& p = s->queue.front();
      if (s->charged + p.charge > s->cfg.hbm_budget_bytes) break;
      int id = -1;
      for (int i = 0; i < s->cfg.max_slots; ++i)
        if (!s->slots[i].used) { id = i; break; }
      if (id < 0) break;
      const size_t off = s->alloc.alloc(p.ws_bytes);
      if (off == SIZE_MAX) break;
      Slot& sl = s->slots[id];
      sl.used = true;
      sl.ticket = p.ticket;
      sl.ws_off = off;
      sl.ws_bytes = p.ws_bytes;
      sl.charge = p.charge;
      s->charged += p.charge;
      s->stats.peak_charged_bytes = std::max(s->stats.peak_charged_bytes, s->charged);
      setup_slot(s, id, p.req);
      s->results[p.ticket].t_admit_ns = now_ns();
      admitted.push_back(id);
      s->hi = std::max(s->hi, id + 1);
      s->active += 1;
      s->queue.pop_front();
    }
    s->stats.peak_active = std::max(s->stats.peak_active, s->active);
    hi = s->hi;
    // updates performed by this tick: running slots at a non-negative step
    for (int i = 0; i < hi; ++i)
      if (s->slots[i].used && s->hstate[i].status == kSlotRunning && s->hstate[i].step >= 0)
        s->stats.updates += 1;
  }
  if (hi == 0) {
    if (active_out) *active_out = 0;
    return TR_OK;
  }
  auto fail_tick = [&](cudaError_t e, const char* what) {
    cudaGetLastError();
    tr_status r = sfail(s, TR_ERR_CUDA, "%s failed: %s", what, cudaGetErrorString(e));
    abandon_all(s, TR_ERR_CUDA);
    return r;
  };
  cudaError_t e = cudaSuccess;
  for (int id : admitted) {
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(s->dtab + id, s->htab + id, sizeof(BInst), cudaMemcpyHostToDevice, s->st);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(s->dstate + id, s->hstate + id, sizeof(SlotState),
                          cudaMemcpyHostToDevice, s->st);
    if (e == cudaSuccess) e = cudaMemsetAsync(s->dcounter + id, 0, sizeof(unsigned), s->st);
  }
  if (e != cudaSuccess) return fail_tick(e, "slot upload");
  e = cudaGraphLaunch(s->graphs[bucket_of(s, hi)], s->st);
  if (e != cudaSuccess) return fail_tick(e, "cudaGraphLaunch");
  e = cudaMemcpyAsync(s->hstate, s->dstate, sizeof(SlotState) * hi, cudaMemcpyDeviceToHost, s->st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(s->herr, s->derr, sizeof(unsigned), cudaMemcpyDeviceToHost, s->st);
  if (e == cudaSuccess) e = cudaMemsetAsync(s->derr, 0, sizeof(unsigned), s->st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s->st);
  if (e != cudaSuccess) return fail_tick(e, "tick");
  if (*s->herr & (kErrTimeout | kErrBadIndex)) {
    tr_status r = sfail(s, TR_ERR_CUDA, "device error bits 0x%x in a tick", *s->herr);
    abandon_all(s, TR_ERR_CUDA);
    return r;
  }
  // Retire finished requests. The singular bit is per slot (SlotState::singular).
  const int64_t t_done = now_ns();
  std::vector<std::pair<int, int64_t>> finished;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    for (int i = 0; i < hi; ++i)
      if (s->slots[i].used && s->hstate[i].status != kSlotRunning)
        finished.emplace_back(i, s->slots[i].ticket);
  }
  if (!finished.empty()) {
    for (auto& f : finished) {
      const size_t o = static_cast<size_t>(f.first) * kMaxServedSweeps;
      e = cudaMemcpyAsync(s->hhist + o, s->dhist + o, sizeof(double) * kMaxServedSweeps,
                          cudaMemcpyDeviceToHost, s->st);
      if (e != cudaSuccess) return fail_tick(e, "fit history copy");
    }
    e = cudaStreamSynchronize(s->st);
    if (e != cudaSuccess) return fail_tick(e, "fit history copy");
  }
  for (auto& f : finished) {
    const int id = f.first;
    const double* hist = s->hhist + static_cast<size_t>(id) * kMaxServedSweeps;
    const SlotState& ss = s->hstate[id];
    std::lock_guard<std::mutex> lk(s->mu);
    tr_result& res = s->results[f.second];
    res.done = 1;
    res.status = status_of(ss.status);
    res.sweeps = ss.sweeps;
    res.singular_updates = ss.singular;
    res.fit = ss.fit;
    res.fit_change = std::fabs(ss.fit - ss.fit_prev);
    res.t_done_ns = t_done;
    const int nh = std::min(ss.sweeps, kMaxServedSweeps);
    for (int q = 0; q < kMaxServedSweeps; ++q) res.fit_history[q] = q < nh ? hist[q] : 0.0;
    Slot& sl = s->slots[id];
    s->alloc.release(sl.ws_off, sl.ws_bytes);
    s->charged -= sl.charge;
    sl = Slot{};
    s->active -= 1;
    s->stats.completed += 1;
  }
  {
    std::lock_guard<std::mutex> lk(s->mu);
    while (s->hi > 0 && !s->slots[s->hi - 1].used) s->hi -= 1;
    s->stats.ticks += 1;
    s->stats.tick_ns += now_ns() - t0;
    if (active_out) *active_out = s->active;
  }
  if (!finished.empty()) s->cv_done.notify_all();
  return TR_OK;
}

void worker_loop(tr_server* s) {
  for (;;) {
    {
      std::unique_lock<std::mutex> lk(s->mu);
      s->cv_work.wait(lk, [&] { return s->stopping || !s->queue.empty() || s->active > 0; });
      if (s->stopping) return;
      if (s->failed) return;
    }
    if (run_tick(s, nullptr) != TR_OK) return;
  }
}

tr_status check_request(tr_server* s, const tr_request& r) {
  const tr_server_config& c = s->cfg;
  if (!r.X) return sfail(s, TR_ERR_INVALID_ARG, "X is NULL");
  if (r.N < 2 || r.N > c.max_modes)
    return sfail(s, TR_ERR_INVALID_ARG, "N=%d outside [2, %d]", r.N, c.max_modes);
  for (int k = 0; k < r.N; ++k) {
    if (r.dims[k] < 1 || r.dims[k] > c.max_dim)
      return sfail(s, TR_ERR_INVALID_ARG, "dims[%d]=%lld outside [1, %lld]", k,
                   static_cast<long long>(r.dims[k]), static_cast<long long>(c.max_dim));
    if (r.ranks[k] < 1 || r.ranks[k] > c.max_rank)
      return sfail(s, TR_ERR_INVALID_ARG, "ranks[%d]=%d outside [1, %d]", k, r.ranks[k],
                   c.max_rank);
    if (!r.cores[k]) return sfail(s, TR_ERR_INVALID_ARG, "cores[%d] is NULL", k);
  }
  if (r.J < 1 || r.J > c.max_samples)
    return sfail(s, TR_ERR_INVALID_ARG, "J=%lld outside [1, %lld]", static_cast<long long>(r.J),
                 static_cast<long long>(c.max_samples));
  if (r.max_sweeps < 0 || r.max_sweeps > kMaxServedSweeps)
    return sfail(s, TR_ERR_INVALID_ARG, "max_sweeps=%d outside [0, %d]", r.max_sweeps,
                 kMaxServedSweeps);
  return TR_OK;
}

}  // namespace

extern "C" {

tr_status tr_server_create(const tr_server_config* cfg, tr_server** out) {
  if (!cfg || !out) return sfail(nullptr, TR_ERR_INVALID_ARG, "NULL config or output");
  *out = nullptr;
  const tr_server_config& c = *cfg;
  if (c.max_slots < 1 || c.max_slots > 4096)
    return sfail(nullptr, TR_ERR_INVALID_ARG, "max_slots=%d outside [1, 4096]", c.max_slots);
  if (c.max_modes < 2 || c.max_modes > kMaxModes)
    return sfail(nullptr, TR_ERR_INVALID_ARG, "max_modes=%d outside [2, %d]", c.max_modes,
                 kMaxModes);
  if (c.max_rank < 1 || c.max_rank > 16)
    return sfail(nullptr, TR_ERR_INVALID_ARG, "max_rank=%d outside [1, 16]", c.max_rank);
  if (c.max_dim < 1 || c.max_dim > INT32_MAX || c.max_samples < 1 || c.max_samples > INT32_MAX)
    return sfail(nullptr, TR_ERR_INVALID_ARG, "max_dim or max_samples out of range");
  if (c.max_sweeps < 1 || c.max_sweeps > kMaxServedSweeps)
    return sfail(nullptr, TR_ERR_INVALID_ARG, "max_sweeps=%d outside [1, %d]", c.max_sweeps,
                 kMaxServedSweeps);
  if (!(c.fit_tol >= 0.0)) return sfail(nullptr, TR_ERR_INVALID_ARG, "fit_tol must be >= 0");
  if (c.X_dtype != TR_F32 && c.X_dtype != TR_F64)
    return sfail(nullptr, TR_ERR_INVALID_ARG, "bad X dtype");
  if (c.prec != TR_PREC_FP64 && c.prec != TR_PREC_MIXED)
    return sfail(nullptr, TR_ERR_INVALID_ARG, "bad precision");
  if (c.arena_bytes < 256 || c.arena_bytes > c.hbm_budget_bytes)
    return sfail(nullptr, TR_ERR_INVALID_ARG, "arena_bytes must be in [256, hbm_budget_bytes]");
  int count = 0;
  if (cudaGetDeviceCount(&count) != cudaSuccess || c.device < 0 || c.device >= count) {
    cudaGetLastError();
    return sfail(nullptr, TR_ERR_INVALID_ARG, "no CUDA device %d", c.device);
  }
  tr_server* s = new tr_server;
  s->cfg = c;
  s->f64 = c.prec == TR_PREC_FP64;
  s->xf64 = c.X_dtype == TR_F64;
  DeviceGuard g(c.device);
  const int S = c.max_slots;
  const char* which = "";
  cudaError_t e = g.ok ? init_kernel_attributes(&which) : cudaErrorInvalidDevice;
  auto step = [&](cudaError_t r) { if (e == cudaSuccess) e = r; };
  step(cudaMalloc(&s->arena, c.arena_bytes));
  step(cudaMalloc(&s->dtab, sizeof(BInst) * S));
  step(cudaMalloc(&s->dstate, sizeof(SlotState) * S));
  step(cudaMalloc(&s->dfitp, sizeof(double) * 2 * kFitParts * S));
  step(cudaMalloc(&s->dhist, sizeof(double) * kMaxServedSweeps * S));
  step(cudaMalloc(&s->dcounter, sizeof(unsigned) * S));
  step(cudaMalloc(&s->derr, sizeof(unsigned)));
  step(cudaMallocHost(&s->htab, sizeof(BInst) * S));
  step(cudaMallocHost(&s->hstate, sizeof(SlotState) * S));
  step(cudaMallocHost(&s->hhist, sizeof(double) * kMaxServedSweeps * S));
  step(cudaMallocHost(&s->herr, sizeof(unsigned)));
  step(cudaStreamCreateWithFlags(&s->st, cudaStreamNonBlocking));
  step(cudaStreamCreateWithFlags(&s->side, cudaStreamNonBlocking));
  step(cudaEventCreateWithFlags(&s->ev_fork, cudaEventDisableTiming));
  step(cudaEventCreateWithFlags(&s->ev_info, cudaEventDisableTiming));
  step(cudaEventCreateWithFlags(&s->ev_join, cudaEventDisableTiming));
  if (e == cudaSuccess) {
    step(cudaMemset(s->dtab, 0, sizeof(BInst) * S));
    step(cudaMemset(s->dstate, 0, sizeof(SlotState) * S));
    step(cudaMemset(s->dhist, 0, sizeof(double) * kMaxServedSweeps * S));
    step(cudaMemset(s->derr, 0, sizeof(unsigned)));
  }
  if (e != cudaSuccess) {
    sfail(nullptr, TR_ERR_CUDA, "server set-up failed %s: %s", which, cudaGetErrorString(e));
    cudaGetLastError();
    free_all(s);
    delete s;
    return e == cudaErrorMemoryAllocation ? TR_ERR_OOM : TR_ERR_CUDA;
  }
  std::memset(s->htab, 0, sizeof(BInst) * S);
  std::memset(s->hstate, 0, sizeof(SlotState) * S);
  s->slots.assign(S, Slot{});
  s->alloc.reset(c.arena_bytes);
  // Launch geometry from the limits (independent of the requests in flight).
  const int Lmax = c.max_rank * c.max_rank;
  s->geo.f64 = s->f64;
  s->geo.xf64 = s->xf64;
  s->geo.Jmax = c.max_samples;
  s->geo.Lmax = Lmax;
  s->geo.Imax = c.max_dim;
  s->geo.n1max = static_cast<int>(std::min<int64_t>(c.max_dim, Lmax));
  s->geo.n2max = static_cast<int>(std::min<int64_t>(c.max_dim, Lmax - 1));
  for (int b = 8; b < S; b *= 2) s->buckets.push_back(b);
  s->buckets.push_back(S);
  for (int b : s->buckets) {
    cudaGraph_t gr = nullptr;
    cudaGraphExec_t ge = nullptr;
    e = cudaStreamBeginCapture(s->st, cudaStreamCaptureModeThreadLocal);
    cudaError_t e2 = e == cudaSuccess ? issue_tick(s, b, s->st) : e;
    if (e == cudaSuccess) e = cudaStreamEndCapture(s->st, &gr);
    if (e == cudaSuccess) e = e2;
    if (e == cudaSuccess) e = cudaGraphInstantiate(&ge, gr, 0);
    if (gr) cudaGraphDestroy(gr);
    if (e != cudaSuccess) {
      sfail(nullptr, TR_ERR_CUDA, "tick graph capture (%d slots) failed: %s", b,
            cudaGetErrorString(e));
      cudaGetLastError();
      free_all(s);
      delete s;
      return TR_ERR_CUDA;
    }
    s->graphs.push_back(ge);
  }
  *out = s;
  return TR_OK;
}

void tr_server_destroy(tr_server* s) {
  if (!s) return;
  tr_server_stop(s);
  DeviceGuard g(s->cfg.device);
  cudaStreamSynchronize(s->st);
  cudaStreamSynchronize(s->side);
  free_all(s);
  delete s;
}

const char* tr_server_last_error(const tr_server* s) {
  return s ? s->last_error.c_str() : g_server_error.c_str();
}

tr_status tr_server_submit(tr_server* s, const tr_request* req, int64_t* ticket) {
  if (!s || !req || !ticket) return TR_ERR_INVALID_ARG;
  const tr_request& r = *req;
  const tr_status chk = check_request(s, r);
  if (chk != TR_OK) {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stats.rejected += 1;
    return chk;
  }
  const size_t ws = request_ws(r, s->f64, s->xf64);
  const size_t charge = request_charge(r, s->xf64, ws);
  if (ws > s->cfg.arena_bytes || charge > s->cfg.hbm_budget_bytes) {
    {
      std::lock_guard<std::mutex> lk(s->mu);
      s->stats.rejected += 1;
    }
    return sfail(s, TR_ERR_BUDGET, "request needs %zu bytes (workspace %zu); budget %zu, arena %zu",
                 charge, ws, s->cfg.hbm_budget_bytes, s->cfg.arena_bytes);
  }
  {
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->failed) {
      s->last_error = "the server failed earlier";
      return TR_ERR_CUDA;
    }
    const int64_t t = s->next_ticket++;
    tr_result res{};
    res.t_submit_ns = now_ns();
    s->results[t] = res;
    s->queue.push_back(Pending{t, r, ws, charge});
    s->stats.submitted += 1;
    *ticket = t;
  }
  s->cv_work.notify_one();
  return TR_OK;
}

tr_status tr_server_tick(tr_server* s, int* active) {
  if (!s) return TR_ERR_INVALID_ARG;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->worker_on) {
      s->last_error = "tr_server_tick while the worker runs";
      return TR_ERR_INVALID_ARG;
    }
  }
  return run_tick(s, active);
}

tr_status tr_server_start(tr_server* s) {
  if (!s) return TR_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(s->mu);
  if (s->worker_on) return TR_OK;
  s->stopping = false;
  s->worker_on = true;
  s->worker = std::thread(worker_loop, s);
  return TR_OK;
}

tr_status tr_server_stop(tr_server* s) {
  if (!s) return TR_ERR_INVALID_ARG;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    if (!s->worker_on) return TR_OK;
    s->stopping = true;
  }
  s->cv_work.notify_all();
  if (s->worker.joinable()) s->worker.join();
  std::lock_guard<std::mutex> lk(s->mu);
  s->worker_on = false;
  s->stopping = false;
  return TR_OK;
}

tr_status tr_server_poll(tr_server* s, int64_t ticket, tr_result* out) {
  if (!s || !out) return TR_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->results.find(ticket);
  if (it == s->results.end()) return TR_ERR_INVALID_ARG;
  *out = it->second;
  return TR_OK;
}

tr_status tr_server_wait(tr_server* s, int64_t ticket, int64_t timeout_ms, tr_result* out) {
  if (!s || !out) return TR_ERR_INVALID_ARG;
  const auto deadline = std::chrono::steady_clock::now() + std::chrono::milliseconds(timeout_ms);
  for (;;) {
    bool worker;
    {
      std::unique_lock<std::mutex> lk(s->mu);
      auto it = s->results.find(ticket);
      if (it == s->results.end()) return TR_ERR_INVALID_ARG;
      worker = s->worker_on;
      if (worker) {
        const bool ok = s->cv_done.wait_until(lk, deadline, [&] {
          auto jt = s->results.find(ticket);
          return jt == s->results.end() || jt->second.done;
        });
        auto jt = s->results.find(ticket);
        if (jt == s->results.end()) return TR_ERR_INVALID_ARG;
        *out = jt->second;
        return ok ? TR_OK : TR_ERR_TIMEOUT;
      }
      if (it->second.done) {
        *out = it->second;
        return TR_OK;
      }
    }
    if (std::chrono::steady_clock::now() >= deadline) {
      tr_server_poll(s, ticket, out);
      return TR_ERR_TIMEOUT;
    }
    const tr_status st = run_tick(s, nullptr);
    if (st != TR_OK) {
      tr_server_poll(s, ticket, out);
      return st;
    }
  }
}

tr_status tr_server_release(tr_server* s, int64_t ticket) {
  if (!s) return TR_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->results.find(ticket);
  if (it == s->results.end() || !it->second.done) return TR_ERR_INVALID_ARG;
  s->results.erase(it);
  return TR_OK;
}

tr_status tr_server_get_stats(tr_server* s, tr_server_stats* out) {
  if (!s || !out) return TR_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(s->mu);
  *out = s->stats;
  out->active = s->active;
  out->queued = static_cast<int>(s->queue.size());
  out->charged_bytes = s->charged;
  return TR_OK;
}

}  // extern "C"
