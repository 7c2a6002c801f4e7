// Continuous-batching reconstruction server.
//
// Requests (a capture description plus caller-owned device input and output
// buffers) are queued by any thread and served by one scheduler thread:
//   - plans are created and autotuned once per distinct description (outside
//     the queue's lock, so running work is not held up) and stay resident on
//     the device;
//   - the memory budget covers both the resident plans (tables, twiddles,
//     radial kernels, tensor-core operand stores, dense kernels) and the
//     workspaces of the requests on the device; a new plan that does not fit
//     evicts idle plans (no request queued or running) in least-recently-used
//     order;
//   - a request is admitted, in arrival order, as soon as a slot (a stream)
//     is free and its workspace (the padded volume's footprint) fits in what
//     the budget leaves next to the resident plans and running requests;
//   - the scheduler launches outside the lock, on the slot's stream, so work
//     that arrives while others run overlaps with them on the GPU; the
//     stream's priority ranks the request by age (one level below the
//     lowest-priority request running at its admission, the highest when
//     none runs), so a later arrival takes the SMs an older, larger request
//     leaves idle instead of slowing it;
//   - workspaces come from the stream-ordered allocator (cudaMallocAsync /
//     cudaFreeAsync on the slot's stream), so admissions never force a
//     device-wide synchronisation;
//   - completion is signalled by a host function enqueued behind each
//     request on its stream (no polling); a request's latency is the host
//     time from submission to that signal.
// Each request's arithmetic is exactly that of a standalone reconstruction
// with the same plan, so results are the same alone and in the mix.
#include <algorithm>
#include <chrono>
#include <cstdint>
#include <condition_variable>
#include <cstdio>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "nlos.h"
#include "nlos_internal.h"

namespace nlos {
size_t plan_workspace_bytes(const nlos_plan_s* p);
size_t plan_resident_bytes(const nlos_plan_s* p);
nlos_status_t plan_run(nlos_plan_s* p, const void* H, void* vol, void* ws, cudaStream_t s);
nlos_status_t set_error(nlos_status_t st, const char* msg);
}  // namespace nlos

namespace {

using Clock = std::chrono::steady_clock;

struct PlanEntry {
  nlos_plan_t plan = nullptr;
  size_t bytes = 0;        // resident device memory of the plan
  uint64_t last_use = 0;   // LRU stamp
  int users = 0;           // requests queued or running with this plan
};

struct Request {
  uint64_t id = 0;
  PlanEntry* entry = nullptr;
  const void* in = nullptr;
  void* out = nullptr;
  size_t need = 0;
  Clock::time_point t_submit;
  double latency_ms = 0.0;
  int state = 0;   // 0 queued, 1 running, 2 done, 3 failed
  int status = NLOS_OK;
};

struct Slot;
struct Done {
  nlos_server_s* sv = nullptr;
  Slot* slot = nullptr;
};

// Stream priority levels a slot can run at: a request is admitted at the
// level of how many requests already run (the oldest runs at the highest
// priority), so later arrivals fill the SMs the older ones leave idle
// instead of slowing them down.
constexpr int kPrioLevels = 4;

struct Slot {
  cudaStream_t prio[kPrioLevels] = {};   // one stream per level, highest first
  cudaStream_t stream = nullptr;         // the running request's stream
  int level = 0;                         // and its level
  Request* req = nullptr;
  Done done;
};

std::string desc_key(const nlos_plan_desc_t& d) {
  char buf[512];
  snprintf(buf, sizeof buf, "%d %d %d %.17g %.17g %.17g %d %d %d %.17g %.17g %d %.17g %.17g %d %d %.17g %d", d.nx,
           d.ny, d.nt, d.bin_width_s, d.wall_w_m, d.wall_h_m, d.method, d.storage, d.pad_factor, d.wavelength_m,
           d.cycles, d.n_depths, d.depth_min_m, d.depth_max_m, d.sigma_s, d.sigma_t, d.delta_m, d.output);
  return buf;
}

}  // namespace

struct nlos_server_s {
  size_t budget = 0;
  size_t in_use = 0;       // workspaces of running requests
  size_t resident = 0;     // resident plans
  uint64_t evictions = 0;
  uint64_t lru = 0;
  std::vector<Slot> slots;
  std::map<std::string, PlanEntry*> plans;
  std::deque<Request*> queue;
  std::unordered_map<uint64_t, Request*> reqs;
  std::vector<double> latencies;
  uint64_t next_id = 1;
  uint64_t completed = 0;
  Clock::time_point t_first, t_last;
  bool have_first = false;
  bool stop = false;
  int device = 0;
  std::mutex mu;           // queue, slots, accounting, plan entries
  std::mutex plan_mu;      // serialises plan creation and eviction (device work, outside mu)
  std::condition_variable cv_work, cv_done;
  std::thread th;
};

namespace {

// Completion of a request; called with sv->mu held.
void finish(nlos_server_s* sv, Slot& sl, bool ok) {
  Request* r = sl.req;
  const auto now = Clock::now();
  r->latency_ms = std::chrono::duration<double, std::milli>(now - r->t_submit).count();
  r->state = ok ? 2 : 3;
  sv->in_use -= r->need;
  --r->entry->users;
  sv->latencies.push_back(r->latency_ms);
  ++sv->completed;
  sv->t_last = now;
  sl.req = nullptr;
}

// Host function behind each request on its slot's stream (a CUDA runtime
// thread runs it; it makes no CUDA calls).
void CUDART_CB on_done(void* arg) {
  Done* d = static_cast<Done*>(arg);
  nlos_server_s* sv = d->sv;
  {
    std::lock_guard<std::mutex> lk(sv->mu);
    if (d->slot->req) finish(sv, *d->slot, d->slot->req->status == NLOS_OK);
  }
  sv->cv_done.notify_all();
  sv->cv_work.notify_one();
}

// Evict idle plans (least recently used first) until `extra` more bytes fit
// in the budget; the evicted plans are appended to `victims` for the caller
// to destroy outside the lock. Called with sv->mu held.
void evict_idle(nlos_server_s* sv, size_t extra, std::vector<nlos_plan_t>& victims) {
  while (sv->resident + sv->in_use + extra > sv->budget) {
    auto victim = sv->plans.end();
    for (auto it = sv->plans.begin(); it != sv->plans.end(); ++it)
      if (it->second->users == 0 && (victim == sv->plans.end() || it->second->last_use < victim->second->last_use))
        victim = it;
    if (victim == sv->plans.end()) return;
    victims.push_back(victim->second->plan);
    sv->resident -= victim->second->bytes;
    ++sv->evictions;
    delete victim->second;
    sv->plans.erase(victim);
  }
}

void scheduler(nlos_server_s* sv) {
  cudaSetDevice(sv->device);
  std::unique_lock<std::mutex> lk(sv->mu);
  std::vector<nlos_plan_t> victims;
  while (true) {
    // admit the head of the queue when a slot is free and its workspace fits
    // (idle resident plans give way to it)
    Request* r = nullptr;
    Slot* slot = nullptr;
    if (!sv->queue.empty()) {
      Request* head = sv->queue.front();
      for (Slot& sl : sv->slots)
        if (!sl.req) {
          slot = &sl;
          break;
        }
      if (slot) evict_idle(sv, head->need, victims);
      if (slot && sv->resident + sv->in_use + head->need <= sv->budget) {
        // one level below the lowest-priority running request (the highest
        // level when none runs)
        int level = 0;
        for (Slot& sl : sv->slots)
          if (sl.req) level = std::max(level, std::min(sl.level + 1, kPrioLevels - 1));
        r = head;
        sv->queue.pop_front();
        r->state = 1;
        slot->req = r;
        slot->level = level;
        slot->stream = slot->prio[level];
        sv->in_use += r->need;
      }
    }
    if (r || !victims.empty()) {
      // device work outside the lock: submitters and completions proceed meanwhile
      lk.unlock();
      for (nlos_plan_t v : victims) nlos_plan_destroy(v);
      victims.clear();
      if (!r) {
        lk.lock();
        continue;
      }
      void* ws = nullptr;
      nlos_status_t st = cudaMallocAsync(&ws, r->need, slot->stream) == cudaSuccess ? NLOS_OK : NLOS_ERR_OUT_OF_MEMORY;
      if (st == NLOS_OK) st = nlos::plan_run(r->entry->plan, r->in, r->out, ws, slot->stream);
      if (ws) cudaFreeAsync(ws, slot->stream);
      r->status = st;
      if (st == NLOS_OK && cudaLaunchHostFunc(slot->stream, on_done, &slot->done) != cudaSuccess)
        r->status = st = NLOS_ERR_CUDA;
      lk.lock();
      if (st != NLOS_OK) {
        finish(sv, *slot, false);
        sv->cv_done.notify_all();
      }
      continue;
    }
    bool busy = false;
    for (Slot& sl : sv->slots) busy = busy || sl.req;
    if (sv->stop && !busy && sv->queue.empty()) break;
    sv->cv_work.wait(lk);   // woken by a submission, a completion or shutdown
  }
}

double percentile(std::vector<double> v, double q) {
  if (v.empty()) return 0.0;
  std::sort(v.begin(), v.end());
  const size_t i = (size_t)std::min<double>(v.size() - 1, q * (v.size() - 1) + 0.5);
  return v[i];
}

// The entry of desc's plan with one more user, creating the plan (and
// evicting idle plans in LRU order to make room for it and a workspace of
// `ws_floor` bytes) if it is not resident. Called with sv->plan_mu held and
// sv->mu not held.
nlos_status_t acquire_plan(nlos_server_s* sv, const nlos_plan_desc_t& d, PlanEntry** out) {
  const std::string key = desc_key(d);
  {
    std::lock_guard<std::mutex> lk(sv->mu);
    auto it = sv->plans.find(key);
    if (it != sv->plans.end()) {
      ++it->second->users;
      it->second->last_use = ++sv->lru;
      *out = it->second;
      return NLOS_OK;
    }
  }
  nlos_plan_t p = nullptr;
  nlos_status_t st = nlos_plan_create_ex(&d, NLOS_PLAN_NO_WORKSPACE, &p);
  if (st != NLOS_OK) return st;
  const size_t bytes = nlos::plan_resident_bytes(p), need = nlos::plan_workspace_bytes(p);
  if (bytes + need > sv->budget) {
    nlos_plan_destroy(p);
    char msg[200];
    snprintf(msg, sizeof msg, "plan (%zu bytes) and workspace (%zu bytes) exceed the budget of %zu bytes", bytes,
             need, sv->budget);
    return nlos::set_error(NLOS_ERR_OUT_OF_MEMORY, msg);
  }
  // launch shapes picked once per description (the process-wide autotune
  // cache): a resident plan serves every later request with the tuned shapes
  if ((st = nlos_plan_autotune(p, nullptr)) != NLOS_OK) {
    nlos_plan_destroy(p);
    return st;
  }
  std::vector<nlos_plan_t> victims;
  {
    std::unique_lock<std::mutex> lk(sv->mu);
    while (true) {
      // evict idle plans, least recently used first, until the new plan and
      // one request's workspace fit next to what is resident and running
      evict_idle(sv, bytes + need, victims);
      if (sv->resident + sv->in_use + bytes + need <= sv->budget) break;
      // every resident plan is in use: wait for requests to finish
      bool busy = !sv->queue.empty();
      for (Slot& sl : sv->slots) busy = busy || sl.req;
      if (!busy) break;   // nothing will free memory: admit over what fits (it runs alone)
      sv->cv_done.wait_for(lk, std::chrono::milliseconds(50));
    }
    PlanEntry* e = new PlanEntry();
    e->plan = p;
    e->bytes = bytes;
    e->users = 1;
    e->last_use = ++sv->lru;
    sv->plans[key] = e;
    sv->resident += bytes;
    *out = e;
  }
  for (nlos_plan_t v : victims) nlos_plan_destroy(v);
  return NLOS_OK;
}

}  // namespace

extern "C" {

nlos_status_t nlos_server_create(size_t memory_budget_bytes, int n_slots, nlos_server_t* out) {
  using namespace nlos;
  if (!out) return set_error(NLOS_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (memory_budget_bytes == 0 || n_slots <= 0 || n_slots > 64)
    return set_error(NLOS_ERR_INVALID_ARG, "budget must be > 0 and slots in [1, 64]");
  nlos_server_s* sv = new nlos_server_s();
  sv->budget = memory_budget_bytes;
  cudaGetDevice(&sv->device);
  // keep freed workspaces in the stream-ordered pool instead of returning them
  cudaMemPool_t pool;
  if (cudaDeviceGetDefaultMemPool(&pool, sv->device) == cudaSuccess) {
    uint64_t keep = UINT64_MAX;
    cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
  }
  sv->slots.resize(n_slots);
  int least = 0, greatest = 0;
  if (cudaDeviceGetStreamPriorityRange(&least, &greatest) != cudaSuccess) least = greatest = 0;
  for (Slot& sl : sv->slots) {
    sl.done.sv = sv;
    sl.done.slot = &sl;
    bool ok = true;
    for (int k = 0; k < kPrioLevels && ok; ++k) {
      // greatest is the numerically lowest value; levels past the range repeat the least
      const int prio = std::min(greatest + k, least);
      ok = cudaStreamCreateWithPriority(&sl.prio[k], cudaStreamNonBlocking, prio) == cudaSuccess;
    }
    sl.stream = sl.prio[0];
    if (!ok) {
      for (Slot& t : sv->slots)
        for (cudaStream_t st : t.prio)
          if (st) cudaStreamDestroy(st);
      delete sv;
      return set_error(NLOS_ERR_CUDA, "server streams");
    }
  }
  sv->th = std::thread(scheduler, sv);
  *out = sv;
  return NLOS_OK;
}

nlos_status_t nlos_server_preload(nlos_server_t sv, const nlos_plan_desc_t* desc) {
  using namespace nlos;
  if (!sv || !desc) return set_error(NLOS_ERR_INVALID_ARG, "NULL argument");
  std::lock_guard<std::mutex> pk(sv->plan_mu);
  PlanEntry* e = nullptr;
  nlos_status_t st = acquire_plan(sv, *desc, &e);
  if (st != NLOS_OK) return st;
  std::lock_guard<std::mutex> lk(sv->mu);
  --e->users;
  return NLOS_OK;
}

nlos_status_t nlos_server_submit(nlos_server_t sv, const nlos_plan_desc_t* desc, const void* transient,
                                 void* volume, uint64_t* ticket) {
  using namespace nlos;
  if (!sv || !desc || !transient || !volume || !ticket) return set_error(NLOS_ERR_INVALID_ARG, "NULL argument");
  {
    std::lock_guard<std::mutex> lk(sv->mu);
    if (sv->stop) return set_error(NLOS_ERR_INVALID_ARG, "server is shutting down");
  }
  PlanEntry* e = nullptr;
  {
    std::lock_guard<std::mutex> pk(sv->plan_mu);
    nlos_status_t st = acquire_plan(sv, *desc, &e);
    if (st != NLOS_OK) return st;
  }
  Request* r = new Request();
  r->entry = e;
  r->in = transient;
  r->out = volume;
  r->need = plan_workspace_bytes(e->plan);
  r->t_submit = Clock::now();
  {
    std::lock_guard<std::mutex> lk(sv->mu);
    r->id = sv->next_id++;
    if (!sv->have_first) {
      sv->have_first = true;
      sv->t_first = r->t_submit;
    }
    sv->reqs[r->id] = r;
    sv->queue.push_back(r);
    *ticket = r->id;
  }
  sv->cv_work.notify_one();
  return NLOS_OK;
}

nlos_status_t nlos_server_wait(nlos_server_t sv, uint64_t ticket, double timeout_s, double* latency_ms) {
  using namespace nlos;
  if (!sv) return set_error(NLOS_ERR_INVALID_ARG, "server is NULL");
  std::unique_lock<std::mutex> lk(sv->mu);
  auto it = sv->reqs.find(ticket);
  if (it == sv->reqs.end()) return set_error(NLOS_ERR_INVALID_ARG, "unknown ticket");
  Request* r = it->second;
  const auto deadline = Clock::now() + std::chrono::duration<double>(timeout_s > 0 ? timeout_s : 3600.0);
  while (r->state < 2) {
    if (sv->cv_done.wait_until(lk, deadline) == std::cv_status::timeout && r->state < 2)
      return set_error(NLOS_ERR_TIMEOUT, "request not finished before the timeout");
  }
  if (latency_ms) *latency_ms = r->latency_ms;
  const int status = r->status;
  sv->reqs.erase(it);
  delete r;
  if (status != NLOS_OK) return set_error((nlos_status_t)status, "request failed on the device");
  return NLOS_OK;
}

nlos_status_t nlos_server_stats(nlos_server_t sv, double* p50_ms, double* p99_ms, double* volumes_per_s,
                                unsigned long long* completed, int reset) {
  using namespace nlos;
  if (!sv) return set_error(NLOS_ERR_INVALID_ARG, "server is NULL");
  std::lock_guard<std::mutex> lk(sv->mu);
  if (p50_ms) *p50_ms = percentile(sv->latencies, 0.50);
  if (p99_ms) *p99_ms = percentile(sv->latencies, 0.99);
  if (completed) *completed = sv->completed;
  if (volumes_per_s) {
    const double span = sv->have_first ? std::chrono::duration<double>(sv->t_last - sv->t_first).count() : 0.0;
    *volumes_per_s = span > 0 ? sv->completed / span : 0.0;
  }
  if (reset) {
    sv->latencies.clear();
    sv->completed = 0;
    sv->have_first = false;
  }
  return NLOS_OK;
}

nlos_status_t nlos_server_memory(nlos_server_t sv, size_t* plan_bytes, size_t* workspace_bytes,
                                 unsigned long long* evictions) {
  using namespace nlos;
  if (!sv) return set_error(NLOS_ERR_INVALID_ARG, "server is NULL");
  std::lock_guard<std::mutex> lk(sv->mu);
  if (plan_bytes) *plan_bytes = sv->resident;
  if (workspace_bytes) *workspace_bytes = sv->in_use;
  if (evictions) *evictions = sv->evictions;
  return NLOS_OK;
}

nlos_status_t nlos_server_destroy(nlos_server_t sv) {
  using namespace nlos;
  if (!sv) return set_error(NLOS_ERR_INVALID_ARG, "server is NULL");
  {
    std::lock_guard<std::mutex> lk(sv->mu);
    sv->stop = true;
  }
  sv->cv_work.notify_all();
  sv->th.join();
  for (Slot& sl : sv->slots)
    for (cudaStream_t st : sl.prio) {
      cudaStreamSynchronize(st);
      cudaStreamDestroy(st);
    }
  for (auto& kv : sv->plans) {
    nlos_plan_destroy(kv.second->plan);
    delete kv.second;
  }
  for (auto& kv : sv->reqs) delete kv.second;
  delete sv;
  return NLOS_OK;
}

}  // extern "C"
