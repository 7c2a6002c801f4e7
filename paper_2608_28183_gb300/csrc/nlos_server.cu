// Continuous-batching reconstruction server.
//
// Requests (a capture description plus caller-owned device input and output
// buffers) are queued by any thread and served by one scheduler thread:
//   - plans are created once per distinct description and stay resident on
//     the device (tables, twiddles, radial kernels) for the server's life;
//   - a request is admitted, in arrival order, as soon as a slot (a stream)
//     is free and its workspace (the padded volume's footprint) fits in the
//     memory budget next to the requests already on the device;
//   - admitted requests run on their slot's stream, so work that arrives while
//     others are running overlaps with them on the GPU;
//   - workspaces come from the stream-ordered allocator (cudaMallocAsync /
//     cudaFreeAsync on the slot's stream), so admissions never force a
//     device-wide synchronisation;
//   - completion is detected with events; a request's latency is the host time
//     from submission to the scheduler observing its completion event.
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
nlos_status_t plan_run(nlos_plan_s* p, const void* H, void* vol, void* ws, cudaStream_t s);
nlos_status_t set_error(nlos_status_t st, const char* msg);
}  // namespace nlos

namespace {

using Clock = std::chrono::steady_clock;

struct Request {
  uint64_t id = 0;
  nlos_plan_t plan = nullptr;
  const void* in = nullptr;
  void* out = nullptr;
  size_t need = 0;
  Clock::time_point t_submit;
  double latency_ms = 0.0;
  int state = 0;   // 0 queued, 1 running, 2 done, 3 failed
  int status = NLOS_OK;
};

struct Slot {
  cudaStream_t stream = nullptr;
  cudaEvent_t done = nullptr;
  Request* req = nullptr;
  void* ws = nullptr;
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
  size_t in_use = 0;
  std::vector<Slot> slots;
  std::map<std::string, nlos_plan_t> plans;
  std::deque<Request*> queue;
  std::unordered_map<uint64_t, Request*> reqs;
  std::vector<double> latencies;
  uint64_t next_id = 1;
  uint64_t completed = 0;
  Clock::time_point t_first, t_last;
  bool have_first = false;
  bool stop = false;
  int device = 0;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::thread th;
};

namespace {

// plan lookup/creation; called with the server lock held
nlos_status_t get_plan(nlos_server_s* sv, const nlos_plan_desc_t& d, nlos_plan_t* out) {
  const std::string key = desc_key(d);
  auto it = sv->plans.find(key);
  if (it != sv->plans.end()) {
    *out = it->second;
    return NLOS_OK;
  }
  nlos_plan_t p = nullptr;
  nlos_status_t st = nlos_plan_create_ex(&d, NLOS_PLAN_NO_WORKSPACE, &p);
  if (st != NLOS_OK) return st;
  sv->plans[key] = p;
  *out = p;
  return NLOS_OK;
}

void finish(nlos_server_s* sv, Slot& sl, bool ok) {
  Request* r = sl.req;
  const auto now = Clock::now();
  r->latency_ms = std::chrono::duration<double, std::milli>(now - r->t_submit).count();
  r->state = ok ? 2 : 3;
  sv->in_use -= r->need;
  sv->latencies.push_back(r->latency_ms);
  ++sv->completed;
  sv->t_last = now;
  sl.req = nullptr;
  sl.ws = nullptr;
}

void scheduler(nlos_server_s* sv) {
  cudaSetDevice(sv->device);
  std::unique_lock<std::mutex> lk(sv->mu);
  while (true) {
    bool changed = false;
    // completions
    for (Slot& sl : sv->slots) {
      if (!sl.req) continue;
      const cudaError_t q = cudaEventQuery(sl.done);
      if (q == cudaErrorNotReady) continue;
      if (q != cudaSuccess) sl.req->status = NLOS_ERR_CUDA;
      finish(sv, sl, q == cudaSuccess);
      changed = true;
    }
    // admissions, in arrival order
    while (!sv->queue.empty()) {
      Request* r = sv->queue.front();
      Slot* free_slot = nullptr;
      for (Slot& sl : sv->slots)
        if (!sl.req) {
          free_slot = &sl;
          break;
        }
      if (!free_slot || sv->in_use + r->need > sv->budget) break;
      sv->queue.pop_front();
      Slot& sl = *free_slot;
      void* ws = nullptr;
      cudaError_t e = cudaMallocAsync(&ws, r->need, sl.stream);
      nlos_status_t st = e == cudaSuccess ? NLOS_OK : NLOS_ERR_OUT_OF_MEMORY;
      if (st == NLOS_OK) st = nlos::plan_run(r->plan, r->in, r->out, ws, sl.stream);
      if (ws) cudaFreeAsync(ws, sl.stream);
      if (st == NLOS_OK && cudaEventRecord(sl.done, sl.stream) != cudaSuccess) st = NLOS_ERR_CUDA;
      r->state = 1;
      sl.req = r;
      sl.ws = ws;
      sv->in_use += r->need;
      if (st != NLOS_OK) {
        r->status = st;
        finish(sv, sl, false);
      }
      changed = true;
    }
    if (changed) sv->cv_done.notify_all();
    bool busy = false;
    for (Slot& sl : sv->slots) busy = busy || sl.req;
    if (sv->stop && !busy && sv->queue.empty()) break;
    if (!busy && sv->queue.empty())
      sv->cv_work.wait(lk);
    else
      sv->cv_work.wait_for(lk, std::chrono::microseconds(20));
  }
}

double percentile(std::vector<double> v, double q) {
  if (v.empty()) return 0.0;
  std::sort(v.begin(), v.end());
  const size_t i = (size_t)std::min<double>(v.size() - 1, q * (v.size() - 1) + 0.5);
  return v[i];
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
  for (Slot& sl : sv->slots) {
    if (cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&sl.done, cudaEventDisableTiming) != cudaSuccess) {
      for (Slot& t : sv->slots) {
        if (t.stream) cudaStreamDestroy(t.stream);
        if (t.done) cudaEventDestroy(t.done);
      }
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
  std::lock_guard<std::mutex> lk(sv->mu);
  nlos_plan_t p;
  return get_plan(sv, *desc, &p);
}

nlos_status_t nlos_server_submit(nlos_server_t sv, const nlos_plan_desc_t* desc, const void* transient,
                                 void* volume, uint64_t* ticket) {
  using namespace nlos;
  if (!sv || !desc || !transient || !volume || !ticket) return set_error(NLOS_ERR_INVALID_ARG, "NULL argument");
  std::lock_guard<std::mutex> lk(sv->mu);
  if (sv->stop) return set_error(NLOS_ERR_INVALID_ARG, "server is shutting down");
  nlos_plan_t p;
  nlos_status_t st = get_plan(sv, *desc, &p);
  if (st != NLOS_OK) return st;
  const size_t need = plan_workspace_bytes(p);
  if (need > sv->budget) {
    char msg[160];
    snprintf(msg, sizeof msg, "request needs %zu bytes of workspace; the budget is %zu", need, sv->budget);
    return set_error(NLOS_ERR_OUT_OF_MEMORY, msg);
  }
  Request* r = new Request();
  r->id = sv->next_id++;
  r->plan = p;
  r->in = transient;
  r->out = volume;
  r->need = need;
  r->t_submit = Clock::now();
  if (!sv->have_first) {
    sv->have_first = true;
    sv->t_first = r->t_submit;
  }
  sv->reqs[r->id] = r;
  sv->queue.push_back(r);
  *ticket = r->id;
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

nlos_status_t nlos_server_destroy(nlos_server_t sv) {
  using namespace nlos;
  if (!sv) return set_error(NLOS_ERR_INVALID_ARG, "server is NULL");
  {
    std::lock_guard<std::mutex> lk(sv->mu);
    sv->stop = true;
    sv->cv_work.notify_all();
  }
  sv->th.join();
  for (Slot& sl : sv->slots) {
    cudaStreamSynchronize(sl.stream);
    cudaStreamDestroy(sl.stream);
    cudaEventDestroy(sl.done);
  }
  for (auto& kv : sv->plans) nlos_plan_destroy(kv.second);
  for (auto& kv : sv->reqs) delete kv.second;
  delete sv;
  return NLOS_OK;
}

}  // extern "C"
