// nlos_reconstruct_noalloc: a reconstruction that allocates nothing.
//
// Some callers cannot call cudaMalloc when they reconstruct: real-time
// capture loops, where an allocation may synchronise the device and stall a
// frame for an unbounded time; host applications that hand this library a
// fixed share of device memory and own the rest through their own pool, so
// that any further allocation fails or competes with them; and code that is
// not allowed to allocate at that point of its control flow. For them this
// entry point runs a plan's stage sequence with its scratch taken from a
// fixed array in device memory instead of the plan's workspace. The plan
// itself (and its tables) must have been created earlier.
//
// The scratch is a file-scope __device__ array of kNoAllocScratchBytes
// (32 MiB). Every GPU that loads this library holds its own copy until the
// process exits. Host code only sees a host-side stand-in for the array's
// name, so the device address is looked up with cudaGetSymbolAddress once per
// device (with that device current) and cached; that synchronous lookup
// happens in the first call on each device only. Plans whose workspace
// exceeds the array are rejected with
// NLOS_ERR_INVALID_ARG. Every call shares the array and it keeps the previous
// call's contents: each stage writes its scratch before reading it, and the
// only accumulator (the phasor-field depth sum) is cleared by the sequence
// itself on every call. Calls that overlap on the GPU (for example, calls on
// different streams) race on the array and must be serialised by the caller.
// The device error word of the bounded waits lives inside the array, which
// nlos_workspace_check does not read: a wait that gives up on this path is
// not reported (the call still returns its launch status).
#include <stdio.h>

#include <mutex>

#include "nlos.h"
#include "nlos_internal.h"

namespace nlos {
size_t plan_workspace_bytes(const nlos_plan_s* p);
bool plan_profiling(const nlos_plan_s* p);
nlos_status_t plan_run(nlos_plan_s* p, const void* H, void* vol, void* ws, cudaStream_t s);
nlos_status_t set_error(nlos_status_t st, const char* msg);
}  // namespace nlos

namespace {
constexpr size_t kNoAllocScratchBytes = size_t(32) << 20;
constexpr int kMaxDevices = 64;
std::mutex g_scratch_mu;
void* g_scratch_ptr[kMaxDevices] = {};
}  // namespace

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

extern "C" nlos_status_t nlos_reconstruct_noalloc(nlos_plan_t plan, const void* transient, void* volume,
                                                  void* stream) {
  using namespace nlos;
  char msg[256];
  if (!plan) return set_error(NLOS_ERR_INVALID_ARG, "plan is NULL");
  if (!transient || !volume) return set_error(NLOS_ERR_INVALID_ARG, "transient/volume is NULL");
  const size_t need = plan_workspace_bytes(plan);
  if (need > kNoAllocScratchBytes) {
    snprintf(msg, sizeof msg, "plan needs %zu bytes of scratch; the fixed scratch holds %zu bytes", need,
             kNoAllocScratchBytes);
    return set_error(NLOS_ERR_INVALID_ARG, msg);
  }
  if (plan_profiling(plan))
    return set_error(NLOS_ERR_INVALID_ARG, "stage tracing creates events; disable it before this call");
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) {
    snprintf(msg, sizeof msg, "cudaGetDevice: %s", cudaGetErrorString(e));
    return set_error(NLOS_ERR_CUDA, msg);
  }
  if (dev < 0 || dev >= kMaxDevices) return set_error(NLOS_ERR_UNSUPPORTED, "device ordinal out of range");
  void* scratch = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_scratch_mu);
    if (!g_scratch_ptr[dev]) {
      void* p = nullptr;
      e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
      if (e != cudaSuccess) {
        snprintf(msg, sizeof msg, "cudaGetSymbolAddress(scratch): %s", cudaGetErrorString(e));
        return set_error(NLOS_ERR_CUDA, msg);
      }
      g_scratch_ptr[dev] = p;
    }
    scratch = g_scratch_ptr[dev];
  }
  return plan_run(plan, transient, volume, scratch, static_cast<cudaStream_t>(stream));
}
