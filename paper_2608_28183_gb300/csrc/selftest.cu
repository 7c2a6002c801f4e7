// Device self-test of the bounded-wait path used by the TMA-staged kernels:
// a barrier that nothing ever arrives on must make the wait give up after its
// iteration limit and record a timeout in the error word, leaving the context
// usable.
#include "nlos.h"
#include "nlos_internal.h"
#include "nlos_tma.cuh"

namespace nlos {
nlos_status_t set_error(nlos_status_t st, const char* msg);
}  // namespace nlos

namespace {
__global__ void bounded_wait_probe_kernel(int limit, int* err) {
  __shared__ uint64_t bar;
  if (threadIdx.x == 0) {
    nlos::mbar_init(&bar, 1);
    nlos::mbar_fence_init();
  }
  __syncthreads();
  const bool done = nlos::mbar_wait_bounded(&bar, 0, limit);   // no arrival is ever made
  if (!done && threadIdx.x == 0) atomicExch(err, nlos::kDevErrTmaTimeout);
}
}  // namespace

extern "C" nlos_status_t nlos_selftest_bounded_wait(int limit, int* code) {
  using namespace nlos;
  if (limit <= 0 || !code) return set_error(NLOS_ERR_INVALID_ARG, "limit must be > 0 and code non-NULL");
  int* d = nullptr;
  if (cudaMalloc(&d, sizeof(int)) != cudaSuccess) return set_error(NLOS_ERR_OUT_OF_MEMORY, "self-test word");
  cudaMemset(d, 0, sizeof(int));
  bounded_wait_probe_kernel<<<1, 32>>>(limit, d);
  cudaError_t e = cudaDeviceSynchronize();
  int v = 0;
  if (e == cudaSuccess) e = cudaMemcpy(&v, d, sizeof v, cudaMemcpyDeviceToHost);
  cudaFree(d);
  if (e != cudaSuccess) return set_error(NLOS_ERR_CUDA, cudaGetErrorString(e));
  *code = v;
  if (v == kDevErrTmaTimeout) return set_error(NLOS_ERR_TIMEOUT, "wait gave up at its iteration limit");
  return NLOS_OK;
}
