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

// ---------------------------------------------------------------------------
// Tensor-core self-check: one CTA computes D = A B^T (M = 128, N columns,
// K = 64) with tcgen05 MMAs from shared-memory descriptors into tensor
// memory, then reads D back. A and B hold small integers (exact in f16 and
// in the f32 sums), so the host can compare element by element.
// ---------------------------------------------------------------------------
#include <cuda_fp16.h>

#include "nlos_umma.cuh"

namespace {
constexpr int kUmmaM = 128, kUmmaK = 64;

__device__ __forceinline__ float umma_probe_a(int r, int k) { return (float)((r * 3 + k * 5) % 7 - 3); }
__device__ __forceinline__ float umma_probe_b(int n, int k) { return (float)((n * 2 + k * 7) % 5 - 2); }

__global__ void __launch_bounds__(128) umma_probe_kernel(int N, float* out, int* err) {
  using namespace nlos;
  extern __shared__ __align__(128) unsigned char ub_sm[];
  __shared__ uint64_t bar;
  __shared__ uint32_t tbase;
  unsigned char* A = ub_sm;
  unsigned char* B = ub_sm + kUmmaM * kUmmaK * 2;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  for (int i = tid; i < kUmmaM * kUmmaK; i += blockDim.x) {
    const int r = i / kUmmaK, k = i % kUmmaK;
    *reinterpret_cast<__half*>(A + umma_kmajor_offset(r, k, kUmmaK)) = __float2half(umma_probe_a(r, k));
  }
  for (int i = tid; i < N * kUmmaK; i += blockDim.x) {
    const int n = i / kUmmaK, k = i % kUmmaK;
    *reinterpret_cast<__half*>(B + umma_kmajor_offset(n, k, kUmmaK)) = __float2half(umma_probe_b(n, k));
  }
  fence_proxy_async_smem();
  if (warp == 0) tmem_alloc(&tbase, 256);
  if (tid == 0) {
    mbar_init(&bar, 1);
    mbar_fence_init();
  }
  tc_fence_before_sync();
  __syncthreads();
  tc_fence_after_sync();
  const uint32_t d = tbase;
  if (tid == 0) {
    const uint32_t idesc = umma_idesc_f16<false>(kUmmaM, N);
    for (int kk = 0; kk < kUmmaK / 16; ++kk) {
      const uint64_t ad = umma_smem_desc(smem_u32(A) + kk * 256, 128, (kUmmaK / 8) * 128);
      const uint64_t bd = umma_smem_desc(smem_u32(B) + kk * 256, 128, (kUmmaK / 8) * 128);
      umma_f16(d, ad, bd, idesc, kk > 0);
    }
    umma_commit(&bar);
  }
  const bool ok = mbar_wait_bounded(&bar, 0, 1 << 20);
  tc_fence_after_sync();
  for (int c = 0; c < N; c += 16) {
    uint32_t v[16];
    tmem_ld16(d + ((uint32_t)(32 * warp) << 16) + (uint32_t)c, v);
    tmem_wait_ld();
    const int row = 32 * warp + lane;
#pragma unroll
    for (int j = 0; j < 16; ++j) out[row * N + c + j] = __uint_as_float(v[j]);
  }
  tc_fence_before_sync();
  __syncthreads();
  if (warp == 0) tmem_dealloc(d, 256);
  if (!ok && tid == 0) atomicExch(err, nlos::kDevErrTmaTimeout);
}
}  // namespace

extern "C" nlos_status_t nlos_selftest_umma(int n_cols, float* out, int* code) {
  using namespace nlos;
  if (!out || !code || n_cols < 16 || n_cols > 256 || n_cols % 16)
    return set_error(NLOS_ERR_INVALID_ARG, "n_cols must be a multiple of 16 in [16, 256]; out/code non-NULL");
  int* d = nullptr;
  if (cudaMalloc(&d, sizeof(int)) != cudaSuccess) return set_error(NLOS_ERR_OUT_OF_MEMORY, "self-test word");
  cudaMemset(d, 0, sizeof(int));
  const int smem = (kUmmaM + n_cols) * kUmmaK * 2;
  cudaError_t e = cudaFuncSetAttribute(umma_probe_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e == cudaSuccess) {
    umma_probe_kernel<<<1, 128, smem>>>(n_cols, out, d);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  int v = 0;
  if (e == cudaSuccess) e = cudaMemcpy(&v, d, sizeof v, cudaMemcpyDeviceToHost);
  cudaFree(d);
  if (e != cudaSuccess) return set_error(NLOS_ERR_CUDA, cudaGetErrorString(e));
  *code = v;
  if (v) return set_error(NLOS_ERR_TIMEOUT, "tensor-core MMA did not complete within the wait limit");
  return NLOS_OK;
}

// ---------------------------------------------------------------------------
// FP32 FMA throughput: every thread runs 8 independent chains of
// x <- x * b + c, 16 steps per chain per iteration. The chains' sum is written
// only if it equals a value it cannot reach, so nothing is stored but the
// compiler keeps every FMA. The host times the launch with events; the
// measured rate is the denominator of the rooflines of FMA-bound kernels.
// ---------------------------------------------------------------------------
namespace {
__global__ void __launch_bounds__(256) ffma_rate_kernel(const float* in, float* out, int iters) {
  const float b = in[0], c = in[1];
  float x[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) x[k] = in[2] + 1e-3f * (float)(threadIdx.x + k);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int u = 0; u < 16; ++u) {
#pragma unroll
      for (int k = 0; k < 8; ++k) x[k] = fmaf(x[k], b, c);
    }
  }
  float s = 0.f;
#pragma unroll
  for (int k = 0; k < 8; ++k) s += x[k];
  if (s == -1.2345e30f) out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}
}  // namespace

extern "C" nlos_status_t nlos_ffma_rate_launch(const float* params, float* sink, int blocks, int iters,
                                               double* flops, void* stream) {
  using namespace nlos;
  if (!params || !sink || !flops || blocks <= 0 || iters <= 0)
    return set_error(NLOS_ERR_INVALID_ARG, "params/sink/flops non-NULL; blocks and iters > 0");
  ffma_rate_kernel<<<blocks, 256, 0, static_cast<cudaStream_t>(stream)>>>(params, sink, iters);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return set_error(NLOS_ERR_CUDA, cudaGetErrorString(e));
  *flops = 2.0 * 8 * 16 * (double)iters * blocks * 256;
  return NLOS_OK;
}

// ---------------------------------------------------------------------------
// Bounds-check self-test: one thread checks an index one past the end of a
// 4-element buffer and the last valid one. The check never performs the
// access, so nothing is read or written out of bounds; the bounds-checked
// build records kDevErrBounds for the first, the normal build records nothing.
// ---------------------------------------------------------------------------
#include "nlos_bounds.cuh"

namespace {
__global__ void bounds_probe_kernel(float* buf, int* err) {
  if (nlos::bchk(4, 4, err)) buf[0] = 1.0f;      // index 4 of 4 elements: outside, skipped
  if (nlos::bchk(3, 4, err)) buf[3] = 2.0f;      // inside
}
}  // namespace

extern "C" nlos_status_t nlos_selftest_bounds(int* code) {
  using namespace nlos;
  if (!code) return set_error(NLOS_ERR_INVALID_ARG, "code is NULL");
  int* d = nullptr;
  float* buf = nullptr;
  if (cudaMalloc(&d, sizeof(int)) != cudaSuccess) return set_error(NLOS_ERR_OUT_OF_MEMORY, "self-test word");
  if (cudaMalloc(&buf, 4 * sizeof(float)) != cudaSuccess) {
    cudaFree(d);
    return set_error(NLOS_ERR_OUT_OF_MEMORY, "self-test buffer");
  }
  cudaMemset(d, 0, sizeof(int));
  bounds_probe_kernel<<<1, 1>>>(buf, d);
  cudaError_t e = cudaDeviceSynchronize();
  int v = 0;
  if (e == cudaSuccess) e = cudaMemcpy(&v, d, sizeof v, cudaMemcpyDeviceToHost);
  cudaFree(d);
  cudaFree(buf);
  if (e != cudaSuccess) return set_error(NLOS_ERR_CUDA, cudaGetErrorString(e));
  *code = v;
  return NLOS_OK;
}
