// Photon binning (Sec. 4.1): SPAD photon records -> transient histogram, or
// directly -> the compact phasor field of the phasor-field pipeline.
//
// A record is a wall index x * ny + y and a timestamp in integer ticks; the
// bin is (ticks - t0) / ticks_per_bin in integers. Records before t0, past
// the last bin or off the grid are dropped.
//
// Phasors: one warp takes 32 records (one coalesced load per lane) and walks
// them in order, broadcasting each by shuffle; its lanes cover 32 band
// frequencies at a time. A photon in bin b adds exp(-2 pi i k_f b / n), read
// from a phase table of n entries staged in shared memory at index
// (k_f b) mod n. Consecutive records of the same wall point (a scanning
// capture emits them in runs) are summed in registers, so the warp issues
// one vector atomic per run and frequency instead of one per photon.
//
// For large photon counts the plan code takes another route to the same
// phasors: an atomic histogram in the plan's workspace followed by the band
// transform of the phasor pipeline (a temporal FFT per wall point), whose
// cost grows with the grid rather than with photons x frequencies.
#include <algorithm>
#include <cstdint>

#include "nlos.h"
#include "nlos_bounds.cuh"
#include "nlos_internal.h"

namespace nlos {

nlos_status_t set_error(nlos_status_t st, const char* msg);

namespace {

__device__ __forceinline__ bool photon_bin(uint32_t p, uint32_t t, uint32_t npix, uint32_t nt, uint32_t t0,
                                           uint32_t tpb, uint32_t* bin) {
  if (p >= npix || t < t0) return false;
  const uint32_t b = (t - t0) / tpb;
  *bin = b;
  return b < nt;
}

__global__ void bin_transient_kernel(const uint32_t* __restrict__ pixel, const uint32_t* __restrict__ ticks,
                                     long long count, uint32_t npix, uint32_t nt, uint32_t t0, uint32_t tpb,
                                     float* __restrict__ H) {
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < count; i += stride) {
    uint32_t b;
    const uint32_t p = __ldg(pixel + i);
    if (photon_bin(p, __ldg(ticks + i), npix, nt, t0, tpb, &b)) atomicAdd(H + (size_t)p * nt + b, 1.0f);
  }
}

constexpr int kBinThreads = 256;

__global__ void __launch_bounds__(kBinThreads)
bin_phasor_kernel(const PhasorBinParams q) {
  extern __shared__ float2 phase_sm[];
  for (int m = threadIdx.x; m < q.n; m += blockDim.x) phase_sm[m] = q.phase[m];
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const long long warp = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
  const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
  const uint32_t npix = q.npix, mask = (uint32_t)q.n - 1;
  float2* P = q.P;
  for (long long base = warp * 32; base < q.count; base += nwarps * 32) {
    const long long i = base + lane;
    uint32_t p = npix, b = 0;
    if (i < q.count) {
      const uint32_t pp = __ldg(q.pixel + i);
      if (!photon_bin(pp, __ldg(q.ticks + i), npix, (uint32_t)q.nt, q.t0, q.tpb, &b)) p = npix;
      else p = pp;
    }
    const int nrec = (int)min(32LL, q.count - base);
    for (int f0 = 0; f0 < q.F; f0 += 32) {
      const int f = f0 + lane;
      const uint32_t k = (uint32_t)(q.k_lo + f);
      const float w = f < q.F ? __ldg(q.w + f) : 0.f;
      float2 acc = make_float2(0.f, 0.f);
      uint32_t cur = npix;
      for (int j = 0; j < nrec; ++j) {
        const uint32_t pj = __shfl_sync(0xffffffffu, p, j);
        const uint32_t bj = __shfl_sync(0xffffffffu, b, j);
        if (pj != cur) {                       // warp-uniform: a new run of one wall point
          if (cur < npix && f < q.F && bchk((long long)cur * q.F + f, (long long)npix * q.F, q.err))
            atomicAdd(P + (size_t)cur * q.F + f, make_float2(acc.x * w, acc.y * w));
          acc = make_float2(0.f, 0.f);
          cur = pj;
        }
        if (pj < npix) {
          const float2 e = phase_sm[(k * bj) & mask];
          acc.x += e.x;
          acc.y += e.y;
        }
      }
      if (cur < npix && f < q.F && bchk((long long)cur * q.F + f, (long long)npix * q.F, q.err))
        atomicAdd(P + (size_t)cur * q.F + f, make_float2(acc.x * w, acc.y * w));
    }
  }
}

int sm_count() {
  static int sms = 0;
  if (sms == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (sms <= 0) sms = 1;
  }
  return sms;
}

}  // namespace

cudaError_t launch_bin_transient(const uint32_t* pixel, const uint32_t* ticks, long long count, uint32_t npix,
                                 uint32_t nt, uint32_t t0, uint32_t tpb, float* H, cudaStream_t s) {
  if (count <= 0) return cudaSuccess;
  const long long blocks = std::min<long long>((count + 255) / 256, (long long)sm_count() * 16);
  bin_transient_kernel<<<(unsigned)blocks, 256, 0, s>>>(pixel, ticks, count, npix, nt, t0, tpb, H);
  return cudaGetLastError();
}

cudaError_t launch_bin_phasors(const PhasorBinParams& q, cudaStream_t s) {
  const size_t smem = sizeof(float2) * (size_t)q.n;
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(bin_phasor_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  const long long warps = (q.count + 31) / 32;
  const long long blocks_needed = (warps * 32 + kBinThreads - 1) / kBinThreads;
  const long long blocks = std::min<long long>(std::max<long long>(blocks_needed, 1), (long long)sm_count() * 8);
  bin_phasor_kernel<<<(unsigned)blocks, kBinThreads, smem, s>>>(q);
  return cudaGetLastError();
}

}  // namespace nlos

extern "C" nlos_status_t nlos_bin_transient(const uint32_t* pixel, const uint32_t* ticks, long long count, int nx,
                                            int ny, int nt, uint32_t t0_ticks, uint32_t ticks_per_bin,
                                            int accumulate, float* transient, void* stream) {
  using namespace nlos;
  if (!transient || count < 0 || (count > 0 && (!pixel || !ticks)) || nx <= 0 || ny <= 0 || nt <= 0 ||
      ticks_per_bin == 0 || (long long)nx * ny > 0xffffffffLL)
    return set_error(NLOS_ERR_INVALID_ARG, "bad binning arguments");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaGetLastError();
  if (!accumulate) {
    const cudaError_t e = cudaMemsetAsync(transient, 0, sizeof(float) * (size_t)nx * ny * nt, s);
    if (e != cudaSuccess) return set_error(NLOS_ERR_CUDA, cudaGetErrorString(e));
  }
  cudaError_t e = launch_bin_transient(pixel, ticks, count, (uint32_t)((long long)nx * ny), (uint32_t)nt, t0_ticks,
                                       ticks_per_bin, transient, s);
  if (e == cudaSuccess) e = cudaGetLastError();
  if (e != cudaSuccess) return set_error(NLOS_ERR_CUDA, cudaGetErrorString(e));
  return NLOS_OK;
}
