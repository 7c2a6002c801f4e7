// Post-processing of reconstructions (Sec. 4.4 background-noise removal and
// the display reduction of Sec. 4.2): max-over-depth images, the mixture of
// experts of Eq. 10, coherence-weighted merging of Eqs. 8-9 and the
// depth-dependent average.
#include <cstdio>

#include "nlos.h"
#include "nlos_internal.h"

namespace nlos {
nlos_status_t set_error(nlos_status_t st, const char* msg);
}  // namespace nlos

namespace {

using nlos::set_error;

// one warp per (x, y) pencil, lanes stride along the contiguous depth axis
__global__ void max_image_kernel(const float* __restrict__ v, long long nxy, int nz, int take_sqrt,
                                 float* __restrict__ img) {
  const long long w = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (w >= nxy) return;
  const float* p = v + w * nz;
  float m = -INFINITY;
  for (int z = lane; z < nz; z += 32) m = fmaxf(m, p[z]);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
  if (lane == 0) img[w] = take_sqrt ? sqrtf(fmaxf(m, 0.f)) : m;
}

__device__ float block_max(float v, float* red) {
  for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x < 32) {
    float r = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : -INFINITY;
    for (int o = 16; o > 0; o >>= 1) r = fmaxf(r, __shfl_xor_sync(0xffffffffu, r, o));
    if (threadIdx.x == 0) red[32] = r;
  }
  __syncthreads();
  const float r = red[32];
  __syncthreads();
  return r;
}

// Eq. 10 on max-normalised images, result normalised to its peak (one CTA)
__global__ void __launch_bounds__(1024) moe_kernel(const float* a, const float* b, long long n, float beta, float eps,
                                                   float* out) {
  __shared__ float red[33];
  float ma = -INFINITY, mb = -INFINITY;
  for (long long i = threadIdx.x; i < n; i += blockDim.x) {
    ma = fmaxf(ma, a[i]);
    mb = fmaxf(mb, b[i]);
  }
  ma = block_max(ma, red);
  mb = block_max(mb, red);
  const float ia = ma > 0.f ? 1.f / ma : 1.f, ib = mb > 0.f ? 1.f / mb : 1.f;
  float mf = -INFINITY;
  for (long long i = threadIdx.x; i < n; i += blockDim.x) {
    const float f = a[i] * ia * powf(b[i] * ib + eps, beta);
    out[i] = f;
    mf = fmaxf(mf, f);
  }
  mf = block_max(mf, red);
  const float im = mf > 0.f ? 1.f / mf : 1.f;
  for (long long i = threadIdx.x; i < n; i += blockDim.x) out[i] *= im;
}

constexpr int kMaxFrames = 16;
struct FramePtrs {
  const void* p[kMaxFrames];
};

// Eqs. 8-9: C = |sum f| / (eps + sum |f|), merged = C |sum f| / N_w
__global__ void coherence_kernel(FramePtrs fr, int nw, long long n, float eps, float* merged, float* coh) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    float sx = 0.f, sy = 0.f, sa = 0.f;
    for (int j = 0; j < nw; ++j) {
      const float2 f = static_cast<const float2*>(fr.p[j])[i];
      sx += f.x;
      sy += f.y;
      sa += sqrtf(fmaf(f.x, f.x, f.y * f.y));
    }
    const float s = sqrtf(fmaf(sx, sx, sy * sy));
    const float c = s / (eps + sa);
    merged[i] = c * s / (float)nw;
    if (coh) coh[i] = c;
  }
}

// depth-dependent average: plane z averages the newest N(z) = min(N_w, 1 + N_w z / n_z) frames
__global__ void dda_kernel(FramePtrs fr, int nw, long long nxy, int nz, float* out) {
  const long long n = nxy * nz;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const int z = (int)(i % nz);
    const int cnt = min(nw, 1 + (int)(((long long)nw * z) / nz));
    float s = 0.f;
    for (int j = 0; j < cnt; ++j) s += static_cast<const float*>(fr.p[j])[i];
    out[i] = s / (float)cnt;
  }
}

nlos_status_t launch_status(const char* what) {
  const cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) return NLOS_OK;
  char msg[160];
  snprintf(msg, sizeof msg, "%s: %s", what, cudaGetErrorString(e));
  return set_error(NLOS_ERR_CUDA, msg);
}

}  // namespace

extern "C" {

nlos_status_t nlos_max_image(const float* volume, int nx, int ny, int nz, int take_sqrt, float* image, void* stream) {
  if (!volume || !image || nx <= 0 || ny <= 0 || nz <= 0) return set_error(NLOS_ERR_INVALID_ARG, "bad image arguments");
  cudaGetLastError();
  const long long nxy = (long long)nx * ny;
  const long long threads = nxy * 32;
  max_image_kernel<<<(unsigned)((threads + 255) / 256), 256, 0, static_cast<cudaStream_t>(stream)>>>(volume, nxy, nz,
                                                                                                    take_sqrt, image);
  return launch_status("max image");
}

nlos_status_t nlos_moe_mix(const float* img_fk, const float* img_rsd, long long count, float beta, float eps, float* out,
                           void* stream) {
  if (!img_fk || !img_rsd || !out || count <= 0 || !(eps >= 0.f))
    return set_error(NLOS_ERR_INVALID_ARG, "bad mixture arguments");
  cudaGetLastError();
  moe_kernel<<<1, 1024, 0, static_cast<cudaStream_t>(stream)>>>(img_fk, img_rsd, count, beta, eps, out);
  return launch_status("mixture of experts");
}

nlos_status_t nlos_coherence_merge(const void* const* frames, int nw, long long count, float eps, float* merged,
                                   float* coherence, void* stream) {
  if (!frames || nw < 1 || nw > kMaxFrames || count <= 0 || !merged || !(eps > 0.f))
    return set_error(NLOS_ERR_INVALID_ARG, "bad coherence arguments (1 <= N_w <= 16, eps > 0)");
  FramePtrs fp{};
  for (int j = 0; j < nw; ++j) {
    if (!frames[j]) return set_error(NLOS_ERR_INVALID_ARG, "NULL frame");
    fp.p[j] = frames[j];
  }
  cudaGetLastError();
  coherence_kernel<<<1024, 256, 0, static_cast<cudaStream_t>(stream)>>>(fp, nw, count, eps, merged, coherence);
  return launch_status("coherence merge");
}

nlos_status_t nlos_dda(const float* const* frames, int nw, long long nxy, int nz, float* out, void* stream) {
  if (!frames || nw < 1 || nw > kMaxFrames || nxy <= 0 || nz <= 0 || !out)
    return set_error(NLOS_ERR_INVALID_ARG, "bad depth-dependent average arguments (1 <= N_w <= 16)");
  FramePtrs fp{};
  for (int j = 0; j < nw; ++j) {
    if (!frames[j]) return set_error(NLOS_ERR_INVALID_ARG, "NULL frame");
    fp.p[j] = frames[j];
  }
  cudaGetLastError();
  dda_kernel<<<1024, 256, 0, static_cast<cudaStream_t>(stream)>>>(fp, nw, nxy, nz, out);
  return launch_status("depth-dependent average");
}

}  // extern "C"
