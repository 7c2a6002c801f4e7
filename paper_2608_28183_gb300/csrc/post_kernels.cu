// Post-processing of reconstructions (Sec. 4.4 background-noise removal and
// the display reduction of Sec. 4.2): max-over-depth images, the mixture of
// experts of Eq. 10, coherence-weighted merging of Eqs. 8-9 and the
// depth-dependent average.
#include <algorithm>
#include <cstdint>
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
// passed as a __grid_constant__ parameter: the per-frame loops index it in
// the parameter bank instead of copying it to the stack
struct FramePtrs {
  const void* p[kMaxFrames];
};

// Eqs. 8-9: C = |sum f| / (eps + sum |f|), merged = C |sum f| / N_w
__device__ __forceinline__ void coherence_one(float sx, float sy, float sa, float eps, float inv_nw, float* m, float* c) {
  const float s = sqrtf(fmaf(sx, sx, sy * sy));
  *c = s / (eps + sa);
  *m = *c * s * inv_nw;
}

// scalar path: any count and alignment
__global__ void coherence_kernel(const __grid_constant__ FramePtrs fr, int nw, long long n, float eps, float* merged, float* coh) {
  const float inv_nw = 1.0f / (float)nw;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    float sx = 0.f, sy = 0.f, sa = 0.f;
    for (int j = 0; j < nw; ++j) {
      const float2 f = static_cast<const float2*>(fr.p[j])[i];
      sx += f.x;
      sy += f.y;
      sa += sqrtf(fmaf(f.x, f.x, f.y * f.y));
    }
    float m, c;
    coherence_one(sx, sy, sa, eps, inv_nw, &m, &c);
    merged[i] = m;
    if (coh) coh[i] = c;
  }
}

// vector path: two voxels per thread (one 16-byte load per frame, four
// frames' loads in flight), for even counts and 16-byte aligned frames
__global__ void coherence_vec_kernel(const __grid_constant__ FramePtrs fr, int nw, long long n2, float eps, float2* merged, float2* coh) {
  const float inv_nw = 1.0f / (float)nw;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n2; i += (long long)gridDim.x * blockDim.x) {
    float ax = 0.f, ay = 0.f, aa = 0.f, bx = 0.f, by = 0.f, ba = 0.f;
    int j = 0;
    for (; j + 4 <= nw; j += 4) {
      float4 f[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) f[u] = __ldcs(static_cast<const float4*>(fr.p[j + u]) + i);
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        ax += f[u].x;
        ay += f[u].y;
        aa += sqrtf(fmaf(f[u].x, f[u].x, f[u].y * f[u].y));
        bx += f[u].z;
        by += f[u].w;
        ba += sqrtf(fmaf(f[u].z, f[u].z, f[u].w * f[u].w));
      }
    }
    for (; j < nw; ++j) {
      const float4 f = __ldcs(static_cast<const float4*>(fr.p[j]) + i);
      ax += f.x;
      ay += f.y;
      aa += sqrtf(fmaf(f.x, f.x, f.y * f.y));
      bx += f.z;
      by += f.w;
      ba += sqrtf(fmaf(f.z, f.z, f.w * f.w));
    }
    float2 m, c;
    coherence_one(ax, ay, aa, eps, inv_nw, &m.x, &c.x);
    coherence_one(bx, by, ba, eps, inv_nw, &m.y, &c.y);
    __stcs(merged + i, m);
    if (coh) __stcs(coh + i, c);
  }
}

// depth-dependent average: plane z averages the newest N(z) = min(N_w, 1 + N_w z / n_z) frames
// 32-bit arithmetic: the host keeps nz below 2^27, so nw * z < 2^31
__device__ __forceinline__ int dda_count(int nw, int z, int nz) {
  return min(nw, 1 + (int)((unsigned)(nw * z) / (unsigned)nz));
}

__global__ void dda_kernel(const __grid_constant__ FramePtrs fr, int nw, long long nxy, int nz, float* out) {
  const long long n = nxy * nz;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const int z = (int)(i % nz);
    const int cnt = dda_count(nw, z, nz);
    float s = 0.f;
    for (int j = 0; j < cnt; ++j) s += static_cast<const float*>(fr.p[j])[i];
    out[i] = s / (float)cnt;
  }
}

// vector path: four consecutive planes per thread (nz a multiple of 4,
// 16-byte aligned frames); the thread index splits into (pencil, plane
// quad) with 32-bit arithmetic
__global__ void dda_vec_kernel(const __grid_constant__ FramePtrs fr, int nw, long long nxy, int nz, float4* out) {
  const int q = nz / 4;
  const long long n4 = nxy * q;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n4; i += (long long)gridDim.x * blockDim.x) {
    const int z0 = 4 * (int)((unsigned)i % (unsigned)q);       // the host keeps n4 below 2^32
    int cnt[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) cnt[e] = dda_count(nw, z0 + e, nz);
    float4 s = make_float4(0.f, 0.f, 0.f, 0.f);
    auto add = [&](const float4& f, int j) {
      if (j < cnt[0]) s.x += f.x;
      if (j < cnt[1]) s.y += f.y;
      if (j < cnt[2]) s.z += f.z;
      s.w += f.w;
    };
    int j = 0;                                 // counts grow with z: cnt[3] is the largest
    for (; j + 4 <= cnt[3]; j += 4) {
      float4 f[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) f[u] = __ldcs(static_cast<const float4*>(fr.p[j + u]) + i);
#pragma unroll
      for (int u = 0; u < 4; ++u) add(f[u], j + u);
    }
    for (; j < cnt[3]; ++j) add(__ldcs(static_cast<const float4*>(fr.p[j]) + i), j);
    __stcs(out + i, make_float4(s.x / (float)cnt[0], s.y / (float)cnt[1], s.z / (float)cnt[2], s.w / (float)cnt[3]));
  }
}

bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15) == 0; }

int grid_for(long long work) {
  static int sms = 0;
  if (sms == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (sms <= 0) sms = 1;
  }
  const long long want = (work + 255) / 256;
  return (int)std::max<long long>(1, std::min<long long>(want, (long long)sms * 8));
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
  bool vec = count % 2 == 0 && aligned16(merged) && (!coherence || aligned16(coherence));
  for (int j = 0; j < nw; ++j) vec = vec && aligned16(frames[j]);
  cudaGetLastError();
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (vec)
    coherence_vec_kernel<<<grid_for(count / 2), 256, 0, s>>>(fp, nw, count / 2, eps, reinterpret_cast<float2*>(merged),
                                                            reinterpret_cast<float2*>(coherence));
  else
    coherence_kernel<<<grid_for(count), 256, 0, s>>>(fp, nw, count, eps, merged, coherence);
  return launch_status("coherence merge");
}

nlos_status_t nlos_dda(const float* const* frames, int nw, long long nxy, int nz, float* out, void* stream) {
  if (!frames || nw < 1 || nw > kMaxFrames || nxy <= 0 || nz <= 0 || nz >= (1 << 27) || !out)
    return set_error(NLOS_ERR_INVALID_ARG, "bad depth-dependent average arguments (1 <= N_w <= 16, nz < 2^27)");
  FramePtrs fp{};
  for (int j = 0; j < nw; ++j) {
    if (!frames[j]) return set_error(NLOS_ERR_INVALID_ARG, "NULL frame");
    fp.p[j] = frames[j];
  }
  bool vec = nz % 4 == 0 && aligned16(out) && nxy * (nz / 4) < (1LL << 32);
  for (int j = 0; j < nw; ++j) vec = vec && aligned16(frames[j]);
  cudaGetLastError();
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (vec)
    dda_vec_kernel<<<grid_for(nxy * (nz / 4)), 256, 0, s>>>(fp, nw, nxy, nz, reinterpret_cast<float4*>(out));
  else
    dda_kernel<<<grid_for(nxy * nz), 256, 0, s>>>(fp, nw, nxy, nz, out);
  return launch_status("depth-dependent average");
}

}  // extern "C"
