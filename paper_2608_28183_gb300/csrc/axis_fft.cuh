// Strided-axis FFT kernel: transforms along the middle axis of a
// [outer][L][inner] array with `inner` contiguous. A CTA owns IC consecutive
// inner columns of one outer slice, so every global access is a run of IC
// consecutive elements (coalesced); the IC transforms run side by side with
// TPC = L/16 threads each, exchanging through shared memory laid out as
// [padded row][IC].
#pragma once
#include <algorithm>
#include <cstdio>
#include <cstdlib>

#include "nlos_bounds.cuh"
#include "nlos_fft.cuh"
#include "nlos_internal.h"
#include "nlos_tma.cuh"

namespace nlos {

// NLOS_DEBUG=1: print each axis launch's path and CUDA result to stderr
inline bool axis_debug() {
  static int on = -1;
  if (on < 0) on = getenv("NLOS_DEBUG") ? 1 : 0;
  return on == 1;
}
inline cudaError_t axis_report(const char* path, int L, int ic, int threads, size_t smem, long long gx, long long gy,
                               cudaError_t e) {
  if (axis_debug())
    fprintf(stderr, "[nlos axis] %s L=%d IC=%d threads=%d smem=%zu grid=(%lld,%lld) -> %s\n", path, L, ic, threads,
            smem, gx, gy, cudaGetErrorString(e));
  return e;
}

template <int L, int IC_> struct AxisTile {
  static constexpr int IC = IC_;
  static constexpr int THREADS = IC * (L / 16);
  static constexpr size_t SMEM = (L > 16) ? sizeof(float2) * FftShape<L>::SMEM * IC : 0;
};

template <int L, int IC_, int LD, int ST, class TS>
struct AxisCtx {
  using TR = typename RealOf<TS>::T;
  static constexpr int IC = IC_;
  static constexpr int SSTRIDE = IC;
  static constexpr bool kSmemInput = false;
  const void* in;
  void* out;
  const float2* tw;
  float2* smem;
  long long in_base, out_base;     // offsets of (outer, axis 0, inner column)
  long long in_axis, out_axis;
  int L_in, L_out, c, t_len, inverse;
  bool valid;
  float ldmul, stmul, tmul;
  long long in_n = 0, out_n = 0;   // extents (bounds-checked build)
  int* err = nullptr;

  __device__ __forceinline__ void load(int l, float2 (&x)[1]) const {
    x[0] = make_float2(0.f, 0.f);
    if (!valid || l >= L_in) return;
    if (!bchk(in_base + l * in_axis, in_n, err)) return;
    if constexpr (LD == kLoadReal) {
      float v = Real<TR>::get(static_cast<const TR*>(in) + in_base + l * in_axis) * ldmul;
      x[0] = make_float2(v * tmul, 0.f);
    } else {
      float2 v = cscale(Cpx<TS>::get(static_cast<const TS*>(in) + in_base + l * in_axis), ldmul);
      x[0] = inverse ? cconj(v) : v;
    }
  }
  __device__ __forceinline__ float2* sm(int) const { return smem + c; }
  __device__ __forceinline__ void store(int l, const float2 (&x)[1]) const {
    float2 v = x[0];
    if (!valid || l >= L_out) return;
    const long long o = out_base + l * out_axis;
    if (!bchk(o, out_n, err)) return;
    if constexpr (ST == kStoreCpx) {
      if (inverse) v = cconj(v);
      Cpx<TS>::put(static_cast<TS*>(out) + o, cscale(v, stmul));
    } else if constexpr (ST == kStoreCpx32) {
      if (inverse) v = cconj(v);
      static_cast<float2*>(out)[o] = cscale(v, stmul);
    } else if constexpr (ST == kStoreAbs2) {
      static_cast<float*>(out)[o] = fmaf(v.x, v.x, v.y * v.y) * stmul;
    } else {
      static_cast<float*>(out)[o] = sqrtf(fmaf(v.x, v.x, v.y * v.y)) * stmul;
    }
  }
};

// ---------------------------------------------------------------------------
// Real input, two columns per transform: the tile covers 2*IC inner columns;
// column c and column c + IC ride as the real and imaginary parts of one
// complex transform. The spectrum stays in shared memory, and the two real
// columns' spectra are split from Z[k] and Z[L-k]:
//   X_c[k] = (Z[k] + conj Z[L-k]) / 2,  X_{c+IC}[k] = (Z[k] - conj Z[L-k]) / (2i).
// ---------------------------------------------------------------------------
template <int L, int IC, class TS>
struct AxisPairCtx {
  using TR = typename RealOf<TS>::T;
  static constexpr int SSTRIDE = IC;
  static constexpr bool kSmemInput = false;
  const TR* in;
  float2* smem;
  const float2* tw;
  long long base0, base1, in_axis;
  int L_in, c;
  bool v0, v1;
  float m0, m1;
  long long in_n = 0;
  int* err = nullptr;
  __device__ __forceinline__ void load(int l, float2 (&x)[1]) const {
    x[0] = make_float2(0.f, 0.f);
    if (l >= L_in) return;
    if (v0 && bchk(base0 + l * in_axis, in_n, err)) x[0].x = Real<TR>::get(in + base0 + l * in_axis) * m0;
    if (v1 && bchk(base1 + l * in_axis, in_n, err)) x[0].y = Real<TR>::get(in + base1 + l * in_axis) * m1;
  }
  __device__ __forceinline__ float2* sm(int) const { return smem + c; }
  __device__ __forceinline__ void store(int l, const float2 (&x)[1]) const { smem[pad16(l) * IC + c] = x[0]; }
};

template <int L, int IC, class TS, bool kHalfIn>
__global__ void __launch_bounds__(AxisTile<L, IC>::THREADS)
axis_fft_realpair_kernel(const AxisParams p) {
  extern __shared__ float2 pair_sm[];
  constexpr int TPC = L / 16;
  const int c = threadIdx.x % IC;
  const int j0 = threadIdx.x / IC;
  const long long ii0 = (long long)blockIdx.x * (2 * IC) + c;
  const long long ii1 = ii0 + IC;
  const long long outer = blockIdx.y;
  const float ldmul = p.ld_dev_scale ? *p.ld_dev_scale : 1.0f;
  AxisPairCtx<L, IC, TS> ctx;
  ctx.in = static_cast<const typename RealOf<TS>::T*>(p.in);
  ctx.smem = pair_sm;
  ctx.tw = p.tw;
  ctx.base0 = outer * p.in_outer + ii0;
  ctx.base1 = outer * p.in_outer + ii1;
  ctx.in_axis = p.in_axis;
  ctx.L_in = p.L_in;
  ctx.c = c;
  ctx.v0 = ii0 < p.inner;
  ctx.v1 = ii1 < p.inner;
  ctx.m0 = ldmul * (p.t_len > 0 ? (float)(int)(ii0 % p.t_len) * p.t_scale : 1.0f);
  ctx.m1 = ldmul * (p.t_len > 0 ? (float)(int)(ii1 % p.t_len) * p.t_scale : 1.0f);
  ctx.in_n = p.in_n;
  ctx.err = p.err;
  fftn_run<L, 1, kHalfIn, false>(ctx, j0);
  __syncthreads();
  const float h = 0.5f * p.scale * (p.st_dev_scale ? *p.st_dev_scale : 1.0f);
  TS* out = static_cast<TS*>(p.out);
  for (int k = j0; k < p.L_out; k += TPC) {
    const float2 zk = pair_sm[pad16(k) * IC + c];
    const float2 zm = pair_sm[pad16((L - k) & (L - 1)) * IC + c];
    const long long o0 = outer * p.out_outer + ii0 + k * p.out_axis, o1 = outer * p.out_outer + ii1 + k * p.out_axis;
    if (ctx.v0 && bchk(o0, p.out_n, p.err)) Cpx<TS>::put(out + o0, make_float2((zk.x + zm.x) * h, (zk.y - zm.y) * h));
    if (ctx.v1 && bchk(o1, p.out_n, p.err)) Cpx<TS>::put(out + o1, make_float2((zk.y + zm.y) * h, (zm.x - zk.x) * h));
  }
}

template <int L, int IC, class TS, bool kHalfIn>
cudaError_t launch_axis_pair_ic(const AxisLaunch& l, cudaStream_t s) {
  using Tile = AxisTile<L, IC>;
  constexpr size_t smem = sizeof(float2) * FftShape<L>::SMEM * IC;
  auto k = axis_fft_realpair_kernel<L, IC, TS, kHalfIn>;
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  dim3 grid((unsigned)((l.p.inner + 2 * IC - 1) / (2 * IC)), (unsigned)l.n_outer);
  k<<<grid, Tile::THREADS, smem, s>>>(l.p);
  return axis_report("realpair", L, IC, Tile::THREADS, smem, grid.x, grid.y, cudaGetLastError());
}

template <int L, int IC, int LD, int ST, class TS, bool kHalfIn, bool kHalfOut>
__global__ void __launch_bounds__(AxisTile<L, IC>::THREADS)
axis_fft_kernel(const AxisParams p) {
  extern __shared__ float2 axis_sm[];
  AxisCtx<L, IC, LD, ST, TS> ctx;
  const int c = threadIdx.x % IC;
  const int j0 = threadIdx.x / IC;
  const long long ii = (long long)blockIdx.x * IC + c;
  const long long outer = blockIdx.y;
  ctx.in = p.in;
  ctx.out = p.out;
  ctx.tw = p.tw;
  ctx.smem = axis_sm;
  ctx.c = c;
  ctx.valid = ii < p.inner;
  ctx.in_base = outer * p.in_outer + ii;
  ctx.out_base = outer * p.out_outer + ii;
  ctx.in_axis = p.in_axis;
  ctx.out_axis = p.out_axis;
  ctx.L_in = p.L_in;
  ctx.L_out = p.L_out;
  ctx.inverse = p.inverse;
  ctx.t_len = p.t_len;
  ctx.ldmul = p.ld_dev_scale ? *p.ld_dev_scale : 1.0f;
  ctx.stmul = p.scale * (p.st_dev_scale ? *p.st_dev_scale : 1.0f);
  ctx.tmul = p.t_len > 0 ? (float)(int)(ii % p.t_len) * p.t_scale : 1.0f;
  ctx.in_n = p.in_n;
  ctx.out_n = p.out_n;
  ctx.err = p.err;
  fftn_run<L, 1, kHalfIn, kHalfOut>(ctx, j0);
}

// ---------------------------------------------------------------------------
// TMA-staged variant: persistent CTAs walk the tiles; while one tile is
// transformed in shared memory, the TMA engine fetches the next one into the
// other buffer (double buffering on two mbarriers). The first pass reads the
// dense staged tile; the transform then continues in place in the same buffer.
// ---------------------------------------------------------------------------
template <int L, int IC, int LD, int ST, class TS>
struct AxisTmaCtx : AxisCtx<L, IC, LD, ST, TS> {
  using Base = AxisCtx<L, IC, LD, ST, TS>;
  using TR = typename Base::TR;
  static constexpr bool kSmemInput = true;
  const void* tile;     // staged tile, [row][IC] of the input element type
  __device__ __forceinline__ void load(int l, float2 (&x)[1]) const {
    x[0] = make_float2(0.f, 0.f);
    if (l >= this->L_in) return;
    if constexpr (LD == kLoadReal) {
      const float v = Real<TR>::get(static_cast<const TR*>(tile) + l * IC + this->c) * this->ldmul;
      x[0] = make_float2(v * this->tmul, 0.f);
    } else {
      const float2 v = cscale(Cpx<TS>::get(static_cast<const TS*>(tile) + l * IC + this->c), this->ldmul);
      x[0] = this->inverse ? cconj(v) : v;
    }
  }
};

template <int L, int IC, int LD, class TS> struct AxisTmaTile {
  using TR = typename RealOf<TS>::T;
  static constexpr size_t ELEM = LD == kLoadReal ? sizeof(TR) : sizeof(TS);
  static constexpr size_t BUF = sizeof(float2) * FftShape<L>::SMEM * IC;   // bytes per buffer (multiple of 128)
  static constexpr size_t SMEM = 2 * BUF + 2 * sizeof(uint64_t);
  static constexpr int THREADS = IC * (L / 16);
};

constexpr int kTmaWaitLimit = 1 << 21;   // polls; each may suspend briefly, ~1 s in all

template <int L, int IC, int LD, int ST, class TS, bool kHalfIn, bool kHalfOut>
__global__ void __launch_bounds__(AxisTile<L, IC>::THREADS)
axis_fft_tma_kernel(const __grid_constant__ CUtensorMap tmap, const AxisParams p, const int tiles_inner,
                    const long long ntiles, int* err) {
  using T = AxisTmaTile<L, IC, LD, TS>;
  extern __shared__ __align__(128) unsigned char tma_sm[];
  auto buf = [&](int slot) { return reinterpret_cast<float2*>(tma_sm + slot * T::BUF); };
  uint64_t* bar = reinterpret_cast<uint64_t*>(tma_sm + 2 * T::BUF);
  const int c = threadIdx.x % IC;
  const int j0 = threadIdx.x / IC;
  const int rows = p.L_in;
  const uint32_t tile_bytes = (uint32_t)(rows * IC * T::ELEM);
  if (threadIdx.x == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    mbar_fence_init();
  }
  __syncthreads();
  auto issue = [&](long long tile, int slot) {
    const int ti = (int)(tile % tiles_inner);
    const int to = (int)(tile / tiles_inner);
    fence_proxy_async_smem();
    mbar_arrive_expect_tx(&bar[slot], tile_bytes);
    for (int r0 = 0; r0 < rows; r0 += 256)
      tma_load_3d(reinterpret_cast<unsigned char*>(buf(slot)) + (size_t)r0 * IC * T::ELEM, &tmap, &bar[slot],
                  ti * IC, r0, to);
  };
  long long tile = blockIdx.x;
  if (threadIdx.x == 0 && tile < ntiles) issue(tile, 0);
  const float ldmul = p.ld_dev_scale ? *p.ld_dev_scale : 1.0f;
  const float stmul = p.scale * (p.st_dev_scale ? *p.st_dev_scale : 1.0f);
  for (int k = 0; tile < ntiles; ++k, tile += gridDim.x) {
    const int slot = k & 1;
    const long long next = tile + gridDim.x;
    if (threadIdx.x == 0 && next < ntiles) issue(next, slot ^ 1);
    if (!mbar_wait_bounded(&bar[slot], (k >> 1) & 1, kTmaWaitLimit)) {
      if (err) atomicExch(err, kDevErrTmaTimeout);
      // give the copies still in flight into this CTA's buffers a last
      // bounded chance to land before the CTA exits
      mbar_wait_bounded(&bar[slot], (k >> 1) & 1, kTmaWaitLimit);
      if (next < ntiles) mbar_wait_bounded(&bar[slot ^ 1], ((k + 1) >> 1) & 1, kTmaWaitLimit);
      return;
    }
    const int ti = (int)(tile % tiles_inner);
    const long long outer = tile / tiles_inner;
    const long long ii = (long long)ti * IC + c;
    AxisTmaCtx<L, IC, LD, ST, TS> ctx;
    ctx.tile = buf(slot);
    ctx.in = p.in;
    ctx.out = p.out;
    ctx.tw = p.tw;
    ctx.smem = buf(slot);
    ctx.c = c;
    ctx.valid = ii < p.inner;
    ctx.in_base = outer * p.in_outer + ii;
    ctx.out_base = outer * p.out_outer + ii;
    ctx.in_axis = p.in_axis;
    ctx.out_axis = p.out_axis;
    ctx.L_in = p.L_in;
    ctx.L_out = p.L_out;
    ctx.inverse = p.inverse;
    ctx.t_len = p.t_len;
    ctx.ldmul = ldmul;
    ctx.stmul = stmul;
    ctx.tmul = p.t_len > 0 ? (float)(int)(ii % p.t_len) * p.t_scale : 1.0f;
    ctx.out_n = p.out_n;
    ctx.err = p.err;
    fftn_run<L, 1, kHalfIn, kHalfOut>(ctx, j0);
    __syncthreads();   // the buffer is free before the next issue into it
  }
}

template <int L, int IC, int LD, int ST, class TS, bool kHalfIn, bool kHalfOut>
cudaError_t launch_axis_tma(const AxisLaunch& l, cudaStream_t s) {
  using T = AxisTmaTile<L, IC, LD, TS>;
  auto k = axis_fft_tma_kernel<L, IC, LD, ST, TS, kHalfIn, kHalfOut>;
  static int blocks_per_sm = 0;
  static int sms = 0;
  if (blocks_per_sm == 0) {
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)T::SMEM);
    if (e != cudaSuccess) return e;
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks_per_sm, k, T::THREADS, T::SMEM);
    if (e != cudaSuccess) return e;
    if (blocks_per_sm < 1) blocks_per_sm = 1;
  }
  const int tiles_inner = (int)((l.p.inner + IC - 1) / IC);
  const long long ntiles = (long long)tiles_inner * l.n_outer;
  const long long grid = std::min<long long>(ntiles, (long long)sms * blocks_per_sm);
  k<<<(unsigned)grid, T::THREADS, T::SMEM, s>>>(l.tmap, l.p, tiles_inner, ntiles, l.err);
  return axis_report("tma", L, IC, T::THREADS, T::SMEM, grid, ntiles, cudaGetLastError());
}

// ---------------------------------------------------------------------------
// TMA-staged real pairs: the persistent double-buffered loop of the TMA
// kernel above with tiles of 2*IC real columns; columns c and c + IC ride as
// the real and imaginary parts of one transform and are split after it, as
// in axis_fft_realpair_kernel.
// ---------------------------------------------------------------------------
template <int L, int IC, class TS>
struct AxisTmaPairCtx {
  using TR = typename RealOf<TS>::T;
  static constexpr int SSTRIDE = IC;
  static constexpr bool kSmemInput = true;
  const TR* tile;       // staged tile, [row][2 IC] reals
  float2* smem;
  const float2* tw;
  int L_in, c;
  float m0, m1;
  __device__ __forceinline__ void load(int l, float2 (&x)[1]) const {
    x[0] = make_float2(0.f, 0.f);
    if (l >= L_in) return;
    x[0].x = Real<TR>::get(tile + l * (2 * IC) + c) * m0;
    x[0].y = Real<TR>::get(tile + l * (2 * IC) + IC + c) * m1;
  }
  __device__ __forceinline__ float2* sm(int) const { return smem + c; }
  __device__ __forceinline__ void store(int l, const float2 (&x)[1]) const { smem[pad16(l) * IC + c] = x[0]; }
};

template <int L, int IC, class TS, bool kHalfIn>
__global__ void __launch_bounds__(AxisTile<L, IC>::THREADS)
axis_fft_tma_pair_kernel(const __grid_constant__ CUtensorMap tmap, const AxisParams p, const int tiles_inner,
                         const long long ntiles, int* err) {
  using TR = typename RealOf<TS>::T;
  constexpr size_t BUF = sizeof(float2) * FftShape<L>::SMEM * IC;
  constexpr int TPC = L / 16;
  extern __shared__ __align__(128) unsigned char tp_sm[];
  auto buf = [&](int slot) { return reinterpret_cast<float2*>(tp_sm + slot * BUF); };
  uint64_t* bar = reinterpret_cast<uint64_t*>(tp_sm + 2 * BUF);
  const int c = threadIdx.x % IC;
  const int j0 = threadIdx.x / IC;
  const int rows = p.L_in;
  const uint32_t tile_bytes = (uint32_t)(rows * 2 * IC * sizeof(TR));
  if (threadIdx.x == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    mbar_fence_init();
  }
  __syncthreads();
  auto issue = [&](long long tile, int slot) {
    const int ti = (int)(tile % tiles_inner);
    const int to = (int)(tile / tiles_inner);
    fence_proxy_async_smem();
    mbar_arrive_expect_tx(&bar[slot], tile_bytes);
    for (int r0 = 0; r0 < rows; r0 += 256)
      tma_load_3d(reinterpret_cast<unsigned char*>(buf(slot)) + (size_t)r0 * 2 * IC * sizeof(TR), &tmap, &bar[slot],
                  ti * 2 * IC, r0, to);
  };
  long long tile = blockIdx.x;
  if (threadIdx.x == 0 && tile < ntiles) issue(tile, 0);
  const float ldmul = p.ld_dev_scale ? *p.ld_dev_scale : 1.0f;
  const float h = 0.5f * p.scale * (p.st_dev_scale ? *p.st_dev_scale : 1.0f);
  TS* out = static_cast<TS*>(p.out);
  for (int k = 0; tile < ntiles; ++k, tile += gridDim.x) {
    const int slot = k & 1;
    const long long next = tile + gridDim.x;
    if (threadIdx.x == 0 && next < ntiles) issue(next, slot ^ 1);
    if (!mbar_wait_bounded(&bar[slot], (k >> 1) & 1, kTmaWaitLimit)) {
      if (err) atomicExch(err, kDevErrTmaTimeout);
      // give the copies still in flight into this CTA's buffers a last
      // bounded chance to land before the CTA exits
      mbar_wait_bounded(&bar[slot], (k >> 1) & 1, kTmaWaitLimit);
      if (next < ntiles) mbar_wait_bounded(&bar[slot ^ 1], ((k + 1) >> 1) & 1, kTmaWaitLimit);
      return;
    }
    const int ti = (int)(tile % tiles_inner);
    const long long outer = tile / tiles_inner;
    const long long ii0 = (long long)ti * (2 * IC) + c;
    const long long ii1 = ii0 + IC;
    AxisTmaPairCtx<L, IC, TS> ctx;
    ctx.tile = reinterpret_cast<const TR*>(buf(slot));
    ctx.smem = buf(slot);
    ctx.tw = p.tw;
    ctx.L_in = rows;
    ctx.c = c;
    ctx.m0 = ldmul * (p.t_len > 0 ? (float)(int)(ii0 % p.t_len) * p.t_scale : 1.0f);
    ctx.m1 = ldmul * (p.t_len > 0 ? (float)(int)(ii1 % p.t_len) * p.t_scale : 1.0f);
    fftn_run<L, 1, kHalfIn, false>(ctx, j0);
    __syncthreads();
    const float2* z = buf(slot);
    const bool v0 = ii0 < p.inner, v1 = ii1 < p.inner;
    for (int q = j0; q < p.L_out; q += TPC) {
      const float2 zk = z[pad16(q) * IC + c];
      const float2 zm = z[pad16((L - q) & (L - 1)) * IC + c];
      const long long o0 = outer * p.out_outer + ii0 + q * p.out_axis, o1 = outer * p.out_outer + ii1 + q * p.out_axis;
      if (v0 && bchk(o0, p.out_n, p.err)) Cpx<TS>::put(out + o0, make_float2((zk.x + zm.x) * h, (zk.y - zm.y) * h));
      if (v1 && bchk(o1, p.out_n, p.err)) Cpx<TS>::put(out + o1, make_float2((zk.y + zm.y) * h, (zm.x - zk.x) * h));
    }
    __syncthreads();   // the buffer is free before the next issue into it
  }
}

template <int L, int IC, class TS, bool kHalfIn>
cudaError_t launch_axis_tma_pair(const AxisLaunch& l, cudaStream_t s) {
  constexpr size_t BUF = sizeof(float2) * FftShape<L>::SMEM * IC;
  constexpr size_t SMEM = 2 * BUF + 2 * sizeof(uint64_t);
  constexpr int THREADS = AxisTile<L, IC>::THREADS;
  auto k = axis_fft_tma_pair_kernel<L, IC, TS, kHalfIn>;
  static int blocks_per_sm = 0;
  static int sms = 0;
  if (blocks_per_sm == 0) {
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SMEM);
    if (e != cudaSuccess) return e;
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks_per_sm, k, THREADS, SMEM);
    if (e != cudaSuccess) return e;
    if (blocks_per_sm < 1) blocks_per_sm = 1;
  }
  const int tiles_inner = (int)((l.p.inner + 2 * IC - 1) / (2 * IC));
  const long long ntiles = (long long)tiles_inner * l.n_outer;
  const long long grid = std::min<long long>(ntiles, (long long)sms * blocks_per_sm);
  k<<<(unsigned)grid, THREADS, SMEM, s>>>(l.tmap, l.p, tiles_inner, ntiles, l.err);
  return axis_report("tma-pair", L, IC, THREADS, SMEM, grid, ntiles, cudaGetLastError());
}

// real-pair variants: tiles [0, n) direct loads, [2n, 3n) TMA staging (n
// column widths); tiles [n, 2n) of a real-input stage are single columns
template <int L, class TS, bool kHalfIn>
cudaError_t launch_axis_pair(const AxisLaunch& l, cudaStream_t s) {
  const int nic = axis_ic_count(L);
  const int v = l.tile >= 0 ? l.tile % nic : 0;
  if (l.has_tmap && l.tile >= 2 * nic) {
    if (v == 0) return launch_axis_tma_pair<L, axis_ic(L, 0), TS, kHalfIn>(l, s);
    if (v == 1) return launch_axis_tma_pair<L, axis_ic(L, 1), TS, kHalfIn>(l, s);
    return launch_axis_tma_pair<L, axis_ic(L, 2), TS, kHalfIn>(l, s);
  }
  if (v == 0) return launch_axis_pair_ic<L, axis_ic(L, 0), TS, kHalfIn>(l, s);
  if (v == 1) return launch_axis_pair_ic<L, axis_ic(L, 1), TS, kHalfIn>(l, s);
  return launch_axis_pair_ic<L, axis_ic(L, 2), TS, kHalfIn>(l, s);
}

template <int L, int IC, int LD, int ST, class TS, bool kHalfIn, bool kHalfOut>
cudaError_t launch_axis_ic(const AxisLaunch& l, cudaStream_t s) {
  const bool tma = l.has_tmap && l.tile >= axis_ic_count(L);
  if (tma) return launch_axis_tma<L, IC, LD, ST, TS, kHalfIn, kHalfOut>(l, s);
  using Tile = AxisTile<L, IC>;
  auto k = axis_fft_kernel<L, IC, LD, ST, TS, kHalfIn, kHalfOut>;
  if (Tile::SMEM > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Tile::SMEM);
    if (e != cudaSuccess) return e;
  }
  dim3 grid((unsigned)((l.p.inner + Tile::IC - 1) / Tile::IC), (unsigned)l.n_outer);
  k<<<grid, Tile::THREADS, Tile::SMEM, s>>>(l.p);
  return axis_report("direct", L, IC, Tile::THREADS, Tile::SMEM, grid.x, grid.y, cudaGetLastError());
}

template <int L, int LD, int ST, class TS, bool kHalfIn, bool kHalfOut>
cudaError_t launch_axis_one(const AxisLaunch& l, cudaStream_t s) {
  if constexpr (LD == kLoadRealPair) {
    return launch_axis_pair<L, TS, kHalfIn>(l, s);
  } else {
    const int v = (l.tile >= 0 && l.tile < axis_tile_count(L)) ? l.tile % axis_ic_count(L) : 0;
    if (v == 0) return launch_axis_ic<L, axis_ic(L, 0), LD, ST, TS, kHalfIn, kHalfOut>(l, s);
    if (v == 1) return launch_axis_ic<L, axis_ic(L, 1), LD, ST, TS, kHalfIn, kHalfOut>(l, s);
    return launch_axis_ic<L, axis_ic(L, 2), LD, ST, TS, kHalfIn, kHalfOut>(l, s);
  }
}

// Each translation unit instantiates one length range (0: 16-64, 1: 128-256,
// 2: 512-2048) so the builds run in parallel. The range is a template
// parameter, so the units' dispatchers are distinct functions (a macro alone
// would give different bodies to one symbol).
template <int RANGE, int LD, int ST, class TS, bool kHalfIn, bool kHalfOut>
cudaError_t launch_axis_len(const AxisLaunch& l, cudaStream_t s) {
  switch (l.L) {
#if defined(AXIS_RANGE) && AXIS_RANGE == 0
    case 16: return launch_axis_one<16, LD, ST, TS, kHalfIn, kHalfOut>(l, s);
    case 32: return launch_axis_one<32, LD, ST, TS, kHalfIn, kHalfOut>(l, s);
    case 64: return launch_axis_one<64, LD, ST, TS, kHalfIn, kHalfOut>(l, s);
#endif
#if defined(AXIS_RANGE) && AXIS_RANGE == 1
    case 128: return launch_axis_one<128, LD, ST, TS, kHalfIn, kHalfOut>(l, s);
    case 256: return launch_axis_one<256, LD, ST, TS, kHalfIn, kHalfOut>(l, s);
#endif
#if defined(AXIS_RANGE) && AXIS_RANGE == 2
    case 512: return launch_axis_one<512, LD, ST, TS, kHalfIn, kHalfOut>(l, s);
    case 1024: return launch_axis_one<1024, LD, ST, TS, kHalfIn, kHalfOut>(l, s);
    case 2048: return launch_axis_one<2048, LD, ST, TS, kHalfIn, kHalfOut>(l, s);
#endif
    default: return axis_report("no-length", l.L, 0, 0, 0, 0, 0, cudaErrorInvalidValue);
  }
}

// The sequences use five shapes: forward passes read a zero-padded upper half
// (L_in = L/2) and keep every output, inverse passes read every input and keep
// the lower half (L_out = L/2); the real-input x pass keeps kx in [0, L/2].
template <class TS, int RANGE>
cudaError_t launch_axis_typed(const AxisLaunch& l, cudaStream_t s) {
  if (l.n_outer <= 0 || l.n_outer > 65535 || l.p.inner <= 0)
    return axis_report("bad-shape", l.L, 0, 0, 0, l.p.inner, l.n_outer, cudaErrorInvalidValue);
  const bool half_in = 2 * l.p.L_in <= l.L, half_out = 2 * l.p.L_out <= l.L;   // zero beyond L_in
  if (axis_debug())
    fprintf(stderr, "[nlos axis] dispatch L=%d load=%d store=%d L_in=%d L_out=%d tile=%d tmap=%d\n", l.L, l.load_mode,
            l.store_mode, l.p.L_in, l.p.L_out, l.tile, l.has_tmap);
  if (l.load_mode == kLoadReal && l.store_mode == kStoreCpx && half_in && !half_out)
    return launch_axis_len<RANGE, kLoadReal, kStoreCpx, TS, true, false>(l, s);
  if (l.load_mode == kLoadRealPair && l.store_mode == kStoreCpx && half_in && 2 * l.p.L_out <= l.L + 2)
    return launch_axis_len<RANGE, kLoadRealPair, kStoreCpx, TS, true, false>(l, s);
  // unpadded transforms: every input present, every output kept (the real
  // x pass keeps the L/2 + 1 non-redundant outputs)
  const bool full_in = l.p.L_in == l.L;
  if (l.load_mode == kLoadReal && l.store_mode == kStoreCpx && full_in && 2 * l.p.L_out <= l.L + 2)
    return launch_axis_len<RANGE, kLoadReal, kStoreCpx, TS, false, false>(l, s);
  if (l.load_mode == kLoadRealPair && l.store_mode == kStoreCpx && full_in && 2 * l.p.L_out <= l.L + 2)
    return launch_axis_len<RANGE, kLoadRealPair, kStoreCpx, TS, false, false>(l, s);
  if (l.load_mode == kLoadCpx && l.store_mode == kStoreCpx && full_in && l.p.L_out == l.L)
    return launch_axis_len<RANGE, kLoadCpx, kStoreCpx, TS, false, false>(l, s);
  if (l.load_mode == kLoadCpx && l.store_mode == kStoreAbs2 && full_in && l.p.L_out == l.L)
    return launch_axis_len<RANGE, kLoadCpx, kStoreAbs2, TS, false, false>(l, s);
  if (l.load_mode == kLoadCpx && l.store_mode == kStoreCpx && half_in && !half_out)
    return launch_axis_len<RANGE, kLoadCpx, kStoreCpx, TS, true, false>(l, s);
  if (l.load_mode == kLoadCpx && l.store_mode == kStoreCpx && l.p.L_in == l.L && half_out)
    return launch_axis_len<RANGE, kLoadCpx, kStoreCpx, TS, false, true>(l, s);
  if (l.load_mode == kLoadCpx && l.store_mode == kStoreAbs2 && l.p.L_in == l.L && half_out)
    return launch_axis_len<RANGE, kLoadCpx, kStoreAbs2, TS, false, true>(l, s);
  if (l.load_mode == kLoadCpx && l.store_mode == kStoreAbs && l.p.L_in == l.L && half_out)
    return launch_axis_len<RANGE, kLoadCpx, kStoreAbs, TS, false, true>(l, s);
  if (l.load_mode == kLoadCpx && l.store_mode == kStoreCpx32 && l.p.L_in == l.L && half_out)
    return launch_axis_len<RANGE, kLoadCpx, kStoreCpx32, TS, false, true>(l, s);
  return axis_report("no-variant", l.L, 0, 0, 0, l.load_mode, l.store_mode, cudaErrorInvalidValue);
}

}  // namespace nlos
