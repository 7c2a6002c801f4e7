// Strided-axis FFT kernel: transforms along the middle axis of a
// [outer][L][inner] array with `inner` contiguous. A CTA owns IC consecutive
// inner columns of one outer slice, so every global access is a run of IC
// consecutive elements (coalesced); the IC transforms run side by side with
// TPC = L/16 threads each, exchanging through shared memory laid out as
// [padded row][IC].
#pragma once
#include "nlos_fft.cuh"
#include "nlos_internal.h"

namespace nlos {

template <class TS> struct RealOf;
template <> struct RealOf<float2> { using T = float; };
template <> struct RealOf<__half2> { using T = __half; };
template <> struct RealOf<__nv_bfloat162> { using T = __nv_bfloat16; };

// Column-tile variants per length (selected by AxisLaunch::tile; index 0 is
// the default, the autotuner may pick another).
__host__ __device__ constexpr int axis_ic(int L, int v) {
  return L <= 32 ? (v == 0 ? 32 : 64)
       : L <= 64 ? (v == 0 ? 32 : 16)
       : L <= 256 ? (v == 0 ? 16 : (v == 1 ? 8 : 32))
       : L <= 512 ? (v == 0 ? 8 : (v == 1 ? 4 : 16))
       : L <= 1024 ? (v == 0 ? 8 : 4)
       : (v == 0 ? 4 : 2);
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
  const void* in;
  void* out;
  const float2* tw;
  float2* smem;
  long long in_base, out_base;     // offsets of (outer, axis 0, inner column)
  long long in_axis, out_axis;
  int L_in, L_out, c, t_len, inverse;
  bool valid;
  float ldmul, stmul, tmul;

  __device__ __forceinline__ void load(int l, float2 (&x)[1]) const {
    x[0] = make_float2(0.f, 0.f);
    if (!valid || l >= L_in) return;
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
    if constexpr (ST == kStoreCpx) {
      if (inverse) v = cconj(v);
      Cpx<TS>::put(static_cast<TS*>(out) + o, cscale(v, stmul));
    } else if constexpr (ST == kStoreAbs2) {
      static_cast<float*>(out)[o] = fmaf(v.x, v.x, v.y * v.y) * stmul;
    } else {
      static_cast<float*>(out)[o] = sqrtf(fmaf(v.x, v.x, v.y * v.y)) * stmul;
    }
  }
};

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
  fftn_run<L, 1, kHalfIn, kHalfOut>(ctx, j0);
}

template <int L, int IC, int LD, int ST, class TS, bool kHalfIn, bool kHalfOut>
cudaError_t launch_axis_ic(const AxisLaunch& l, cudaStream_t s) {
  using Tile = AxisTile<L, IC>;
  auto k = axis_fft_kernel<L, IC, LD, ST, TS, kHalfIn, kHalfOut>;
  if (Tile::SMEM > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Tile::SMEM);
    if (e != cudaSuccess) return e;
  }
  dim3 grid((unsigned)((l.p.inner + Tile::IC - 1) / Tile::IC), (unsigned)l.n_outer);
  k<<<grid, Tile::THREADS, Tile::SMEM, s>>>(l.p);
  return cudaGetLastError();
}

template <int L, int LD, int ST, class TS, bool kHalfIn, bool kHalfOut>
cudaError_t launch_axis_one(const AxisLaunch& l, cudaStream_t s) {
  const int v = (l.tile >= 0 && l.tile < axis_tile_count(L)) ? l.tile : 0;
  if (v == 0) return launch_axis_ic<L, axis_ic(L, 0), LD, ST, TS, kHalfIn, kHalfOut>(l, s);
  if (v == 1) return launch_axis_ic<L, axis_ic(L, 1), LD, ST, TS, kHalfIn, kHalfOut>(l, s);
  return launch_axis_ic<L, axis_ic(L, 2), LD, ST, TS, kHalfIn, kHalfOut>(l, s);
}

// AXIS_SMALL / AXIS_LARGE select the length range a translation unit
// instantiates (lengths <= 256 and >= 512), so the builds run in parallel.
template <int LD, int ST, class TS, bool kHalfIn, bool kHalfOut>
cudaError_t launch_axis_len(const AxisLaunch& l, cudaStream_t s) {
  switch (l.L) {
#if defined(AXIS_SMALL)
    case 16: return launch_axis_one<16, LD, ST, TS, kHalfIn, kHalfOut>(l, s);
    case 32: return launch_axis_one<32, LD, ST, TS, kHalfIn, kHalfOut>(l, s);
    case 64: return launch_axis_one<64, LD, ST, TS, kHalfIn, kHalfOut>(l, s);
    case 128: return launch_axis_one<128, LD, ST, TS, kHalfIn, kHalfOut>(l, s);
    case 256: return launch_axis_one<256, LD, ST, TS, kHalfIn, kHalfOut>(l, s);
#endif
#if defined(AXIS_LARGE)
    case 512: return launch_axis_one<512, LD, ST, TS, kHalfIn, kHalfOut>(l, s);
    case 1024: return launch_axis_one<1024, LD, ST, TS, kHalfIn, kHalfOut>(l, s);
    case 2048: return launch_axis_one<2048, LD, ST, TS, kHalfIn, kHalfOut>(l, s);
#endif
    default: return cudaErrorInvalidValue;
  }
}

// The sequences use five shapes: forward passes read a zero-padded upper half
// (L_in = L/2) and keep every output, inverse passes read every input and keep
// the lower half (L_out = L/2); the real-input x pass keeps kx in [0, L/2].
template <class TS>
cudaError_t launch_axis_typed(const AxisLaunch& l, cudaStream_t s) {
  if (l.n_outer <= 0 || l.n_outer > 65535 || l.p.inner <= 0) return cudaErrorInvalidValue;
  const bool half_in = 2 * l.p.L_in == l.L, half_out = 2 * l.p.L_out <= l.L;
  if (l.load_mode == kLoadReal && l.store_mode == kStoreCpx && half_in && !half_out)
    return launch_axis_len<kLoadReal, kStoreCpx, TS, true, false>(l, s);
  if (l.load_mode == kLoadCpx && l.store_mode == kStoreCpx && half_in && !half_out)
    return launch_axis_len<kLoadCpx, kStoreCpx, TS, true, false>(l, s);
  if (l.load_mode == kLoadCpx && l.store_mode == kStoreCpx && l.p.L_in == l.L && half_out)
    return launch_axis_len<kLoadCpx, kStoreCpx, TS, false, true>(l, s);
  if (l.load_mode == kLoadCpx && l.store_mode == kStoreAbs2 && l.p.L_in == l.L && half_out)
    return launch_axis_len<kLoadCpx, kStoreAbs2, TS, false, true>(l, s);
  if (l.load_mode == kLoadCpx && l.store_mode == kStoreAbs && l.p.L_in == l.L && half_out)
    return launch_axis_len<kLoadCpx, kStoreAbs, TS, false, true>(l, s);
  return cudaErrorInvalidValue;
}

}  // namespace nlos
