// Device-side FFT building blocks for the NLOS kernels (sm_103a).
//
// Every transform here is a power-of-two Stockham FFT (self-sorting, natural
// order in and out) executed by TPC = L/E threads, each holding E = 16 or 32
// complex values in registers. A pass of radix R (E, or a smaller power of two for the remainder)
// gathers R values per butterfly at stride L/R, multiplies by the pass
// twiddles W_{Ns R}^{k r}, runs an in-register radix-R DFT and scatters to
// (j/Ns) Ns R + j%Ns + r Ns. Between passes data goes through shared memory
// in place (read, barrier, write, barrier). The first pass reads straight from
// global memory through a caller-supplied functor (zero padding, scaling and
// type conversion fused there) and the last pass writes straight to global
// memory through another (cropping, magnitude, band selection fused there).
//
// Inverse transforms use conj(DFT(conj(x))), so a context conjugates on load
// and on store; there is one butterfly implementation.
//
// Twiddle tables come from the plan (generated in float64 on the host,
// stored as float2): for pass p the table T_p[r * Ns + k] = exp(-2 pi i k r /
// (Ns R)), laid out with k fastest so that lanes with consecutive k read
// consecutive addresses.
#pragma once

#include <cuda_runtime.h>
#include <cuda_fp16.h>
#include <cuda_bf16.h>
#include <stdint.h>

namespace nlos {

// ---------------------------------------------------------------------------
// complex helpers
// ---------------------------------------------------------------------------
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ float2 cconj(float2 a) { return make_float2(a.x, -a.y); }
__device__ __forceinline__ float2 cscale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }
// a * (-i)
__device__ __forceinline__ float2 cmul_mi(float2 a) { return make_float2(a.y, -a.x); }

// cos(2 pi m / 32) for m = 0..8 (values of the circle function, listed).
__device__ __forceinline__ float cos32_q(int m) {
  switch (m) {
    case 0: return 1.0f;
    case 1: return 0.98078528040323043f;
    case 2: return 0.92387953251128674f;
    case 3: return 0.83146961230254524f;
    case 4: return 0.70710678118654752f;
    case 5: return 0.55557023301960218f;
    case 6: return 0.38268343236508984f;
    case 7: return 0.19509032201612833f;
    default: return 0.0f;
  }
}
__device__ __forceinline__ float cos32(int m) {
  m &= 31;
  if (m <= 8) return cos32_q(m);
  if (m <= 16) return -cos32_q(16 - m);
  if (m <= 24) return -cos32_q(m - 16);
  return cos32_q(32 - m);
}
__device__ __forceinline__ float sin32(int m) { return cos32(m - 8); }

// a * exp(-2 pi i m / 32); m is a compile-time constant after unrolling, so
// the branches and table reads fold away.
__device__ __forceinline__ float2 mul_w32(float2 a, int m) {
  m &= 31;
  if (m == 0) return a;
  if (m == 8) return make_float2(a.y, -a.x);
  if (m == 16) return make_float2(-a.x, -a.y);
  if (m == 24) return make_float2(-a.y, a.x);
  const float c = cos32(m), s = sin32(m);
  return make_float2(fmaf(a.x, c, a.y * s), fmaf(a.y, c, -a.x * s));
}

// ---------------------------------------------------------------------------
// in-register radix-R DFTs, natural order in and out, forward sign e^{-i}
// ---------------------------------------------------------------------------
template <int R> struct Dft;

template <> struct Dft<1> {
  static __device__ __forceinline__ void run(float2*) {}
};
template <> struct Dft<2> {
  static __device__ __forceinline__ void run(float2* v) {
    const float2 t = v[0];
    v[0] = cadd(t, v[1]);
    v[1] = csub(t, v[1]);
  }
};
template <> struct Dft<4> {
  static __device__ __forceinline__ void run(float2* v) {
    const float2 a = cadd(v[0], v[2]), b = csub(v[0], v[2]);
    const float2 c = cadd(v[1], v[3]), d = cmul_mi(csub(v[1], v[3]));
    v[0] = cadd(a, c);
    v[2] = csub(a, c);
    v[1] = cadd(b, d);
    v[3] = csub(b, d);
  }
};
// R = R1 * R2 with n = n1 + R1 n2 and k = k2 + R2 k1:
//   X[k2 + R2 k1] = sum_n1 W_R^{n1 k2} W_R1^{n1 k1} (sum_n2 x[n1 + R1 n2] W_R2^{n2 k2})
template <int R> struct Dft {
  static constexpr int R1 = (R >= 16) ? 4 : 2;
  static constexpr int R2 = R / R1;
  static __device__ __forceinline__ void run(float2* v) {
    float2 y[R1][R2];
#pragma unroll
    for (int n1 = 0; n1 < R1; ++n1) {
#pragma unroll
      for (int n2 = 0; n2 < R2; ++n2) y[n1][n2] = v[n1 + R1 * n2];
      Dft<R2>::run(y[n1]);
#pragma unroll
      for (int k2 = 0; k2 < R2; ++k2) y[n1][k2] = mul_w32(y[n1][k2], (32 / R) * n1 * k2);
    }
#pragma unroll
    for (int k2 = 0; k2 < R2; ++k2) {
      float2 t[R1];
#pragma unroll
      for (int n1 = 0; n1 < R1; ++n1) t[n1] = y[n1][k2];
      Dft<R1>::run(t);
#pragma unroll
      for (int k1 = 0; k1 < R1; ++k1) v[k2 + R2 * k1] = t[k1];
    }
  }
};

// ---------------------------------------------------------------------------
// pass schedule of an L-point transform
// ---------------------------------------------------------------------------
__host__ __device__ constexpr int ilog2c(int x) { return x <= 1 ? 0 : 1 + ilog2c(x / 2); }

// E complex values per thread (16: radix-16 passes, 32: radix-32 passes; a
// radix-2^(log2 L mod log2 E) remainder pass closes the schedule)
template <int L, int E_ = 16> struct FftShape {
  static_assert(L >= E_ && (L & (L - 1)) == 0, "power-of-two length >= E");
  static_assert(E_ == 16 || E_ == 32, "16 or 32 values per thread");
  static constexpr int E = E_;            // complex values held per thread
  static constexpr int LE = ilog2c(E_);
  static constexpr int TPC = L / E;       // threads per transform
  static constexpr int LOG = ilog2c(L);
  static constexpr int NFULL = LOG / LE;
  static constexpr int REM = LOG % LE;
  static constexpr int NPASS = NFULL + (REM ? 1 : 0);
  static constexpr int SMEM = L + L / E;  // padded shared-memory elements per transform
  __host__ __device__ static constexpr int radix(int p) { return p < NFULL ? E : (1 << REM); }
  __host__ __device__ static constexpr int span(int p) { return p == 0 ? 1 : span(p - 1) * radix(p - 1); }
  __host__ __device__ static constexpr int twoff(int p) {
    return p == 0 ? 0 : twoff(p - 1) + span(p - 1) * radix(p - 1);
  }
  static constexpr int TWSIZE = twoff(NPASS);
};

// Barrier between the passes of a transform: the whole CTA, or - for a
// context that declares kBarThreads - the warp (kBarThreads = 32: every
// transform of the context lies within one warp) or named barrier 1 over the
// first kBarThreads threads (warp-specialised kernels whose other warps do
// not take part in the transforms).
template <class C, class = void> struct CtxBar {
  static constexpr int threads = 0;
};
template <class C> struct CtxBar<C, decltype((void)C::kBarThreads)> {
  static constexpr int threads = C::kBarThreads;
};
// Where a context's twiddle table lives: global memory read through the
// read-only path (default), or - for a context that declares kTwShared - a
// copy in shared memory.
template <class C, class = void> struct CtxTwShared {
  static constexpr bool value = false;
};
template <class C> struct CtxTwShared<C, decltype((void)C::kTwShared)> {
  static constexpr bool value = C::kTwShared;
};

template <class Ctx> __device__ __forceinline__ void fft_sync() {
  if constexpr (CtxBar<Ctx>::threads == 0) {
    __syncthreads();
  } else if constexpr (CtxBar<Ctx>::threads == 32) {
    __syncwarp();
  } else {
    asm volatile("bar.sync 1, %0;" ::"r"(CtxBar<Ctx>::threads) : "memory");
  }
}

// One padding element per 16 (per E) keeps the radix-16 (radix-E) scatter of
// the first pass (stride E) and the contiguous gathers free of bank conflicts.
__device__ __forceinline__ int pad16(int l) { return l + (l >> 4); }
template <int E> __device__ __forceinline__ int padE(int l) { return l + l / E; }

// Radix-16 DFT whose inputs 8..15 are zero (first pass of a transform whose
// upper half is zero padding): the first radix-4 stage sees (x0, x1, 0, 0).
__device__ __forceinline__ void dft16_half(float2* v) {
  float2 y[4][4];
#pragma unroll
  for (int n1 = 0; n1 < 4; ++n1) {
    const float2 x0 = v[n1], x1 = v[n1 + 4];
    const float2 mi = cmul_mi(x1);
    y[n1][0] = cadd(x0, x1);
    y[n1][2] = csub(x0, x1);
    y[n1][1] = cadd(x0, mi);
    y[n1][3] = csub(x0, mi);
#pragma unroll
    for (int k2 = 0; k2 < 4; ++k2) y[n1][k2] = mul_w32(y[n1][k2], 2 * n1 * k2);
  }
#pragma unroll
  for (int k2 = 0; k2 < 4; ++k2) {
    float2 t[4];
#pragma unroll
    for (int n1 = 0; n1 < 4; ++n1) t[n1] = y[n1][k2];
    Dft<4>::run(t);
#pragma unroll
    for (int k1 = 0; k1 < 4; ++k1) v[k2 + 4 * k1] = t[k1];
  }
}

// Radix-8 and radix-32 DFTs whose upper half of inputs is zero (first pass of
// a radix-32 transform whose upper half is zero padding). Radix 8 = 2 x 4:
// the radix-4 DFTs see (x0, x1, 0, 0); radix 32 = 4 x 8 with the radix-8
// DFTs pruned that way.
__device__ __forceinline__ void dft8_half(float2* v) {
  float2 y[2][4];
#pragma unroll
  for (int n1 = 0; n1 < 2; ++n1) {
    const float2 x0 = v[n1], x1 = v[n1 + 2];
    const float2 mi = cmul_mi(x1);
    y[n1][0] = cadd(x0, x1);
    y[n1][2] = csub(x0, x1);
    y[n1][1] = cadd(x0, mi);
    y[n1][3] = csub(x0, mi);
#pragma unroll
    for (int k2 = 0; k2 < 4; ++k2) y[n1][k2] = mul_w32(y[n1][k2], 4 * n1 * k2);
  }
#pragma unroll
  for (int k2 = 0; k2 < 4; ++k2) {
    float2 t[2] = {y[0][k2], y[1][k2]};
    Dft<2>::run(t);
    v[k2] = t[0];
    v[k2 + 4] = t[1];
  }
}
__device__ __forceinline__ void dft32_half(float2* v) {
  float2 y[4][8];
#pragma unroll
  for (int n1 = 0; n1 < 4; ++n1) {
#pragma unroll
    for (int n2 = 0; n2 < 8; ++n2) y[n1][n2] = v[n1 + 4 * n2];   // n2 >= 4 are the zero inputs
    dft8_half(y[n1]);
#pragma unroll
    for (int k2 = 0; k2 < 8; ++k2) y[n1][k2] = mul_w32(y[n1][k2], n1 * k2);
  }
#pragma unroll
  for (int k2 = 0; k2 < 8; ++k2) {
    float2 t[4];
#pragma unroll
    for (int n1 = 0; n1 < 4; ++n1) t[n1] = y[n1][k2];
    Dft<4>::run(t);
#pragma unroll
    for (int k1 = 0; k1 < 4; ++k1) v[k2 + 8 * k1] = t[k1];
  }
}

// Runs passes P..NPASS-1 of NT L-point transforms that share one schedule
// (same thread mapping and twiddles) for one thread.
//   kHalfIn:  inputs l >= L/2 are zero (not loaded; pruned first butterfly)
//   kHalfOut: only outputs l < L/2 are stored (dead outputs are not computed)
// Ctx provides:
//   void load(int l, float2 (&x)[NT])        input element l of every transform (first pass)
//   void store(int l, const float2 (&x)[NT]) output element l of every transform (last pass)
//   float2* sm(int t)                        shared-memory base of transform t; element l
//                                            lives at sm(t)[pad16(l) * SSTRIDE]
//   static constexpr int SSTRIDE
//   static constexpr bool kSmemInput         load() reads the shared buffer the passes reuse
//   const float2* tw                         twiddle table of the plan for length L
template <int L, int NT, bool kHalfIn, bool kHalfOut, int P, class Ctx, int E = 16>
__device__ __forceinline__ void fftn_passes(Ctx& ctx, const int j0, float2 (&v)[NT][E]) {
  using S = FftShape<L, E>;
  constexpr int R = S::radix(P);
  constexpr int NS = S::span(P);
  constexpr int BPT = E / R;
  constexpr int Q = L / R;
  constexpr int SS = Ctx::SSTRIDE;
  constexpr bool kFirst = (P == 0);
  constexpr bool kLast = (P == S::NPASS - 1);
#pragma unroll
  for (int i = 0; i < BPT; ++i) {
    const int j = j0 + i * S::TPC;
    if constexpr (kFirst) {
#pragma unroll
      for (int r = 0; r < R; ++r) {
        if (kHalfIn && 2 * r >= R) {
#pragma unroll
          for (int t = 0; t < NT; ++t) v[t][i * R + r] = make_float2(0.f, 0.f);
        } else {
          float2 x[NT];
          ctx.load(j + r * Q, x);
#pragma unroll
          for (int t = 0; t < NT; ++t) v[t][i * R + r] = x[t];
        }
      }
    } else if constexpr (Q % E == 0) {
      const int pj = padE<E>(j) * SS;
#pragma unroll
      for (int t = 0; t < NT; ++t) {
        const float2* s = ctx.sm(t) + pj;
#pragma unroll
        for (int r = 0; r < R; ++r) v[t][i * R + r] = s[r * (Q + Q / E) * SS];
      }
    } else {
#pragma unroll
      for (int t = 0; t < NT; ++t)
#pragma unroll
        for (int r = 0; r < R; ++r) v[t][i * R + r] = ctx.sm(t)[padE<E>(j + r * Q) * SS];
    }
  }
  // in-place: every read of this pass completes before the first write (a
  // first pass whose input was staged in the same shared buffer needs it too)
  if constexpr (!kFirst || Ctx::kSmemInput) fft_sync<Ctx>();
#pragma unroll
  for (int i = 0; i < BPT; ++i) {
    const int j = j0 + i * S::TPC;
    if constexpr (!kFirst) {
      const float2* tp = ctx.tw + S::twoff(P) + (j & (NS - 1));
#pragma unroll
      for (int r = 1; r < R; ++r) {
        const float2 w = CtxTwShared<Ctx>::value ? tp[r * NS] : __ldg(tp + r * NS);
#pragma unroll
        for (int t = 0; t < NT; ++t) v[t][i * R + r] = cmul(v[t][i * R + r], w);
      }
    }
#pragma unroll
    for (int t = 0; t < NT; ++t) {
      if constexpr (kFirst && kHalfIn && R == 16) dft16_half(&v[t][i * R]);
      else if constexpr (kFirst && kHalfIn && R == 32) dft32_half(&v[t][i * R]);
      else Dft<R>::run(&v[t][i * R]);
    }
  }
#pragma unroll
  for (int i = 0; i < BPT; ++i) {
    const int j = j0 + i * S::TPC;
    const int base = (j / NS) * NS * R + (j & (NS - 1));
    if constexpr (kLast) {
#pragma unroll
      for (int r = 0; r < R; ++r) {
        if (kHalfOut && 2 * r >= R) continue;
        float2 x[NT];
#pragma unroll
        for (int t = 0; t < NT; ++t) x[t] = v[t][i * R + r];
        ctx.store(base + r * NS, x);
      }
    } else if constexpr (NS == 1 && R == E) {
      const int pb = (E + 1) * j * SS;     // padE(E j + r) = (E + 1) j + r
#pragma unroll
      for (int t = 0; t < NT; ++t) {
        float2* s = ctx.sm(t) + pb;
#pragma unroll
        for (int r = 0; r < R; ++r) s[r * SS] = v[t][i * R + r];
      }
    } else if constexpr (NS % E == 0) {
      const int pb = padE<E>(base) * SS;
#pragma unroll
      for (int t = 0; t < NT; ++t) {
        float2* s = ctx.sm(t) + pb;
#pragma unroll
        for (int r = 0; r < R; ++r) s[r * (NS + NS / E) * SS] = v[t][i * R + r];
      }
    } else {
#pragma unroll
      for (int t = 0; t < NT; ++t)
#pragma unroll
        for (int r = 0; r < R; ++r) ctx.sm(t)[padE<E>(base + r * NS) * SS] = v[t][i * R + r];
    }
  }
  if constexpr (!kLast) {
    fft_sync<Ctx>();
    fftn_passes<L, NT, kHalfIn, kHalfOut, P + 1, Ctx, E>(ctx, j0, v);
  }
}

template <int L, int NT, bool kHalfIn, bool kHalfOut, class Ctx, int E = 16>
__device__ __forceinline__ void fftn_run(Ctx& ctx, const int j0) {
  float2 v[NT][E];
  fftn_passes<L, NT, kHalfIn, kHalfOut, 0, Ctx, E>(ctx, j0, v);
}

// ---------------------------------------------------------------------------
// storage types for complex intermediates and real inputs
// ---------------------------------------------------------------------------
template <class T> struct Cpx;
template <> struct Cpx<float2> {
  static __device__ __forceinline__ float2 get(const float2* p) { return *p; }
  static __device__ __forceinline__ void put(float2* p, float2 v) { *p = v; }
};
template <> struct Cpx<__half2> {
  static __device__ __forceinline__ float2 get(const __half2* p) { return __half22float2(*p); }
  static __device__ __forceinline__ void put(__half2* p, float2 v) { *p = __float22half2_rn(v); }
};
template <> struct Cpx<__nv_bfloat162> {
  static __device__ __forceinline__ float2 get(const __nv_bfloat162* p) { return __bfloat1622float2(*p); }
  static __device__ __forceinline__ void put(__nv_bfloat162* p, float2 v) { *p = __float22bfloat162_rn(v); }
};

// real element type of each complex storage type
template <class TS> struct RealOf;
template <> struct RealOf<float2> { using T = float; };
template <> struct RealOf<__half2> { using T = __half; };
template <> struct RealOf<__nv_bfloat162> { using T = __nv_bfloat16; };

template <class T> struct Real;
template <> struct Real<float> {
  static __device__ __forceinline__ float get(const float* p) { return *p; }
};
template <> struct Real<__half> {
  static __device__ __forceinline__ float get(const __half* p) { return __half2float(*p); }
};
template <> struct Real<__nv_bfloat16> {
  static __device__ __forceinline__ float get(const __nv_bfloat16* p) { return __bfloat162float(*p); }
};

}  // namespace nlos
