// f-k with the inverse temporal transform taken last (Sec. 4.2, Alg. 1).
//
// The inverse 3D transform of the Stolt-resampled spectrum factors into 1D
// transforms that commute, and only x < a, y < b of its result are kept. So
// the inverse along z can run after the lateral inverses, on the a x b kept
// pencils instead of on all (2a) x (2b) spectral pencils:
//
//   FK3 (fk_stolt_kernel): per stored pencil (kx, ky) the forward temporal
//       transform U (length L = 2n, the upper half of the input zero), then
//       the resampled spectra of the pencil and of its Hermitian partner,
//       V(m) = lerp(U at the Stolt source) * m / mu for 1 <= m < L/2 and its
//       partner's conj(lerp(U at minus the source)) * m / mu, both written to
//       global memory as they are ([kx][ky][m], m < n = L/2; V = 0 for m <= 0
//       and above L/2);
//   FK4: the lateral inverses (y then x, crop) of V, complex (the fused pair
//       of fk_chain.cuh);
//   FK5 (fk_zinv_kernel): per kept pencil (x, y) the inverse temporal
//       transform (length L, input m < L/2, output z < n) and |.|^2 with the
//       1/(Lx Ly Lt) normalisation, or the complex value.
//
// FK3 then runs one temporal transform per stored pencil instead of three,
// and FK5 one per kept pencil: the temporal transforms drop from
// 3 (a + 1) 2b to (a + 1) 2b + a b per volume, for 24V more bytes moved
// (V's 32V written and read once more at a quarter of its size: 8V, plus the
// complex intermediate of FK4). Any storage type (the 16-bit forms keep the
// per-pass scales of the other stages), L = 2n.
#pragma once
#include "fk_stolt.cuh"
#include "fk_zstage.cuh"
#include "nlos_bounds.cuh"
#include "nlos_fft.cuh"
#include "nlos_internal.h"

namespace nlos {

// Barrier threads of a transform context: a warp where the transform is one
// warp (L / E = 32 threads, each pencil's buffer private to its warp), else
// the CTA.
template <int L, int E> constexpr int fk_lite_bar() { return FftShape<L, E>::TPC == 32 ? 32 : 0; }

// forward transform of the stored pencil in place in its buffer (the
// transform's last pass reads all of the buffer before it writes). The last
// pass stores the spectrum unpadded, U[l]: its lanes write consecutive l, and
// the Stolt gather then indexes U without the padding arithmetic. The load
// scale of the non-ramped form is applied after the transform (it is linear).
template <int L, class TS, bool kRamp, int E>
struct FkLiteFwdCtx {
  static constexpr int SSTRIDE = 1;
  static constexpr bool kSmemInput = false;
  static constexpr int kBarThreads = fk_lite_bar<L, E>();
  const TS* g;
  float2* U;
  const float2* tw;
  bool valid;
  float ldmul, t_ramp;
  long long g_off, g_n;
  int* err;
  __device__ __forceinline__ void load(int l, float2 (&x)[1]) const {
    if (!(valid && bchk(g_off + l, g_n, err))) {
      x[0] = make_float2(0.f, 0.f);
    } else if constexpr (kRamp) {
      x[0] = cscale(Cpx<TS>::get(g + l), ldmul * (float)l * t_ramp);
    } else {
      x[0] = Cpx<TS>::get(g + l);
    }
  }
  __device__ __forceinline__ float2* sm(int) const { return U; }
  __device__ __forceinline__ void store(int l, const float2 (&x)[1]) const { U[l] = x[0]; }
};

// E: values per thread of the transforms (16: radix-16 passes, 32: radix-32)
// MINB: CTAs per SM the register allocation must allow (0: left to the
// compiler). The radix-32 length-1024 form (one warp per transform) keeps to
// 80 registers per thread: six 128-thread CTAs, which its shared memory also
// allows.
template <int L, int PPC, int E> struct FkLiteTile {
  static constexpr int THREADS = PPC * (L / E);
  static constexpr size_t SMEM = sizeof(float2) * PPC * FftShape<L, E>::SMEM;
  static constexpr int MINB = (E == 32 && L == 1024 && THREADS * 80 <= 65536) ? 65536 / (THREADS * 80) : 0;
};

template <int L, int PPC, class TS, bool kRamp, int E>
__global__ void __launch_bounds__(FkLiteTile<L, PPC, E>::THREADS, FkLiteTile<L, PPC, E>::MINB) fk_stolt_kernel(const FkZParams p) {
  using S = FftShape<L, E>;
  extern __shared__ float2 fl_sm[];
  const int w = threadIdx.x / S::TPC;
  const int j0 = threadIdx.x % S::TPC;
  const long long pid = (long long)blockIdx.x * PPC + w;
  const bool valid = pid < p.npencils;
  const int twob = p.b_pad;
  const int kx = valid ? (int)(pid / twob) : 0;
  const int ky = valid ? (int)(pid % twob) : 0;
  float2* U = fl_sm + w * S::SMEM;
  const float ldmul = p.ld_scale * (p.ld_dev_scale ? *p.ld_dev_scale : 1.0f);
  {
    const long long q = valid ? pid : 0;
    FkLiteFwdCtx<L, TS, kRamp, E> ctx{static_cast<const TS*>(p.G) + q * p.n, U, E == 32 ? p.tw32 : p.tw, valid,
                                      ldmul, p.t_ramp, q * p.n, p.G_n, p.err};
    fftn_run<L, 1, true, false, FkLiteFwdCtx<L, TS, kRamp, E>, E>(ctx, j0);
  }
  if constexpr (fk_lite_bar<L, E>() == 32) __syncwarp();
  else __syncthreads();
  if (!valid) return;
  const float2 ax = p.ax[kx];
  const float2 ay = p.ay[ky];
  float2 A = two_sum(ax.x, ay.x);
  A = fast_two_sum(A.x, A.y + (ax.y + ay.y));
  TS* V = static_cast<TS*>(p.psi);
  const long long o0 = ((long long)kx * twob + ky) * p.n;
  const int mkx = (kx == 0) ? 0 : p.a_pad - kx;
  const int mky = (twob - ky) & (twob - 1);
  const long long o1 = ((long long)mkx * twob + mky) * p.n;
  // the partner is stored only where it is not itself a stored pencil
  const bool partner = kx > 0 && 2 * kx < p.a_pad;
  const float st = kRamp ? p.st_scale : p.st_scale * ldmul;
  const StoltSplitA As = stolt_split_a(A.x, A.y);
  float fm = (float)j0;
  for (int m = j0; m < L / 2; m += S::TPC, fm += (float)S::TPC) {
    float2 d = make_float2(0.f, 0.f), e = d;
    if (m >= 1) {
      const StoltCoord c = stolt_coord_split(As, m, fm, L / 2);
      if (c.valid) {
        // k0 + 1 <= L/2 is in the spectrum; at k0 = L/2 - 1 its weight alpha is 0
        const int k1 = c.k1;
        const float2 u0 = U[c.k0], u1 = U[k1];
        const float2 w0 = U[(L - c.k0) & (L - 1)], w1 = U[(L - k1) & (L - 1)];
        // (1 - alpha) u0 + alpha u1, times the Jacobian m/mu and the scale
        const float b1 = c.jac * st * c.alpha;
        const float b0 = fmaf(c.jac, st, -b1);
        d = make_float2(fmaf(b1, u1.x, b0 * u0.x), fmaf(b1, u1.y, b0 * u0.y));
        e = make_float2(fmaf(b1, w1.x, b0 * w0.x), -fmaf(b1, w1.y, b0 * w0.y));
      }
    }
    if (bchk(o0 + m, p.psi_n, p.err)) Cpx<TS>::put(V + o0 + m, d);
    if (partner && bchk(o1 + m, p.psi_n, p.err)) Cpx<TS>::put(V + o1 + m, e);
  }
}

// inverse temporal transform of a kept pencil as conj(DFT(conj(V))): input
// m < L/2 (the upper half is zero), output z < L/2
template <int L, class TS, bool kCpx, int E>
struct FkZInvCtx {
  static constexpr int SSTRIDE = 1;
  static constexpr bool kSmemInput = false;
  static constexpr int kBarThreads = fk_lite_bar<L, E>();
  const TS* in;
  void* out;
  float2* W;
  const float2* tw;
  bool valid;
  float scale;
  long long in_off, in_n, out_off, out_n;
  int* err;
  __device__ __forceinline__ void load(int l, float2 (&x)[1]) const {
    x[0] = (valid && bchk(in_off + l, in_n, err)) ? cconj(Cpx<TS>::get(in + l)) : make_float2(0.f, 0.f);
  }
  __device__ __forceinline__ float2* sm(int) const { return W; }
  __device__ __forceinline__ void store(int l, const float2 (&x)[1]) const {
    if (!valid || !bchk(out_off + l, out_n, err)) return;
    if (kCpx) static_cast<float2*>(out)[l] = make_float2(x[0].x * scale, -x[0].y * scale);
    else static_cast<float*>(out)[l] = scale * fmaf(x[0].x, x[0].x, x[0].y * x[0].y);
  }
};

template <int L, int PPC, class TS, bool kCpx, int E>
__global__ void __launch_bounds__(FkLiteTile<L, PPC, E>::THREADS, FkLiteTile<L, PPC, E>::MINB) fk_zinv_kernel(const FkZInvParams p) {
  using S = FftShape<L, E>;
  extern __shared__ float2 zi_sm[];
  const int w = threadIdx.x / S::TPC;
  const int j0 = threadIdx.x % S::TPC;
  const long long pid = (long long)blockIdx.x * PPC + w;
  const bool valid = pid < p.npencils;
  const long long q = valid ? pid : 0;
  void* out = kCpx ? static_cast<void*>(static_cast<float2*>(p.out) + q * p.n)
                   : static_cast<void*>(static_cast<float*>(p.out) + q * p.n);
  const float scale = p.scale * (p.dev_scale ? *p.dev_scale : 1.0f);
  FkZInvCtx<L, TS, kCpx, E> ctx{static_cast<const TS*>(p.in) + q * p.n, out, zi_sm + w * S::SMEM,
                             E == 32 ? p.tw32 : p.tw, valid, scale, q * p.n, p.in_n, q * p.n, p.out_n, p.err};
  fftn_run<L, 1, true, true, FkZInvCtx<L, TS, kCpx, E>, E>(ctx, j0);
}

template <int L, int PPC, class TS, bool kRamp, int E = 16>
cudaError_t launch_fk_stolt_one(const FkZParams& p, cudaStream_t s) {
  using T = FkLiteTile<L, PPC, E>;
  auto k = fk_stolt_kernel<L, PPC, TS, kRamp, E>;
  if (T::SMEM > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)T::SMEM);
    if (e != cudaSuccess) return e;
  }
  const long long blocks = (p.npencils + PPC - 1) / PPC;
  k<<<(unsigned)blocks, T::THREADS, T::SMEM, s>>>(p);
  return cudaGetLastError();
}

template <int L, int PPC, class TS, bool kCpx, int E = 16>
cudaError_t launch_fk_zinv_one(const FkZInvParams& p, cudaStream_t s) {
  using T = FkLiteTile<L, PPC, E>;
  auto k = fk_zinv_kernel<L, PPC, TS, kCpx, E>;
  if (T::SMEM > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)T::SMEM);
    if (e != cudaSuccess) return e;
  }
  const long long blocks = (p.npencils + PPC - 1) / PPC;
  k<<<(unsigned)blocks, T::THREADS, T::SMEM, s>>>(p);
  return cudaGetLastError();
}

// launch shapes 0 / 1: radix-16 passes at the two pencils-per-CTA counts of
// fk_ppc; 2 / 3: radix-32 passes (32 values per thread) at twice those
// counts (the same threads per CTA). The ramped form, float32 only, takes shape 0.
template <int L, class TS>
cudaError_t launch_fk_stolt_len(const FkZParams& p, int tile, cudaStream_t s) {
  constexpr int P0 = fk_ppc(L, 0), P1 = fk_ppc(L, 1);
  if (p.t_ramp != 0.f) {
    if constexpr (std::is_same<TS, float2>::value) return launch_fk_stolt_one<L, P0, TS, true>(p, s);
    else return cudaErrorInvalidValue;
  }
  switch (tile) {
    case 1: return launch_fk_stolt_one<L, P1, TS, false>(p, s);
    case 2: return launch_fk_stolt_one<L, 2 * P0, TS, false, 32>(p, s);
    case 3: return launch_fk_stolt_one<L, 2 * P1, TS, false, 32>(p, s);
    default: return launch_fk_stolt_one<L, P0, TS, false>(p, s);
  }
}

template <int L, class TS>
cudaError_t launch_fk_zinv_len(const FkZInvParams& p, int tile, cudaStream_t s) {
  constexpr int P0 = fk_ppc(L, 0), P1 = fk_ppc(L, 1);
  if (p.complex_out) {
    switch (tile) {
      case 1: return launch_fk_zinv_one<L, P1, TS, true>(p, s);
      case 2: return launch_fk_zinv_one<L, 2 * P0, TS, true, 32>(p, s);
      case 3: return launch_fk_zinv_one<L, 2 * P1, TS, true, 32>(p, s);
      default: return launch_fk_zinv_one<L, P0, TS, true>(p, s);
    }
  }
  switch (tile) {
    case 1: return launch_fk_zinv_one<L, P1, TS, false>(p, s);
    case 2: return launch_fk_zinv_one<L, 2 * P0, TS, false, 32>(p, s);
    case 3: return launch_fk_zinv_one<L, 2 * P1, TS, false, 32>(p, s);
    default: return launch_fk_zinv_one<L, P0, TS, false>(p, s);
  }
}

}  // namespace nlos
