// f-k migration, temporal-frequency stage (Sec. 4.2, Alg. 1 Stolt step).
//
// The x/y transforms before this stage keep only kx in [0, Lx/2] of the real
// input's spectrum (Hermitian half along x). Each stored pencil (kx, ky) is
// transformed along t (length L >= 2n, zero beyond the n samples) into
// U(kx, ky, m), held in shared memory. The Stolt step reads U at the source
// coordinate mu = sqrt(A + m^2), A = (L s_x p~/Lx)^2 + (L s_y q~/Ly)^2 (for
// L = 2n, Lx = 2a: (n s_x p~/a)^2 ...), with a two-tap linear interpolation
// along the contiguous axis, weights it by Z/Z' = m/mu and keeps
// 1 <= m <= L/2-1 with mu <= L/2-1 (Z > 0 and interpn's zero fill).
// The same pencil also yields its Hermitian partner (-kx, -ky): there
// U(-p~, -q~, k) = conj(U(p~, q~, -k)), so the partner's resampled spectrum is
// conj(lerp(U[-k0], U[-k1])) * m/mu. Both resampled spectra are inverse
// transformed (length L, only z < n kept) and written, so the Stolt output
// never round-trips through global memory.
//
// mu is computed in float-float: A comes from float64 per-plan tables split
// into (hi, lo) floats, m^2 is exact, and the square root gets one Newton
// correction from an exact FMA residual. Plain float would put the
// interpolation weight off by up to 6e-5 near m ~ 1000.
#pragma once
#include <type_traits>
#include "fk_stolt.cuh"
#include "fk_zwarp.cuh"
#include "nlos_bounds.cuh"
#include "nlos_fft.cuh"
#include "nlos_internal.h"

namespace nlos {

// forward transform of the stored pencil; its upper half is zero padding
// (kGuard: the pencil is shorter than L / 2, loads past it read zero;
// kRamp: sample t is also multiplied by t * t_ramp)
template <int L, class TS, bool kGuard, bool kRamp>
struct FkFwdCtx {
  static constexpr int SSTRIDE = 1;
  static constexpr bool kSmemInput = false;
  const TS* g;
  float2* U;
  float2* W;
  const float2* tw;
  bool valid;
  float ldmul;
  int n_in;                  // stored samples of the pencil (the rest is zero padding)
  long long g_off, g_n;      // offset of g in its buffer, the buffer's extent (bounds-checked build)
  int* err;
  float t_ramp;
  __device__ __forceinline__ void load(int l, float2 (&x)[1]) const {
    const float m = kRamp ? ldmul * (float)l * t_ramp : ldmul;
    x[0] = (valid && (!kGuard || l < n_in) && bchk(g_off + l, g_n, err)) ? cscale(Cpx<TS>::get(g + l), m)
                                                                         : make_float2(0.f, 0.f);
  }
  __device__ __forceinline__ float2* sm(int) const { return W; }
  __device__ __forceinline__ void store(int l, const float2 (&x)[1]) const { U[pad16(l)] = x[0]; }
};

// both inverse transforms at once: t = 0 the stored pencil, t = 1 its
// Hermitian partner; one Stolt coordinate per m feeds both. kAliasU: the
// pencil's transform runs in U's own buffer, so the first pass must finish
// reading U before it writes (kSmemInput adds that barrier).
template <int L, class TS, bool kAliasU, bool kGuard>
struct FkInvCtx {
  static constexpr int SSTRIDE = 1;
  static constexpr bool kSmemInput = kAliasU;
  const float2* U;
  float2* W0;
  float2* W1;
  const float2* tw;
  TS* out0;
  TS* out1;
  int n;                     // Stolt source bound: indices below L/2
  float Ahi, Alo;
  bool st0, st1;
  float stmul;
  int n_out;                 // kept outputs z < n_out
  long long off0, off1, psi_n;   // offsets of out0 / out1 in their buffer, its extent (bounds-checked build)
  int* err;
  __device__ __forceinline__ void load(int m, float2 (&x)[2]) const {
    x[0] = x[1] = make_float2(0.f, 0.f);
    if (m < 1) return;                                // m < L/2 (upper half is pruned)
    const StoltCoord c = stolt_coord(Ahi, Alo, m, n);
    if (!c.valid) return;
    const float2 u0 = U[pad16(c.k0)], u1 = U[pad16(c.k1)];
    const float2 w0 = U[pad16((L - c.k0) & (L - 1))], w1 = U[pad16((L - c.k1) & (L - 1))];
    const float2 d = make_float2(fmaf(c.alpha, u1.x - u0.x, u0.x), fmaf(c.alpha, u1.y - u0.y, u0.y));
    const float2 e = make_float2(fmaf(c.alpha, w1.x - w0.x, w0.x), fmaf(c.alpha, w1.y - w0.y, w0.y));
    // inverse DFT as conj(DFT(conj(V))): the pencil loads conj(V); the
    // partner's V is conj(lerp) * m/mu, whose conjugate is lerp * m/mu
    x[0] = cconj(cscale(d, c.jac));
    x[1] = cscale(e, c.jac);
  }
  __device__ __forceinline__ float2* sm(int t) const { return t == 0 ? W0 : W1; }
  __device__ __forceinline__ void store(int l, const float2 (&x)[2]) const {   // every l the schedule keeps
    if (kGuard && l >= n_out) return;
    if (st0 && bchk(off0 + l, psi_n, err)) Cpx<TS>::put(out0 + l, cscale(cconj(x[0]), stmul));
    if (st1 && bchk(off1 + l, psi_n, err)) Cpx<TS>::put(out1 + l, cscale(cconj(x[1]), stmul));
  }
};

// pencils-per-CTA variants per length (index 0 is the default)
__host__ __device__ constexpr int fk_ppc(int L, int v) {
  return L <= 128 ? (v == 0 ? 16 : 32)
       : L <= 256 ? (v == 0 ? 8 : 16)
       : L <= 512 ? (v == 0 ? 4 : 8)
       : L <= 1024 ? (v == 0 ? 2 : 4)
       : L <= 4096 ? (v == 0 ? 2 : 1) : 1;
}

// kAlias: two shared buffers per pencil instead of three (the pencil's
// inverse transform reuses the spectrum's buffer) and a register cap of
// about 100 per thread, so that more CTAs fit on an SM.
template <int L, int PPC_, bool kAlias = false> struct FkTile {
  static constexpr int PPC = PPC_;   // pencils per CTA
  static constexpr int THREADS = PPC * (L / 16);
  static constexpr int NBUF = kAlias ? 2 : 3;
  static constexpr size_t SMEM = sizeof(float2) * NBUF * PPC * FftShape<L>::SMEM;
  static constexpr int MIN_BLOCKS_RAW = 65536 / (THREADS * 96);
  static constexpr int MIN_BLOCKS = !kAlias ? 1 : MIN_BLOCKS_RAW < 1 ? 1 : MIN_BLOCKS_RAW > 16 ? 16 : MIN_BLOCKS_RAW;
};

// kPad2: the temporal axis is zero-padded to L >= 2n (the forward input's
// upper half is zero and only z < n is kept); otherwise L = n and every
// output is kept. Either way the Stolt source must stay below L/2.
// kGuard: L > 2n (a time axis that is not a power of two): loads beyond the
// pencil and stores beyond z = n are masked; otherwise the pruned passes
// already stop there.
// kRamp: the spectrum was taken without f-k's t/(n-1) ramp, which the
// forward loads apply (float32 shared-spectrum plans, launch shape 0 only)
template <int L, int PPC, class TS, bool kPad2, bool kAlias, bool kGuard, bool kRamp = false>
__global__ void __launch_bounds__(FkTile<L, PPC, kAlias>::THREADS, FkTile<L, PPC, kAlias>::MIN_BLOCKS)
fk_zstage_kernel(const FkZParams p) {
  using S = FftShape<L>;
  extern __shared__ float2 fk_sm[];
  const int w = threadIdx.x / S::TPC;
  const int j0 = threadIdx.x % S::TPC;
  const long long pid = (long long)blockIdx.x * PPC + w;
  const bool valid = pid < p.npencils;
  const int twob = p.b_pad;
  const int kx = valid ? (int)(pid / twob) : 0;
  const int ky = valid ? (int)(pid % twob) : 0;
  float2* U = fk_sm + w * S::SMEM;
  float2* W0 = kAlias ? U : fk_sm + (PPC + w) * S::SMEM;
  float2* W1 = fk_sm + ((kAlias ? 1 : 2) * PPC + w) * S::SMEM;
  const float ldmul = p.ld_scale * (p.ld_dev_scale ? *p.ld_dev_scale : 1.0f);
  {
    FkFwdCtx<L, TS, kGuard, kRamp> ctx{static_cast<const TS*>(p.G) + (valid ? pid : 0) * p.n, U, W0, p.tw, valid,
                                       ldmul, p.n, (valid ? pid : 0) * p.n, p.G_n, p.err, p.t_ramp};
    fftn_run<L, 1, kPad2, false>(ctx, j0);
  }
  __syncthreads();
  const float2 ax = p.ax[kx];
  const float2 ay = p.ay[ky];
  float2 A = two_sum(ax.x, ay.x);
  A = fast_two_sum(A.x, A.y + (ax.y + ay.y));
  TS* psi = static_cast<TS*>(p.psi);
  const long long o_direct = ((long long)kx * twob + ky) * p.n;
  const int mkx = (kx == 0) ? 0 : p.a_pad - kx;
  const int mky = (twob - ky) & (twob - 1);
  const long long o_mirror = ((long long)mkx * twob + mky) * p.n;
  // the partner is stored only where it is not itself a stored pencil
  FkInvCtx<L, TS, kAlias, kGuard> ctx{U, W0, W1, p.tw, psi + o_direct, psi + o_mirror, L / 2, A.x, A.y,
                      valid, valid && kx > 0 && 2 * kx < p.a_pad, p.st_scale, p.n, o_direct, o_mirror, p.psi_n, p.err};
  fftn_run<L, 2, true, kPad2>(ctx, j0);
}

template <int L, int PPC, class TS, bool kAlias, bool kRamp = false>
cudaError_t launch_fk_ppc(const FkZParams& p, cudaStream_t s) {
  using T = FkTile<L, PPC, kAlias>;
  auto k = p.pad != 2 ? fk_zstage_kernel<L, PPC, TS, false, kAlias, false, kRamp>
           : p.L == 2 * p.n ? fk_zstage_kernel<L, PPC, TS, true, kAlias, false, kRamp>
                            : fk_zstage_kernel<L, PPC, TS, true, kAlias, true, kRamp>;
  if (T::SMEM > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)T::SMEM);
    if (e != cudaSuccess) return e;
  }
  const long long blocks = (p.npencils + T::PPC - 1) / T::PPC;
  k<<<(unsigned)blocks, T::THREADS, T::SMEM, s>>>(p);
  return cudaGetLastError();
}

// tiles 0/1: the two CTA sizes; 2/3: the same with aliased buffers
template <int L, class TS>
cudaError_t launch_fk_one(const FkZParams& p, int tile, cudaStream_t s) {
  if (p.t_ramp != 0.f) {
    // ramp applied at the loads: float32 storage, launch shape 0
    if constexpr (std::is_same<TS, float2>::value) return launch_fk_ppc<L, fk_ppc(L, 0), TS, false, true>(p, s);
    else return cudaErrorInvalidValue;
  }
  switch (tile) {
    case 4:
      if constexpr (L == 1024) return launch_fk_warp<L, TS>(p, s);
      else return cudaErrorInvalidValue;
    case 1: return launch_fk_ppc<L, fk_ppc(L, 1), TS, false>(p, s);
    case 2: return launch_fk_ppc<L, fk_ppc(L, 0), TS, true>(p, s);
    case 3: return launch_fk_ppc<L, fk_ppc(L, 1), TS, true>(p, s);
    default: return launch_fk_ppc<L, fk_ppc(L, 0), TS, false>(p, s);
  }
}

// Each translation unit instantiates one length range (0: 16-256,
// 1: 512-1024, 2: 2048-8192); RANGE keeps the units' dispatchers distinct.
template <class TS, int RANGE>
cudaError_t launch_fk_typed(const FkZParams& p, int tile, cudaStream_t s) {
  if (p.npencils <= 0) return cudaErrorInvalidValue;
  switch (p.L) {
#if defined(FK_RANGE) && FK_RANGE == 0
    case 16: return launch_fk_one<16, TS>(p, tile, s);
    case 32: return launch_fk_one<32, TS>(p, tile, s);
    case 64: return launch_fk_one<64, TS>(p, tile, s);
    case 128: return launch_fk_one<128, TS>(p, tile, s);
    case 256: return launch_fk_one<256, TS>(p, tile, s);
#endif
#if defined(FK_RANGE) && FK_RANGE == 1
    case 512: return launch_fk_one<512, TS>(p, tile, s);
    case 1024: return launch_fk_one<1024, TS>(p, tile, s);
#endif
#if defined(FK_RANGE) && FK_RANGE == 2
    case 2048: return launch_fk_one<2048, TS>(p, tile, s);
    case 4096: return launch_fk_one<4096, TS>(p, tile, s);
    case 8192: return launch_fk_one<8192, TS>(p, tile, s);
#endif
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace nlos
