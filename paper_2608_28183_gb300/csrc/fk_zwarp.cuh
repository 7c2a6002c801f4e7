// f-k temporal-frequency stage with one warp per transform (Sec. 4.2, Alg. 1
// Stolt step; the arithmetic is that of fk_zstage.cuh).
//
// A CTA of two warps owns the stored pencils P0 = (kx, ky) and P1 = (kx, -ky)
// (for ky = 0 and ky = Ly/2 the two coincide and warp 1 only repeats warp 0,
// without storing). Both share the Stolt constant
// A = (L s_x p~/Lx)^2 + (L s_y q~/Ly)^2, so the source coordinate of every m
// is computed once per CTA into a table that the four inverse transforms
// read. Per warp (radix-32 transforms, 32 values per thread, only warp-local
// barriers between passes):
//   1. forward transform of its pencil, in place in its buffer U;
//   2. inverse transform of the resampled pencil, lerp(U[k0], U[k1]) m/mu,
//      through a second buffer W;
//   3. inverse transform of the resampled Hermitian partner (-kx, -ky),
//      conj(lerp(U[-k0], U[-k1])) m/mu, in place in U once every gather of it
//      has been read.
// Inverse transforms run as conj(DFT(conj(V))).
//
// Coordinate table: mu = sqrt(A + m^2) in float-float (stolt_coord) stored as
// fixed point, k0 in the upper bits and the fraction alpha in the lower
// FRAC = 32 - log2(L/2) bits (alpha to 2^-23 at L = 1024), or an all-ones
// word where the source lies beyond L/2 - 1 or m < 1; the weight m/mu beside
// it as a float.
#pragma once
#include "fk_stolt.cuh"
#include "nlos_bounds.cuh"
#include "nlos_fft.cuh"
#include "nlos_internal.h"

namespace nlos {

constexpr unsigned kStoltNone = 0xffffffffu;

template <int L> struct FkWarpShape {
  static_assert(L == 1024, "one warp per transform: L / 32 = 32 threads");
  static constexpr int E = 32;
  static constexpr int NB = L / 2;                       // Stolt source bound
  static constexpr int FRAC = 32 - ilog2c(NB);           // fraction bits of the table
  static constexpr int BUF = FftShape<L, E>::SMEM;       // float2 per buffer
  static constexpr size_t SMEM = sizeof(float2) * 4 * BUF + (sizeof(unsigned) + sizeof(float)) * NB;
};

template <int L, class TS, bool kGuard>
struct FkWarpFwdCtx {
  static constexpr int SSTRIDE = 1;
  static constexpr bool kSmemInput = false;
  static constexpr int kBarThreads = 32;
  const TS* g;
  float2* U;
  const float2* tw;
  float ldmul;
  int n_in;
  long long g_off, g_n;      // offset of g in its buffer, the buffer's extent (bounds-checked build)
  int* err;
  __device__ __forceinline__ void load(int l, float2 (&x)[1]) const {
    x[0] = ((!kGuard || l < n_in) && bchk(g_off + l, g_n, err)) ? cscale(Cpx<TS>::get(g + l), ldmul)
                                                                : make_float2(0.f, 0.f);
  }
  __device__ __forceinline__ float2* sm(int) const { return U; }
  __device__ __forceinline__ void store(int l, const float2 (&x)[1]) const { U[padE<32>(l)] = x[0]; }
};

// kPartner: gathers at -k0, -k1 (the Hermitian partner) instead of k0, k1
template <int L, class TS, bool kGuard, bool kPartner>
struct FkWarpInvCtx {
  using Sh = FkWarpShape<L>;
  static constexpr int SSTRIDE = 1;
  static constexpr bool kSmemInput = kPartner;   // the partner runs in place in U
  static constexpr int kBarThreads = 32;
  const float2* U;
  float2* buf;
  const unsigned* coord;
  const float* jac;
  const float2* tw;
  TS* out;
  bool st;
  float stmul;
  int n_out;
  long long out_off, psi_n;  // offset of out in its buffer, the buffer's extent (bounds-checked build)
  int* err;
  __device__ __forceinline__ void load(int m, float2 (&x)[1]) const {
    x[0] = make_float2(0.f, 0.f);
    const unsigned e = coord[m];                  // m < L/2: the upper half is pruned
    if (e == kStoltNone) return;
    const int k0 = (int)(e >> Sh::FRAC);
    const int k1 = min(k0 + 1, Sh::NB - 1);
    const float al = (float)(e & ((1u << Sh::FRAC) - 1u)) * (1.0f / (float)(1u << Sh::FRAC));
    const float j = jac[m];
    float2 u0, u1;
    if (kPartner) {
      u0 = U[padE<32>((L - k0) & (L - 1))];
      u1 = U[padE<32>((L - k1) & (L - 1))];
    } else {
      u0 = U[padE<32>(k0)];
      u1 = U[padE<32>(k1)];
    }
    const float2 d = make_float2(fmaf(al, u1.x - u0.x, u0.x), fmaf(al, u1.y - u0.y, u0.y));
    // the pencil loads conj(V) = conj(d) m/mu; the partner's V is conj(d) m/mu
    // as well (d gathered at -k), whose conjugate d m/mu it loads
    x[0] = kPartner ? cscale(d, j) : make_float2(d.x * j, -d.y * j);
  }
  __device__ __forceinline__ float2* sm(int) const { return buf; }
  __device__ __forceinline__ void store(int l, const float2 (&x)[1]) const {
    if (kGuard && l >= n_out) return;
    if (st && bchk(out_off + l, psi_n, err)) Cpx<TS>::put(out + l, make_float2(x[0].x * stmul, -x[0].y * stmul));
  }
};

// kPad2 / kGuard as in fk_zstage_kernel.
template <int L, class TS, bool kPad2, bool kGuard>
__global__ void __launch_bounds__(64) fk_zwarp_kernel(const FkZParams p) {
  using Sh = FkWarpShape<L>;
  extern __shared__ float2 zw_sm[];
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  float2* U = zw_sm + w * Sh::BUF;
  float2* W = zw_sm + (2 + w) * Sh::BUF;
  unsigned* coord = reinterpret_cast<unsigned*>(zw_sm + 4 * Sh::BUF);
  float* jac = reinterpret_cast<float*>(coord + Sh::NB);
  const int hb = p.b_pad / 2 + 1;
  const int kx = (int)(blockIdx.x / hb);
  const int ky0 = (int)(blockIdx.x % hb);
  const int ky1 = (p.b_pad - ky0) & (p.b_pad - 1);
  const bool single = ky1 == ky0;
  const int ky = w ? ky1 : ky0;
  const long long pid = (long long)kx * p.b_pad + ky;
  const float ldmul = p.ld_scale * (p.ld_dev_scale ? *p.ld_dev_scale : 1.0f);
  {
    FkWarpFwdCtx<L, TS, kGuard> ctx{static_cast<const TS*>(p.G) + pid * p.n, U, p.tw32, ldmul, p.n, pid * p.n, p.G_n,
                                    p.err};
    fftn_run<L, 1, kPad2, false, FkWarpFwdCtx<L, TS, kGuard>, 32>(ctx, lane);
  }
  {
    // A is even in q~, so both pencils take ay[ky0]
    const float2 ax = p.ax[kx];
    const float2 ay = p.ay[ky0];
    float2 A = two_sum(ax.x, ay.x);
    A = fast_two_sum(A.x, A.y + (ax.y + ay.y));
    for (int m = threadIdx.x; m < Sh::NB; m += 64) {
      unsigned e = kStoltNone;
      float j = 0.f;
      if (m >= 1) {
        const StoltCoord c = stolt_coord(A.x, A.y, m, Sh::NB);
        if (c.valid) {
          const unsigned fr = min(__float2uint_rz(c.alpha * (float)(1u << Sh::FRAC)), (1u << Sh::FRAC) - 1u);
          e = ((unsigned)c.k0 << Sh::FRAC) | fr;
          j = c.jac;
        }
      }
      coord[m] = e;
      jac[m] = j;
    }
  }
  __syncthreads();   // the table, and each warp's spectrum
  TS* psi = static_cast<TS*>(p.psi);
  const bool own = w == 0 || !single;
  {
    FkWarpInvCtx<L, TS, kGuard, false> ctx{U, W, coord, jac, p.tw32, psi + pid * p.n, own, p.st_scale, p.n, pid * p.n,
                                           p.psi_n, p.err};
    fftn_run<L, 1, true, kPad2, FkWarpInvCtx<L, TS, kGuard, false>, 32>(ctx, lane);
  }
  {
    // the partner is stored only where it is not itself a stored pencil
    const int mkx = (kx == 0) ? 0 : p.a_pad - kx;
    const int mky = (p.b_pad - ky) & (p.b_pad - 1);
    const bool st = own && kx > 0 && 2 * kx < p.a_pad;
    const long long mo = ((long long)mkx * p.b_pad + mky) * p.n;
    FkWarpInvCtx<L, TS, kGuard, true> ctx{U, U, coord, jac, p.tw32, psi + mo, st, p.st_scale, p.n, mo, p.psi_n, p.err};
    fftn_run<L, 1, true, kPad2, FkWarpInvCtx<L, TS, kGuard, true>, 32>(ctx, lane);
  }
}

template <int L, class TS>
cudaError_t launch_fk_warp(const FkZParams& p, cudaStream_t s) {
  using Sh = FkWarpShape<L>;
  if (!p.tw32) return cudaErrorInvalidValue;
  auto k = p.pad != 2 ? fk_zwarp_kernel<L, TS, false, false>
           : p.L == 2 * p.n ? fk_zwarp_kernel<L, TS, true, false>
                            : fk_zwarp_kernel<L, TS, true, true>;
  if (Sh::SMEM > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Sh::SMEM);
    if (e != cudaSuccess) return e;
  }
  const long long units = (long long)(p.a_pad / 2 + 1) * (p.b_pad / 2 + 1);
  k<<<(unsigned)units, 64, Sh::SMEM, s>>>(p);
  return cudaGetLastError();
}

}  // namespace nlos
