// Phasor-field (radial RSD) kernels: temporal band transform, depth sum over
// the radial kernel, plan-time float64 construction of the radial kernel, and
// the per-volume scale used by reduced-precision storage.
#include "nlos_bounds.cuh"
#include "nlos_fft.cuh"
#include "nlos_internal.h"
#include "nlos_tma.cuh"
#include "nlos_umma.cuh"

namespace nlos {

// ---------------------------------------------------------------------------
// PF1: P[x][y][f] = w(f) * sum_t H[x][y][t] exp(-2 pi i (k_lo + f) t / n)
// (Sec. 3.1 phasor field; w(f) is the virtual wave's spectrum, folded here
// instead of inside the depth sum.)
// Two real pencils share one complex transform: z = h0 + i h1, Z = DFT(z),
// then X0[k] = (Z[k] + conj Z[L - k]) / 2 and X1[k] = (Z[k] - conj Z[L - k]) / (2i).
// The transform keeps the band bins and their mirrors in shared memory; the
// pair's threads then split them and store both pencils' bands.
// ---------------------------------------------------------------------------
template <int L, class TR, bool kStaged>
struct PfBandCtx {
  static constexpr int SSTRIDE = 1;
  // staged: the pair's samples sit at the start of the transform's own
  // buffer, so the first pass reads them all before it writes
  static constexpr bool kSmemInput = kStaged;
  const TR* h0;                // global pencil, or (staged) the pair's samples in shared memory
  bool has1;                   // the pair's second pencil exists
  float2* O;                   // [2F]: Z[k_lo + f], then Z[L - k_lo - f]
  float2* W;
  const float2* tw;
  int k_lo, F;
  float ldmul;
  int n_in;                    // samples of the pencil; the DFT runs over L >= n_in
  long long h_off, H_n;        // offset of h0 in H, H's extent (bounds-checked build)
  int* err;
  __device__ __forceinline__ void load(int l, float2 (&x)[1]) const {
    const bool in = l < n_in;
    float re = 0.f, im = 0.f;
    if (kStaged) {
      if (in) re = Real<TR>::get(h0 + l) * ldmul;
      if (in && has1) im = Real<TR>::get(h0 + n_in + l) * ldmul;
    } else {
      if (in && bchk(h_off + l, H_n, err)) re = Real<TR>::get(h0 + l) * ldmul;
      if (in && has1 && bchk(h_off + n_in + l, H_n, err)) im = Real<TR>::get(h0 + n_in + l) * ldmul;
    }
    x[0] = make_float2(re, im);
  }
  __device__ __forceinline__ float2* sm(int) const { return W; }
  __device__ __forceinline__ void store(int l, const float2 (&x)[1]) const {
    const int f = l - k_lo;
    if (f >= 0 && f < F) O[f] = x[0];
    const int g = ((L - l) & (L - 1)) - k_lo;
    if (g >= 0 && g < F) O[F + g] = x[0];
  }
};

template <int L> struct PfBandTile {
  // transforms (pencil pairs) per CTA
  static constexpr int PPC = L <= 256 ? 8 : 2;
  static constexpr int THREADS = PPC * (L / 16);
  static constexpr size_t BUF = sizeof(float2) * PPC * FftShape<L>::SMEM;   // one slot of transform buffers
  // slots of transform buffers (two when staged), the band bins, two barriers
  static constexpr size_t smem(int F, bool staged) {
    return (staged ? 2 : 1) * BUF + sizeof(float2) * PPC * 2 * F + 2 * sizeof(uint64_t);
  }
};

constexpr int kBandWaitLimit = 1 << 21;   // polls of a staged-load barrier (~1 s in all)

// split the transform of one pencil pair into both pencils' bands (w(f) and
// the store scale applied) and store them; returns the largest |component| stored
template <class TS>
__device__ __forceinline__ float band_split_store(const PfBandParams& p, const float2* O, long long q, bool has1,
                                                  int j0, int TPC) {
  float m = 0.f;
  TS* P0 = static_cast<TS*>(p.P) + q * p.F;
  TS* P1 = P0 + p.F;
  for (int f = j0; f < p.F; f += TPC) {
    const float2 z = O[f], c = cconj(O[p.F + f]);
    const float s = 0.5f * __ldg(p.w + f) * p.st_scale;
    float2 x0 = make_float2(s * (z.x + c.x), s * (z.y + c.y));
    float2 x1 = make_float2(s * (z.y - c.y), -s * (z.x - c.x));   // (z - c) / (2i)
    if (bchk(q * p.F + f, p.P_n, p.err)) {
      if (p.accumulate) x0 = cadd(x0, Cpx<TS>::get(P0 + f));
      Cpx<TS>::put(P0 + f, x0);
      m = fmaxf(m, fmaxf(fabsf(x0.x), fabsf(x0.y)));
    }
    if (has1 && bchk((q + 1) * p.F + f, p.P_n, p.err)) {
      if (p.accumulate) x1 = cadd(x1, Cpx<TS>::get(P1 + f));
      Cpx<TS>::put(P1 + f, x1);
      m = fmaxf(m, fmaxf(fabsf(x1.x), fabsf(x1.y)));
    }
  }
  return m;
}

template <int L>
__device__ __forceinline__ void band_amax(const PfBandParams& p, float m) {
  if (!p.amax) return;
  // the bound the float32 depth sum scales its phasors by (see PfBandParams)
  // (blocks of short transforms have fewer than 32 threads: reduce over
  // the lanes that exist)
  constexpr int TH = PfBandTile<L>::THREADS;
  constexpr int WID = TH < 32 ? TH : 32;
  constexpr unsigned MASK = TH < 32 ? ((1u << TH) - 1u) : 0xffffffffu;
#pragma unroll
  for (int o = WID / 2; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(MASK, m, o, WID));
  if ((threadIdx.x % WID) == 0) atomicMax(p.amax, __float_as_uint(m));
}

// one pass over the pairs, samples loaded by each thread from global memory
template <int L, class TR, class TS>
__global__ void __launch_bounds__(PfBandTile<L>::THREADS)
pf_band_kernel(const PfBandParams p) {
  using S = FftShape<L>;
  using T = PfBandTile<L>;
  extern __shared__ __align__(16) unsigned char pfb_sm[];
  const int w = threadIdx.x / S::TPC;
  const int j0 = threadIdx.x % S::TPC;
  const long long q0 = 2 * ((long long)blockIdx.x * T::PPC + w);    // the pair's first pencil
  const bool v0 = q0 < p.npencils, v1 = q0 + 1 < p.npencils;
  const long long q = v0 ? q0 : 0;
  const float ldmul = p.ld_scale * (p.ld_dev_scale ? *p.ld_dev_scale : 1.0f);
  float2* W = reinterpret_cast<float2*>(pfb_sm) + w * S::SMEM;
  float2* O = reinterpret_cast<float2*>(pfb_sm + T::BUF) + (size_t)w * 2 * p.F;
  PfBandCtx<L, TR, false> ctx{static_cast<const TR*>(p.H) + q * p.n, v1, O, W, p.tw, p.k_lo, p.F, ldmul, p.n,
                              q * p.n, p.H_n, p.err};
  fftn_run<L, 1, false, false>(ctx, j0);
  __syncthreads();
  const float m = v0 ? band_split_store<TS>(p, O, q, v1, j0, S::TPC) : 0.f;
  band_amax<L>(p, m);
}

// persistent CTAs over sets of PPC pairs (2 PPC consecutive pencils): one
// thread stages the next set's samples with bulk copies into the other slot
// of transform buffers while the CTA transforms the current set
template <int L, class TR, class TS>
__global__ void __launch_bounds__(PfBandTile<L>::THREADS)
pf_band_staged_kernel(const PfBandParams p, const long long nsets) {
  using S = FftShape<L>;
  using T = PfBandTile<L>;
  extern __shared__ __align__(128) unsigned char pfb_sm[];
  uint64_t* bar = reinterpret_cast<uint64_t*>(pfb_sm + 2 * T::BUF + sizeof(float2) * T::PPC * 2 * p.F);
  const int w = threadIdx.x / S::TPC;
  const int j0 = threadIdx.x % S::TPC;
  const size_t pbytes = (size_t)p.n * sizeof(TR);                 // one pencil (a multiple of 16)
  auto slot_buf = [&](int slot, int t) {
    return reinterpret_cast<float2*>(pfb_sm + slot * T::BUF) + t * S::SMEM;
  };
  if (threadIdx.x == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    mbar_fence_init();
  }
  __syncthreads();
  const TR* H = static_cast<const TR*>(p.H);
  auto issue = [&](long long set, int slot) {
    const long long first = 2 * T::PPC * set;
    const long long cnt = p.npencils - first < 2 * T::PPC ? p.npencils - first : 2 * T::PPC;
    mbar_arrive_expect_tx(&bar[slot], (uint32_t)(cnt * pbytes));
    for (int t = 0; 2 * t < cnt; ++t) {
      const long long k = cnt - 2 * t < 2 ? cnt - 2 * t : 2;
      bulk_load(slot_buf(slot, t), H + (first + 2 * t) * p.n, (uint32_t)(k * pbytes), &bar[slot]);
    }
  };
  long long set = blockIdx.x;
  if (threadIdx.x == 0 && set < nsets) issue(set, 0);
  const float ldmul = p.ld_scale * (p.ld_dev_scale ? *p.ld_dev_scale : 1.0f);
  float2* O = reinterpret_cast<float2*>(pfb_sm + 2 * T::BUF) + (size_t)w * 2 * p.F;
  float m = 0.f;
  for (int k = 0; set < nsets; ++k, set += gridDim.x) {
    const int slot = k & 1;
    const long long next = set + gridDim.x;
    if (threadIdx.x == 0 && next < nsets) issue(next, slot ^ 1);
    // every thread waits for the slot; a wait that gives up anywhere sends
    // the whole CTA out (after a last bounded wait for its copies in flight)
    const bool ok = __syncthreads_and(mbar_wait_bounded(&bar[slot], (k >> 1) & 1, kBandWaitLimit));
    if (!ok) {
      if (threadIdx.x == 0) {
        if (p.err) atomicExch(p.err, kDevErrTmaTimeout);
        mbar_wait_bounded(&bar[slot], (k >> 1) & 1, kBandWaitLimit);
        if (next < nsets) mbar_wait_bounded(&bar[slot ^ 1], ((k + 1) >> 1) & 1, kBandWaitLimit);
      }
      return;
    }
    const long long q0 = 2 * (set * T::PPC + w);
    const bool v0 = q0 < p.npencils, v1 = q0 + 1 < p.npencils;
    float2* W = slot_buf(slot, w);
    PfBandCtx<L, TR, true> ctx{reinterpret_cast<const TR*>(W), v1, O, W, p.tw, p.k_lo, p.F, ldmul, p.n, 0, 0, p.err};
    fftn_run<L, 1, false, false>(ctx, j0);
    __syncthreads();
    if (v0) m = fmaxf(m, band_split_store<TS>(p, O, q0, v1, j0, S::TPC));
    // the slot and the band bins are rewritten next: order this iteration's
    // shared-memory accesses before the coming bulk copies and transforms
    fence_proxy_async_smem();
    __syncthreads();
  }
  band_amax<L>(p, m);
}

static int band_sm_count() {
  static int sms = 0;
  if (sms == 0) {
    int dev = 0, v = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
    sms = v > 0 ? v : 1;
  }
  return sms;
}

template <int L, class TR, class TS>
static cudaError_t launch_band_one(const PfBandParams& p, cudaStream_t s) {
  using T = PfBandTile<L>;
  const long long pairs = (p.npencils + 1) / 2;
  const long long nsets = (pairs + T::PPC - 1) / T::PPC;
  // staged bulk copies need 16-byte aligned pencils; a pair must fit the
  // transform buffer it is staged in
  const bool staged = (sizeof(float2) * FftShape<L>::SMEM) % 16 == 0 && (reinterpret_cast<uintptr_t>(p.H) & 15) == 0 &&
                      ((size_t)p.n * sizeof(TR)) % 16 == 0 &&
                      2 * (size_t)p.n * sizeof(TR) <= sizeof(float2) * FftShape<L>::SMEM;
  if (staged) {
    auto k = pf_band_staged_kernel<L, TR, TS>;
    const size_t smem = T::smem(p.F, true);
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int per = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k, T::THREADS, smem);
    if (e != cudaSuccess) return e;
    const long long grid = std::min<long long>(nsets, (long long)band_sm_count() * std::max(per, 1));
    k<<<(unsigned)grid, T::THREADS, smem, s>>>(p, nsets);
    return cudaGetLastError();
  }
  auto k = pf_band_kernel<L, TR, TS>;
  const size_t smem = T::smem(p.F, false);
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  k<<<(unsigned)nsets, T::THREADS, smem, s>>>(p);
  return cudaGetLastError();
}

template <class TR, class TS>
static cudaError_t launch_band_typed(const PfBandParams& p, cudaStream_t s) {
  switch (p.L) {
    case 16: return launch_band_one<16, TR, TS>(p, s);
    case 32: return launch_band_one<32, TR, TS>(p, s);
    case 64: return launch_band_one<64, TR, TS>(p, s);
    case 128: return launch_band_one<128, TR, TS>(p, s);
    case 256: return launch_band_one<256, TR, TS>(p, s);
    case 512: return launch_band_one<512, TR, TS>(p, s);
    case 1024: return launch_band_one<1024, TR, TS>(p, s);
    case 2048: return launch_band_one<2048, TR, TS>(p, s);
    case 4096: return launch_band_one<4096, TR, TS>(p, s);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_pf_band(const PfBandParams& p, int storage, cudaStream_t s) {
  if (p.npencils <= 0 || p.F <= 0) return cudaErrorInvalidValue;
  switch (storage) {
    case kF32: return launch_band_typed<float, float2>(p, s);
    case kF16: return launch_band_typed<__half, __half2>(p, s);
    case kBF16: return launch_band_typed<__nv_bfloat16, __nv_bfloat162>(p, s);
    default: return cudaErrorInvalidValue;
  }
}

// ---------------------------------------------------------------------------
// PF1 + PF2 from the shared lateral spectrum (Sec. 4.4 mixture of experts):
// one temporal DFT per stored pencil (kx, ky), kx in [0, Lx/2], writes the
// band of (kx, ky) and, from the mirrored bins, that of (Lx - kx, -ky); the
// rows kx = 0 and kx = Lx/2 are their own partners' rows and store once.
// ---------------------------------------------------------------------------
template <int L>
struct PfSpecCtx {
  static constexpr int SSTRIDE = 1;
  static constexpr bool kSmemInput = false;
  const float2* g;
  float2* P0;                  // band row of (kx, ky)
  float2* P1;                  // band row of the partner, or null
  float2* W;
  const float2* tw;
  const float* w;
  int k_lo, F, n_in;
  bool valid;
  long long g_off, G_n, off0, off1, P_n;   // offsets and extents (bounds-checked build)
  int* err;
  mutable float m = 0.f;       // max |component| of what this thread stored
  __device__ __forceinline__ void load(int l, float2 (&x)[1]) const {
    x[0] = (valid && l < n_in && bchk(g_off + l, G_n, err)) ? __ldg(g + l) : make_float2(0.f, 0.f);
  }
  __device__ __forceinline__ float2* sm(int) const { return W; }
  __device__ __forceinline__ void store(int l, const float2 (&x)[1]) const {
    if (!valid) return;
    int f = l - k_lo;
    float2 v;
    if (f >= 0 && f < F) {
      if (!bchk(off0 + f, P_n, err)) return;
      v = cscale(x[0], __ldg(w + f));
      P0[f] = v;
    } else {
      f = ((L - l) & (L - 1)) - k_lo;
      if (!P1 || f < 0 || f >= F || !bchk(off1 + f, P_n, err)) return;
      v = cscale(cconj(x[0]), __ldg(w + f));
      P1[f] = v;
    }
    m = fmaxf(m, fmaxf(fabsf(v.x), fabsf(v.y)));
  }
};

template <int L>
__global__ void __launch_bounds__(PfBandTile<L>::THREADS)
pf_band_spectrum_kernel(const PfSpecParams p) {
  using S = FftShape<L>;
  constexpr int PPC = PfBandTile<L>::PPC;
  extern __shared__ float2 pfs_sm[];
  const int w = threadIdx.x / S::TPC;
  const int j0 = threadIdx.x % S::TPC;
  const long long np = (long long)(p.Lx / 2 + 1) * p.Ly;
  const long long pid = (long long)blockIdx.x * PPC + w;
  const bool valid = pid < np;
  const long long q = valid ? pid : 0;
  const int kx = (int)(q / p.Ly);
  const int ky = (int)(q % p.Ly);
  const long long o0 = q * p.F;                     // (kx Ly + ky) F
  const long long o1 = ((long long)(p.Lx - kx) * p.Ly + ((p.Ly - ky) & (p.Ly - 1))) * p.F;
  const bool partner = kx > 0 && 2 * kx < p.Lx;
  PfSpecCtx<L> ctx{p.G + q * p.n, p.Phat + o0, partner ? p.Phat + o1 : nullptr, pfs_sm + w * S::SMEM, p.tw, p.w,
                   p.k_lo, p.F, p.n, valid, q * p.n, p.G_n, o0, o1, p.Phat_n, p.err};
  fftn_run<L, 1, false, false>(ctx, j0);
  if (p.amax) {
    constexpr int TH = PfBandTile<L>::THREADS;
    constexpr int WID = TH < 32 ? TH : 32;
    constexpr unsigned MASK = TH < 32 ? ((1u << TH) - 1u) : 0xffffffffu;
    float m = ctx.m;
#pragma unroll
    for (int o = WID / 2; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(MASK, m, o, WID));
    if ((threadIdx.x % WID) == 0) atomicMax(p.amax, __float_as_uint(m));
  }
}

template <int L>
static cudaError_t launch_spec_one(const PfSpecParams& p, cudaStream_t s) {
  using T = PfBandTile<L>;
  auto k = pf_band_spectrum_kernel<L>;
  const size_t smem = sizeof(float2) * T::PPC * FftShape<L>::SMEM;
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  const long long np = (long long)(p.Lx / 2 + 1) * p.Ly;
  const long long blocks = (np + T::PPC - 1) / T::PPC;
  k<<<(unsigned)blocks, T::THREADS, smem, s>>>(p);
  return cudaGetLastError();
}

cudaError_t launch_pf_band_spectrum(const PfSpecParams& p, cudaStream_t s) {
  if (p.F <= 0 || p.n <= 0 || p.n > p.L || p.Lx < 2 || p.Ly < 1 || (p.Ly & (p.Ly - 1)) ||
      p.k_lo < 1 || p.k_lo + p.F > p.L / 2)
    return cudaErrorInvalidValue;
  switch (p.L) {
    case 16: return launch_spec_one<16>(p, s);
    case 32: return launch_spec_one<32>(p, s);
    case 64: return launch_spec_one<64>(p, s);
    case 128: return launch_spec_one<128>(p, s);
    case 256: return launch_spec_one<256>(p, s);
    case 512: return launch_spec_one<512>(p, s);
    case 1024: return launch_spec_one<1024>(p, s);
    case 2048: return launch_spec_one<2048>(p, s);
    case 4096: return launch_spec_one<4096>(p, s);
    default: return cudaErrorInvalidValue;
  }
}

// ---------------------------------------------------------------------------
// PF3: depth sum (Alg. 4 inner loop; Sec. 4.3 propagation sum). One CTA owns a
// chunk of up to 16 pixels that share the radial index pair (i0, i1) and 128
// depths; each thread keeps 16 complex accumulators (one per pixel) for its
// depth, so every radial-kernel sample read from memory feeds 16 pixels. The
// lerp is K0 + alpha (K1 - K0) and the taper multiplies the finished sum.
// Accumulation is float32 whatever the storage type.
// ---------------------------------------------------------------------------
constexpr int kDepthThreads = 64;                 // threads per CTA
constexpr int kDepthPerThread = 2;                // depths per thread (d and d + 64)
constexpr int kDepthBlock = kDepthThreads * kDepthPerThread;

template <class TS, class TK>
__global__ void __launch_bounds__(kDepthThreads)
pf_depth_kernel(const PfDepthParams p) {
  extern __shared__ float4 ps4[];   // [F][kPfChunk / 2] pairs of the chunk's phasors
  __shared__ int pix[kPfChunk];
  __shared__ float sal[kPfChunk], sac[kPfChunk];
  const int ch = blockIdx.x;
  const int d0 = blockIdx.y * kDepthBlock + threadIdx.x;
  if (threadIdx.x < kPfChunk) {
    pix[threadIdx.x] = p.chunk_pix[ch * kPfChunk + threadIdx.x];
    sal[threadIdx.x] = p.chunk_alpha[ch * kPfChunk + threadIdx.x];
    sac[threadIdx.x] = p.chunk_acut[ch * kPfChunk + threadIdx.x];
  }
  __syncthreads();
  const int F = p.F;
  const TS* Ph = static_cast<const TS*>(p.Phat);
  float2* ps = reinterpret_cast<float2*>(ps4);
  for (int idx = threadIdx.x; idx < kPfChunk * F; idx += kDepthThreads) {
    const int q = idx / F, f = idx - q * F;
    const int px = pix[q];
    ps[f * kPfChunk + q] = px >= 0 ? Cpx<TS>::get(Ph + (long long)px * F + f) : make_float2(0.f, 0.f);
  }
  __syncthreads();
  float alpha[kPfChunk];
#pragma unroll
  for (int q = 0; q < kPfChunk; ++q) alpha[q] = sal[q];
  float2 acc[kDepthPerThread][kPfChunk];
#pragma unroll
  for (int e = 0; e < kDepthPerThread; ++e)
#pragma unroll
    for (int q = 0; q < kPfChunk; ++q) acc[e][q] = make_float2(0.f, 0.f);
  const int2 i01 = p.chunk_i01[ch];
  const TK* K = static_cast<const TK*>(p.K);
  const long long row0 = (long long)i01.x * F * p.D, row1 = (long long)i01.y * F * p.D;
  bool dv[kDepthPerThread];
  int dd[kDepthPerThread];
#pragma unroll
  for (int e = 0; e < kDepthPerThread; ++e) {
    dd[e] = d0 + e * kDepthThreads;
    dv[e] = dd[e] < p.D;
  }
#pragma unroll 2
  for (int f = 0; f < F; ++f) {
    float2 k0[kDepthPerThread], dk[kDepthPerThread];
#pragma unroll
    for (int e = 0; e < kDepthPerThread; ++e) {
      const long long o = (long long)f * p.D + (dv[e] ? dd[e] : 0);
      const float2 a = Cpx<TK>::get(K + row0 + o), b = Cpx<TK>::get(K + row1 + o);
      k0[e] = a;
      dk[e] = csub(b, a);
    }
    const float4* pf = ps4 + f * (kPfChunk / 2);
#pragma unroll
    for (int q2 = 0; q2 < kPfChunk / 2; ++q2) {
      const float4 xx = pf[q2];
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int q = 2 * q2 + h;
        const float2 x = h == 0 ? make_float2(xx.x, xx.y) : make_float2(xx.z, xx.w);
#pragma unroll
        for (int e = 0; e < kDepthPerThread; ++e) {
          const float2 kl = make_float2(fmaf(alpha[q], dk[e].x, k0[e].x), fmaf(alpha[q], dk[e].y, k0[e].y));
          acc[e][q].x = fmaf(x.x, kl.x, fmaf(-x.y, kl.y, acc[e][q].x));
          acc[e][q].y = fmaf(x.x, kl.y, fmaf(x.y, kl.x, acc[e][q].y));
        }
      }
    }
  }
  const float sc = p.scale * (p.dev_scale ? *p.dev_scale : 1.0f);
  TS* C = static_cast<TS*>(p.C);
#pragma unroll
  for (int q = 0; q < kPfChunk; ++q) {
    const int px = pix[q];
    if (px < 0) continue;
#pragma unroll
    for (int e = 0; e < kDepthPerThread; ++e)
      if (dv[e]) Cpx<TS>::put(C + (long long)px * p.D + dd[e], cscale(acc[e][q], sac[q] * sc));
  }
}

template <class TS, class TK>
static cudaError_t launch_depth_typed(const PfDepthParams& p, cudaStream_t s) {
  auto k = pf_depth_kernel<TS, TK>;
  const size_t smem = sizeof(float2) * kPfChunk * p.F;
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  dim3 grid((unsigned)p.nchunks, (unsigned)((p.D + kDepthBlock - 1) / kDepthBlock));
  k<<<grid, kDepthThreads, smem, s>>>(p);
  return cudaGetLastError();
}

cudaError_t launch_pf_depth(const PfDepthParams& p, int storage, int kstorage, cudaStream_t s) {
  if (p.nchunks <= 0) return cudaSuccess;
  if (p.F <= 0 || p.D <= 0 || p.D > 65535 * kDepthBlock) return cudaErrorInvalidValue;
  if (storage == kF32 && kstorage == kF32) return launch_depth_typed<float2, float2>(p, s);
  if (storage == kF16 && kstorage == kF16) return launch_depth_typed<__half2, __half2>(p, s);
  if (storage == kBF16 && kstorage == kBF16) return launch_depth_typed<__nv_bfloat162, __nv_bfloat162>(p, s);
  if (storage == kF16 && kstorage == kF32) return launch_depth_typed<__half2, float2>(p, s);
  if (storage == kBF16 && kstorage == kF32) return launch_depth_typed<__nv_bfloat162, float2>(p, s);
  return cudaErrorInvalidValue;
}

// ---------------------------------------------------------------------------
// Plan-time radial kernel (Eqs. 4-6) in float64.
// ---------------------------------------------------------------------------
__global__ void kr_phase_kernel(const KrBuildParams p) {
  const long long total = (long long)p.n_r * p.F * p.D;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
       idx += (long long)gridDim.x * blockDim.x) {
    const int dd = (int)(idx % p.D);
    const long long rest = idx / p.D;
    const int f = (int)(rest % p.F);
    const int j = (int)(rest / p.F);
    const double r = p.r[j], z = p.depth[dd];
    const double ph = p.sigma_s * p.kappa[f] * sqrt(r * r + z * z);
    double sn, cs;
    sincos(ph, &sn, &cs);
    p.A[idx] = make_double2(cs, sn);
  }
}

// K64[i][fd] = mod(f, d) * sum_j B[i][j] A[j][fd]; 64 x 64 output tile per
// CTA, 4 x 4 per thread.
__global__ void __launch_bounds__(256) kr_gemm_kernel(const KrBuildParams p) {
  __shared__ double Bs[16][64];
  __shared__ double2 As[16][64];
  const int NFD = p.F * p.D;
  const int i_base = blockIdx.y * 64, fd_base = blockIdx.x * 64;
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  double2 acc[4][4];
#pragma unroll
  for (int u = 0; u < 4; ++u)
#pragma unroll
    for (int v = 0; v < 4; ++v) acc[u][v] = make_double2(0.0, 0.0);
  for (int j0 = 0; j0 < p.n_r; j0 += 16) {
    for (int e = threadIdx.x; e < 16 * 64; e += 256) {
      const int jj = e / 64, q = e % 64;
      const int i = i_base + q, j = j0 + jj, fd = fd_base + q;
      Bs[jj][q] = (i < p.n_rho && j < p.n_r) ? p.B[(long long)i * p.n_r + j] : 0.0;
      As[jj][q] = (fd < NFD && j < p.n_r) ? p.A[(long long)j * NFD + fd] : make_double2(0.0, 0.0);
    }
    __syncthreads();
#pragma unroll 4
    for (int jj = 0; jj < 16; ++jj) {
      double bv[4];
      double2 av[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) bv[u] = Bs[jj][ty + 16 * u];
#pragma unroll
      for (int v = 0; v < 4; ++v) av[v] = As[jj][tx + 16 * v];
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) {
          acc[u][v].x = fma(bv[u], av[v].x, acc[u][v].x);
          acc[u][v].y = fma(bv[u], av[v].y, acc[u][v].y);
        }
    }
    __syncthreads();
  }
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const int i = i_base + ty + 16 * u;
    if (i >= p.n_rho) continue;
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      const int fd = fd_base + tx + 16 * v;
      if (fd >= NFD) continue;
      const int f = fd / p.D, dd = fd % p.D;
      const double ph = p.kappa[f] * (p.sigma_t * p.depth[dd] + p.delta);
      double sn, cs;
      sincos(ph, &sn, &cs);
      const double2 a = acc[u][v];
      p.K64[(long long)i * NFD + fd] = make_double2(a.x * cs - a.y * sn, a.x * sn + a.y * cs);
    }
  }
}

cudaError_t launch_kr_build(const KrBuildParams& p, cudaStream_t s) {
  kr_phase_kernel<<<1024, 256, 0, s>>>(p);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const int NFD = p.F * p.D;
  dim3 grid((unsigned)((NFD + 63) / 64), (unsigned)((p.n_rho + 63) / 64));
  kr_gemm_kernel<<<grid, 256, 0, s>>>(p);
  return cudaGetLastError();
}

template <class TK>
__global__ void kr_store_kernel(const double2* K64, TK* K, long long count, double scale) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < count;
       i += (long long)gridDim.x * blockDim.x) {
    const double2 v = K64[i];
    Cpx<TK>::put(K + i, make_float2((float)(v.x * scale), (float)(v.y * scale)));
  }
}

cudaError_t launch_kr_store(const double2* K64, void* K, long long count, int storage, double scale,
                            cudaStream_t s) {
  switch (storage) {
    case kF32: kr_store_kernel<float2><<<1024, 256, 0, s>>>(K64, static_cast<float2*>(K), count, scale); break;
    case kF16: kr_store_kernel<__half2><<<1024, 256, 0, s>>>(K64, static_cast<__half2*>(K), count, scale); break;
    case kBF16:
      kr_store_kernel<__nv_bfloat162><<<1024, 256, 0, s>>>(K64, static_cast<__nv_bfloat162*>(K), count, scale);
      break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Per-volume scale for reduced-precision storage (two-stage, deterministic).
// ---------------------------------------------------------------------------
// eight consecutive elements per thread and iteration (n is a multiple of 8,
// so they share one pencil and their ramp is t0 .. t0 + 7), read as one
// 16-byte vector (two for float) when the array is 16-byte aligned; the ramp
// index advances by the grid stride modulo n instead of a division per step
template <class TR> struct Eight;
template <> struct Eight<float> {
  static __device__ __forceinline__ void get(const float* p, bool vec, float (&v)[8]) {
    if (vec) {
      const float4 a = reinterpret_cast<const float4*>(p)[0], b = reinterpret_cast<const float4*>(p)[1];
      v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w; v[4] = b.x; v[5] = b.y; v[6] = b.z; v[7] = b.w;
    } else {
#pragma unroll
      for (int k = 0; k < 8; ++k) v[k] = p[k];
    }
  }
};
template <class T2, class TR> struct EightHalf {
  static __device__ __forceinline__ void get(const TR* p, bool vec, float (&v)[8]) {
    if (vec) {
      const uint4 u = reinterpret_cast<const uint4*>(p)[0];
      const T2* h = reinterpret_cast<const T2*>(&u);
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const float2 f = Cpx<T2>::get(h + k);
        v[2 * k] = f.x;
        v[2 * k + 1] = f.y;
      }
    } else {
#pragma unroll
      for (int k = 0; k < 8; ++k) v[k] = Real<TR>::get(p + k);
    }
  }
};
template <> struct Eight<__half> : EightHalf<__half2, __half> {};
template <> struct Eight<__nv_bfloat16> : EightHalf<__nv_bfloat162, __nv_bfloat16> {};

// The last CTA to finish (a counter in the partials' array, reset by that
// CTA) sums the partials in index order and writes the scale, its inverse
// and the inverse square: the result does not depend on CTA timing.
template <class TR>
__global__ void sumsq_partial_kernel(const TR* H, long long count, int n, float t_scale, bool vec, float* partial,
                                     unsigned* counter, float target, float* out) {
  __shared__ float red[256];
  __shared__ double dred[256];
  __shared__ bool last;
  float acc = 0.f;
  const long long chunks = count / 8;
  const long long q0 = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const long long stride = (long long)gridDim.x * blockDim.x;
  int t0 = (int)((q0 * 8) % n);
  const int step = (int)((stride * 8) % n);
  constexpr int U = 4;                       // independent loads in flight per thread
  long long q = q0;
  for (; q + (U - 1) * stride < chunks; q += U * stride) {
    float v[U][8];
#pragma unroll
    for (int u = 0; u < U; ++u) Eight<TR>::get(H + (q + u * stride) * 8, vec, v[u]);
#pragma unroll
    for (int u = 0; u < U; ++u) {
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        const float x = t_scale != 0.f ? v[u][k] * ((float)(t0 + k) * t_scale) : v[u][k];
        acc = fmaf(x, x, acc);
      }
      t0 += step;
      if (t0 >= n) t0 -= n;
    }
  }
  for (; q < chunks; q += stride) {
    float v[8];
    Eight<TR>::get(H + q * 8, vec, v);
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      const float x = t_scale != 0.f ? v[k] * ((float)(t0 + k) * t_scale) : v[k];
      acc = fmaf(x, x, acc);
    }
    t0 += step;
    if (t0 >= n) t0 -= n;
  }
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int sft = 128; sft > 0; sft >>= 1) {
    if (threadIdx.x < sft) red[threadIdx.x] += red[threadIdx.x + sft];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    partial[blockIdx.x] = red[0];
    __threadfence();
    last = atomicAdd(counter, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  double dacc = 0.0;
  for (int i = threadIdx.x; i < (int)gridDim.x; i += blockDim.x) dacc += ((volatile float*)partial)[i];
  dred[threadIdx.x] = dacc;
  __syncthreads();
  for (int sft = 128; sft > 0; sft >>= 1) {
    if (threadIdx.x < sft) dred[threadIdx.x] += dred[threadIdx.x + sft];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const double nrm = sqrt(dred[0]);
    const float sc = nrm > 0.0 ? (float)(target / nrm) : 1.0f;
    out[0] = sc;
    out[1] = 1.0f / sc;
    out[2] = (float)(1.0 / ((double)sc * (double)sc));
  }
}

cudaError_t launch_volume_scale(const void* H, long long count, int n, float t_scale, int storage,
                                float target, float* partial, int npartial, float* out, cudaStream_t s) {
  // four CTAs per SM (enough bytes in flight with 16-byte loads); the count
  // of partials only changes the summation tree, not determinism. The last
  // partial slot holds the CTAs' completion counter.
  int blocks = npartial - 1 < 152 * 4 ? npartial - 1 : 152 * 4;
  if (blocks < 1) return cudaErrorInvalidValue;
  unsigned* counter = reinterpret_cast<unsigned*>(partial + npartial - 1);
  // a caller's workspace may hold anything there on its first use
  cudaError_t e0 = cudaMemsetAsync(counter, 0, sizeof(unsigned), s);
  if (e0 != cudaSuccess) return e0;
  const bool vec = (reinterpret_cast<uintptr_t>(H) & 15) == 0;
  switch (storage) {
    case kF32:
      sumsq_partial_kernel<float><<<blocks, 256, 0, s>>>(static_cast<const float*>(H), count, n, t_scale, vec, partial,
                                                         counter, target, out);
      break;
    case kF16:
      sumsq_partial_kernel<__half><<<blocks, 256, 0, s>>>(static_cast<const __half*>(H), count, n, t_scale, vec,
                                                          partial, counter, target, out);
      break;
    case kBF16:
      sumsq_partial_kernel<__nv_bfloat16><<<blocks, 256, 0, s>>>(static_cast<const __nv_bfloat16*>(H), count, n,
                                                                 t_scale, vec, partial, counter, target, out);
      break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Dense phasor-field method (Alg. 3): the propagation kernel of every
// (frequency, depth) pair stored in Fourier form over the padded grid. The
// spatial kernel is generated here with its phase in float64 (the phase runs
// to hundreds of radians), then transformed by the axis FFTs at plan time.
// ---------------------------------------------------------------------------
__global__ void dense_gen_kernel(const DenseGenParams p) {
  const long long FD = (long long)p.F * p.D;
  const long long total = (long long)p.Nu * p.Nv * FD;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const int dd = (int)(i % p.D);
    const int f = (int)((i / p.D) % p.F);
    const long long pix = i / FD;
    const int x = (int)(pix / p.Nv), y = (int)(pix % p.Nv);
    const double sx = (x < p.Nu / 2 ? x : x - p.Nu) * p.dx;
    const double sy = (y < p.Nv / 2 ? y : y - p.Nv) * p.dy;
    const double z = p.depth[dd];
    const double R = sqrt(sx * sx + sy * sy + z * z);
    double sn, cs;
    sincos(p.kappa[f] * (p.sigma_s * R + p.sigma_t * z + p.delta), &sn, &cs);
    p.k[i] = make_float2((float)cs, (float)sn);
  }
}

cudaError_t launch_dense_gen(const DenseGenParams& p, cudaStream_t s) {
  dense_gen_kernel<<<152 * 16, 256, 0, s>>>(p);
  return cudaGetLastError();
}

// One CTA per padded pixel, threads over depths; the pixel's F phasors sit in
// shared memory and each thread streams its column of the kernel (read once,
// evict first), four frequencies in flight.
__global__ void __launch_bounds__(128) pf_dense_kernel(const PfDenseParams p) {
  extern __shared__ float2 ph_sm[];
  const long long pix = blockIdx.x;
  for (int f = threadIdx.x; f < p.F; f += blockDim.x) ph_sm[f] = p.Phat[pix * p.F + f];
  __syncthreads();
  const float2* K = p.K + pix * p.F * (long long)p.D;
  for (int d = threadIdx.x; d < p.D; d += blockDim.x) {
    float2 acc = make_float2(0.f, 0.f);
    int f = 0;
    for (; f + 4 <= p.F; f += 4) {
      float2 k[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) k[u] = __ldcs(K + (long long)(f + u) * p.D + d);
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const float2 x = ph_sm[f + u];
        acc.x = fmaf(x.x, k[u].x, fmaf(-x.y, k[u].y, acc.x));
        acc.y = fmaf(x.x, k[u].y, fmaf(x.y, k[u].x, acc.y));
      }
    }
    for (; f < p.F; ++f) {
      const float2 k = __ldcs(K + (long long)f * p.D + d), x = ph_sm[f];
      acc.x = fmaf(x.x, k.x, fmaf(-x.y, k.y, acc.x));
      acc.y = fmaf(x.x, k.y, fmaf(x.y, k.x, acc.y));
    }
    p.C[pix * p.D + d] = acc;
  }
}

// max |x| of a float array: grid-stride 16-byte loads when the array is
// 16-byte aligned (a scalar tail covers the rest), warp maximum, one atomicMax
// of the float bits per warp (bits of non-negative floats order like the values)
__global__ void absmax_kernel(const float* x, long long count, bool aligned, unsigned* out) {
  float m = 0.f;
  const long long n4 = aligned ? count / 4 : 0;
  const long long stride = (long long)gridDim.x * blockDim.x;
  const float4* x4 = reinterpret_cast<const float4*>(x);
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n4; i += stride) {
    const float4 v = x4[i];
    m = fmaxf(m, fmaxf(fmaxf(fabsf(v.x), fabsf(v.y)), fmaxf(fabsf(v.z), fabsf(v.w))));
  }
  for (long long i = 4 * n4 + blockIdx.x * (long long)blockDim.x + threadIdx.x; i < count; i += stride)
    m = fmaxf(m, fabsf(x[i]));
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) atomicMax(out, __float_as_uint(m));
}

cudaError_t launch_absmax(const float* x, long long count, unsigned* out, cudaStream_t s) {
  if (count <= 0) return cudaSuccess;
  const long long blocks = (count / 4 + 255) / 256;
  const bool aligned = (reinterpret_cast<uintptr_t>(x) & 15) == 0;
  absmax_kernel<<<(unsigned)(blocks < 152 * 4 ? (blocks < 1 ? 1 : blocks) : 152 * 4), 256, 0, s>>>(x, count, aligned,
                                                                                                   out);
  return cudaGetLastError();
}


// one warp per listed row (first list, then second): 4-byte stores across the lanes
__global__ void clear_rows2_kernel(unsigned* C, const int* l1, long long n1, const int* l2, long long n2,
                                   long long row_words) {
  const long long w = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (w >= n1 + n2) return;
  const int pix = w < n1 ? l1[w] : l2[w - n1];
  if (pix < 0) return;
  unsigned* row = C + (long long)pix * row_words;
  for (long long i = lane; i < row_words; i += 32) row[i] = 0u;
}

cudaError_t launch_clear_rows2(void* C, const int* l1, long long n1, const int* l2, long long n2, size_t row_bytes,
                               cudaStream_t s) {
  if (n1 < 0 || n2 < 0) return cudaErrorInvalidValue;
  if (n1 + n2 == 0) return cudaSuccess;
  if (!C || (n1 && !l1) || (n2 && !l2) || row_bytes % 4) return cudaErrorInvalidValue;
  const long long threads = (n1 + n2) * 32;
  clear_rows2_kernel<<<(unsigned)((threads + 255) / 256), 256, 0, s>>>(static_cast<unsigned*>(C), l1, n1, l2, n2,
                                                                      (long long)(row_bytes / 4));
  return cudaGetLastError();
}

cudaError_t launch_clear_rows(void* C, const int* list, long long n, size_t row_bytes, cudaStream_t s) {
  return launch_clear_rows2(C, list, n, nullptr, 0, row_bytes, s);
}

cudaError_t launch_pf_dense(const PfDenseParams& p, cudaStream_t s) {
  if (p.npix <= 0 || p.F <= 0 || p.D <= 0) return cudaErrorInvalidValue;
  const int threads = p.D <= 64 ? 64 : 128;
  const size_t smem = sizeof(float2) * p.F;
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(pf_dense_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  pf_dense_kernel<<<(unsigned)p.npix, threads, smem, s>>>(p);
  return cudaGetLastError();
}

}  // namespace nlos
