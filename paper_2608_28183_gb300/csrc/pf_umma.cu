// Phasor-field depth sum on the 5th-generation tensor cores (Eq. 7, Alg. 4,
// 16-bit storage). Pixels that share the radial pair (i0, i1) form tiles of
// up to 128 rows; for one tile the sum over the band frequencies of
// Phat * lerp(K_r[i0], K_r[i1], alpha) is two real matrix products with a
// shared accumulator:
//
//   Y = A0 B0^T + A1 B1^T,  A0 = (1 - alpha) Phat,  A1 = alpha Phat,
//
// with the complex phasors as interleaved (Re, Im) columns of A and B the real
// form of K_r[i0] / K_r[i1] interleaved to match (a Re output row holds
// (Kr, -Ki) per frequency, an Im output row (Ki, Kr)), so Y's first Db
// columns are Re C and the next Db are Im C for a block of Db depths. A row of
// A is a scaled copy of a phasor row, built in shared memory; B arrives by 1D
// bulk copies in the operand layout the plan stored; kind::f16 MMAs
// (M = 128, N = 2 Db, K = 16) accumulate in tensor memory; warps read the
// accumulator back (warp w owns rows 32 (w % 4) .. + 31) to apply the taper
// and scale. Inputs are f16 with their per-volume and per-pass scales, the
// accumulator is f32.
//
// Two schedules:
//  * pf_umma_ws_kernel: one persistent CTA per SM, warp-specialised - a
//    producer warp keeps kStages operand stages in flight, four warps build A
//    and run the epilogue, one thread issues the MMAs - with two accumulators
//    so a tile's epilogue overlaps the next tile's MMAs;
//  * pf_umma_kernel: one CTA per tile, one stage.
#include <cuda_fp16.h>

#include "nlos_internal.h"
#include "nlos_umma.cuh"

namespace nlos {

namespace {

constexpr int kWaitLimit = 1 << 26;                    // probes of a barrier (a few hundred ms)
constexpr int kQ = kUmmaKChunk / 2;                    // frequencies per chunk
constexpr uint32_t kSbo = (kUmmaKChunk / 8) * 128;     // row-group stride of a chunk operand

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// A chunk kc of a tile: element (row r, frequency f = kc * kQ + q) of
// (1 - alpha_r) Phat / alpha_r Phat as the column pair (2q, 2q + 1). A warp
// instruction covers 8 rows x 4 consecutive q: the 32 lanes hit 32 distinct
// shared-memory banks and read 8 runs of 16 bytes of the phasor rows. NT
// threads (a multiple of 32) share the chunk.
template <int NT>
struct AChunk {
  static constexpr int kBlocks = (kUmmaTile / 8) * (kQ / 4);
  static constexpr int kIters = kBlocks / (NT / 32);
  __device__ static __forceinline__ void coords(int i, int t, int& r, int& q) {
    const int T = i * (NT / 32) + (t >> 5);
    r = (T / (kQ / 4)) * 8 + (t & 7);
    q = (T % (kQ / 4)) * 4 + ((t & 31) >> 3);
  }
  __device__ static __forceinline__ void load(__half2 (&h)[kIters], const __half2* Phat, int F, const int* spix,
                                              int kc, int t) {
#pragma unroll
    for (int i = 0; i < kIters; ++i) {
      int r, q;
      coords(i, t, r, q);
      const int f = kc * kQ + q;
      const int pix = spix[r];
      h[i] = (pix >= 0 && f < F) ? Phat[(size_t)pix * F + f] : __floats2half2_rn(0.f, 0.f);
    }
  }
  __device__ static __forceinline__ void store(unsigned char* A0, unsigned char* A1, const __half2 (&h)[kIters],
                                               const float* salpha, int t) {
#pragma unroll
    for (int i = 0; i < kIters; ++i) {
      int r, q;
      coords(i, t, r, q);
      const uint32_t off = umma_kmajor_offset(r, 2 * q, kUmmaKChunk);
      const float2 v = __half22float2(h[i]);
      const float al = salpha[r], w0 = 1.f - al;
      *reinterpret_cast<__half2*>(A0 + off) = __floats2half2_rn(w0 * v.x, w0 * v.y);
      *reinterpret_cast<__half2*>(A1 + off) = __floats2half2_rn(al * v.x, al * v.y);
    }
  }
};

// MMAs of one chunk into accumulator `acc` (first: the chunk starts the sum)
__device__ __forceinline__ void mma_chunk(uint32_t acc, uint32_t idesc, const unsigned char* A0,
                                          const unsigned char* A1, const unsigned char* B0, const unsigned char* B1,
                                          bool first) {
#pragma unroll
  for (int kk = 0; kk < kUmmaKChunk / 16; ++kk) {
    const uint32_t ko = kk * 256;     // two 8-column core matrices per K = 16 slab
    umma_f16(acc, umma_smem_desc(smem_u32(A0) + ko, 128, kSbo), umma_smem_desc(smem_u32(B0) + ko, 128, kSbo), idesc,
             (first && kk == 0) ? 0u : 1u);
    umma_f16(acc, umma_smem_desc(smem_u32(A1) + ko, 128, kSbo), umma_smem_desc(smem_u32(B1) + ko, 128, kSbo), idesc,
             1u);
  }
}

// accumulator rows of one warp -> C (taper and scale), columns [c0, c0 + ncols)
template <int Db>
__device__ __forceinline__ void epilogue_cols(uint32_t acc, int warp, int pix, float gsc, __half2* crow, int blk,
                                              int D, int c0, int ncols) {
  const uint32_t lane_base = acc + ((uint32_t)(32 * (warp & 3)) << 16);
  for (int c = c0; c < c0 + ncols; c += 16) {
    uint32_t re[16], im[16];
    tmem_ld16(lane_base + (uint32_t)c, re);
    tmem_ld16(lane_base + (uint32_t)(Db + c), im);
    tmem_wait_ld();
    if (pix >= 0) {
      __half2 o[16];
#pragma unroll
      for (int q = 0; q < 16; ++q) o[q] = __floats2half2_rn(gsc * __uint_as_float(re[q]), gsc * __uint_as_float(im[q]));
      if (blk * Db + c + 16 <= D && (reinterpret_cast<uintptr_t>(crow + c) & 15) == 0) {
        uint4* dst = reinterpret_cast<uint4*>(crow + c);          // 16-byte stores: 4 depths each
#pragma unroll
        for (int v = 0; v < 4; ++v) dst[v] = reinterpret_cast<const uint4*>(o)[v];
      } else {
#pragma unroll
        for (int q = 0; q < 16; ++q)
          if (blk * Db + c + q < D) crow[c + q] = o[q];
      }
    }
  }
}

template <int Db>
struct Sizes {
  static constexpr int N = 2 * Db;
  static constexpr uint32_t A_BYTES = kUmmaTile * kUmmaKChunk * 2;   // one A operand chunk
  static constexpr uint32_t B_BYTES = N * kUmmaKChunk * 2;           // one B operand chunk
  static constexpr uint32_t STAGE = 2 * A_BYTES + 2 * B_BYTES;        // A0 A1 B0 B1
  static constexpr uint32_t ACC_COLS = N <= 32 ? 32 : N <= 64 ? 64 : N <= 128 ? 128 : 256;
};

// ---------------------------------------------------------------------------
// Warp-specialised persistent schedule
// ---------------------------------------------------------------------------
constexpr int kStages = 4;
constexpr int kWsBuilders = 256;                 // warps 0-7: A build, epilogue
constexpr int kWsThreads = kWsBuilders + 64;     // warp 8: producer, warp 9: MMA issue
constexpr int kProducerWarp = kWsBuilders / 32, kMmaWarp = kProducerWarp + 1;

template <int Db>
__global__ void __launch_bounds__(kWsThreads, 1) pf_umma_ws_kernel(const PfUmmaParams p) {
  using S = Sizes<Db>;
  using A = AChunk<kWsBuilders>;
  extern __shared__ __align__(128) unsigned char ws_sm[];
  __shared__ uint64_t full_b[kStages], full_a[kStages], empty[kStages], acc_full[2], acc_empty[2];
  __shared__ uint32_t tbase;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  auto A0 = [&](int s) { return ws_sm + s * S::STAGE; };
  auto A1 = [&](int s) { return ws_sm + s * S::STAGE + S::A_BYTES; };
  auto B0 = [&](int s) { return ws_sm + s * S::STAGE + 2 * S::A_BYTES; };
  auto B1 = [&](int s) { return ws_sm + s * S::STAGE + 2 * S::A_BYTES + S::B_BYTES; };
  if (warp == kMmaWarp) tmem_alloc(&tbase, 2 * S::ACC_COLS);
  if (tid == 0) {
    for (int s = 0; s < kStages; ++s) {
      mbar_init(&full_b[s], 1);
      mbar_init(&full_a[s], kWsBuilders);
      mbar_init(&empty[s], 1);
    }
    for (int a = 0; a < 2; ++a) {
      mbar_init(&acc_full[a], 1);
      mbar_init(&acc_empty[a], kWsBuilders);
    }
    mbar_fence_init();
  }
  tc_fence_before_sync();
  __syncthreads();
  tc_fence_after_sync();
  const uint32_t tm = tbase;
  const int ntiles_mine = (p.ntiles - (int)blockIdx.x + (int)gridDim.x - 1) / (int)gridDim.x;
  const int U = ntiles_mine * p.nblk;           // units: (tile, depth block)
  const int G = U * p.KC;                       // chunks
  auto unit_tile = [&](int u) { return (int)blockIdx.x + (u / p.nblk) * (int)gridDim.x; };
  int err = 0;

  if (warp == kProducerWarp) {
    // producer: B operand stages, up to kStages chunks ahead of the MMAs
    if (lane == 0) {
      const size_t blk_bytes = (size_t)p.KC * S::B_BYTES;
      const unsigned char* Bg = static_cast<const unsigned char*>(p.B);
      for (int g = 0; g < G && !err; ++g) {
        const int s = g % kStages, r = g / kStages, u = g / p.KC, kc = g % p.KC;
        if (r >= 1 && !mbar_spin_bounded(&empty[s], (r - 1) & 1, kWaitLimit)) {
          err = 1;
          break;
        }
        const int tl = unit_tile(u), blk = u % p.nblk;
        const int2 i01 = p.tile_i01[tl];
        mbar_arrive_expect_tx(&full_b[s], 2 * S::B_BYTES);
        bulk_load(B0(s), Bg + ((size_t)i01.x * p.nblk + blk) * blk_bytes + (size_t)kc * S::B_BYTES, S::B_BYTES,
                  &full_b[s]);
        bulk_load(B1(s), Bg + ((size_t)i01.y * p.nblk + blk) * blk_bytes + (size_t)kc * S::B_BYTES, S::B_BYTES,
                  &full_b[s]);
      }
    }
  } else if (warp == kMmaWarp) {
    // MMA issue
    if (lane == 0) {
      const uint32_t idesc = umma_idesc_f16<false>(kUmmaTile, S::N);
      for (int g = 0; g < G && !err; ++g) {
        const int s = g % kStages, r = g / kStages, u = g / p.KC, kc = g % p.KC;
        const int a = u & 1;
        if (kc == 0 && u >= 2 && !mbar_spin_bounded(&acc_empty[a], ((u - 2) >> 1) & 1, kWaitLimit)) err = 1;
        if (!err && !mbar_spin_bounded(&full_b[s], r & 1, kWaitLimit)) err = 1;
        if (!err && !mbar_spin_bounded(&full_a[s], r & 1, kWaitLimit)) err = 1;
        if (err) break;
        tc_fence_after_sync();
        mma_chunk(tm + (uint32_t)(a * S::ACC_COLS), idesc, A0(s), A1(s), B0(s), B1(s), kc == 0);
        umma_commit(&empty[s]);
        if (kc == p.KC - 1) umma_commit(&acc_full[a]);
      }
    }
  } else {
    // builders: A stages, then the epilogue of the previous unit
    const int t = tid;
    const __half2* Ph = static_cast<const __half2*>(p.Phat);
    auto epilogue = [&](int u) {
      const int a = u & 1, tl = unit_tile(u), blk = u % p.nblk;
      if (!mbar_spin_bounded(&acc_full[a], (u >> 1) & 1, kWaitLimit)) err = 1;
      tc_fence_after_sync();
      // warps w and w + 4 own the rows of lane quarter w % 4 and split the depths
      const int row = t & (kUmmaTile - 1), half = t >> 7;
      const int pix = p.tile_pix[(size_t)tl * kUmmaTile + row];
      const float ac = p.tile_acut[(size_t)tl * kUmmaTile + row];
      __half2* crow = static_cast<__half2*>(p.C) + (size_t)(pix >= 0 ? pix : 0) * p.D + (size_t)blk * Db;
      const uint32_t acc = tm + (uint32_t)(a * S::ACC_COLS);
      if (!err) {
        if (Db >= 32) epilogue_cols<Db>(acc, warp, pix, p.scale * ac, crow, blk, p.D, half * (Db / 2), Db / 2);
        else if (half == 0) epilogue_cols<Db>(acc, warp, pix, p.scale * ac, crow, blk, p.D, 0, Db);
      }
      tc_fence_before_sync();
      mbar_arrive(&acc_empty[a]);
    };
    // a builder touches kIters rows: their pixel and weight are held in
    // registers per tile, and the next chunk's phasors are loaded before the
    // current chunk is stored
    int rp[A::kIters];
    float ra[A::kIters];
    auto load_rows = [&](int u) {
      const int tl = unit_tile(u);
#pragma unroll
      for (int i = 0; i < A::kIters; ++i) {
        int r, q;
        A::coords(i, t, r, q);
        rp[i] = p.tile_pix[(size_t)tl * kUmmaTile + r];
        ra[i] = p.tile_alpha[(size_t)tl * kUmmaTile + r];
      }
    };
    auto load_h = [&](__half2 (&h)[A::kIters], int kc) {
#pragma unroll
      for (int i = 0; i < A::kIters; ++i) {
        int r, q;
        A::coords(i, t, r, q);
        const int f = kc * kQ + q;
        h[i] = (rp[i] >= 0 && f < p.F) ? Ph[(size_t)rp[i] * p.F + f] : __floats2half2_rn(0.f, 0.f);
      }
    };
    __half2 hc[A::kIters], hn[A::kIters];
    if (U > 0) {
      load_rows(0);
      load_h(hc, 0);
    }
    for (int u = 0; u < U && !err; ++u) {
      for (int kc = 0; kc < p.KC; ++kc) {
        const int g = u * p.KC + kc;
        const int s = g % kStages, r = g / kStages;
        const bool next_unit = kc + 1 == p.KC;
        if (r >= 1 && !mbar_spin_bounded(&empty[s], (r - 1) & 1, kWaitLimit)) {
          err = 1;
          break;
        }
#pragma unroll
        for (int i = 0; i < A::kIters; ++i) {
          int rr, q;
          A::coords(i, t, rr, q);
          const uint32_t off = umma_kmajor_offset(rr, 2 * q, kUmmaKChunk);
          const float2 v = __half22float2(hc[i]);
          const float w0 = 1.f - ra[i];
          *reinterpret_cast<__half2*>(A0(s) + off) = __floats2half2_rn(w0 * v.x, w0 * v.y);
          *reinterpret_cast<__half2*>(A1(s) + off) = __floats2half2_rn(ra[i] * v.x, ra[i] * v.y);
        }
        fence_proxy_async_smem();
        mbar_arrive(&full_a[s]);
        // next chunk (of this unit or the next one) in flight
        if (!next_unit) {
          load_h(hn, kc + 1);
        } else if (u + 1 < U) {
          load_rows(u + 1);
          load_h(hn, 0);
        }
#pragma unroll
        for (int i = 0; i < A::kIters; ++i) hc[i] = hn[i];
      }
      if (err) break;
      if (u >= 1) epilogue(u - 1);
    }
    if (U >= 1 && !err) epilogue(U - 1);
  }
  if (err && p.err) atomicExch(p.err, kDevErrTmaTimeout);
  // on success every MMA has completed once the builders saw the last
  // accumulator full; on a timeout the waits above have given up
  tc_fence_before_sync();
  __syncthreads();
  if (warp == kMmaWarp) tmem_dealloc(tm, 2 * S::ACC_COLS);
}

// ---------------------------------------------------------------------------
// One CTA per tile, one stage
// ---------------------------------------------------------------------------
constexpr int kThreads = 256;

template <int Db>
__global__ void __launch_bounds__(kThreads) pf_umma_kernel(const PfUmmaParams p) {
  using S = Sizes<Db>;
  using A = AChunk<kThreads>;
  extern __shared__ __align__(128) unsigned char um_sm[];
  __shared__ uint64_t bar_load, bar_mma;
  __shared__ uint32_t tbase;
  __shared__ int spix[kUmmaTile];
  __shared__ float salpha[kUmmaTile];
  unsigned char* A0 = um_sm;
  unsigned char* A1 = um_sm + S::A_BYTES;
  unsigned char* B0 = um_sm + 2 * S::A_BYTES;
  unsigned char* B1 = B0 + S::B_BYTES;
  const int tid = threadIdx.x, warp = tid >> 5;
  const int row = tid & (kUmmaTile - 1), half = tid >> 7;
  const int tile = blockIdx.x;
  const int2 i01 = p.tile_i01[tile];
  const int pix = p.tile_pix[(size_t)tile * kUmmaTile + row];
  const float ac = p.tile_acut[(size_t)tile * kUmmaTile + row];
  if (tid < kUmmaTile) {
    spix[tid] = p.tile_pix[(size_t)tile * kUmmaTile + tid];
    salpha[tid] = p.tile_alpha[(size_t)tile * kUmmaTile + tid];
  }
  const __half2* Ph = static_cast<const __half2*>(p.Phat);
  if (warp == 0) tmem_alloc(&tbase, S::ACC_COLS);
  if (tid == 0) {
    mbar_init(&bar_load, 1);
    mbar_init(&bar_mma, 1);
    mbar_fence_init();
  }
  tc_fence_before_sync();
  __syncthreads();
  tc_fence_after_sync();
  __half2 hcur[A::kIters], hnext[A::kIters];
  A::load(hcur, Ph, p.F, spix, 0, tid);
  const uint32_t dt = tbase;
  const uint32_t idesc = umma_idesc_f16<false>(kUmmaTile, S::N);
  const size_t blk_bytes = (size_t)p.KC * S::B_BYTES;
  const unsigned char* Bg = static_cast<const unsigned char*>(p.B);
  int phase = 0;
  bool ok = true;
  for (int blk = 0; blk < p.nblk && ok; ++blk) {
    const unsigned char* b0g = Bg + ((size_t)i01.x * p.nblk + blk) * blk_bytes;
    const unsigned char* b1g = Bg + ((size_t)i01.y * p.nblk + blk) * blk_bytes;
    for (int kc = 0; kc < p.KC; ++kc) {
      if (tid == 0) {
        fence_proxy_async_smem();
        mbar_arrive_expect_tx(&bar_load, 2 * S::B_BYTES);
        bulk_load(B0, b0g + (size_t)kc * S::B_BYTES, S::B_BYTES, &bar_load);
        bulk_load(B1, b1g + (size_t)kc * S::B_BYTES, S::B_BYTES, &bar_load);
      }
      A::store(A0, A1, hcur, salpha, tid);
      // the next chunk's phasors are in flight while this chunk's MMAs run
      A::load(hnext, Ph, p.F, spix, kc + 1 < p.KC ? kc + 1 : 0, tid);
      fence_proxy_async_smem();
      __syncthreads();
      if (tid == 0) {
        ok = mbar_spin_bounded(&bar_load, phase, kWaitLimit);
        tc_fence_after_sync();
        if (ok) mma_chunk(dt, idesc, A0, A1, B0, B1, kc == 0);
        umma_commit(&bar_mma);
      }
      // the MMAs read A and B; they finish before the next chunk overwrites them
      const bool done = mbar_spin_bounded(&bar_mma, phase, kWaitLimit);
      ok = __syncthreads_and(ok && done ? 1 : 0) != 0;
      phase ^= 1;
#pragma unroll
      for (int i = 0; i < A::kIters; ++i) hcur[i] = hnext[i];
      if (!ok) break;
    }
    if (!ok) break;
    // epilogue: warps w and w + 4 share the rows of lane quarter w % 4
    tc_fence_after_sync();
    __half2* crow = static_cast<__half2*>(p.C) + (size_t)(pix >= 0 ? pix : 0) * p.D + (size_t)blk * Db;
    if (Db >= 32) epilogue_cols<Db>(dt, warp, pix, p.scale * ac, crow, blk, p.D, half * (Db / 2), Db / 2);
    else if (half == 0) epilogue_cols<Db>(dt, warp, pix, p.scale * ac, crow, blk, p.D, 0, Db);
    tc_fence_before_sync();
    __syncthreads();
    tc_fence_after_sync();
  }
  if (!ok && tid == 0) {
    if (p.err) atomicExch(p.err, kDevErrTmaTimeout);
    // a bounded last chance for copies still in flight into this CTA's buffers
    mbar_spin_bounded(&bar_load, phase ^ 1, kWaitLimit);
    mbar_spin_bounded(&bar_mma, phase ^ 1, kWaitLimit);
  }
  tc_fence_before_sync();
  __syncthreads();
  if (warp == 0) tmem_dealloc(dt, S::ACC_COLS);
}

// B operand blocks from the float64 radial kernel: block (bin, blk), chunk kc,
// row n (output column: Re of depth blk Db + n for n < Db, Im of depth
// blk Db + n - Db otherwise), column k = 2 f + part (part 0 multiplies Re Phat,
// part 1 Im Phat):
//   Re row: (Kr, -Ki),  Im row: (Ki, Kr),  zero beyond F and beyond D.
__global__ void kr_store_umma_kernel(const double2* K64, __half* B, int n_rho, int F, int D, int Db, int nblk,
                                     int KC, double scale) {
  const long long N = 2LL * Db;
  const long long per_chunk = N * kUmmaKChunk;
  const long long total = (long long)n_rho * nblk * KC * per_chunk;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const long long chunk = i / per_chunk;
    const int e = (int)(i % per_chunk);
    const int n = e / kUmmaKChunk, kj = e % kUmmaKChunk;
    const int kc = (int)(chunk % KC);
    const int blk = (int)((chunk / KC) % nblk);
    const int bin = (int)(chunk / ((long long)KC * nblk));
    const int k = kc * kUmmaKChunk + kj;
    const bool im_row = n >= Db;
    const int d = blk * Db + (im_row ? n - Db : n);
    double v = 0.0;
    const int f = k >> 1, part = k & 1;
    if (d < D && f < F) {
      const double2 kv = K64[((size_t)bin * F + f) * D + d];
      if (!im_row) v = part == 0 ? kv.x : -kv.y;
      else v = part == 0 ? kv.y : kv.x;
    }
    const size_t off = (size_t)chunk * per_chunk * 2 + umma_kmajor_offset(n, kj, kUmmaKChunk);   // bytes
    B[off / 2] = __double2half(v * scale);
  }
}

template <int Db>
cudaError_t launch_simple(const PfUmmaParams& p, cudaStream_t s) {
  constexpr uint32_t smem = 2 * Sizes<Db>::A_BYTES + 2 * Sizes<Db>::B_BYTES;
  auto k = pf_umma_kernel<Db>;
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  k<<<(unsigned)p.ntiles, kThreads, smem, s>>>(p);
  return cudaGetLastError();
}

template <int Db>
cudaError_t launch_ws(const PfUmmaParams& p, cudaStream_t s) {
  constexpr uint32_t smem = kStages * Sizes<Db>::STAGE;
  auto k = pf_umma_ws_kernel<Db>;
  static int sms = 0;
  if (sms == 0) {
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (sms <= 0) sms = 1;
  }
  const int grid = p.ntiles < sms ? p.ntiles : sms;   // one persistent CTA per SM
  k<<<grid, kWsThreads, smem, s>>>(p);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_pf_umma(const PfUmmaParams& p, bool pipelined, cudaStream_t s) {
  if (p.ntiles <= 0) return cudaSuccess;
  switch (p.Db) {
    case 16: return pipelined ? launch_ws<16>(p, s) : launch_simple<16>(p, s);
    case 32: return pipelined ? launch_ws<32>(p, s) : launch_simple<32>(p, s);
    case 64: return pipelined ? launch_ws<64>(p, s) : launch_simple<64>(p, s);
    case 128: return pipelined ? launch_ws<128>(p, s) : launch_simple<128>(p, s);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_kr_store_umma(const double2* K64, void* B, int n_rho, int F, int D, int Db, int nblk, int KC,
                                 double scale, cudaStream_t s) {
  kr_store_umma_kernel<<<152 * 8, 256, 0, s>>>(K64, static_cast<__half*>(B), n_rho, F, D, Db, nblk, KC, scale);
  return cudaGetLastError();
}

}  // namespace nlos
