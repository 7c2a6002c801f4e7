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
// A is a scaled copy of a phasor row, built in shared memory by the CTA's
// threads (row r = pixel r of the tile); B arrives by 1D bulk copies in the
// operand layout the plan stored, one elected thread issues kind::f16 MMAs (M = 128, N = 2 Db,
// K = 16 each) into a tensor-memory accumulator, and the four warps read it
// back (warp w owns rows 32 w .. 32 w + 31) to apply the taper and scale.
// Inputs are f16 with their per-volume and per-pass scales, the accumulator
// is f32.
#include <cuda_fp16.h>

#include "nlos_internal.h"
#include "nlos_umma.cuh"

namespace nlos {

namespace {

constexpr int kThreads = 256;               // 8 warps; the epilogue gives two warps per 32 rows
constexpr int kWaitLimit = 1 << 21;

// A chunk kc of a tile: element (row r, frequency f = kc * 32 + q) of
// (1 - alpha_r) Phat / alpha_r Phat as the column pair (2q, 2q + 1). Each warp
// instruction covers 8 rows x 4 consecutive q: the 32 lanes hit 32 distinct
// shared-memory banks and read 8 runs of 16 bytes from the phasor rows.
__device__ __forceinline__ void build_a_chunk(unsigned char* A0, unsigned char* A1, const __half2* Phat, int F,
                                              const int* tpix, const float* talpha, int kc, int tid) {
  const int warp = tid >> 5, lane = tid & 31;
  constexpr int kIters = kUmmaTile * (kUmmaKChunk / 2) / (32 * kThreads / 32);   // 16
  __half2 h[kIters];
  float al[kIters];
#pragma unroll
  for (int i = 0; i < kIters; ++i) {
    const int T = i * (kThreads / 32) + warp;                 // 8-row x 4-q block
    const int r = (T >> 3) * 8 + (lane & 7), q = (T & 7) * 4 + (lane >> 3);
    const int f = kc * (kUmmaKChunk / 2) + q;
    const int pix = __ldg(tpix + r);
    al[i] = __ldg(talpha + r);
    h[i] = (pix >= 0 && f < F) ? Phat[(size_t)pix * F + f] : __floats2half2_rn(0.f, 0.f);
  }
#pragma unroll
  for (int i = 0; i < kIters; ++i) {
    const int T = i * (kThreads / 32) + warp;
    const int r = (T >> 3) * 8 + (lane & 7), q = (T & 7) * 4 + (lane >> 3);
    const uint32_t off = umma_kmajor_offset(r, 2 * q, kUmmaKChunk);
    const float2 v = __half22float2(h[i]);
    const float w0 = 1.f - al[i];
    *reinterpret_cast<__half2*>(A0 + off) = __floats2half2_rn(w0 * v.x, w0 * v.y);
    *reinterpret_cast<__half2*>(A1 + off) = __floats2half2_rn(al[i] * v.x, al[i] * v.y);
  }
}

template <int Db>
struct UmmaSmem {
  static constexpr int N = 2 * Db;
  static constexpr uint32_t A_BYTES = kUmmaTile * kUmmaKChunk * 2;   // one A operand chunk
  static constexpr uint32_t B_BYTES = N * kUmmaKChunk * 2;           // one B operand chunk
  static constexpr uint32_t TOTAL = 2 * A_BYTES + 2 * B_BYTES;
  static constexpr uint32_t TMEM_COLS = N <= 32 ? 32 : N <= 64 ? 64 : N <= 128 ? 128 : 256;
};

template <int Db>
__global__ void __launch_bounds__(kThreads) pf_umma_kernel(const PfUmmaParams p) {
  using S = UmmaSmem<Db>;
  extern __shared__ __align__(128) unsigned char um_sm[];
  __shared__ uint64_t bar_load, bar_mma;
  __shared__ uint32_t tbase;
  unsigned char* A0 = um_sm;
  unsigned char* A1 = um_sm + S::A_BYTES;
  unsigned char* B0 = um_sm + 2 * S::A_BYTES;
  unsigned char* B1 = B0 + S::B_BYTES;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int row = tid & (kUmmaTile - 1), half = tid >> 7;   // tile row; which half of each chunk
  const int tile = blockIdx.x;
  const int2 i01 = p.tile_i01[tile];
  const int pix = p.tile_pix[(size_t)tile * kUmmaTile + row];
  const float ac = p.tile_acut[(size_t)tile * kUmmaTile + row];
  const int* tpix = p.tile_pix + (size_t)tile * kUmmaTile;
  const float* talpha = p.tile_alpha + (size_t)tile * kUmmaTile;
  const __half2* Ph = static_cast<const __half2*>(p.Phat);

  if (warp == 0) tmem_alloc(&tbase, S::TMEM_COLS);
  if (tid == 0) {
    mbar_init(&bar_load, 1);
    mbar_init(&bar_mma, 1);
    mbar_fence_init();
  }
  tc_fence_before_sync();
  __syncthreads();
  tc_fence_after_sync();
  const uint32_t dt = tbase;
  const uint32_t idesc = umma_idesc_f16<false>(kUmmaTile, S::N);
  const size_t blk_bytes = (size_t)p.KC * S::B_BYTES;                  // one depth block of one bin
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
      build_a_chunk(A0, A1, Ph, p.F, tpix, talpha, kc, tid);
      fence_proxy_async_smem();
      __syncthreads();
      if (tid == 0) {
        ok = mbar_wait_bounded(&bar_load, phase, kWaitLimit);
        tc_fence_after_sync();
        if (ok) {
#pragma unroll
          for (int kk = 0; kk < kUmmaKChunk / 16; ++kk) {
            const uint32_t ko = kk * 256;     // two 8-column core matrices per K = 16 slab
            umma_f16(dt, umma_smem_desc(smem_u32(A0) + ko, 128, 1024), umma_smem_desc(smem_u32(B0) + ko, 128, 1024),
                     idesc, (kc > 0 || kk > 0) ? 1u : 0u);
            umma_f16(dt, umma_smem_desc(smem_u32(A1) + ko, 128, 1024), umma_smem_desc(smem_u32(B1) + ko, 128, 1024),
                     idesc, 1u);
          }
        }
        umma_commit(&bar_mma);
      }
      // the MMAs read A and B; they finish before the next chunk overwrites them
      const bool done = mbar_wait_bounded(&bar_mma, phase, kWaitLimit);
      ok = __syncthreads_and(ok && done ? 1 : 0) != 0;
      phase ^= 1;
      if (!ok) break;
    }
    if (!ok) break;
    // epilogue: rows of this warp, Re in columns [0, Db), Im in [Db, 2 Db)
    tc_fence_after_sync();
    __half2* crow = static_cast<__half2*>(p.C) + (size_t)(pix >= 0 ? pix : 0) * p.D + (size_t)blk * Db;
    const float g = p.scale * ac;
    const uint32_t lane_base = dt + ((uint32_t)(32 * (warp & 3)) << 16);
    constexpr int kCols = Db >= 32 ? Db / 2 : Db;          // depth columns per warp half
    const int c0 = Db >= 32 ? half * kCols : 0;
    const bool writer = Db >= 32 || half == 0;
#pragma unroll
    for (int c = c0; c < c0 + kCols; c += 16) {
      uint32_t re[16], im[16];
      tmem_ld16(lane_base + (uint32_t)c, re);
      tmem_ld16(lane_base + (uint32_t)(Db + c), im);
      tmem_wait_ld();
      if (pix >= 0 && writer) {
#pragma unroll
        for (int q = 0; q < 16; ++q) {
          const int d = blk * Db + c + q;
          if (d < p.D) crow[c + q] = __floats2half2_rn(g * __uint_as_float(re[q]), g * __uint_as_float(im[q]));
        }
      }
    }
    (void)lane;
    // every warp has read the accumulator before the next block's MMAs
    tc_fence_before_sync();
    __syncthreads();
    tc_fence_after_sync();
  }
  if (!ok && tid == 0) {
    if (p.err) atomicExch(p.err, kDevErrTmaTimeout);
    // a bounded last chance for copies still in flight into this CTA's buffers
    mbar_wait_bounded(&bar_load, phase ^ 1, kWaitLimit);
    mbar_wait_bounded(&bar_mma, phase ^ 1, kWaitLimit);
  }
  tc_fence_before_sync();
  __syncthreads();
  if (warp == 0) tmem_dealloc(dt, S::TMEM_COLS);
}

// Persistent, double-buffered form: one CTA per SM walks its tiles; the
// operand buffers and the tensor-memory accumulator are doubled so that the
// bulk copies and the A build of the next chunk overlap the MMAs of the
// current one, and a tile's epilogue overlaps the next tile's first chunk.
template <int Db>
struct PipeSmem {
  static constexpr int N = 2 * Db;
  static constexpr uint32_t A_BYTES = kUmmaTile * kUmmaKChunk * 2;
  static constexpr uint32_t B_BYTES = N * kUmmaKChunk * 2;
  static constexpr uint32_t STAGE = 2 * A_BYTES + 2 * B_BYTES;        // A0 A1 B0 B1
  static constexpr uint32_t TOTAL = 2 * STAGE;
  static constexpr uint32_t ACC_COLS = N <= 32 ? 32 : N <= 64 ? 64 : N <= 128 ? 128 : 256;
  static constexpr uint32_t TMEM_COLS = 2 * ACC_COLS;
};

template <int Db>
__global__ void __launch_bounds__(kThreads, 1) pf_umma_pipe_kernel(const PfUmmaParams p) {
  using S = PipeSmem<Db>;
  extern __shared__ __align__(128) unsigned char up_sm[];
  __shared__ uint64_t bar_load[2], bar_mma[2];
  __shared__ uint32_t tbase;
  const int tid = threadIdx.x, warp = tid >> 5;
  const int row = tid & (kUmmaTile - 1), half = tid >> 7;
  auto A0 = [&](int st) { return up_sm + st * S::STAGE; };
  auto A1 = [&](int st) { return up_sm + st * S::STAGE + S::A_BYTES; };
  auto B0 = [&](int st) { return up_sm + st * S::STAGE + 2 * S::A_BYTES; };
  auto B1 = [&](int st) { return up_sm + st * S::STAGE + 2 * S::A_BYTES + S::B_BYTES; };
  if (warp == 0) tmem_alloc(&tbase, S::TMEM_COLS);
  if (tid == 0) {
    for (int i = 0; i < 2; ++i) {
      mbar_init(&bar_load[i], 1);
      mbar_init(&bar_mma[i], 1);
    }
    mbar_fence_init();
  }
  tc_fence_before_sync();
  __syncthreads();
  tc_fence_after_sync();
  const uint32_t tm = tbase;
  const uint32_t idesc = umma_idesc_f16<false>(kUmmaTile, S::N);
  const size_t blk_bytes = (size_t)p.KC * S::B_BYTES;
  const unsigned char* Bg = static_cast<const unsigned char*>(p.B);
  // this CTA's work: units (tile, depth block), each KC chunks
  const int units = (p.ntiles - (int)blockIdx.x + (int)gridDim.x - 1) / (int)gridDim.x * p.nblk;
  const int G = units * p.KC;
  auto unit_tile = [&](int u) { return (int)blockIdx.x + (u / p.nblk) * (int)gridDim.x; };
  // chunk g: unit g / KC, chunk kc = g % KC; stage g & 1, k-th use of its stage: g >> 1
  auto prepare = [&](int g) {               // bulk copies and A build of chunk g into stage g & 1
    const int st = g & 1, u = g / p.KC, kc = g % p.KC;
    const int tl = unit_tile(u), blk = u % p.nblk;
    const int2 i01 = p.tile_i01[tl];
    if (tid == 0) {
      fence_proxy_async_smem();
      mbar_arrive_expect_tx(&bar_load[st], 2 * S::B_BYTES);
      bulk_load(B0(st), Bg + ((size_t)i01.x * p.nblk + blk) * blk_bytes + (size_t)kc * S::B_BYTES, S::B_BYTES,
                &bar_load[st]);
      bulk_load(B1(st), Bg + ((size_t)i01.y * p.nblk + blk) * blk_bytes + (size_t)kc * S::B_BYTES, S::B_BYTES,
                &bar_load[st]);
    }
    build_a_chunk(A0(st), A1(st), static_cast<const __half2*>(p.Phat), p.F, p.tile_pix + (size_t)tl * kUmmaTile,
                  p.tile_alpha + (size_t)tl * kUmmaTile, kc, tid);
    fence_proxy_async_smem();
  };
  bool ok = true;
  if (G > 0) prepare(0);
  for (int g = 0; g < G && ok; ++g) {
    const int st = g & 1, use = g >> 1;
    const int u = g / p.KC, kc = g % p.KC;
    const uint32_t acc = tm + (uint32_t)((u & 1) * S::ACC_COLS);
    __syncthreads();                          // chunk g's A is built by every thread
    if (tid == 0) {
      ok = mbar_wait_bounded(&bar_load[st], use & 1, kWaitLimit);
      tc_fence_after_sync();
      if (ok) {
#pragma unroll
        for (int kk = 0; kk < kUmmaKChunk / 16; ++kk) {
          const uint32_t ko = kk * 256;
          umma_f16(acc, umma_smem_desc(smem_u32(A0(st)) + ko, 128, 1024),
                   umma_smem_desc(smem_u32(B0(st)) + ko, 128, 1024), idesc, (kc > 0 || kk > 0) ? 1u : 0u);
          umma_f16(acc, umma_smem_desc(smem_u32(A1(st)) + ko, 128, 1024),
                   umma_smem_desc(smem_u32(B1(st)) + ko, 128, 1024), idesc, 1u);
        }
      }
      umma_commit(&bar_mma[st]);
    }
    // stage st ^ 1 is free once chunk g - 1's MMAs are done; fill it with chunk g + 1
    if (g + 1 < G) {
      if (g >= 1) {
        const bool d = mbar_wait_bounded(&bar_mma[st ^ 1], ((g - 1) >> 1) & 1, kWaitLimit);
        if (!d) ok = false;
      }
      prepare(g + 1);
    }
    if (kc == p.KC - 1) {
      // last chunk of unit u: its MMAs done, then read accumulator (u & 1)
      const bool d = mbar_wait_bounded(&bar_mma[st], use & 1, kWaitLimit);
      tc_fence_after_sync();
      const int tl = unit_tile(u), blk = u % p.nblk;
      const int pix = p.tile_pix[(size_t)tl * kUmmaTile + row];
      const float ac = p.tile_acut[(size_t)tl * kUmmaTile + row];
      __half2* crow = static_cast<__half2*>(p.C) + (size_t)(pix >= 0 ? pix : 0) * p.D + (size_t)blk * Db;
      const float gsc = p.scale * ac;
      const uint32_t lane_base = acc + ((uint32_t)(32 * (warp & 3)) << 16);
      constexpr int kCols = Db >= 32 ? Db / 2 : Db;
      const int c0 = Db >= 32 ? half * kCols : 0;
      const bool writer = Db >= 32 || half == 0;
#pragma unroll
      for (int c = c0; c < c0 + kCols; c += 16) {
        uint32_t re[16], im[16];
        tmem_ld16(lane_base + (uint32_t)c, re);
        tmem_ld16(lane_base + (uint32_t)(Db + c), im);
        tmem_wait_ld();
        if (pix >= 0 && writer && d) {
#pragma unroll
          for (int q = 0; q < 16; ++q) {
            const int dd = blk * Db + c + q;
            if (dd < p.D) crow[c + q] = __floats2half2_rn(gsc * __uint_as_float(re[q]), gsc * __uint_as_float(im[q]));
          }
        }
      }
      if (!d) ok = false;
      tc_fence_before_sync();
    }
    ok = __syncthreads_and(ok ? 1 : 0) != 0;
  }
  if (!ok && tid == 0) {
    if (p.err) atomicExch(p.err, kDevErrTmaTimeout);
    for (int i = 0; i < 2; ++i) {               // bounded last chance for copies in flight
      mbar_wait_bounded(&bar_load[i], 0, kWaitLimit);
      mbar_wait_bounded(&bar_load[i], 1, kWaitLimit);
    }
  }
  // every issued MMA has completed before the accumulator is freed
  if (ok && G > 0 && tid == 0) {
    mbar_wait_bounded(&bar_mma[(G - 1) & 1], ((G - 1) >> 1) & 1, kWaitLimit);
    if (G > 1) mbar_wait_bounded(&bar_mma[(G - 2) & 1], ((G - 2) >> 1) & 1, kWaitLimit);
  }
  tc_fence_before_sync();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tm, S::TMEM_COLS);
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
cudaError_t launch_umma_db(const PfUmmaParams& p, cudaStream_t s) {
  using S = UmmaSmem<Db>;
  auto k = pf_umma_kernel<Db>;
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)S::TOTAL);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  k<<<(unsigned)p.ntiles, kThreads, S::TOTAL, s>>>(p);
  return cudaGetLastError();
}

template <int Db>
cudaError_t launch_pipe_db(const PfUmmaParams& p, cudaStream_t s) {
  using S = PipeSmem<Db>;
  auto k = pf_umma_pipe_kernel<Db>;
  static int sms = 0;
  if (sms == 0) {
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)S::TOTAL);
    if (e != cudaSuccess) return e;
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (sms <= 0) sms = 1;
  }
  const int grid = p.ntiles < sms ? p.ntiles : sms;   // one persistent CTA per SM
  k<<<grid, kThreads, S::TOTAL, s>>>(p);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_pf_umma(const PfUmmaParams& p, bool pipelined, cudaStream_t s) {
  if (p.ntiles <= 0) return cudaSuccess;
  switch (p.Db) {
    case 16: return pipelined ? launch_pipe_db<16>(p, s) : launch_umma_db<16>(p, s);
    case 32: return pipelined ? launch_pipe_db<32>(p, s) : launch_umma_db<32>(p, s);
    case 64: return pipelined ? launch_pipe_db<64>(p, s) : launch_umma_db<64>(p, s);
    case 128: return pipelined ? launch_pipe_db<128>(p, s) : launch_umma_db<128>(p, s);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_kr_store_umma(const double2* K64, void* B, int n_rho, int F, int D, int Db, int nblk, int KC,
                                 double scale, cudaStream_t s) {
  kr_store_umma_kernel<<<152 * 8, 256, 0, s>>>(K64, static_cast<__half*>(B), n_rho, F, D, Db, nblk, KC, scale);
  return cudaGetLastError();
}

}  // namespace nlos
