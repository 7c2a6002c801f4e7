// Phasor-field depth sum on the 5th-generation tensor cores (Eq. 7, Alg. 4).
// Pixels that share the radial pair (i0, i1) form tiles of up to 128 rows;
// for one tile the sum over the band frequencies of
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
// bulk copies in the operand layout the plan stored; MMAs (M = 128, N = 2 Db)
// accumulate in tensor memory; warps read the accumulator back (warp w owns
// rows 32 (w % 4) .. + 31) to apply the taper and scale.
//
// Operand kinds (both stage 64-byte operand rows per chunk):
//  * OpF16 (16-bit storage): f16 A and B, kind::f16 MMAs (K = 16), 32 columns
//    (16 frequencies) per chunk;
//  * OpTf32x3 (float32 storage): A and B split into tf32 parts hi = tf32(x),
//    lo = tf32(x - hi); each product is A_hi B_hi^T + A_hi B_lo^T +
//    A_lo B_hi^T in kind::tf32 MMAs (K = 8), 16 columns (8 frequencies) per
//    chunk. The parts carry 22 significant bits of every operand, so the sum
//    keeps float32 accuracy at three tf32 products per term.
//
// Two schedules:
//  * pf_umma_ws_kernel: one persistent CTA per SM, warp-specialised - a
//    producer warp keeps up to four operand stages in flight, eight warps
//    build A and run the epilogue, one thread issues the MMAs - with two
//    accumulators so a tile's epilogue overlaps the next tile's MMAs;
//  * pf_umma_kernel: one CTA per tile, one stage.
#include <cuda_fp16.h>

#include "nlos_internal.h"
#include "nlos_umma.cuh"

namespace nlos {

namespace {

constexpr int kWaitLimit = 1 << 26;                    // probes of a barrier (a few hundred ms)
constexpr uint32_t kSbo = (kUmmaRowBytes / 16) * 128;  // row-group stride of a chunk operand
constexpr uint32_t kABytes = kUmmaTile * kUmmaRowBytes;  // one A operand part of a chunk
constexpr uint32_t kSmemBudget = 200 * 1024;           // dynamic shared memory of the stages

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// byte offset of the complex value of frequency q (within the chunk) of
// operand row r: columns (2q, 2q + 1), elements of `elem` bytes, 64-byte rows
// in 8 x 16-byte core matrices
__host__ __device__ constexpr uint32_t chunk_offset(int r, int q, int elem) {
  return (uint32_t)(((r >> 3) * (kUmmaRowBytes / 16) + ((2 * q * elem) >> 4)) * 128 + (r & 7) * 16 +
                    ((2 * q * elem) & 15));
}

struct OpF16 {
  using In = __half2;    // phasor element
  using Out = __half2;   // depth-sum element
  static constexpr int kKind = kUmmaF16, kElem = 2, kParts = 1, kSlab = 16;
  static constexpr int kQ = kUmmaRowBytes / (2 * kElem);   // frequencies per chunk
  __device__ static __forceinline__ float2 load(In v) { return __half22float2(v); }
  __device__ static __forceinline__ In zero() { return __floats2half2_rn(0.f, 0.f); }
  // A operand parts of one weight at byte offset off
  __device__ static __forceinline__ void put(unsigned char* a, uint32_t off, float x, float y) {
    *reinterpret_cast<__half2*>(a + off) = __floats2half2_rn(x, y);
  }
  __device__ static __forceinline__ uint32_t idesc(int N) { return umma_idesc_f16<false>(kUmmaTile, N); }
  __device__ static __forceinline__ void mma(uint32_t d, uint64_t a, uint64_t b, uint32_t id, uint32_t acc) {
    umma_f16(d, a, b, id, acc);
  }
  __device__ static __forceinline__ Out out(float x, float y) { return __floats2half2_rn(x, y); }
};

struct OpTf32x3 {
  using In = float2;
  using Out = float2;
  static constexpr int kKind = kUmmaTf32x3, kElem = 4, kParts = 2, kSlab = 8;
  static constexpr int kQ = kUmmaRowBytes / (2 * kElem);
  __device__ static __forceinline__ float2 load(In v) { return v; }
  __device__ static __forceinline__ In zero() { return make_float2(0.f, 0.f); }
  __device__ static __forceinline__ void put(unsigned char* a, uint32_t off, float x, float y) {
    const float hx = to_tf32(x), hy = to_tf32(y);
    *reinterpret_cast<float2*>(a + off) = make_float2(hx, hy);
    *reinterpret_cast<float2*>(a + kABytes + off) = make_float2(to_tf32(x - hx), to_tf32(y - hy));
  }
  __device__ static __forceinline__ uint32_t idesc(int N) { return umma_idesc_tf32(kUmmaTile, N); }
  __device__ static __forceinline__ void mma(uint32_t d, uint64_t a, uint64_t b, uint32_t id, uint32_t acc) {
    umma_tf32(d, a, b, id, acc);
  }
  __device__ static __forceinline__ Out out(float x, float y) { return make_float2(x, y); }
};

// Stage layout: A(w, part) for weights w = 0 (1 - alpha), 1 (alpha), then
// B(bin, part) for bins i0, i1; the parts of one B block are contiguous in the
// stage and in the plan's operand store, so one bulk copy brings a bin.
template <class Op, int Db>
struct Sizes {
  static constexpr int N = 2 * Db;
  static constexpr uint32_t B_BYTES = N * kUmmaRowBytes;                      // one B part of a chunk
  static constexpr uint32_t B_BLOCK = Op::kParts * B_BYTES;                    // all parts of one bin
  static constexpr uint32_t B_OFF = 2 * Op::kParts * kABytes;
  static constexpr uint32_t STAGE = B_OFF + 2 * B_BLOCK;
  static constexpr int STAGES = kSmemBudget / STAGE >= 4 ? 4 : (int)(kSmemBudget / STAGE);
  static constexpr uint32_t ACC_COLS = N <= 32 ? 32 : N <= 64 ? 64 : N <= 128 ? 128 : 256;
  static_assert(STAGES >= 1, "a stage must fit in shared memory");
};

// A chunk of a tile: frequency q of row r for thread t and iteration i. A
// warp instruction covers 8 rows x 4 consecutive q: the 32 lanes hit 32
// distinct shared-memory banks (f16) or two conflict-free 128-byte wavefronts
// (tf32) and read 8 runs of 4 consecutive phasors. NT threads (a multiple of
// 32) share the chunk.
template <class Op, int NT>
struct AChunk {
  static constexpr int kBlocks = (kUmmaTile / 8) * (Op::kQ / 4);
  static constexpr int kIters = kBlocks / (NT / 32);
  static_assert(kIters * (NT / 32) == kBlocks, "threads must divide the chunk");
  __device__ static __forceinline__ void coords(int i, int t, int& r, int& q) {
    const int T = i * (NT / 32) + (t >> 5);
    r = (T / (Op::kQ / 4)) * 8 + (t & 7);
    q = (T % (Op::kQ / 4)) * 4 + ((t & 31) >> 3);
  }
  // value v of row r with weight alpha into both A operands
  __device__ static __forceinline__ void put(unsigned char* stage, int r, int q, float2 v, float alpha) {
    const uint32_t off = chunk_offset(r, q, Op::kElem);
    const float w0 = 1.f - alpha;
    Op::put(stage, off, w0 * v.x, w0 * v.y);
    Op::put(stage + Op::kParts * kABytes, off, alpha * v.x, alpha * v.y);
  }
};

// MMAs of one chunk into accumulator `acc` (first: the chunk starts the sum)
template <class Op, int Db>
__device__ __forceinline__ void mma_chunk(uint32_t acc, uint32_t idesc, const unsigned char* stage, bool first) {
  using S = Sizes<Op, Db>;
  const uint32_t s0 = smem_u32(stage);
#pragma unroll
  for (int kk = 0; kk < kUmmaRowBytes / (Op::kElem * Op::kSlab); ++kk) {
    const uint32_t ko = kk * 256;     // an MMA reads 32 bytes of K: two 16-byte core-matrix columns
#pragma unroll
    for (int w = 0; w < 2; ++w) {
      const uint32_t a_hi = s0 + w * Op::kParts * kABytes + ko;
      const uint32_t b_hi = s0 + S::B_OFF + w * S::B_BLOCK + ko;
      Op::mma(acc, umma_smem_desc(a_hi, 128, kSbo), umma_smem_desc(b_hi, 128, kSbo), idesc,
              (first && kk == 0 && w == 0) ? 0u : 1u);
      if (Op::kParts == 2) {
        Op::mma(acc, umma_smem_desc(a_hi, 128, kSbo), umma_smem_desc(b_hi + S::B_BYTES, 128, kSbo), idesc, 1u);
        Op::mma(acc, umma_smem_desc(a_hi + kABytes, 128, kSbo), umma_smem_desc(b_hi, 128, kSbo), idesc, 1u);
      }
    }
  }
}

// accumulator rows of one warp -> C (taper and scale), columns [c0, c0 + ncols)
template <class Op, int Db>
__device__ __forceinline__ void epilogue_cols(uint32_t acc, int warp, int pix, float gsc, typename Op::Out* crow,
                                              int blk, int D, int c0, int ncols) {
  using Out = typename Op::Out;
  constexpr int kVec = 16 / sizeof(Out);        // complex values per 16-byte store
  const uint32_t lane_base = acc + ((uint32_t)(32 * (warp & 3)) << 16);
  for (int c = c0; c < c0 + ncols; c += 16) {
    uint32_t re[16], im[16];
    tmem_ld16(lane_base + (uint32_t)c, re);
    tmem_ld16(lane_base + (uint32_t)(Db + c), im);
    tmem_wait_ld();
    if (pix >= 0) {
      Out o[16];
#pragma unroll
      for (int q = 0; q < 16; ++q) o[q] = Op::out(gsc * __uint_as_float(re[q]), gsc * __uint_as_float(im[q]));
      if (blk * Db + c + 16 <= D && (reinterpret_cast<uintptr_t>(crow + c) & 15) == 0) {
        uint4* dst = reinterpret_cast<uint4*>(crow + c);
#pragma unroll
        for (int v = 0; v < 16 / kVec; ++v) dst[v] = reinterpret_cast<const uint4*>(o)[v];
      } else {
#pragma unroll
        for (int q = 0; q < 16; ++q)
          if (blk * Db + c + q < D) crow[c + q] = o[q];
      }
    }
  }
}

// ---------------------------------------------------------------------------
// Warp-specialised persistent schedule
// ---------------------------------------------------------------------------
constexpr int kMaxStages = 4;
constexpr int kWsBuilders = 256;                 // warps 0-7: A build, epilogue
constexpr int kWsThreads = kWsBuilders + 64;     // warp 8: producer, warp 9: MMA issue
constexpr int kProducerWarp = kWsBuilders / 32, kMmaWarp = kProducerWarp + 1;

template <class Op, int Db>
__global__ void __launch_bounds__(kWsThreads, 1) pf_umma_ws_kernel(const PfUmmaParams p) {
  using S = Sizes<Op, Db>;
  using A = AChunk<Op, kWsBuilders>;
  using In = typename Op::In;
  using Out = typename Op::Out;
  constexpr int kStages = S::STAGES;
  extern __shared__ __align__(128) unsigned char ws_sm[];
  __shared__ uint64_t full_b[kMaxStages], full_a[kMaxStages], empty[kMaxStages], acc_full[2], acc_empty[2];
  __shared__ uint32_t tbase;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  auto stage = [&](int s) { return ws_sm + s * S::STAGE; };
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
      const size_t blk_bytes = (size_t)p.KC * S::B_BLOCK;
      const unsigned char* Bg = static_cast<const unsigned char*>(p.B);
      for (int g = 0; g < G && !err; ++g) {
        const int s = g % kStages, r = g / kStages, u = g / p.KC, kc = g % p.KC;
        if (r >= 1 && !mbar_spin_bounded(&empty[s], (r - 1) & 1, kWaitLimit)) {
          err = 1;
          break;
        }
        const int tl = unit_tile(u), blk = u % p.nblk;
        const int2 i01 = p.tile_i01[tl];
        unsigned char* b = stage(s) + S::B_OFF;
        mbar_arrive_expect_tx(&full_b[s], 2 * S::B_BLOCK);
        bulk_load(b, Bg + ((size_t)i01.x * p.nblk + blk) * blk_bytes + (size_t)kc * S::B_BLOCK, S::B_BLOCK,
                  &full_b[s]);
        bulk_load(b + S::B_BLOCK, Bg + ((size_t)i01.y * p.nblk + blk) * blk_bytes + (size_t)kc * S::B_BLOCK,
                  S::B_BLOCK, &full_b[s]);
      }
    }
  } else if (warp == kMmaWarp) {
    // MMA issue
    if (lane == 0) {
      const uint32_t idesc = Op::idesc(S::N);
      for (int g = 0; g < G && !err; ++g) {
        const int s = g % kStages, r = g / kStages, u = g / p.KC, kc = g % p.KC;
        const int a = u & 1;
        if (kc == 0 && u >= 2 && !mbar_spin_bounded(&acc_empty[a], ((u - 2) >> 1) & 1, kWaitLimit)) err = 1;
        if (!err && !mbar_spin_bounded(&full_b[s], r & 1, kWaitLimit)) err = 1;
        if (!err && !mbar_spin_bounded(&full_a[s], r & 1, kWaitLimit)) err = 1;
        if (err) break;
        tc_fence_after_sync();
        mma_chunk<Op, Db>(tm + (uint32_t)(a * S::ACC_COLS), idesc, stage(s), kc == 0);
        umma_commit(&empty[s]);
        if (kc == p.KC - 1) umma_commit(&acc_full[a]);
      }
    }
  } else {
    // builders: A stages, then the epilogue of the previous unit
    const int t = tid;
    const In* Ph = static_cast<const In*>(p.Phat);
    auto epilogue = [&](int u) {
      const int a = u & 1, tl = unit_tile(u), blk = u % p.nblk;
      if (!mbar_spin_bounded(&acc_full[a], (u >> 1) & 1, kWaitLimit)) err = 1;
      tc_fence_after_sync();
      // warps w and w + 4 own the rows of lane quarter w % 4 and split the depths
      const int row = t & (kUmmaTile - 1), half = t >> 7;
      const int pix = p.tile_pix[(size_t)tl * kUmmaTile + row];
      const float ac = p.tile_acut[(size_t)tl * kUmmaTile + row];
      Out* crow = static_cast<Out*>(p.C) + (size_t)(pix >= 0 ? pix : 0) * p.D + (size_t)blk * Db;
      const uint32_t acc = tm + (uint32_t)(a * S::ACC_COLS);
      if (!err) {
        if (Db >= 32) epilogue_cols<Op, Db>(acc, warp, pix, p.scale * ac, crow, blk, p.D, half * (Db / 2), Db / 2);
        else if (half == 0) epilogue_cols<Op, Db>(acc, warp, pix, p.scale * ac, crow, blk, p.D, 0, Db);
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
    auto load_h = [&](In (&h)[A::kIters], int kc) {
#pragma unroll
      for (int i = 0; i < A::kIters; ++i) {
        int r, q;
        A::coords(i, t, r, q);
        const int f = kc * Op::kQ + q;
        h[i] = (rp[i] >= 0 && f < p.F) ? Ph[(size_t)rp[i] * p.F + f] : Op::zero();
      }
    };
    In hc[A::kIters], hn[A::kIters];
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
          A::put(stage(s), rr, q, Op::load(hc[i]), ra[i]);
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

template <class Op, int Db>
__global__ void __launch_bounds__(kThreads) pf_umma_kernel(const PfUmmaParams p) {
  using S = Sizes<Op, Db>;
  using A = AChunk<Op, kThreads>;
  using In = typename Op::In;
  using Out = typename Op::Out;
  extern __shared__ __align__(128) unsigned char um_sm[];
  __shared__ uint64_t bar_load, bar_mma;
  __shared__ uint32_t tbase;
  __shared__ int spix[kUmmaTile];
  __shared__ float salpha[kUmmaTile];
  unsigned char* B = um_sm + S::B_OFF;
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
  const In* Ph = static_cast<const In*>(p.Phat);
  if (warp == 0) tmem_alloc(&tbase, S::ACC_COLS);
  if (tid == 0) {
    mbar_init(&bar_load, 1);
    mbar_init(&bar_mma, 1);
    mbar_fence_init();
  }
  tc_fence_before_sync();
  __syncthreads();
  tc_fence_after_sync();
  auto load_h = [&](In (&h)[A::kIters], int kc) {
#pragma unroll
    for (int i = 0; i < A::kIters; ++i) {
      int r, q;
      A::coords(i, tid, r, q);
      const int f = kc * Op::kQ + q;
      const int px = spix[r];
      h[i] = (px >= 0 && f < p.F) ? Ph[(size_t)px * p.F + f] : Op::zero();
    }
  };
  In hcur[A::kIters], hnext[A::kIters];
  load_h(hcur, 0);
  const uint32_t dt = tbase;
  const uint32_t idesc = Op::idesc(S::N);
  const size_t blk_bytes = (size_t)p.KC * S::B_BLOCK;
  const unsigned char* Bg = static_cast<const unsigned char*>(p.B);
  int phase = 0;
  bool ok = true;
  for (int blk = 0; blk < p.nblk && ok; ++blk) {
    const unsigned char* b0g = Bg + ((size_t)i01.x * p.nblk + blk) * blk_bytes;
    const unsigned char* b1g = Bg + ((size_t)i01.y * p.nblk + blk) * blk_bytes;
    for (int kc = 0; kc < p.KC; ++kc) {
      if (tid == 0) {
        fence_proxy_async_smem();
        mbar_arrive_expect_tx(&bar_load, 2 * S::B_BLOCK);
        bulk_load(B, b0g + (size_t)kc * S::B_BLOCK, S::B_BLOCK, &bar_load);
        bulk_load(B + S::B_BLOCK, b1g + (size_t)kc * S::B_BLOCK, S::B_BLOCK, &bar_load);
      }
#pragma unroll
      for (int i = 0; i < A::kIters; ++i) {
        int r, q;
        A::coords(i, tid, r, q);
        A::put(um_sm, r, q, Op::load(hcur[i]), salpha[r]);
      }
      // the next chunk's phasors are in flight while this chunk's MMAs run
      load_h(hnext, kc + 1 < p.KC ? kc + 1 : 0);
      fence_proxy_async_smem();
      __syncthreads();
      if (tid == 0) {
        ok = mbar_spin_bounded(&bar_load, phase, kWaitLimit);
        tc_fence_after_sync();
        if (ok) mma_chunk<Op, Db>(dt, idesc, um_sm, kc == 0);
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
    Out* crow = static_cast<Out*>(p.C) + (size_t)(pix >= 0 ? pix : 0) * p.D + (size_t)blk * Db;
    if (Db >= 32) epilogue_cols<Op, Db>(dt, warp, pix, p.scale * ac, crow, blk, p.D, half * (Db / 2), Db / 2);
    else if (half == 0) epilogue_cols<Op, Db>(dt, warp, pix, p.scale * ac, crow, blk, p.D, 0, Db);
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
// part, row n (output column: Re of depth blk Db + n for n < Db, Im of depth
// blk Db + n - Db otherwise), column k = 2 f + c (c = 0 multiplies Re Phat,
// c = 1 Im Phat):
//   Re row: (Kr, -Ki),  Im row: (Ki, Kr),  zero beyond F and beyond D.
// f16 kind: one part, the scaled value; tf32 kind: parts hi = tf32(v),
// lo = tf32(v - hi) of the float32 value v.
template <class Op>
__global__ void kr_store_umma_kernel(const double2* K64, unsigned char* B, int n_rho, int F, int D, int Db, int nblk,
                                     int KC, double scale) {
  constexpr int kCols = kUmmaRowBytes / Op::kElem;
  const long long N = 2LL * Db;
  const long long per_chunk = N * kCols;
  const long long total = (long long)n_rho * nblk * KC * per_chunk;
  const size_t part_bytes = (size_t)N * kUmmaRowBytes;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const long long chunk = i / per_chunk;
    const int e = (int)(i % per_chunk);
    const int n = e / kCols, kj = e % kCols;
    const int kc = (int)(chunk % KC);
    const int blk = (int)((chunk / KC) % nblk);
    const int bin = (int)(chunk / ((long long)KC * nblk));
    const int k = kc * kCols + kj;
    const bool im_row = n >= Db;
    const int d = blk * Db + (im_row ? n - Db : n);
    double v = 0.0;
    const int f = k >> 1, c = k & 1;
    if (d < D && f < F) {
      const double2 kv = K64[((size_t)bin * F + f) * D + d];
      if (!im_row) v = c == 0 ? kv.x : -kv.y;
      else v = c == 0 ? kv.y : kv.x;
    }
    // element (n, kj) of a 64-byte-row operand: core matrix (n / 8, byte column / 16)
    const int bc = kj * Op::kElem;
    const size_t off = ((size_t)(n >> 3) * (kUmmaRowBytes / 16) + (bc >> 4)) * 128 + (n & 7) * 16 + (bc & 15);
    unsigned char* base = B + (size_t)chunk * Op::kParts * part_bytes;
    if (Op::kKind == kUmmaF16) {
      *reinterpret_cast<__half*>(base + off) = __double2half(v * scale);
    } else {
      const float x = (float)(v * scale);
      const float hi = to_tf32(x);
      *reinterpret_cast<float*>(base + off) = hi;
      *reinterpret_cast<float*>(base + part_bytes + off) = to_tf32(x - hi);
    }
  }
}

template <class Op, int Db>
cudaError_t launch_simple(const PfUmmaParams& p, cudaStream_t s) {
  constexpr uint32_t smem = Sizes<Op, Db>::STAGE;
  auto k = pf_umma_kernel<Op, Db>;
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  k<<<(unsigned)p.ntiles, kThreads, smem, s>>>(p);
  return cudaGetLastError();
}

template <class Op, int Db>
cudaError_t launch_ws(const PfUmmaParams& p, cudaStream_t s) {
  constexpr uint32_t smem = Sizes<Op, Db>::STAGES * Sizes<Op, Db>::STAGE;
  auto k = pf_umma_ws_kernel<Op, Db>;
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

template <class Op>
cudaError_t launch_kind(const PfUmmaParams& p, bool pipelined, cudaStream_t s) {
  switch (p.Db) {
    case 16: return pipelined ? launch_ws<Op, 16>(p, s) : launch_simple<Op, 16>(p, s);
    case 32: return pipelined ? launch_ws<Op, 32>(p, s) : launch_simple<Op, 32>(p, s);
    case 64: return pipelined ? launch_ws<Op, 64>(p, s) : launch_simple<Op, 64>(p, s);
    case 128: return pipelined ? launch_ws<Op, 128>(p, s) : launch_simple<Op, 128>(p, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace

cudaError_t launch_pf_umma(const PfUmmaParams& p, bool pipelined, cudaStream_t s) {
  if (p.ntiles <= 0) return cudaSuccess;
  if (p.kind == kUmmaF16) return launch_kind<OpF16>(p, pipelined, s);
  if (p.kind == kUmmaTf32x3) return launch_kind<OpTf32x3>(p, pipelined, s);
  return cudaErrorInvalidValue;
}

cudaError_t launch_kr_store_umma(const double2* K64, void* B, int kind, int n_rho, int F, int D, int Db, int nblk,
                                 int KC, double scale, cudaStream_t s) {
  unsigned char* b = static_cast<unsigned char*>(B);
  if (kind == kUmmaF16)
    kr_store_umma_kernel<OpF16><<<152 * 8, 256, 0, s>>>(K64, b, n_rho, F, D, Db, nblk, KC, scale);
  else if (kind == kUmmaTf32x3)
    kr_store_umma_kernel<OpTf32x3><<<152 * 8, 256, 0, s>>>(K64, b, n_rho, F, D, Db, nblk, KC, scale);
  else
    return cudaErrorInvalidValue;
  return cudaGetLastError();
}

}  // namespace nlos
