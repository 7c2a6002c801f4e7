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
// Operand kinds (both stage 64-byte operand rows per chunk: 32 f16 columns,
// 16 frequencies; kind::f16 MMAs, K = 16):
//  * OpF16 (16-bit storage): f16 A and B, one product;
//  * OpF16x3 (float32 storage): A and B split into f16 parts hi = f16(x),
//    lo = f16(x - hi), each product taken as A_hi B_hi^T + A_hi B_lo^T +
//    A_lo B_hi^T. The parts carry 22 significant bits of every operand, so
//    the sum keeps float32 accuracy (the dropped A_lo B_lo^T is ~2^-22 of
//    it) at three f16 products per term. A is scaled into f16 range per
//    volume by a power of two from a bound on |Phat|, B per plan; the
//    epilogue removes both.
//
// Two schedules:
//  * pf_umma_ws_kernel: one persistent CTA per SM, warp-specialised - a
//    producer warp keeps up to four operand stages in flight, eight warps
//    build A, one thread issues the MMAs, four warps run the epilogue - with
//    two accumulators so a tile's epilogue overlaps the next tile's MMAs; the
//    tiles left after the last full round are split along the frequency sum
//    so that no CTA runs a whole extra tile;
//  * pf_umma_kernel: one CTA per tile, one stage.
#include <cuda_fp16.h>

#include "nlos_bounds.cuh"
#include "nlos_internal.h"
#include "nlos_umma.cuh"

namespace nlos {

namespace {

constexpr int kWaitLimit = 1 << 26;                    // probes of a barrier (a few hundred ms)
constexpr uint32_t kSmemBudget = 200 * 1024;           // dynamic shared memory of the stages

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// byte offset of the complex value of frequency q (within the chunk) of
// operand row r: columns (2q, 2q + 1), kRowBytes-byte rows in 8 x 16-byte
// core matrices
template <class Op>
__host__ __device__ constexpr uint32_t chunk_offset(int r, int q) {
  return (uint32_t)(((r >> 3) * (Op::kRowBytes / 16) + ((2 * q * Op::kElem) >> 4)) * 128 + (r & 7) * 16 +
                    ((2 * q * Op::kElem) & 15));
}

struct OpF16 {
  using In = __half2;    // phasor element
  using Out = __half2;   // depth-sum element
  static constexpr int kKind = kUmmaF16, kElem = 2, kParts = 1, kSlab = 16;
  static constexpr bool kScaled = false;     // A scaled per volume by a bound on |Phat|
  // L2 prefetch of B blocks ahead of their copies: it shortens the copies of
  // the two-stage f16x3 ring; the four-stage f16 ring does not gain from it
  static constexpr bool kPrefetchB = false;
  static constexpr uint32_t kRowBytes = 64;                 // bytes of an operand row per chunk
  static constexpr uint32_t kSbo = (kRowBytes / 16) * 128;  // row-group stride of a chunk operand
  static constexpr uint32_t kABytes = kUmmaTile * kRowBytes;  // one A operand part of a chunk
  static constexpr int kQ = kRowBytes / (2 * kElem);        // frequencies per chunk
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

struct OpF16x3 {
  using In = float2;
  using Out = float2;
  static constexpr int kKind = kUmmaF16x3, kElem = 2, kParts = 2, kSlab = 16;
  static constexpr bool kScaled = true;
  static constexpr bool kPrefetchB = true;
  static constexpr uint32_t kRowBytes = 64;
  static constexpr uint32_t kSbo = (kRowBytes / 16) * 128;
  static constexpr uint32_t kABytes = kUmmaTile * kRowBytes;
  static constexpr int kQ = kRowBytes / (2 * kElem);
  __device__ static __forceinline__ float2 load(In v) { return v; }
  __device__ static __forceinline__ In zero() { return make_float2(0.f, 0.f); }
  // x, y already scaled into f16 range: hi = f16(x), lo = f16(x - hi)
  __device__ static __forceinline__ void put(unsigned char* a, uint32_t off, float x, float y) {
    const __half2 hi = __floats2half2_rn(x, y);
    const float2 h = __half22float2(hi);
    *reinterpret_cast<__half2*>(a + off) = hi;
    *reinterpret_cast<__half2*>(a + kABytes + off) = __floats2half2_rn(x - h.x, y - h.y);
  }
  __device__ static __forceinline__ uint32_t idesc(int N) { return umma_idesc_f16<false>(kUmmaTile, N); }
  __device__ static __forceinline__ void mma(uint32_t d, uint64_t a, uint64_t b, uint32_t id, uint32_t acc) {
    umma_f16(d, a, b, id, acc);
  }
  __device__ static __forceinline__ Out out(float x, float y) { return make_float2(x, y); }
};

// Scale of the A operand of a scaled kind: 2^(15 - e(amax) - abound_exp)
// keeps |A| < 2^15 (f16 holds 65504); 1 when the phasors are all zero. sa
// and its inverse are exact powers of two.
template <class Op>
__device__ __forceinline__ void a_scale(const PfUmmaParams& p, float& sa, float& inv_sa) {
  sa = inv_sa = 1.f;
  if (!Op::kScaled) return;
  const float m = __uint_as_float(*p.amax);
  if (!(m > 0.f)) return;
  int e;
  frexpf(m, &e);                                  // m < 2^e
  int k = 15 - e - p.abound_exp;
  k = k < -120 ? -120 : k > 120 ? 120 : k;
  sa = ldexpf(1.f, k);
  inv_sa = ldexpf(1.f, -k);
}

static_assert(OpF16::kRowBytes == umma_row_bytes(kUmmaF16) &&
                  OpF16::kRowBytes / OpF16::kElem == umma_chunk_cols(kUmmaF16),
              "f16 chunk geometry");
static_assert(OpF16x3::kRowBytes == umma_row_bytes(kUmmaF16x3) &&
                  OpF16x3::kRowBytes / OpF16x3::kElem == umma_chunk_cols(kUmmaF16x3),
              "f16x3 chunk geometry");

// Stage layout: A(w, part) for weights w = 0 (1 - alpha), 1 (alpha), then
// B(bin, part) for bins i0, i1; the parts of one B block are contiguous in the
// stage and in the plan's operand store, so one bulk copy brings a bin.
template <class Op, int Db>
struct Sizes {
  static constexpr int N = 2 * Db;
  static constexpr uint32_t B_BYTES = N * Op::kRowBytes;                      // one B part of a chunk
  static constexpr uint32_t B_BLOCK = Op::kParts * B_BYTES;                    // all parts of one bin
  static constexpr uint32_t B_OFF = 2 * Op::kParts * Op::kABytes;
  static constexpr uint32_t STAGE = B_OFF + 2 * B_BLOCK;
  static constexpr int STAGES = kSmemBudget / STAGE >= 4 ? 4 : (int)(kSmemBudget / STAGE);
  static constexpr uint32_t ACC_COLS = N <= 32 ? 32 : N <= 64 ? 64 : N <= 128 ? 128 : 256;
  static_assert(STAGES >= 1, "a stage must fit in shared memory");
};

// A chunk of a tile: frequency q of row r for thread t and iteration i. A
// warp instruction covers 8 rows x 4 consecutive q: the 32 lanes hit 32
// distinct shared-memory banks and read 8 runs of 4 consecutive phasors. NT threads (a multiple of
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
  // value v of row r with weights (1 - alpha) sa, alpha sa into both A operands
  __device__ static __forceinline__ void put(unsigned char* stage, int r, int q, float2 v, float alpha, float sa) {
    const uint32_t off = chunk_offset<Op>(r, q);
    const float w0 = (1.f - alpha) * sa, w1 = alpha * sa;
    Op::put(stage, off, w0 * v.x, w0 * v.y);
    Op::put(stage + Op::kParts * Op::kABytes, off, w1 * v.x, w1 * v.y);
  }
};

// MMAs of one chunk into accumulator `acc` (first: the chunk starts the sum)
template <class Op, int Db>
__device__ __forceinline__ void mma_chunk(uint32_t acc, uint32_t idesc, const unsigned char* stage, bool first) {
  using S = Sizes<Op, Db>;
  const uint32_t s0 = smem_u32(stage);
#pragma unroll
  for (int kk = 0; kk < (int)Op::kRowBytes / (Op::kElem * Op::kSlab); ++kk) {
    const uint32_t ko = kk * 256;     // an MMA reads 32 bytes of K: two 16-byte core-matrix columns
#pragma unroll
    for (int w = 0; w < 2; ++w) {
      const uint32_t a_hi = s0 + w * Op::kParts * Op::kABytes + ko;
      const uint32_t b_hi = s0 + S::B_OFF + w * S::B_BLOCK + ko;
      constexpr uint32_t sbo = Op::kSbo;
      Op::mma(acc, umma_smem_desc(a_hi, 128, sbo), umma_smem_desc(b_hi, 128, sbo), idesc,
              (first && kk == 0 && w == 0) ? 0u : 1u);
      if (Op::kParts == 2) {
        Op::mma(acc, umma_smem_desc(a_hi, 128, sbo), umma_smem_desc(b_hi + S::B_BYTES, 128, sbo), idesc, 1u);
        Op::mma(acc, umma_smem_desc(a_hi + Op::kABytes, 128, sbo), umma_smem_desc(b_hi, 128, sbo), idesc, 1u);
      }
    }
  }
}

// accumulator rows of one warp -> C (taper and scale), columns [c0, c0 + ncols);
// `add`: the accumulator holds part of the frequency sum and is added to C
// (cleared beforehand) with atomics instead of stored
template <class Op, int Db>
__device__ __forceinline__ void epilogue_cols(uint32_t acc, int warp, int pix, float gsc, typename Op::Out* crow,
                                              int blk, int D, int c0, int ncols, bool add = false) {
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
      if (add) {
#pragma unroll
        for (int q = 0; q < 16; ++q)
          if (blk * Db + c + q < D) atomicAdd(crow + c + q, o[q]);
      } else if (blk * Db + c + 16 <= D && (reinterpret_cast<uintptr_t>(crow + c) & 15) == 0) {
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
// parts of a tail unit's frequency sum: with at most two, every element of C
// receives at most two atomic additions onto an exact zero (0 + x is exact,
// x + y = y + x), so the result does not depend on their order
constexpr int kMaxSplit = 2;
constexpr int kWsBuilders = 256;                 // warps 0-7: A build
constexpr int kProducerWarp = kWsBuilders / 32;  // warp 8: B copies
constexpr int kMmaWarp = kProducerWarp + 1;      // warp 9: MMA issue
constexpr int kEpiWarp0 = kMmaWarp + 1;          // warps 10-13: epilogue, one per TMEM lane quarter
constexpr int kEpiThreads = 128;
constexpr int kWsThreads = kWsBuilders + 64 + kEpiThreads;

// The work of CTA b: R = ntiles / grid rounds of whole tiles (tile b + k grid,
// all its depth blocks, every chunk), then the tail - the ntiles - R grid
// remaining tiles' units, each split into `split` chunk ranges - as segments
// b, b + grid, ... of the tail list. A segment that covers part of a unit's
// frequency sum adds its result to C.
struct Seg {
  int tile, blk, k0, k1;
  bool partial;
};
struct WsWork {
  int R, nseg;
  __device__ WsWork(const PfUmmaParams& p) {
    const int b = blockIdx.x, grid = gridDim.x;
    R = p.ntiles / grid;
    const int ntail = (p.ntiles - R * grid) * p.nblk * p.split;
    nseg = R * p.nblk + (ntail > b ? (ntail - b + grid - 1) / grid : 0);
  }
  __device__ Seg seg(const PfUmmaParams& p, int j) const {
    const int b = blockIdx.x, grid = gridDim.x;
    Seg s;
    if (j < R * p.nblk) {
      s.tile = b + (j / p.nblk) * grid;
      s.blk = j % p.nblk;
      s.k0 = 0;
      s.k1 = p.KC;
      s.partial = false;
    } else {
      const int t = b + (j - R * p.nblk) * grid;
      const int tu = t / p.split, part = t % p.split;
      s.tile = R * grid + tu / p.nblk;
      s.blk = tu % p.nblk;
      s.k0 = part * p.KC / p.split;
      s.k1 = (part + 1) * p.KC / p.split;
      s.partial = p.split > 1;
    }
    return s;
  }
};

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
      mbar_init(&acc_empty[a], kEpiThreads);
    }
    mbar_fence_init();
  }
  tc_fence_before_sync();
  __syncthreads();
  tc_fence_after_sync();
  const uint32_t tm = tbase;
  const WsWork W(p);
  float sa, inv_sa;
  a_scale<Op>(p, sa, inv_sa);
  const int nseg = W.nseg;
  int err = 0;

  if (warp == kProducerWarp) {
    // producer: lane 0 keeps B operand stages up to kStages chunks ahead of
    // the MMAs and, for the f16x3 kind (two stages of 96 KB), asks L2 for the
    // B blocks kPrefetch chunks ahead
    const size_t blk_bytes = (size_t)p.KC * S::B_BLOCK;
    const unsigned char* Bg = static_cast<const unsigned char*>(p.B);
    auto b_block = [&](const Seg& sg, int kc, int bin) {
      const int2 i01 = p.tile_i01[sg.tile];
      const int b = bin ? i01.y : i01.x;
      return Bg + ((size_t)b * p.nblk + sg.blk) * blk_bytes + (size_t)kc * S::B_BLOCK;
    };
    // prefetch cursor: kPrefetch chunks ahead of the copies
    constexpr int kPrefetch = 2 * kStages;
    int pj = 0, pk = 0;
    Seg ps{};
    if (nseg > 0) {
      ps = W.seg(p, 0);
      pk = ps.k0;
    }
    auto advance = [&]() {
      if (pj >= nseg) return;
      if (++pk >= ps.k1 && ++pj < nseg) {
        ps = W.seg(p, pj);
        pk = ps.k0;
      }
    };
    for (int i = 0; i < kPrefetch; ++i) advance();
    int g = 0;
    for (int j = 0; j < nseg && !err; ++j) {
      const Seg sg = W.seg(p, j);
      for (int kc = sg.k0; kc < sg.k1; ++kc, ++g) {
        const int s = g % kStages, r = g / kStages;
        if (lane == 0) {
          if (r >= 1 && !mbar_spin_bounded(&empty[s], (r - 1) & 1, kWaitLimit)) err = 1;
          if (!err) {
            unsigned char* b = stage(s) + S::B_OFF;
            mbar_arrive_expect_tx(&full_b[s], 2 * S::B_BLOCK);
            bulk_load(b, b_block(sg, kc, 0), S::B_BLOCK, &full_b[s]);
            bulk_load(b + S::B_BLOCK, b_block(sg, kc, 1), S::B_BLOCK, &full_b[s]);
            if (Op::kPrefetchB && pj < nseg) {
              bulk_prefetch_l2(b_block(ps, pk, 0), S::B_BLOCK);
              bulk_prefetch_l2(b_block(ps, pk, 1), S::B_BLOCK);
            }
          }
        }
        advance();
        err = __shfl_sync(0xffffffffu, err, 0);
        if (err) break;
      }
    }
  } else if (warp == kMmaWarp) {
    // MMA issue
    if (lane == 0) {
      const uint32_t idesc = Op::idesc(S::N);
      int g = 0;
      for (int j = 0; j < nseg && !err; ++j) {
        const Seg sg = W.seg(p, j);
        const int a = j & 1;
        for (int kc = sg.k0; kc < sg.k1; ++kc, ++g) {
          const int s = g % kStages, r = g / kStages;
          if (kc == sg.k0 && j >= 2 && !mbar_spin_bounded(&acc_empty[a], ((j - 2) >> 1) & 1, kWaitLimit)) err = 1;
          if (!err && !mbar_spin_bounded(&full_b[s], r & 1, kWaitLimit)) err = 1;
          if (!err && !mbar_spin_bounded(&full_a[s], r & 1, kWaitLimit)) err = 1;
          if (err) break;
          tc_fence_after_sync();
          mma_chunk<Op, Db>(tm + (uint32_t)(a * S::ACC_COLS), idesc, stage(s), kc == sg.k0);
          umma_commit(&empty[s]);
          if (kc == sg.k1 - 1) umma_commit(&acc_full[a]);
        }
      }
    }
  } else if (warp >= kEpiWarp0) {
    // epilogue: warp w reads TMEM lane quarter w % 4 (thread = tile row) and
    // writes every depth of its row; runs beside the next segment's MMAs
    const int row = 32 * (warp & 3) + lane;
    for (int j = 0; j < nseg; ++j) {
      const Seg sg = W.seg(p, j);
      const int a = j & 1;
      if (!mbar_spin_bounded(&acc_full[a], (j >> 1) & 1, kWaitLimit)) {
        err = 1;
        break;
      }
      tc_fence_after_sync();
      int pix = p.tile_pix[(size_t)sg.tile * kUmmaTile + row];
      if (pix >= 0 && !bchk((long long)pix * p.D + p.D - 1, p.C_n, p.err)) pix = -1;   // the row must lie in C
      const float ac = p.tile_acut[(size_t)sg.tile * kUmmaTile + row];
      Out* crow = static_cast<Out*>(p.C) + (size_t)(pix >= 0 ? pix : 0) * p.D + (size_t)sg.blk * Db;
      epilogue_cols<Op, Db>(tm + (uint32_t)(a * S::ACC_COLS), warp, pix, p.scale * inv_sa * ac, crow, sg.blk, p.D, 0, Db,
                            sg.partial);
      tc_fence_before_sync();
      mbar_arrive(&acc_empty[a]);
    }
  } else {
    // builders: A stages. A builder touches kIters rows: their pixel and
    // weight are held in registers per segment, and the next chunk's phasors
    // are loaded before the current chunk is stored
    const int t = tid;
    const In* Ph = static_cast<const In*>(p.Phat);
    int rp[A::kIters];
    float ra[A::kIters];
    auto load_rows = [&](int tl) {
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
        h[i] = (rp[i] >= 0 && f < p.F && bchk((long long)rp[i] * p.F + f, p.Phat_n, p.err))
                   ? Ph[(size_t)rp[i] * p.F + f] : Op::zero();
      }
    };
    In hc[A::kIters], hn[A::kIters];
    if (nseg > 0) {
      const Seg s0 = W.seg(p, 0);
      load_rows(s0.tile);
      load_h(hc, s0.k0);
    }
    int g = 0;
    for (int j = 0; j < nseg && !err; ++j) {
      const Seg sg = W.seg(p, j);
      for (int kc = sg.k0; kc < sg.k1; ++kc, ++g) {
        const int s = g % kStages, r = g / kStages;
        if (r >= 1 && !mbar_spin_bounded(&empty[s], (r - 1) & 1, kWaitLimit)) {
          err = 1;
          break;
        }
#pragma unroll
        for (int i = 0; i < A::kIters; ++i) {
          int rr, q;
          A::coords(i, t, rr, q);
          A::put(stage(s), rr, q, Op::load(hc[i]), ra[i], sa);
        }
        fence_proxy_async_smem();
        mbar_arrive(&full_a[s]);
        // next chunk (of this segment or the next one) in flight
        if (kc + 1 < sg.k1) {
          load_h(hn, kc + 1);
        } else if (j + 1 < nseg) {
          const Seg nx = W.seg(p, j + 1);
          load_rows(nx.tile);
          load_h(hn, nx.k0);
        }
#pragma unroll
        for (int i = 0; i < A::kIters; ++i) hc[i] = hn[i];
      }
    }
  }
  if (err && p.err) atomicExch(p.err, kDevErrTmaTimeout);
  // on success every MMA has completed once the epilogue warps saw the last
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
  int pix = p.tile_pix[(size_t)tile * kUmmaTile + row];
  if (pix >= 0 && !bchk((long long)pix * p.D + p.D - 1, p.C_n, p.err)) pix = -1;   // the row must lie in C
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
      h[i] = (px >= 0 && f < p.F && bchk((long long)px * p.F + f, p.Phat_n, p.err)) ? Ph[(size_t)px * p.F + f]
                                                                                      : Op::zero();
    }
  };
  In hcur[A::kIters], hnext[A::kIters];
  load_h(hcur, 0);
  float sa, inv_sa;
  a_scale<Op>(p, sa, inv_sa);
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
        A::put(um_sm, r, q, Op::load(hcur[i]), salpha[r], sa);
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
    if (Db >= 32) epilogue_cols<Op, Db>(dt, warp, pix, p.scale * inv_sa * ac, crow, blk, p.D, half * (Db / 2), Db / 2);
    else if (half == 0) epilogue_cols<Op, Db>(dt, warp, pix, p.scale * inv_sa * ac, crow, blk, p.D, 0, Db);
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
// f16 kind: one part, the scaled value; f16x3 kind: parts hi = f16(v),
// lo = f16(v - hi) of the scaled value.
template <class Op>
__global__ void kr_store_umma_kernel(const double2* K64, unsigned char* B, int n_rho, int F, int D, int Db, int nblk,
                                     int KC, double scale) {
  constexpr int kCols = Op::kRowBytes / Op::kElem;
  const long long N = 2LL * Db;
  const long long per_chunk = N * kCols;
  const long long total = (long long)n_rho * nblk * KC * per_chunk;
  const size_t part_bytes = (size_t)N * Op::kRowBytes;
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
    // element (n, kj) of a kRowBytes-row operand: core matrix (n / 8, byte column / 16)
    const int bc = kj * Op::kElem;
    const size_t off = ((size_t)(n >> 3) * (Op::kRowBytes / 16) + (bc >> 4)) * 128 + (n & 7) * 16 + (bc & 15);
    unsigned char* base = B + (size_t)chunk * Op::kParts * part_bytes;
    if (Op::kKind == kUmmaF16) {
      *reinterpret_cast<__half*>(base + off) = __double2half(v * scale);
    } else {
      const __half hi = __double2half(v * scale);
      *reinterpret_cast<__half*>(base + off) = hi;
      *reinterpret_cast<__half*>(base + part_bytes + off) = __double2half(v * scale - (double)__half2float(hi));
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

int sm_count() {
  static int sms = 0;
  if (sms == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (sms <= 0) sms = 1;
  }
  return sms;
}

// Grid and split of the persistent schedule: one CTA per SM; the tiles left
// after the last full round have their units split along the frequency sum
// (at most kMaxSplit parts, at most KC) so that idle CTAs share them.
struct WsShape {
  int grid, split, first_split_tile;
};
WsShape ws_shape(const PfUmmaParams& p) {
  const int sms = sm_count();
  const int units = p.ntiles * p.nblk;
  const int full = p.ntiles / sms;
  const int tail_units = (p.ntiles - full * sms) * p.nblk;
  int split = tail_units > 0 ? sms / tail_units : 1;
  split = split < 1 ? 1 : split > kMaxSplit ? kMaxSplit : split;
  if (split > p.KC) split = p.KC;
  WsShape w;
  w.grid = full > 0 ? sms : (units * split < sms ? units * split : sms);
  const int R = p.ntiles / w.grid;                     // full rounds the kernel runs
  w.split = R * w.grid == p.ntiles ? 1 : split;        // every tile whole: no tail
  w.first_split_tile = w.split > 1 ? R * w.grid : p.ntiles;
  return w;
}

template <class Op, int Db>
cudaError_t launch_ws(const PfUmmaParams& p, cudaStream_t s) {
  constexpr uint32_t smem = Sizes<Op, Db>::STAGES * Sizes<Op, Db>::STAGE;
  auto k = pf_umma_ws_kernel<Op, Db>;
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  const WsShape w = ws_shape(p);
  PfUmmaParams q = p;
  q.split = w.split;
  k<<<w.grid, kWsThreads, smem, s>>>(q);
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

int pf_umma_first_split_tile(const PfUmmaParams& p) {
  if (p.ntiles <= 0) return 0;
  return ws_shape(p).first_split_tile;
}

cudaError_t launch_pf_umma(const PfUmmaParams& p, bool pipelined, cudaStream_t s) {
  if (p.ntiles <= 0) return cudaSuccess;
  if (p.kind == kUmmaF16) return launch_kind<OpF16>(p, pipelined, s);
  if (p.kind == kUmmaF16x3) return launch_kind<OpF16x3>(p, pipelined, s);
  return cudaErrorInvalidValue;
}

cudaError_t launch_kr_store_umma(const double2* K64, void* B, int kind, int n_rho, int F, int D, int Db, int nblk,
                                 int KC, double scale, cudaStream_t s) {
  unsigned char* b = static_cast<unsigned char*>(B);
  if (kind == kUmmaF16)
    kr_store_umma_kernel<OpF16><<<152 * 8, 256, 0, s>>>(K64, b, n_rho, F, D, Db, nblk, KC, scale);
  else if (kind == kUmmaF16x3)
    kr_store_umma_kernel<OpF16x3><<<152 * 8, 256, 0, s>>>(K64, b, n_rho, F, D, Db, nblk, KC, scale);
  else
    return cudaErrorInvalidValue;
  return cudaGetLastError();
}

}  // namespace nlos
