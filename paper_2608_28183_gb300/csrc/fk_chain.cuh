// f-k lateral transforms, fused in pairs (Sec. 4.2, Alg. 1):
//   forward: the real-input x transform (kx in [0, L/2]) and the y transform
//            of the scaled, zero-padded transient (FK1);
//   inverse: the y transform (keep y < b) and the x transform with the crop
//            and |.|^2 (FK4).
// The intermediate of each pair (x-transformed transient, y-inverted
// spectrum) stays in L2. One persistent kernel walks a ticket queue of work
// items over chunks of 16 consecutive t (or z) columns; the second
// transform's items of chunk c need every first-transform item of chunk c.
// Tickets go first(0), first(1), second(0), first(2), second(1), ..., so an
// item only ever depends on items whose tickets were taken before it.
//
// Each item is one or two sub-tiles of IC = 8 columns. Sub-tiles stream
// through two or three shared-memory slots: a producer warp takes the tickets, waits
// for chunk counters and issues the TMA copy of the next sub-tile while the
// other warps transform the current one (the scalar Stockham core of
// nlos_fft.cuh with radix-32 passes, 32 values per thread, in place in the
// slot).
//
// The intermediate of a chunk (about 8 MB at 256 x 256) is read within a few
// microseconds of being written; once its TMA copies have landed, its L2
// lines are dropped without write-back (discard.global.L2; float32 storage,
// where a chunk row is one 128-byte line), so it never reaches DRAM.
#pragma once
#include "axis_fft.cuh"
#include "nlos_bounds.cuh"
#include "nlos_internal.h"
#include "nlos_tma.cuh"

namespace nlos {

constexpr int kChainIC = 8;                // columns per sub-tile
constexpr int kChainE = 32;                // values per thread (radix-32 passes)
constexpr int kChainCols = 2 * kChainIC;   // columns (t or z values) per chunk and item
constexpr int kChainWaitLimit = 1 << 18;   // polls of a chunk counter (~0.1 s with the back-off; below the ~1 s slot waits)

__device__ __forceinline__ int ld_acquire(const int* p) {
  int v;
  asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void l2_discard(const void* p) {
  asm volatile("discard.global.L2 [%0], 128;" ::"l"(p) : "memory");
}
// make global data this thread has acquired visible to its later async-proxy (TMA) reads
__device__ __forceinline__ void fence_proxy_async_global() { asm volatile("fence.proxy.async.global;" ::: "memory"); }
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// ticket order with a lag of D chunks (1 <= D <= nchunks):
//   first(0 .. D-1) | first(c + D), second(c) for c < nchunks - D | second(nchunks - D .. nchunks - 1)
// D is chosen so that the tickets between a chunk's last first-transform
// item and its first second-transform item exceed the CTAs in flight: by the
// time a CTA takes second(c), the items of first(c) are normally finished.
struct ChainItem {
  int second;   // 0: first-transform item, 1: second-transform item
  int chunk, idx;
};
__device__ __forceinline__ ChainItem chain_decode(int t, int n1, int n2, int nchunks, int D) {
  if (t < D * n1) return {0, t / n1, t % n1};
  t -= D * n1;
  const int blk = t / (n1 + n2), off = t % (n1 + n2);
  if (blk < nchunks - D) return off < n1 ? ChainItem{0, blk + D, off} : ChainItem{1, blk, off - n1};
  t -= (nchunks - D) * (n1 + n2);
  return {1, nchunks - D + t / n2, t % n2};
}

// per-slot description of the sub-tile in it (written by the producer before
// the slot's full barrier completes)
struct ChainSlot {
  int state;   // 0: loaded, 1: no more work, 2: skipped (a dependency wait ran out)
  int ticket, sub;
};

template <int L, int NSLOT = 2> struct ChainTile {
  static constexpr int CONSUMERS = kChainIC * (L / kChainE);   // threads that transform
  static constexpr int THREADS = CONSUMERS + 32;               // + the producer warp
  static constexpr size_t BUF = sizeof(float2) * FftShape<L, kChainE>::SMEM * kChainIC;   // multiple of 128 bytes
  static constexpr size_t TW = sizeof(float2) * FftShape<L, kChainE>::TWSIZE;   // the twiddle table's copy
  static constexpr size_t SMEM = NSLOT * BUF + TW + 2 * NSLOT * sizeof(uint64_t) + NSLOT * sizeof(ChainSlot);
  // resident CTAs per SM the register budget is held to (what shared memory allows at L = 512)
  static constexpr int MIN_BLOCKS = L <= 512 ? (NSLOT == 2 ? 3 : 2) : 1;
  // the consumers' named barrier counts whole warps
  static_assert(CONSUMERS % 32 == 0, "consumer threads must be whole warps");
};

// transform contexts of the consumer threads: their barriers are named
// barrier 1 over the consumers only
// (the kernel keeps a copy of the twiddle table in shared memory: its data
// slots take most of the SM's shared memory, leaving little L1 for the
// table's global reads)
template <int L, int IC, int LD, int ST, class TS>
struct ChainTmaCtx : AxisTmaCtx<L, IC, LD, ST, TS> {
  static constexpr int kBarThreads = ChainTile<L>::CONSUMERS;
  static constexpr bool kTwShared = true;
};
template <int L, int IC, class TS>
struct ChainTmaPairCtx : AxisTmaPairCtx<L, IC, TS> {
  static constexpr int kBarThreads = ChainTile<L>::CONSUMERS;
  static constexpr bool kTwShared = true;
  __device__ __forceinline__ void store(int l, const float2 (&x)[1]) const {
    this->smem[padE<kChainE>(l) * IC + this->c] = x[0];
  }
};
// y inverse of the inverse chain: stores the intermediate with an L2
// evict-last policy (it is read back within microseconds, then dropped)
template <int L, int IC, class TS>
struct ChainMidCtx : AxisTmaCtx<L, IC, kLoadCpx, kStoreCpx, TS> {
  static constexpr int kBarThreads = ChainTile<L>::CONSUMERS;
  static constexpr bool kTwShared = true;
  uint64_t keep;
  __device__ __forceinline__ void store(int l, const float2 (&x)[1]) const {
    if (l >= this->L_out) return;
    if (!bchk(this->out_base + l * this->out_axis, this->out_n, this->err)) return;
    const float2 v = make_float2(x[0].x * this->stmul, -x[0].y * this->stmul);   // inverse: conjugate
    TS* o = static_cast<TS*>(this->out) + this->out_base + l * this->out_axis;
    if constexpr (sizeof(TS) == 8) st_global_hint(reinterpret_cast<float2*>(o), v, keep);
    else Cpx<TS>::put(o, v);
  }
};

// the second transform of either chain: its output is not read again while
// the chain runs, so it is stored evict-first and leaves L2 to the intermediate
template <int L, int IC, int ST, class TS>
struct ChainOutCtx : ChainTmaCtx<L, IC, kLoadCpx, ST, TS> {
  uint64_t stream;
  __device__ __forceinline__ void store(int l, const float2 (&x)[1]) const {
    float2 v = x[0];
    if (!this->valid || l >= this->L_out) return;
    const long long o = this->out_base + l * this->out_axis;
    if (!bchk(o, this->out_n, this->err)) return;
    if constexpr (ST == kStoreAbs2) {
      st_global_hint(static_cast<float*>(this->out) + o, fmaf(v.x, v.x, v.y * v.y) * this->stmul, stream);
    } else {
      if (this->inverse) v = cconj(v);
      v = cscale(v, this->stmul);
      if constexpr (ST == kStoreCpx32 || sizeof(TS) == 8) st_global_hint(static_cast<float2*>(this->out) + o, v, stream);
      else Cpx<TS>::put(static_cast<TS*>(this->out) + o, v);
    }
  }
};

template <int L> __device__ __forceinline__ void consumer_sync() {
  asm volatile("bar.sync 1, %0;" ::"r"(ChainTile<L>::CONSUMERS) : "memory");
}

// common fields of a staged complex sub-tile's transform context
template <class Ctx>
__device__ __forceinline__ void chain_ctx(Ctx& ctx, float2* slot, const float2* tw, int c, int inverse) {
  ctx.tile = slot;
  ctx.smem = slot;
  ctx.tw = tw;
  ctx.in = nullptr;
  ctx.c = c;
  ctx.valid = true;
  ctx.in_base = 0;
  ctx.in_axis = 0;
  ctx.inverse = inverse;
  ctx.t_len = 0;
  ctx.ldmul = 1.0f;
  ctx.tmul = 1.0f;
  ctx.in_n = 0;   // the staged tile is read from shared memory
}

// Forward (kFwd) and inverse chains. Per chunk: forward n1 = b x items (one
// wall row y, 16 real t columns, one sub-tile: columns c and c + 8 ride as one
// complex transform) and n2 = L/2 + 1 y items (one kx, two sub-tiles of 8
// complex columns); inverse n1 = L y items (one kx) and n2 = b x items (one
// y), two sub-tiles each.
// map1 / map2: tensor maps of the first / second transform's input.
//
// Warp roles: warps 0 .. CONSUMERS/32 - 1 transform sub-tiles; the last warp
// (one elected lane) takes tickets, waits for chunk counters and issues the
// TMA copies, running up to NSLOT sub-tiles ahead. Per slot a full barrier
// (producer arrival + copy bytes) and an empty barrier (one arrival once no
// consumer touches the slot any more). The producer only
// ever waits for empty slots (the consumers release them without waiting on
// the producer) and for first-transform items of a chunk, all of which were
// issued before (by this or another CTA) and need nothing but their
// consumers: the kernel cannot deadlock, and every wait is bounded.
template <int L, class TS, bool kFwd, int ST, int NSLOT>
__global__ void __launch_bounds__(ChainTile<L, NSLOT>::THREADS, ChainTile<L, NSLOT>::MIN_BLOCKS)
fk_chain_kernel(const __grid_constant__ CUtensorMap map1, const __grid_constant__ CUtensorMap map2,
                const FkChainParams p) {
  using T = ChainTile<L, NSLOT>;
  using TR = typename RealOf<TS>::T;
  constexpr int IC = kChainIC;
  constexpr int E = kChainE;
  constexpr int TPC = L / E;
  extern __shared__ __align__(128) unsigned char cs[];
  auto buf = [&](int slot) { return reinterpret_cast<float2*>(cs + slot * T::BUF); };
  float2* tw = reinterpret_cast<float2*>(cs + NSLOT * T::BUF);
  uint64_t* full = reinterpret_cast<uint64_t*>(cs + NSLOT * T::BUF + T::TW);
  uint64_t* empty = full + NSLOT;
  ChainSlot* desc = reinterpret_cast<ChainSlot*>(cs + NSLOT * T::BUF + T::TW + 2 * NSLOT * sizeof(uint64_t));
  const int hx = L / 2 + 1;
  const int n1 = kFwd ? p.b : L;
  const int n2 = kFwd ? hx : p.b;
  const int total = p.nchunks * (n1 + n2);
  const long long bn = (long long)p.b * p.n;
  int* done = p.sync + 1;
  auto subs_of = [&](const ChainItem& it) { return (kFwd && !it.second) ? 1 : 2; };

  if (threadIdx.x == 0) {
    for (int i = 0; i < NSLOT; ++i) {
      mbar_init(&full[i], 1);
      mbar_init(&empty[i], 1);
    }
    mbar_fence_init();
  }
  for (int i = threadIdx.x; i < FftShape<L, kChainE>::TWSIZE; i += T::THREADS) tw[i] = __ldg(p.tw + i);
  __syncthreads();

  if (threadIdx.x >= T::CONSUMERS) {
    // ------------------------------ producer ------------------------------
    if (threadIdx.x != T::CONSUMERS) return;
    // the inverse's input spectrum is read once: keep L2 for the intermediate
    const uint64_t once = l2_policy_evict_first();
    int t = -1, sub = 0;
    for (int k = 0;; ++k) {
      const int slot = k % NSLOT;
      if (k >= NSLOT && !mbar_wait_bounded(&empty[slot], ((k / NSLOT) - 1) & 1, kTmaWaitLimit)) {
        if (p.err) atomicExch(p.err, kDevErrTmaTimeout);
        return;
      }
      // next sub-tile: the rest of the current item, or a new ticket
      if (t >= 0 && t < total && sub + 1 < subs_of(chain_decode(t, n1, n2, p.nchunks, p.lag))) {
        ++sub;
      } else {
        t = atomicAdd(p.sync, 1);
        sub = 0;
      }
      ChainSlot& d = desc[slot];
      d.ticket = t;
      d.sub = sub;
      if (t >= total) {
        d.state = 1;
        mbar_arrive(&full[slot]);
        return;
      }
      const ChainItem it = chain_decode(t, n1, n2, p.nchunks, p.lag);
      if (it.second && sub == 0) {
        int ok = 1, n = 0;
        while (ld_acquire(done + it.chunk) < n1) {
          if (++n > kChainWaitLimit) {
            ok = 0;
            if (p.err) atomicExch(p.err, kDevErrChainTimeout);
            break;
          }
          __nanosleep(32);
        }
        if (!ok) {
          d.state = 2;
          mbar_arrive(&full[slot]);
          continue;
        }
        fence_proxy_async_global();
      }
      d.state = 0;
      const bool xreal = kFwd && !it.second;
      const int rows = kFwd ? (it.second ? p.b : p.a) : L;
      const size_t row_bytes = (size_t)IC * (xreal ? 2 * sizeof(TR) : sizeof(TS));
      mbar_arrive_expect_tx(&full[slot], (uint32_t)(rows * row_bytes));
      for (int r0 = 0; r0 < rows; r0 += 256) {
        unsigned char* dst = reinterpret_cast<unsigned char*>(buf(slot)) + (size_t)r0 * row_bytes;
        if (xreal)
          tma_load_3d(dst, &map1, &full[slot], it.idx * p.n + it.chunk * kChainCols, r0, 0);
        else if (it.second)
          tma_load_3d(dst, &map2, &full[slot], it.chunk * kChainCols + sub * IC, r0, it.idx);
        else
          tma_load_3d_hint(dst, &map1, &full[slot], it.chunk * kChainCols + sub * IC, r0, it.idx, once);
      }
    }
  }

  // ------------------------------ consumers ------------------------------
  const uint64_t keep = l2_policy_evict_last();
  const uint64_t once = l2_policy_evict_first();
  const int c = threadIdx.x % IC;
  const int j0 = threadIdx.x / IC;
  const float ldm = p.ld_dev_scale ? *p.ld_dev_scale : 1.0f;
  const float std_ = p.st_dev_scale ? *p.st_dev_scale : 1.0f;
  for (int k = 0;; ++k) {
    const int slot = k % NSLOT;
    if (!mbar_wait_bounded(&full[slot], (k / NSLOT) & 1, kTmaWaitLimit)) {
      if (p.err) atomicExch(p.err, kDevErrTmaTimeout);
      return;   // (the producer gives up on its empty waits the same way)
    }
    const ChainSlot d = desc[slot];
    if (d.state == 1) break;
    const ChainItem it = chain_decode(d.ticket, n1, n2, p.nchunks, p.lag);
    const int nsubs = subs_of(it);
    if (d.state == 0) {
      const int col0 = it.chunk * kChainCols + d.sub * IC;
      // drop the consumed intermediate from L2: both sub-tiles of this
      // second-transform item have landed
      if (p.discard && it.second && d.sub == nsubs - 1) {
        const int nl = kFwd ? p.b : L;
        const float2* base = static_cast<const float2*>(p.mid) + (long long)it.chunk * kChainCols;
        for (int r = threadIdx.x; r < nl; r += T::CONSUMERS) {
          const long long o = (long long)it.chunk * kChainCols +
                              (kFwd ? (long long)it.idx * bn + (long long)r * p.n : (long long)r * bn + (long long)it.idx * p.n);
          if (bchk(o + kChainCols - 1, p.mid_n, p.err)) l2_discard(base + (o - (long long)it.chunk * kChainCols));
        }
      }
      if (kFwd && !it.second) {
        // x forward of wall row y = idx: 16 real columns t0 + c, t0 + c + 8
        const int t0 = it.chunk * kChainCols;
        ChainTmaPairCtx<L, IC, TS> ctx;
        ctx.tile = reinterpret_cast<const TR*>(buf(slot));
        ctx.smem = buf(slot);
        ctx.tw = tw;
        ctx.L_in = p.a;
        ctx.c = c;
        ctx.m0 = p.t_scale != 0.f ? ldm * (float)(t0 + c) * p.t_scale : ldm;
        ctx.m1 = p.t_scale != 0.f ? ldm * (float)(t0 + c + IC) * p.t_scale : ldm;
        fftn_run<L, 1, true, false, ChainTmaPairCtx<L, IC, TS>, E>(ctx, j0);
        consumer_sync<L>();
        // split the two real columns: X_c[k] = (Z[k] + conj Z[L-k]) / 2,
        // X_{c+8}[k] = (Z[k] - conj Z[L-k]) / (2i), k in [0, L/2]
        const float h = 0.5f * p.s1;
        const float2* z = buf(slot);
        const long long oo = (long long)it.idx * p.n + t0 + c;
        TS* o0 = static_cast<TS*>(p.mid) + oo;
        for (int q = j0; q < hx; q += TPC) {
          const float2 zk = z[padE<E>(q) * IC + c];
          const float2 zm = z[padE<E>((L - q) & (L - 1)) * IC + c];
          TS* o = o0 + q * bn;
          if (bchk(oo + q * bn + IC, p.mid_n, p.err)) {
            Cpx<TS>::put(o, make_float2((zk.x + zm.x) * h, (zk.y - zm.y) * h));
            Cpx<TS>::put(o + IC, make_float2((zk.y + zm.y) * h, (zm.x - zk.x) * h));
          }
        }
      } else if (kFwd) {
        // y forward of kx = idx: rows y < b, all L outputs (stored evict-first:
        // the spectrum is read by the next stage, after this one)
        ChainOutCtx<L, IC, kStoreCpx, TS> ctx;
        chain_ctx(ctx, buf(slot), tw, c, 0);
        ctx.stream = once;
        ctx.out = p.out;
        ctx.out_n = p.out_n;
        ctx.err = p.err;
        ctx.out_base = (long long)it.idx * L * p.n + col0 + c;
        ctx.out_axis = p.n;
        ctx.L_in = p.b;
        ctx.L_out = L;
        ctx.stmul = p.s2;
        fftn_run<L, 1, true, false, ChainOutCtx<L, IC, kStoreCpx, TS>, E>(ctx, j0);
      } else if (!it.second) {
        // y inverse of kx = idx: keep y < b
        ChainMidCtx<L, IC, TS> ctx;
        chain_ctx(ctx, buf(slot), tw, c, 1);
        ctx.keep = keep;
        ctx.out = p.mid;
        ctx.out_n = p.mid_n;
        ctx.err = p.err;
        ctx.out_base = (long long)it.idx * bn + col0 + c;
        ctx.out_axis = p.n;
        ctx.L_in = L;
        ctx.L_out = p.b;
        ctx.stmul = p.s1;
        fftn_run<L, 1, false, true, ChainMidCtx<L, IC, TS>, E>(ctx, j0);
      } else {
        // x inverse of wall row y = idx: keep x < a, |.|^2 (or complex)
        ChainOutCtx<L, IC, ST, TS> ctx;
        chain_ctx(ctx, buf(slot), tw, c, 1);
        ctx.stream = once;
        ctx.out = p.out;
        ctx.out_n = p.out_n;
        ctx.err = p.err;
        ctx.out_base = (long long)it.idx * p.n + col0 + c;
        ctx.out_axis = bn;
        ctx.L_in = L;
        ctx.L_out = p.a;
        ctx.stmul = p.s2 * std_;
        fftn_run<L, 1, false, true, ChainOutCtx<L, IC, ST, TS>, E>(ctx, j0);
      }
    }
    // no consumer touches the slot any more: order the shared-memory
    // accesses before the next copy into it and release it; a finished
    // first-transform item also publishes its stores
    consumer_sync<L>();
    if (threadIdx.x == 0) {
      fence_proxy_async_smem();
      mbar_arrive(&empty[slot]);
      if (!it.second && d.sub == nsubs - 1) {
        __threadfence();
        atomicAdd(done + it.chunk, 1);
      }
    }
  }
}

template <int L, class TS, int NSLOT>
cudaError_t launch_fk_chain_one(const FkChainLaunch& l, cudaStream_t s) {
  using T = ChainTile<L, NSLOT>;
  const FkChainParams& p = l.p;
  void (*k)(const __grid_constant__ CUtensorMap, const __grid_constant__ CUtensorMap, const FkChainParams) =
      l.fwd ? fk_chain_kernel<L, TS, true, kStoreCpx, NSLOT>
            : l.store_mode == kStoreCpx32 ? fk_chain_kernel<L, TS, false, kStoreCpx32, NSLOT>
            : l.store_mode == kStoreCpx   ? fk_chain_kernel<L, TS, false, kStoreCpx, NSLOT>
                                          : fk_chain_kernel<L, TS, false, kStoreAbs2, NSLOT>;
  // one persistent CTA per resident slot (occupancy queried once per kernel)
  static void* known[4] = {};
  static int slots[4] = {};
  const int key = l.fwd ? 0 : (l.store_mode == kStoreCpx32 ? 2 : l.store_mode == kStoreCpx ? 3 : 1);
  if (known[key] != (void*)k) {
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)T::SMEM);
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 0, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k, T::THREADS, T::SMEM);
    if (e != cudaSuccess) return e;
    slots[key] = sms * (per < 1 ? 1 : per);
    known[key] = (void*)k;
  }
  const int per_chunk = l.fwd ? (p.b + L / 2 + 1) : (L + p.b);
  const long long items = (long long)p.nchunks * per_chunk;
  const int grid = (int)(items < slots[key] ? items : slots[key]);
  FkChainParams q = p;
  q.lag = 1 + (grid + per_chunk - 1) / per_chunk;
  if (q.lag > q.nchunks) q.lag = q.nchunks;
  k<<<grid, T::THREADS, T::SMEM, s>>>(l.map1, l.map2, q);
  return cudaGetLastError();
}

// Each translation unit instantiates one storage type.
template <class TS>
cudaError_t launch_fk_chain_typed(const FkChainLaunch& l, cudaStream_t s) {
  const bool three = l.nslot == 3;
  switch (l.p.L) {
    case 128: return three ? launch_fk_chain_one<128, TS, 3>(l, s) : launch_fk_chain_one<128, TS, 2>(l, s);
    case 256: return three ? launch_fk_chain_one<256, TS, 3>(l, s) : launch_fk_chain_one<256, TS, 2>(l, s);
    case 512: return three ? launch_fk_chain_one<512, TS, 3>(l, s) : launch_fk_chain_one<512, TS, 2>(l, s);
    case 1024: return launch_fk_chain_one<1024, TS, 2>(l, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace nlos
