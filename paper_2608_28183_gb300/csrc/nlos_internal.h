// Internal interfaces between the host plan code and the kernel files.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

namespace nlos {

// Element types of stored intermediates / inputs.
enum Storage : int { kF32 = 0, kF16 = 1, kBF16 = 2 };

// Load/store modes of the strided-axis FFT.
enum AxisLoad : int { kLoadReal = 0, kLoadCpx = 1, kLoadRealPair = 2 };
// kStoreCpx32 writes complex float32 whatever the storage type (complex volumes)
enum AxisStore : int { kStoreCpx = 0, kStoreAbs2 = 1, kStoreAbs = 2, kStoreCpx32 = 3 };

// FFT of length L along one axis of a [outer][L][inner] array (inner
// contiguous). Elements along the axis beyond L_in are zero; outputs with
// index >= L_out are not written. Strides are in elements of the stored type
// (complex elements for complex arrays).
struct AxisParams {
  const void* in;
  void* out;
  const float2* tw;            // twiddles of the plan for length L
  long long inner;
  long long in_outer, in_axis;
  long long out_outer, out_axis;
  int L_in, L_out;
  int inverse;                 // conjugate on load and on store
  float scale;                 // multiplies every stored value (|.|^2 and |.| included)
  const float* ld_dev_scale;   // optional device scalar multiplying loads
  const float* st_dev_scale;   // optional device scalar multiplying stores
  int t_len;                   // real loads: multiply by (inner index % t_len) * t_scale
  float t_scale;
  long long in_n, out_n;       // element extents of in / out (bounds-checked build; 0: unchecked)
  int* err;                    // device error word (bounds-checked build), may be null
};

struct AxisLaunch {
  AxisParams p;
  int tile;                    // launch-shape variant: column tile = tile % n, TMA staging = tile / n
  CUtensorMap tmap;            // input tensor map for TMA staging (valid if has_tmap)
  int has_tmap;
  int* err;                    // device error word (bounded-wait timeouts), may be null
  int L;
  long long n_outer;
  int storage;                 // element type of complex arrays (and of real input)
  int load_mode;               // AxisLoad
  int store_mode;              // AxisStore
};
cudaError_t launch_axis_fft(const AxisLaunch& l, cudaStream_t s);
// Column-tile variants per length (selected by AxisLaunch::tile; index 0 is
// the default, the autotuner may pick another).
__host__ __device__ constexpr int axis_ic(int L, int v) {
  return L <= 32 ? (v == 0 ? 32 : 64)
       : L <= 64 ? (v == 0 ? 32 : 16)
       : L <= 256 ? (v == 0 ? 16 : (v == 1 ? 8 : 32))
       : L <= 512 ? (v == 0 ? 8 : (v == 1 ? 4 : 16))
       : L <= 1024 ? (v == 0 ? 8 : 4)
       : (v == 0 ? 4 : 2);
}

// number of column-tile widths of the axis transform of length L; the launch
// shape variants are these widths, each with direct loads or TMA staging
__host__ __device__ constexpr int axis_ic_count(int L) { return (L >= 128 && L <= 512) ? 3 : 2; }
__host__ __device__ constexpr int axis_tile_count(int L) { return 2 * axis_ic_count(L); }
// error codes written to the device error word
constexpr int kDevErrTmaTimeout = 1;
constexpr int kDevErrChainTimeout = 2;    // a fused lateral stage gave up waiting for a chunk
constexpr int kDevErrBounds = 3;          // bounds-checked build: an index outside its buffer (access skipped)
// launch-shape variants of the f-k temporal stage of length L: 0-3 one pencil
// and its partner per thread group (two CTA sizes, with or without aliased
// buffers), 4 one warp per radix-32 transform (the pencils (kx, +-ky) and
// their partners in one CTA); the default at L = 1024 is 2
// (variant 4 exists for L = 1024 only: one transform of 32 values per thread is one warp)
__host__ __device__ constexpr int fk_tile_count(int L) { return L == 1024 ? 5 : 4; }
__host__ __device__ constexpr int fk_tile_default(int L) { return L == 1024 ? 2 : 0; }

// f-k temporal-frequency stage: forward length-2n FFT of each stored pencil
// G[kx][ky][0..n) (kx in [0, a], ky in [0, 2b)), Stolt resampling with the
// Jacobian and the Z > 0 mask, and inverse length-2n FFTs producing the pencil
// (kx, ky) and, for 0 < kx < a, its Hermitian partner (2a-kx, -ky), keeping
// z < n. Output psi[kx'][ky'][z] for kx' in [0, 2a).
struct FkZParams {
  const void* G;
  void* psi;
  const float2* tw;            // twiddles for the temporal length L
  const float2* tw32;          // twiddles of the radix-32 schedule for L (warp-per-transform variant)
  const float2* ax;            // [a_pad] float-float (hi, lo) of (L s_x p~ / a_pad)^2
  const float2* ay;            // [b_pad] float-float of (L s_y q~ / b_pad)^2
  int a_pad, b_pad, n;         // padded lateral lengths, time bins (pencil stride, kept outputs)
  int L;                       // temporal transform length (power of two)
  int pad;                     // 2: zero-padded (L >= 2n); 1: unpadded (L = n)
  long long npencils;          // (a_pad / 2 + 1) * b_pad
  float ld_scale;              // multiplies forward loads
  const float* ld_dev_scale;   // optional device scalar multiplying forward loads
  float st_scale;              // multiplies stored values
  float t_ramp;                // non-zero: forward loads also multiplied by t * t_ramp (the
                               // spectrum was taken without the t/(n-1) ramp; float32 only,
                               // launch shape 0 whatever `tile` asks)
  long long G_n, psi_n;        // element extents (bounds-checked build; 0: unchecked)
  int* err;                    // device error word (bounds-checked build), may be null
};
cudaError_t launch_fk_zstage(const FkZParams& p, int storage, int tile, cudaStream_t s);

// f-k with the inverse temporal transform last (fk_zsplit.cuh; L = 2n):
// FK3 without its inverses (psi receives the resampled spectra V[kx][ky][m],
// m < n) and FK5, the inverse temporal transform of the a x b kept pencils.
cudaError_t launch_fk_stolt(const FkZParams& p, int storage, int tile, cudaStream_t s);
struct FkZInvParams {
  const void* in;              // [npencils][n] the laterally inverted spectra (storage type), m < n = L/2
  void* out;                   // [npencils][n] float (|.|^2) or float2 (complex_out)
  const float2* tw;            // twiddles for L
  const float2* tw32;          // twiddles of the radix-32 schedule for L
  int L, n;
  long long npencils;          // a * b
  float scale;                 // normalisation (of |.|^2 or of the complex value)
  const float* dev_scale;      // optional device scalar multiplying scale (16-bit storage)
  int complex_out;
  long long in_n, out_n;       // element extents (bounds-checked build; 0: unchecked)
  int* err;                    // device error word (bounds-checked build), may be null
};
cudaError_t launch_fk_zinv(const FkZInvParams& p, int storage, int tile, cudaStream_t s);

// f-k lateral transforms fused in pairs (fk_chain.cuh):
//   forward: in = H [a][b][n] real, mid = [L/2 + 1][b][n], out = G [L/2 + 1][L][n]
//   inverse: in = psi [L][L][n], mid = [L][b][n], out = [a][b][n] float
//            (|.|^2), float2 (complex) or the storage type (complex, the
//            spectrum whose temporal inverse comes last)
struct FkChainParams {
  const void* in;
  void* mid;
  void* out;
  const float2* tw;            // twiddles for L
  int a, b, n, L;
  int nchunks;                 // n / 16
  int lag;                     // chunks between a chunk's first- and second-transform tickets (set by the launcher)
  float t_scale;               // forward: ramp factor 1/(n-1) (value * t * t_scale; 0: no ramp)
  float s1, s2;                // scales of the values the first / second transform stores
  const float* ld_dev_scale;   // forward: optional device scalar multiplying the input
  const float* st_dev_scale;   // inverse: optional device scalar multiplying the output
  int* sync;                   // [1 + nchunks] ints, zero at launch: ticket, finished first-transform items per chunk
  int* err;                    // device error word
  int discard;                 // drop consumed lines of `mid` from L2 (float32 storage)
  long long in_n, mid_n, out_n;  // element extents (bounds-checked build; 0: unchecked)
};
struct FkChainLaunch {
  FkChainParams p;
  CUtensorMap map1, map2;      // TMA maps of the first / second transform's input
  int fwd;                     // 1 forward, 0 inverse
  int store_mode;              // inverse: kStoreAbs2 or kStoreCpx32
  int nslot;                   // shared-memory slots per CTA (2 or 3; 2 at L = 1024)
};
cudaError_t launch_fk_chain(const FkChainLaunch& l, int storage, cudaStream_t s);
// zero-padded f-k with Lx = Ly = L in [128, 1024] (at least one warp of
// transforming threads per CTA), n a multiple of 16, and every TMA box row
// count (a, b, L) at most 256 or a multiple of it
inline bool fk_chain_eligible(int a, int b, int n, int Lx, int Ly, int pad) {
  auto rows_ok = [](int r) { return r <= 256 || r % 256 == 0; };
  return pad == 2 && Lx == Ly && Lx >= 128 && Lx <= 1024 && 2 * a <= Lx && 2 * b <= Ly && n % 16 == 0 && n >= 16 &&
         rows_ok(a) && rows_ok(b);
}

// Phasor-field temporal band transform: per wall pencil H[x][y][0..n) (real),
// length-n DFT, keep bins k_lo..k_lo+F-1, multiply by w(f): P[x][y][f].
struct PfBandParams {
  const void* H;
  void* P;
  const float2* tw;            // twiddles for L
  const float* w;              // [F]
  int n, k_lo, F;              // n: samples per pencil (stride of H)
  int L;                       // DFT length (power of two >= n; samples beyond n are zero)
  long long npencils;          // a * b
  float ld_scale;
  const float* ld_dev_scale;
  float st_scale;
  int accumulate;              // add to P instead of overwriting it
  unsigned* amax;              // when set: atomicMax of max |Re|, |Im| of the stored P (float bits)
  long long H_n, P_n;          // element extents (bounds-checked build; 0: unchecked)
  int* err;                    // device error word (bounds-checked build), may be null
};
cudaError_t launch_pf_band(const PfBandParams& p, int storage, cudaStream_t s);

// PF1 + PF2 from a lateral spectrum shared with f-k (mixture of experts,
// Sec. 4.4): G holds the x then y forward transforms of the transient,
// kx in [0, Lx/2], ky in [0, Ly), n samples per pencil (the f-k forward
// spectrum taken without its ramp). The temporal DFT Z of each pencil (length
// L >= n, zero beyond n) gives Phat(kx, ky, f) = w(f) Z(k_lo + f) and, for
// 0 < kx < Lx/2, the Hermitian partner of the real transient:
// Phat(Lx - kx, -ky, f) = w(f) conj(Z(L - k_lo - f)). Float32 only.
struct PfSpecParams {
  const float2* G;             // [Lx/2 + 1][Ly][n]
  float2* Phat;                // [Lx][Ly][F]
  const float2* tw;            // twiddles for L
  const float* w;              // [F]
  int n, L, k_lo, F, Lx, Ly;
  unsigned* amax;              // when set: atomicMax of max |Re|, |Im| of the stored Phat (float bits)
  long long G_n, Phat_n;       // element extents (bounds-checked build; 0: unchecked)
  int* err;                    // device error word (bounds-checked build), may be null
};
cudaError_t launch_pf_band_spectrum(const PfSpecParams& p, cudaStream_t s);

// Photon binning into the compact phasor field P[pixel][f] (float32 complex):
// P += w_f * exp(-2 pi i (k_lo + f) b / n) per kept photon.
struct PhasorBinParams {
  const uint32_t* pixel;
  const uint32_t* ticks;
  long long count;
  uint32_t npix;
  int nt, n;                   // time bins; phase table length (n == nt)
  uint32_t t0, tpb;
  const float2* phase;         // [n] exp(-2 pi i m / n)
  const float* w;              // [F]
  int k_lo, F;
  float2* P;
  int* err;                    // device error word (bounds-checked build), may be null
};
cudaError_t launch_bin_phasors(const PhasorBinParams& q, cudaStream_t s);
// photon records -> float32 histogram H[pixel][bin] (+= 1 per kept record)
cudaError_t launch_bin_transient(const uint32_t* pixel, const uint32_t* ticks, long long count, uint32_t npix,
                                 uint32_t nt, uint32_t t0, uint32_t tpb, float* H, cudaStream_t s);

// Phasor-field depth sum over pixel chunks sharing a radial index i0:
// C[pix][d] = acut * sum_f Phat[pix][f] * ((1 - alpha) K[i0][f][d] + alpha K[i1][f][d]).
constexpr int kPfChunk = 16;
struct PfDepthParams {
  const void* Phat;            // [Nu*Nv][F] complex (storage type)
  const void* K;               // [N_rho][F][D] complex (kernel storage type)
  void* C;                     // [Nu*Nv][D] complex (storage type)
  const int2* chunk_i01;       // [nchunks] (i0, i1)
  const int* chunk_pix;        // [nchunks][16] pixel index or -1
  const float* chunk_alpha;    // [nchunks][16]
  const float* chunk_acut;     // [nchunks][16]
  int nchunks, F, D;
  float scale;
  const float* dev_scale;      // optional device scalar multiplying C
};
cudaError_t launch_pf_depth(const PfDepthParams& p, int storage, int kernel_storage, cudaStream_t s);

// Plan-time kernel build in float64:
// K[i][f][d] = mod[f][d] * sum_j B[i][j] exp(i sigma_s kappa_f sqrt(r_j^2 + d^2))
struct KrBuildParams {
  const double* B;             // [n_rho][n_r] = q_j 2 pi r_j J0(2 pi r_j rho_i) (0 beyond cutoff)
  const double* r;             // [n_r]
  const double* kappa;         // [F]
  const double* depth;         // [D]
  int n_rho, n_r, F, D;
  double sigma_s, sigma_t, delta;
  double2* A;                  // scratch [n_r][F][D]
  double2* K64;                // out [n_rho][F][D]
};
cudaError_t launch_kr_build(const KrBuildParams& p, cudaStream_t s);
// Convert the float64 kernel to the stored type with a scale.
cudaError_t launch_kr_store(const double2* K64, void* K, long long count, int storage, double scale,
                            cudaStream_t s);

// Tensor-core depth sum: per tile of up to 128 pixels that share the radial
// pair (i0, i1), Y = A0 B(i0)^T + A1 B(i1)^T with A0 = (1 - alpha) [Re Phat |
// Im Phat], A1 = alpha [Re Phat | Im Phat] (built in shared memory) and B(i)
// the real form of K_r[i] ([Kr -Ki; Ki Kr], 2 Db output columns per depth
// block, stored per plan in the operand layout); C = scale * acut * (Y_re +
// i Y_im). Two operand kinds, both kind::f16 MMAs:
//  * kUmmaF16 (16-bit storage): f16 operands, one product;
//  * kUmmaF16x3 (float32 storage): every operand x split into f16 parts
//    x_hi = f16(x), x_lo = f16(x - x_hi), and A B^T taken as
//    A_hi B_hi^T + A_hi B_lo^T + A_lo B_hi^T (the dropped A_lo B_lo^T term is
//    ~2^-22 of the product), fp32 accumulation. A is scaled into f16 range by
//    a power of two derived from a bound on |Phat| (amax, abound_exp below),
//    B by the plan's power-of-two scale; the epilogue removes both.
// Operand rows per chunk: 64 bytes - 32 f16 columns (16 frequencies).
constexpr int kUmmaTile = 128;           // pixels per tile (MMA M)
enum UmmaKind { kUmmaF16 = 0, kUmmaF16x3 = 1 };
__host__ __device__ constexpr int umma_row_bytes(int) { return 64; }
__host__ __device__ constexpr int umma_chunk_cols(int) { return 32; }
__host__ __device__ constexpr int umma_parts(int kind) { return kind == kUmmaF16 ? 1 : 2; }
struct PfUmmaParams {
  const void* Phat;            // [npix][F] half2 (f16 kind) or float2 (f16x3 kind)
  const void* B;               // [n_rho][nblk][KC][parts][2 Db rows x row bytes], operand layout
  void* C;                     // [npix][D] half2 or float2
  const int2* tile_i01;        // [ntiles]
  const int* tile_pix;         // [ntiles][128] pixel or -1
  const float* tile_alpha;     // [ntiles][128]
  const float* tile_acut;      // [ntiles][128]
  int ntiles, F, D, Db, nblk, KC;
  int kind;                    // UmmaKind
  int split;                   // set by the launcher: parts of a tail unit's frequency sum
  // kUmmaF16x3 only: *amax (float bits) bounds |Re|, |Im| of the compact
  // phasors and every |Phat| component is below *amax * 2^abound_exp; A is
  // scaled by 2^(15 - e(*amax) - abound_exp) with *amax < 2^e(*amax)
  const unsigned* amax;
  int abound_exp;
  float scale;
  int* err;                    // device error word (bounded waits)
  long long Phat_n, C_n;       // element extents (bounds-checked build; 0: unchecked)
};
// pipelined: persistent warp-specialised CTAs (one per SM) instead of one CTA per tile
cudaError_t launch_pf_umma(const PfUmmaParams& p, bool pipelined, cudaStream_t s);
// first tile whose frequency sum the persistent schedule splits (its parts
// are added into C, which must be zero there); ntiles when none is split
int pf_umma_first_split_tile(const PfUmmaParams& p);
// zero `row_bytes` (a multiple of 4) at C + pix * row_bytes for every
// pix = list[i] >= 0, i < n
cudaError_t launch_clear_rows(void* C, const int* list, long long n, size_t row_bytes, cudaStream_t s);
// the same for the entries of two lists in one launch
cudaError_t launch_clear_rows2(void* C, const int* l1, long long n1, const int* l2, long long n2, size_t row_bytes,
                               cudaStream_t s);
// max |x| over `count` floats into *out (float bits, atomicMax; *out must be
// cleared beforehand)
cudaError_t launch_absmax(const float* x, long long count, unsigned* out, cudaStream_t s);
// K_r (float64 [n_rho][F][D]) -> B operand blocks of the given kind, scaled
cudaError_t launch_kr_store_umma(const double2* K64, void* B, int kind, int n_rho, int F, int D, int Db, int nblk,
                                 int KC, double scale, cudaStream_t s);

// Dense phasor-field kernel (Alg. 3), spatial form on the signed padded grid:
// k[x][y][f][d] = exp(i kappa_f (sigma_s R + sigma_t d + Delta)),
// R = sqrt((x~ dx)^2 + (y~ dy)^2 + d^2), phase in float64.
struct DenseGenParams {
  const double* kappa;         // [F]
  const double* depth;         // [D]
  int Nu, Nv, F, D;
  double dx, dy, sigma_s, sigma_t, delta;
  float2* k;                   // out [Nu][Nv][F][D]
};
cudaError_t launch_dense_gen(const DenseGenParams& p, cudaStream_t s);
// Dense depth sum: C[pix][d] = sum_f Phat[pix][f] * Khat[pix][f][d] (float32).
struct PfDenseParams {
  const float2* Phat;          // [npix][F]
  const float2* K;             // [npix][F][D]
  float2* C;                   // [npix][D]
  long long npix;
  int F, D;
};
cudaError_t launch_pf_dense(const PfDenseParams& p, cudaStream_t s);

// Per-volume scale for reduced-precision storage: out[0] = target / ||u||_2,
// out[1] = 1 / out[0], out[2] = 1 / out[0]^2, where u = H * (t % n) * t_scale (t_scale = 0: no ramp).
cudaError_t launch_volume_scale(const void* H, long long count, int n, float t_scale, int storage,
                                float target, float* partial, int npartial, float* out,
                                cudaStream_t s);

}  // namespace nlos
