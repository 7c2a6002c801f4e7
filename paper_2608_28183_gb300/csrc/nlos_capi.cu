// Host side of the library: plan creation (float64 tables), the stage
// sequences of f-k migration and phasor-field reconstruction, and the C ABI
// declared in include/nlos.h.
#include <nvtx3/nvToolsExt.h>
#include <math.h>

#include <algorithm>
#include <atomic>
#include <cstdarg>
#include <cstdlib>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "nlos.h"
#include "nlos_internal.h"

namespace nlos {
cudaError_t launch_axis_fft_f32_r0(const AxisLaunch& l, cudaStream_t s);
cudaError_t launch_axis_fft_f32_r1(const AxisLaunch& l, cudaStream_t s);
cudaError_t launch_axis_fft_f32_r2(const AxisLaunch& l, cudaStream_t s);
cudaError_t launch_axis_fft_f16_r0(const AxisLaunch& l, cudaStream_t s);
cudaError_t launch_axis_fft_f16_r1(const AxisLaunch& l, cudaStream_t s);
cudaError_t launch_axis_fft_f16_r2(const AxisLaunch& l, cudaStream_t s);
cudaError_t launch_axis_fft_bf16_r0(const AxisLaunch& l, cudaStream_t s);
cudaError_t launch_axis_fft_bf16_r1(const AxisLaunch& l, cudaStream_t s);
cudaError_t launch_axis_fft_bf16_r2(const AxisLaunch& l, cudaStream_t s);
cudaError_t launch_fk_zstage_f32_r0(const FkZParams& p, int tile, cudaStream_t s);
cudaError_t launch_fk_zstage_f32_r1(const FkZParams& p, int tile, cudaStream_t s);
cudaError_t launch_fk_zstage_f32_r2(const FkZParams& p, int tile, cudaStream_t s);
cudaError_t launch_fk_zstage_f16_r0(const FkZParams& p, int tile, cudaStream_t s);
cudaError_t launch_fk_zstage_f16_r1(const FkZParams& p, int tile, cudaStream_t s);
cudaError_t launch_fk_zstage_f16_r2(const FkZParams& p, int tile, cudaStream_t s);
cudaError_t launch_fk_zstage_bf16_r0(const FkZParams& p, int tile, cudaStream_t s);
cudaError_t launch_fk_zstage_bf16_r1(const FkZParams& p, int tile, cudaStream_t s);
cudaError_t launch_fk_zstage_bf16_r2(const FkZParams& p, int tile, cudaStream_t s);

cudaError_t launch_axis_fft(const AxisLaunch& l, cudaStream_t s) {
  static cudaError_t (*const fn[3][3])(const AxisLaunch&, cudaStream_t) = {
      {launch_axis_fft_f32_r0, launch_axis_fft_f32_r1, launch_axis_fft_f32_r2},
      {launch_axis_fft_f16_r0, launch_axis_fft_f16_r1, launch_axis_fft_f16_r2},
      {launch_axis_fft_bf16_r0, launch_axis_fft_bf16_r1, launch_axis_fft_bf16_r2}};
  if (l.storage < 0 || l.storage > 2) return cudaErrorInvalidValue;
  return fn[l.storage][l.L <= 64 ? 0 : l.L <= 256 ? 1 : 2](l, s);
}

cudaError_t launch_fk_chain_f32(const FkChainLaunch& l, cudaStream_t s);
cudaError_t launch_fk_chain_f16(const FkChainLaunch& l, cudaStream_t s);
cudaError_t launch_fk_chain_bf16(const FkChainLaunch& l, cudaStream_t s);

cudaError_t launch_fk_chain(const FkChainLaunch& l, int storage, cudaStream_t s) {
  switch (storage) {
    case kF32: return launch_fk_chain_f32(l, s);
    case kF16: return launch_fk_chain_f16(l, s);
    case kBF16: return launch_fk_chain_bf16(l, s);
    default: return cudaErrorInvalidValue;
  }
}

#define NLOS_ZSPLIT(t)                                                                   \
  cudaError_t launch_fk_stolt_##t##_r0(const FkZParams& p, int tile, cudaStream_t s);    \
  cudaError_t launch_fk_stolt_##t##_r1(const FkZParams& p, int tile, cudaStream_t s);    \
  cudaError_t launch_fk_zinv_##t##_r0(const FkZInvParams& p, int tile, cudaStream_t s);  \
  cudaError_t launch_fk_zinv_##t##_r1(const FkZInvParams& p, int tile, cudaStream_t s);
NLOS_ZSPLIT(f32)
NLOS_ZSPLIT(f16)
NLOS_ZSPLIT(bf16)
#undef NLOS_ZSPLIT

cudaError_t launch_fk_stolt(const FkZParams& p, int storage, int tile, cudaStream_t s) {
  static cudaError_t (*const fn[3][2])(const FkZParams&, int, cudaStream_t) = {
      {launch_fk_stolt_f32_r0, launch_fk_stolt_f32_r1},
      {launch_fk_stolt_f16_r0, launch_fk_stolt_f16_r1},
      {launch_fk_stolt_bf16_r0, launch_fk_stolt_bf16_r1}};
  if (p.npencils <= 0 || p.L != 2 * p.n || p.pad != 2 || storage < 0 || storage > 2) return cudaErrorInvalidValue;
  return fn[storage][p.L <= 1024 ? 0 : 1](p, tile, s);
}

cudaError_t launch_fk_zinv(const FkZInvParams& p, int storage, int tile, cudaStream_t s) {
  static cudaError_t (*const fn[3][2])(const FkZInvParams&, int, cudaStream_t) = {
      {launch_fk_zinv_f32_r0, launch_fk_zinv_f32_r1},
      {launch_fk_zinv_f16_r0, launch_fk_zinv_f16_r1},
      {launch_fk_zinv_bf16_r0, launch_fk_zinv_bf16_r1}};
  if (p.npencils <= 0 || p.L != 2 * p.n || storage < 0 || storage > 2) return cudaErrorInvalidValue;
  return fn[storage][p.L <= 1024 ? 0 : 1](p, tile, s);
}

cudaError_t launch_fk_zstage(const FkZParams& p, int storage, int tile, cudaStream_t s) {
  static cudaError_t (*const fn[3][3])(const FkZParams&, int, cudaStream_t) = {
      {launch_fk_zstage_f32_r0, launch_fk_zstage_f32_r1, launch_fk_zstage_f32_r2},
      {launch_fk_zstage_f16_r0, launch_fk_zstage_f16_r1, launch_fk_zstage_f16_r2},
      {launch_fk_zstage_bf16_r0, launch_fk_zstage_bf16_r1, launch_fk_zstage_bf16_r2}};
  if (storage < 0 || storage > 2) return cudaErrorInvalidValue;
  return fn[storage][p.L <= 256 ? 0 : p.L <= 1024 ? 1 : 2](p, tile, s);
}
}  // namespace nlos

using namespace nlos;

namespace {

constexpr double kC = 299792458.0;   // speed of light, m/s
constexpr double kPi = 3.14159265358979323846;
constexpr double kTaperBins = 8.0;   // smoothstep width below the radial cutoff
constexpr float kVolumeTarget = 4096.0f;   // ||scaled input||_2 for reduced-precision storage
constexpr int kScalePartials = 2048;
constexpr int kBatchStreams = 8;
constexpr size_t kErrOffset = 64;    // device error word inside the workspace's scalar area
constexpr size_t kAmaxOffset = 128;  // max |component| of the compact phasors (f16x3 depth sum)

thread_local std::string g_err;

nlos_status_t fail(nlos_status_t st, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_err = buf;
  return st;
}

nlos_status_t cuda_fail(cudaError_t e, const char* where) {
  if (e == cudaErrorMemoryAllocation)
    return fail(NLOS_ERR_OUT_OF_MEMORY, "%s: %s", where, cudaGetErrorString(e));
  return fail(NLOS_ERR_CUDA, "%s: %s", where, cudaGetErrorString(e));
}

#define NLOS_CU(call, where)                     \
  do {                                           \
    cudaError_t e_ = (call);                     \
    if (e_ != cudaSuccess) return cuda_fail(e_, where); \
  } while (0)

bool is_pow2(long long v) { return v > 0 && (v & (v - 1)) == 0; }
int ilog2i(long long v) { int k = 0; while ((1LL << k) < v) ++k; return k; }
size_t align256(size_t v) { return (v + 255) & ~size_t(255); }
int ceil_int_guarded(double x) { return (int)ceil(x - 1e-9); }
int pow2_at_least(int x) { int p = 1; while (p < x) p <<= 1; return p; }

// per-pass scale keeping reduced-precision intermediates bounded: the
// nearest power of two at or above 1/sqrt(L)
float pass_scale(int storage, int L) {
  if (storage == kF32) return 1.0f;
  return ldexpf(1.0f, -(ilog2i(L) / 2));
}

size_t complex_bytes(int storage) { return storage == kF32 ? 8 : 4; }
size_t real_bytes(int storage) { return storage == kF32 ? 4 : 2; }

}  // namespace

// Staging for pipelined host-buffer calls: kPipeSlots device input/output
// pairs and three streams, so that the copy in of capture i+1 and the copy
// out of capture i-1 overlap the reconstruction of capture i.
constexpr int kPipeSlots = 3;
struct HostPipe {
  void* d_in[kPipeSlots] = {};
  void* d_out[kPipeSlots] = {};
  cudaStream_t h2d = nullptr, comp = nullptr, d2h = nullptr;
  cudaEvent_t start = nullptr;
  cudaEvent_t in_ready[kPipeSlots] = {}, done[kPipeSlots] = {}, out_free[kPipeSlots] = {};
};

struct nlos_plan_s {
  nlos_plan_desc_t d{};
  int a = 0, b = 0, n = 0;
  int Lx = 0, Ly = 0, Lt = 0;           // transform lengths (padded, powers of two)
  int storage = kF32;
  int nz = 0;
  std::map<int, float2*> tw;            // twiddle table per FFT length
  std::map<int, float2*> tw32;          // twiddles of the radix-32 schedule (32 values per thread)
  // f-k Stolt constants
  float2* ax = nullptr;
  float2* ay = nullptr;
  // phasor-field tables
  int F = 0, D = 0, k_lo = 0, nchunks = 0, kr_storage = kF32;
  float* w = nullptr;
  float2* phase = nullptr;              // [n] exp(-2 pi i m / n) for photon binning
  float2* Kd = nullptr;                 // dense method: Khat [Nu*Nv][F][D]
  // tensor-core depth sum (16-bit storage): B operand blocks and 128-pixel tiles
  void* Bu = nullptr;
  int2* tu_i01 = nullptr;
  int* tu_pix = nullptr;
  float* tu_alpha = nullptr;
  float* tu_acut = nullptr;
  int* clr_pix = nullptr;          // pixels of the padded grid outside every tile (depth sum writes none)
  int nclr = 0;
  int ntiles_u = 0, Db_u = 0, nblk_u = 0, KC_u = 0, kind_u = 0;
  void* Kr = nullptr;
  int2* ch_i01 = nullptr;
  int* ch_pix = nullptr;
  float* ch_alpha = nullptr;
  float* ch_acut = nullptr;
  double kr_scale = 1.0;
  double bu_scale = 1.0;          // power-of-two scale of the tensor-core B operands
  // workspace layout: up to three complex buffers + scale scalars + partials
  size_t off[3] = {0, 0, 0};
  size_t off_scal = 0, off_part = 0;
  size_t off_sync = 0;                  // chunk counters of the fused lateral f-k stages
  bool fused = false;                   // f-k lateral transforms fused in pairs (fk_chain.cuh)
  bool zlast = false;                   // f-k inverse temporal transform last (fk_zsplit.cuh)
  size_t ws_bytes = 0;
  void* ws = nullptr;
  // host-call staging
  void* d_in = nullptr;
  void* d_out = nullptr;
  struct HostPipe* pipe = nullptr;      // pipelined host calls (created on first use)
  std::vector<void*> allocs;
  size_t resident = 0;                  // bytes of device memory the plan holds (tables, kernels, workspace)
  // per-stage tile variant (autotuner) and the transform length it applies to
  std::vector<int> tiles;
  std::vector<int> stage_len;     // 0: stage has no variants
  std::vector<int> stage_kind;    // 1: strided-axis transform, 2: f-k temporal stage, 3: real-input axis,
                                  // 4: depth sum with a tensor-core variant
  bool tuned = false;
  // stage tracing
  std::vector<std::string> stage_names;
  bool prof_on = false;
  std::vector<cudaEvent_t> prof_pool;
  std::vector<int> prof_stage;          // stage index of each recorded event (-1: call start)
  size_t prof_used = 0;
  // shared-spectrum mixture of experts: spectrum ready, phasor branch done (created on first use)
  cudaEvent_t moe_ev[2] = {nullptr, nullptr};
};

namespace {

// failure-path testing hook: the n-th plan allocation from now fails (0: off)
std::atomic<int> g_fail_alloc{0};

nlos_status_t dalloc(nlos_plan_s* p, void** ptr, size_t bytes, const char* what) {
  int k = g_fail_alloc.load();
  while (k > 0 && !g_fail_alloc.compare_exchange_weak(k, k - 1)) {
  }
  if (k == 1) {
    *ptr = nullptr;
    return fail(NLOS_ERR_OUT_OF_MEMORY, "%s: injected allocation failure", what);
  }
  cudaError_t e = cudaMalloc(ptr, bytes ? bytes : 16);
  if (e != cudaSuccess) {
    *ptr = nullptr;
    cudaGetLastError();
    return cuda_fail(e, what);
  }
  p->allocs.push_back(*ptr);
  p->resident += bytes ? bytes : 16;
  return NLOS_OK;
}

template <class T>
nlos_status_t upload(nlos_plan_s* p, T** dst, const std::vector<T>& src, const char* what) {
  void* ptr = nullptr;
  nlos_status_t st = dalloc(p, &ptr, sizeof(T) * src.size(), what);
  if (st != NLOS_OK) return st;
  NLOS_CU(cudaMemcpy(ptr, src.data(), sizeof(T) * src.size(), cudaMemcpyHostToDevice), what);
  *dst = static_cast<T*>(ptr);
  return NLOS_OK;
}

// Stockham pass twiddle tables of an L-point transform (same schedule as
// FftShape<L>): for pass p with span Ns and radix R, T_p[r Ns + k] =
// exp(-2 pi i k r / (Ns R)), float64 then rounded to float.
std::vector<float2> make_twiddles(int L, int E = 16) {
  const int LE = E == 32 ? 5 : 4;
  const int LOG = ilog2i(L), NFULL = LOG / LE, REM = LOG % LE;
  const int npass = NFULL + (REM ? 1 : 0);
  std::vector<float2> t;
  int span = 1;
  for (int pss = 0; pss < npass; ++pss) {
    const int R = pss < NFULL ? E : (1 << REM);
    for (int r = 0; r < R; ++r)
      for (int k = 0; k < span; ++k) {
        const long long m = (long long)k * r;           // exponent over span*R
        const double ang = -2.0 * kPi * (double)m / (double)(span * R);
        t.push_back(make_float2((float)cos(ang), (float)sin(ang)));
      }
    span *= R;
  }
  return t;
}

nlos_status_t ensure_twiddles(nlos_plan_s* p, int L) {
  if (p->tw.count(L)) return NLOS_OK;
  const std::vector<float2> t = make_twiddles(L);
  float2* d = nullptr;
  nlos_status_t st = upload(p, &d, t, "twiddle upload");
  if (st != NLOS_OK) return st;
  p->tw[L] = d;
  // radix-32 schedule (32 values per thread)
  if (L >= 32) {
    float2* d32 = nullptr;
    if ((st = upload(p, &d32, make_twiddles(L, 32), "twiddle upload")) != NLOS_OK) return st;
    p->tw32[L] = d32;
  }
  return NLOS_OK;
}

// (hi, lo) float pair of a float64 value
float2 split_ff(double v) {
  const float hi = (float)v;
  return make_float2(hi, (float)(v - (double)hi));
}

// ---------------------------------------------------------------------------
// f-k plan: Stolt constants A_x(p) = (Lt s_x p~ / Lx)^2 with s_x = c dt / (2 dx)
// (Alg. 1's s per axis), signed index p~ of the Lx-point padded axis; for
// Lx = 2a, Lt = 2n this is Alg. 1's (n s_x p~ / a)^2.
// ---------------------------------------------------------------------------
nlos_status_t build_fk(nlos_plan_s* p) {
  const auto& d = p->d;
  const int Lx = p->Lx, Ly = p->Ly, Lt = p->Lt;
  const double dx = d.wall_w_m / d.nx, dy = d.wall_h_m / d.ny;
  const double sx = kC * d.bin_width_s / (2.0 * dx);
  const double sy = kC * d.bin_width_s / (2.0 * dy);
  // mu^2 = A + m^2 with A = (Lt s_x p~ / Lx)^2 + (Lt s_y q~ / Ly)^2
  std::vector<float2> ax(Lx), ay(Ly);
  for (int i = 0; i < Lx; ++i) {
    const int pt = i < Lx / 2 ? i : i - Lx;
    const double v = (double)Lt * sx * pt / Lx;
    ax[i] = split_ff(v * v);
  }
  for (int i = 0; i < Ly; ++i) {
    const int qt = i < Ly / 2 ? i : i - Ly;
    const double v = (double)Lt * sy * qt / Ly;
    ay[i] = split_ff(v * v);
  }
  nlos_status_t st;
  if ((st = upload(p, &p->ax, ax, "stolt table")) != NLOS_OK) return st;
  if ((st = upload(p, &p->ay, ay, "stolt table")) != NLOS_OK) return st;
  if ((st = ensure_twiddles(p, Lx)) != NLOS_OK) return st;
  if ((st = ensure_twiddles(p, Ly)) != NLOS_OK) return st;
  if ((st = ensure_twiddles(p, Lt)) != NLOS_OK) return st;
  const size_t cb = complex_bytes(p->storage);
  const long long b = p->b, n = p->n, hx = Lx / 2 + 1;
  const size_t b0 = std::max(hx * b * n, (long long)Lx * b * n) * cb;   // G1, then the y-inverse output
  const size_t b1 = hx * Ly * n * cb;                                    // G (kx <= Lx/2)
  const size_t b2 = (size_t)Lx * Ly * n * cb;                             // psi_z
  p->off[0] = 0;
  p->off[1] = align256(b0);
  p->off[2] = p->off[1] + align256(b1);
  p->off_scal = p->off[2] + align256(b2);
  p->off_part = p->off_scal + 256;
  p->off_sync = p->off_part + align256(sizeof(float) * kScalePartials);
  p->ws_bytes = p->off_sync + align256(sizeof(int) * (2 + n / 16));
  p->nz = p->n;
  return NLOS_OK;
}

// ---------------------------------------------------------------------------
// phasor-field plan (Sec. 4.3 Eqs. 4-7, supplementary radial sampling)
// ---------------------------------------------------------------------------
double taper_weight(double rb, double rc) {
  if (rb <= rc - kTaperBins) return 1.0;
  if (rb >= rc) return 0.0;
  const double t = (rc - rb) / kTaperBins;
  return t * t * (3.0 - 2.0 * t);
}

nlos_status_t build_dense(nlos_plan_s* p, const std::vector<double>& kappa, const std::vector<double>& depth,
                          int sig_s, int sig_t, double dx, double dy);
nlos_status_t pf_finish(nlos_plan_s* p, const std::vector<float>& w);

nlos_status_t build_pf(nlos_plan_s* p) {
  const auto& d = p->d;
  const double dx = d.wall_w_m / d.nx, dy = d.wall_h_m / d.ny;
  // virtual-wave band: f0 = c / lambda, sigma_t = cycles / (6 f0), +-5 sigma_f
  const double lam = d.wavelength_m > 0 ? d.wavelength_m : 4.0 * dx;
  const double cyc = d.cycles > 0 ? d.cycles : 5.0;
  const double f0 = kC / lam;
  // temporal DFT length Lt: n, or the next power of two (zero-padded transient)
  const double df = 1.0 / (p->Lt * d.bin_width_s);
  const int k0 = (int)llround(f0 / df);
  const double sigma_f = 1.0 / (2.0 * kPi * (cyc / (6.0 * f0)));
  const int kh = (int)llround(5.0 * sigma_f / df);
  const int lo = std::max(1, k0 - kh), hi = std::min(p->Lt / 2 - 1, k0 + kh);
  if (hi < lo) return fail(NLOS_ERR_INVALID_ARG, "virtual-wave band is empty (k0=%d, n=%d)", k0, p->n);
  p->k_lo = lo;
  p->F = hi - lo + 1;
  std::vector<float> w(p->F);
  std::vector<double> kappa(p->F);
  for (int f = 0; f < p->F; ++f) {
    const double fk = (lo + f) * df;
    w[f] = (float)exp(-(fk - f0) * (fk - f0) / (2.0 * sigma_f * sigma_f));
    kappa[f] = 2.0 * kPi * fk / kC;
  }
  const double lambda_min = kC / (hi * df);
  // radial sampling over the padded aperture
  const int Nu = p->Lx, Nv = p->Ly;
  const double r_max = sqrt(pow(0.5 * Nu * dx, 2) + pow(0.5 * Nv * dy, 2));
  const double rho_max = sqrt(pow(1.0 / (2.0 * dx), 2) + pow(1.0 / (2.0 * dy), 2));
  const int sig_s = d.sigma_s > 0 ? d.sigma_s : 2;
  const int sig_t = (d.sigma_s > 0 || d.sigma_t > 0) ? d.sigma_t : 0;
  const int n_r = std::max(2, pow2_at_least(ceil_int_guarded(2.0 * sig_s * r_max / lambda_min) + 1));
  const int n_rho = pow2_at_least(ceil_int_guarded(2.0 * r_max * rho_max) + 1);
  const double dr = r_max / (n_r - 1);
  const double rho_cut = std::min(rho_max, 0.5 * (n_r - 1) / r_max);
  const double rc_bin = rho_cut * (n_rho - 1) / rho_max;
  p->D = d.n_depths;
  std::vector<double> depth(p->D), r(n_r), rho(n_rho);
  for (int j = 0; j < p->D; ++j)
    depth[j] = p->D == 1 ? d.depth_min_m : d.depth_min_m + j * (d.depth_max_m - d.depth_min_m) / (p->D - 1);
  if (d.method == NLOS_PHASOR_DENSE) {
    nlos_status_t st = build_dense(p, kappa, depth, sig_s, sig_t, dx, dy);
    return st != NLOS_OK ? st : pf_finish(p, w);
  }
  for (int j = 0; j < n_r; ++j) r[j] = j * dr;
  for (int i = 0; i < n_rho; ++i) rho[i] = i * (rho_max / (n_rho - 1));
  // ring basis with trapezoid weights (Eq. 5, Eq. 6), zero beyond the cutoff
  std::vector<double> B((size_t)n_rho * n_r, 0.0);
  for (int i = 0; i < n_rho; ++i) {
    if (rho[i] > rho_cut) continue;
    for (int j = 0; j < n_r; ++j) {
      const double q = (j == 0 || j == n_r - 1) ? 0.5 * dr : dr;
      B[(size_t)i * n_r + j] = q * 2.0 * kPi * r[j] * j0(2.0 * kPi * r[j] * rho[i]);
    }
  }
  // radial kernel on the device in float64
  double *dB = nullptr, *dr_ = nullptr, *dk = nullptr, *ddep = nullptr;
  double2 *dA = nullptr, *dK64 = nullptr;
  const long long NFD = (long long)p->F * p->D;
  std::vector<void*> tmp;
  auto tmp_alloc = [&](void** ptr, size_t bytes) -> cudaError_t {
    cudaError_t e = cudaMalloc(ptr, bytes);
    if (e == cudaSuccess) tmp.push_back(*ptr); else cudaGetLastError();
    return e;
  };
  auto free_tmp = [&]() { for (void* v : tmp) cudaFree(v); tmp.clear(); };
  cudaError_t e = cudaSuccess;
  if ((e = tmp_alloc((void**)&dB, sizeof(double) * B.size())) != cudaSuccess ||
      (e = tmp_alloc((void**)&dr_, sizeof(double) * n_r)) != cudaSuccess ||
      (e = tmp_alloc((void**)&dk, sizeof(double) * p->F)) != cudaSuccess ||
      (e = tmp_alloc((void**)&ddep, sizeof(double) * p->D)) != cudaSuccess ||
      (e = tmp_alloc((void**)&dA, sizeof(double2) * (size_t)n_r * NFD)) != cudaSuccess ||
      (e = tmp_alloc((void**)&dK64, sizeof(double2) * (size_t)n_rho * NFD)) != cudaSuccess) {
    free_tmp();
    return cuda_fail(e, "radial kernel scratch");
  }
  cudaMemcpy(dB, B.data(), sizeof(double) * B.size(), cudaMemcpyHostToDevice);
  cudaMemcpy(dr_, r.data(), sizeof(double) * n_r, cudaMemcpyHostToDevice);
  cudaMemcpy(dk, kappa.data(), sizeof(double) * p->F, cudaMemcpyHostToDevice);
  cudaMemcpy(ddep, depth.data(), sizeof(double) * p->D, cudaMemcpyHostToDevice);
  KrBuildParams kp{dB, dr_, dk, ddep, n_rho, n_r, p->F, p->D, (double)sig_s, (double)sig_t, d.delta_m, dA, dK64};
  e = launch_kr_build(kp, 0);
  // stored kernel: float32 for float32 plans, float16 (scaled into range) otherwise
  p->kr_storage = p->storage;
  p->kr_scale = 1.0;
  if (p->storage != kF32) {
    const double bound = kPi * r_max * r_max;   // >= sum_j q_j 2 pi r_j |J0|
    p->kr_scale = ldexp(1.0, (int)floor(log2(16384.0 / bound)));
  }
  void* Kr = nullptr;
  nlos_status_t st = NLOS_OK;
  if (e == cudaSuccess) {
    st = dalloc(p, &Kr, complex_bytes(p->kr_storage) * (size_t)n_rho * NFD, "radial kernel");
    if (st == NLOS_OK) e = launch_kr_store(dK64, Kr, (long long)n_rho * NFD, p->kr_storage, p->kr_scale, 0);
  }
  if (e == cudaSuccess && st == NLOS_OK && (p->storage == kF16 || p->storage == kF32)) {
    // the same kernel as tensor-core B operands: [Kr -Ki; Ki Kr] per bin and
    // depth block, f16 for 16-bit plans, f16 (hi, lo) parts for float32 plans;
    // both scaled into f16 range by a power of two
    p->kind_u = p->storage == kF16 ? kUmmaF16 : kUmmaF16x3;
    p->bu_scale = p->storage == kF16 ? p->kr_scale
                                     : ldexp(1.0, (int)floor(log2(16384.0 / (kPi * r_max * r_max))));
    const int cols = umma_chunk_cols(p->kind_u);
    p->Db_u = p->D <= 16 ? 16 : p->D <= 32 ? 32 : p->D <= 64 ? 64 : 128;
    p->nblk_u = (p->D + p->Db_u - 1) / p->Db_u;
    p->KC_u = (2 * p->F + cols - 1) / cols;
    const size_t bbytes =
        (size_t)n_rho * p->nblk_u * p->KC_u * umma_parts(p->kind_u) * (2 * p->Db_u) * umma_row_bytes(p->kind_u);
    st = dalloc(p, &p->Bu, bbytes, "tensor-core kernel operands");
    if (st == NLOS_OK)
      e = launch_kr_store_umma(dK64, p->Bu, p->kind_u, n_rho, p->F, p->D, p->Db_u, p->nblk_u, p->KC_u,
                               p->bu_scale, 0);
  }
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  free_tmp();
  if (st != NLOS_OK) return st;
  if (e != cudaSuccess) return cuda_fail(e, "radial kernel build");
  p->Kr = Kr;
  // pixel-to-radius lookup, grouped into chunks sharing (i0, i1)
  struct Pix { int i0, i1, pix; float alpha, acut; };
  std::vector<Pix> px;
  px.reserve((size_t)Nu * Nv);
  const int i_c = (int)floor(rc_bin);
  const int last_base = std::max(0, std::min(i_c - 1, n_rho - 2));
  for (int kx = 0; kx < Nu; ++kx) {
    const double fx = (kx < Nu / 2 ? kx : kx - Nu) / (Nu * dx);
    for (int ky = 0; ky < Nv; ++ky) {
      const double fy = (ky < Nv / 2 ? ky : ky - Nv) / (Nv * dy);
      const double rb = sqrt(fx * fx + fy * fy) * (n_rho - 1) / rho_max;
      const double ac = taper_weight(rb, rc_bin);
      if (ac <= 0.0) continue;
      const int i0 = std::max(0, std::min((int)floor(rb), last_base));
      const int i1 = std::min(i0 + 1, i_c);
      px.push_back({i0, i1, kx * Nv + ky, (float)(rb - i0), (float)ac});
    }
  }
  {
    // pixels beyond the cutoff: their depth-sum output is zero
    std::vector<char> inside((size_t)Nu * Nv, 0);
    for (const Pix& q : px) inside[q.pix] = 1;
    std::vector<int> outside;
    for (int k = 0; k < Nu * Nv; ++k)
      if (!inside[k]) outside.push_back(k);
    p->nclr = (int)outside.size();
    if (p->nclr > 0 && (st = upload(p, &p->clr_pix, outside, "cutoff list")) != NLOS_OK) return st;
  }
  std::stable_sort(px.begin(), px.end(), [](const Pix& u, const Pix& v) {
    return u.i0 != v.i0 ? u.i0 < v.i0 : u.i1 < v.i1;
  });
  std::vector<int2> ci;
  std::vector<int> cp;
  std::vector<float> ca, cc;
  for (size_t s = 0; s < px.size();) {
    size_t e2 = s;
    while (e2 < px.size() && px[e2].i0 == px[s].i0 && px[e2].i1 == px[s].i1) ++e2;
    for (size_t c = s; c < e2; c += kPfChunk) {
      ci.push_back(make_int2(px[s].i0, px[s].i1));
      for (int q = 0; q < kPfChunk; ++q) {
        const size_t idx = c + q;
        const bool ok = idx < e2;
        cp.push_back(ok ? px[idx].pix : -1);
        ca.push_back(ok ? px[idx].alpha : 0.f);
        cc.push_back(ok ? px[idx].acut : 0.f);
      }
    }
    s = e2;
  }
  p->nchunks = (int)ci.size();
  if (p->nchunks > 0) {
    if ((st = upload(p, &p->ch_i01, ci, "chunk table")) != NLOS_OK) return st;
    if ((st = upload(p, &p->ch_pix, cp, "chunk table")) != NLOS_OK) return st;
    if ((st = upload(p, &p->ch_alpha, ca, "chunk table")) != NLOS_OK) return st;
    if ((st = upload(p, &p->ch_acut, cc, "chunk table")) != NLOS_OK) return st;
  }
  if (p->Bu) {
    // 128-pixel tiles of pixels sharing (i0, i1) for the tensor-core depth sum
    std::vector<int2> ti;
    std::vector<int> tp;
    std::vector<float> ta, tc;
    for (size_t s0 = 0; s0 < px.size();) {
      size_t e2 = s0;
      while (e2 < px.size() && px[e2].i0 == px[s0].i0 && px[e2].i1 == px[s0].i1) ++e2;
      for (size_t c = s0; c < e2; c += kUmmaTile) {
        ti.push_back(make_int2(px[s0].i0, px[s0].i1));
        for (int q = 0; q < kUmmaTile; ++q) {
          const size_t idx = c + q;
          const bool ok = idx < e2;
          tp.push_back(ok ? px[idx].pix : -1);
          ta.push_back(ok ? px[idx].alpha : 0.f);
          tc.push_back(ok ? px[idx].acut : 0.f);
        }
      }
      s0 = e2;
    }
    p->ntiles_u = (int)ti.size();
    if (p->ntiles_u > 0) {
      if ((st = upload(p, &p->tu_i01, ti, "tile table")) != NLOS_OK) return st;
      if ((st = upload(p, &p->tu_pix, tp, "tile table")) != NLOS_OK) return st;
      if ((st = upload(p, &p->tu_alpha, ta, "tile table")) != NLOS_OK) return st;
      if ((st = upload(p, &p->tu_acut, tc, "tile table")) != NLOS_OK) return st;
    }
  }
  return pf_finish(p, w);
}

// band weights, phase table, twiddles and the workspace layout of a
// phasor-field plan (both kernel representations)
nlos_status_t pf_finish(nlos_plan_s* p, const std::vector<float>& w) {
  nlos_status_t st;
  const int Nu = p->Lx, Nv = p->Ly;
  if ((st = upload(p, &p->w, w, "band weights")) != NLOS_OK) return st;
  std::vector<float2> phase(p->Lt);
  for (int m = 0; m < p->Lt; ++m) {
    const double t = 2.0 * kPi * m / p->Lt;
    phase[m] = make_float2((float)cos(t), (float)-sin(t));
  }
  if ((st = upload(p, &p->phase, phase, "phase table")) != NLOS_OK) return st;
  if ((st = ensure_twiddles(p, p->Lt)) != NLOS_OK) return st;
  if ((st = ensure_twiddles(p, Nu)) != NLOS_OK) return st;
  if ((st = ensure_twiddles(p, Nv)) != NLOS_OK) return st;
  const size_t cb = complex_bytes(p->storage);
  const long long a = p->a, b = p->b, F = p->F, D = p->D;
  const long long U = Nu, V = Nv;
  const size_t b0 = std::max(a * b * F, U * b * D) * cb;           // P, then the y-inverse output
  const size_t b1 = std::max(a * V * F, U * V * D) * cb;           // y-transformed P, then C
  const size_t b2 = U * V * F * cb;                                // Phat
  p->off[0] = 0;
  p->off[1] = align256(b0);
  p->off[2] = p->off[1] + align256(b1);
  p->off_scal = p->off[2] + align256(b2);
  p->off_part = p->off_scal + 256;
  p->off_sync = p->off_part + align256(sizeof(float) * kScalePartials);
  p->ws_bytes = p->off_sync + 256;
  p->nz = p->D;
  return NLOS_OK;
}

// records a tracing event after `stage` (or a call start for stage -1)
// With stage tracing on, each stage is also an NVTX range named after it
// (host-side enqueue ranges, visible to ncu's --nvtx filters): mark(-1) opens
// stage 0, mark(i) closes stage i and opens stage i + 1.
nlos_status_t mark(nlos_plan_s* p, cudaStream_t s, int stage) {
  if (!p->prof_on) return NLOS_OK;
  if (stage >= 0) nvtxRangePop();
  if (stage + 1 < (int)p->stage_names.size()) nvtxRangePushA(p->stage_names[stage + 1].c_str());
  if (p->prof_used == p->prof_pool.size()) {
    cudaEvent_t e;
    NLOS_CU(cudaEventCreate(&e), "profiling event");
    p->prof_pool.push_back(e);
  }
  NLOS_CU(cudaEventRecord(p->prof_pool[p->prof_used], s), "profiling event");
  p->prof_stage.push_back(stage);
  ++p->prof_used;
  return NLOS_OK;
}

#define NLOS_MARK(p, s, stage)                     \
  do {                                             \
    nlos_status_t m_ = mark((p), (s), (stage));    \
    if (m_ != NLOS_OK) return m_;                  \
  } while (0)

// cuTensorMapEncodeTiled through the runtime's driver entry point (no link
// dependency on the driver library)
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
  static EncodeTiledFn fn = nullptr;
  static bool tried = false;
  if (!tried) {
    tried = true;
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(f);
    else
      cudaGetLastError();   // do not leave a failed lookup as the thread's pending error
  }
  return fn;
}

// Prepare TMA staging for an axis launch whose variant asks for it: a 3D map
// (inner, axis rows, outer) over the input with a box of one column tile by
// min(L_in, 256) rows. Leaves the launch on direct loads when the layout does
// not meet TMA's 16-byte rules (e.g. an odd number of band frequencies).
void attach_tmap(AxisLaunch& l) {
  l.has_tmap = 0;
  const int nic = axis_ic_count(l.L);
  if (l.tile < nic) return;
  EncodeTiledFn fn = encode_fn();
  if (!fn) return;
  const bool real_in = l.load_mode == kLoadReal || l.load_mode == kLoadRealPair;
  const size_t elem = real_in ? real_bytes(l.storage) : complex_bytes(l.storage);
  const int IC = axis_ic(l.L, l.tile % nic) * (l.load_mode == kLoadRealPair ? 2 : 1);   // columns per box
  const unsigned long long s1 = (unsigned long long)l.p.in_axis * elem;
  const unsigned long long s2 =
      l.n_outer > 1 ? (unsigned long long)l.p.in_outer * elem : (unsigned long long)l.p.L_in * s1;
  if (s1 % 16 || s2 % 16 || (IC * elem) % 16 || (reinterpret_cast<uintptr_t>(l.p.in) % 16)) return;
  if (l.p.L_in > 256 && l.p.L_in % 256) return;
  const CUtensorMapDataType dt = elem == 8 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT64
                               : elem == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32
                                           : CU_TENSOR_MAP_DATA_TYPE_UINT16;
  const cuuint64_t dims[3] = {(cuuint64_t)l.p.inner, (cuuint64_t)l.p.L_in, (cuuint64_t)l.n_outer};
  const cuuint64_t strides[2] = {s1, s2};
  const cuuint32_t box[3] = {(cuuint32_t)IC, (cuuint32_t)std::min(l.p.L_in, 256), 1};
  const cuuint32_t estr[3] = {1, 1, 1};
  if (fn(&l.tmap, dt, 3, const_cast<void*>(l.p.in), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
         CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) ==
      CUDA_SUCCESS)
    l.has_tmap = 1;
}

// 3D tiled map over `base` with dims (d0 contiguous, d1, d2), byte strides
// s1, s2 of dims 1 and 2, box (b0, b1, 1) of `elem`-byte elements.
bool encode_3d(CUtensorMap* m, const void* base, size_t elem, unsigned long long d0, unsigned long long d1,
               unsigned long long d2, unsigned long long s1, unsigned long long s2, unsigned b0, unsigned b1,
               bool promote) {
  EncodeTiledFn fn = encode_fn();
  if (!fn) return false;
  if (s1 % 16 || s2 % 16 || (b0 * elem) % 16 || reinterpret_cast<uintptr_t>(base) % 16) return false;
  const CUtensorMapDataType dt = elem == 8 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT64
                               : elem == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32
                                           : CU_TENSOR_MAP_DATA_TYPE_UINT16;
  const cuuint64_t dims[3] = {d0, d1, d2};
  const cuuint64_t strides[2] = {s1, s2};
  const cuuint32_t box[3] = {b0, b1, 1};
  const cuuint32_t estr[3] = {1, 1, 1};
  return fn(m, dt, 3, const_cast<void*>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
            CU_TENSOR_MAP_SWIZZLE_NONE, promote ? CU_TENSOR_MAP_L2_PROMOTION_L2_256B : CU_TENSOR_MAP_L2_PROMOTION_NONE,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

AxisLaunch axis(int storage, int L, long long n_outer, const void* in, void* out, long long inner,
                long long in_outer, long long in_axis, long long out_outer, long long out_axis, int L_in,
                int L_out, int inverse, float scale, const float2* tw, int tile) {
  AxisLaunch l{};
  l.tile = tile;
  l.storage = storage;
  l.L = L;
  l.n_outer = n_outer;
  l.load_mode = kLoadCpx;
  l.store_mode = kStoreCpx;
  l.p.in = in;
  l.p.out = out;
  l.p.tw = tw;
  l.p.inner = inner;
  l.p.in_outer = in_outer;
  l.p.in_axis = in_axis;
  l.p.out_outer = out_outer;
  l.p.out_axis = out_axis;
  l.p.L_in = L_in;
  l.p.L_out = L_out;
  l.p.inverse = inverse;
  l.p.scale = scale;
  return l;
}

// element extents of the workspace's three complex buffers (bounds-checked build)
long long ws_extent(const nlos_plan_s* p, int k) {
  const size_t end = k == 0 ? p->off[1] : k == 1 ? p->off[2] : p->off_scal;
  return (long long)((end - p->off[k]) / complex_bytes(p->storage));
}
void set_extents(AxisLaunch& l, long long in_n, long long out_n) {
  l.p.in_n = in_n;
  l.p.out_n = out_n;
  l.p.err = l.err;
}

// part: 0 the whole reconstruction; 1 only the lateral forward transforms,
// without the t/(n-1) ramp (the spectrum shared with a phasor-field plan,
// float32 plans only); 2 the rest after part 1, the ramp applied as the
// temporal stage loads the spectrum (it commutes with the lateral transforms).
nlos_status_t run_fk(nlos_plan_s* p, const void* H, void* vol, char* ws, cudaStream_t s, int part) {
  const int st = p->storage;
  const long long a = p->a, b = p->b, n = p->n;
  void* b0 = ws + p->off[0];
  void* b1 = ws + p->off[1];
  void* b2 = ws + p->off[2];
  float* scal = reinterpret_cast<float*>(ws + p->off_scal);
  int* err = reinterpret_cast<int*>(ws + p->off_scal + kErrOffset);
  const float* s_in = nullptr;
  const float* inv_s = nullptr;
  const float* inv_s2 = nullptr;
  int sid = 0;
  if (part != 2) NLOS_MARK(p, s, -1);
  const float ramp = 1.0f / (float)(n - 1);
  if (st != kF32) {
    NLOS_CU(launch_volume_scale(H, a * b * n, (int)n, 1.0f / (float)(n - 1), st, kVolumeTarget,
                                reinterpret_cast<float*>(ws + p->off_part), kScalePartials, scal, s),
            "volume scale");
    NLOS_MARK(p, s, sid++);
    s_in = scal;
    inv_s = scal + 1;
    inv_s2 = scal + 2;
  }
  const long long pf = p->d.pad_factor, Lx = p->Lx, Ly = p->Ly, Lt = p->Lt, hx = Lx / 2 + 1;
  const float g2a = pass_scale(st, (int)Lx), g2b = pass_scale(st, (int)Ly), g2n = pass_scale(st, (int)Lt);
  // inverse normalisation: pass scales applied before the last transform (it applies none of its own)
  const double N = (double)Lx * Ly * Lt;
  const double gprod = (double)g2a * g2b * g2n * g2n * g2b;
  const bool cpx = p->d.output == NLOS_OUT_COMPLEX;
  const float fscale = (float)(cpx ? 1.0 / (N * gprod) : 1.0 / (N * N * gprod * gprod));
  FkChainParams ch{};
  int* sync = reinterpret_cast<int*>(ws + p->off_sync);
  const size_t sync_bytes = sizeof(int) * (size_t)(1 + n / 16);
  const size_t cb = complex_bytes(st), rb = real_bytes(st);
  if (p->fused) {
    ch.tw = p->tw32[(int)Lx];   // radix-32 schedule
    ch.a = (int)a;
    ch.b = (int)b;
    ch.n = (int)n;
    ch.L = (int)Lx;
    ch.nchunks = (int)(n / 16);
    ch.sync = sync;
    ch.err = err;
    ch.discard = 0;   // per stage below (variant 0 on float32 storage)
  }
  AxisLaunch l{};
  if (part == 2) {
    sid = p->fused ? 1 : 2;
  } else if (p->fused) {
    // FK1 fused: x forward (real input, t/(n-1), zero-padded, kx in [0, Lx/2]) then y forward
    FkChainLaunch c{};
    c.p = ch;
    c.p.in = H;
    c.p.mid = b0;
    c.p.out = b1;
    c.p.t_scale = part == 1 ? 0.0f : ramp;
    c.p.s1 = g2a;
    c.p.s2 = g2b;
    c.p.ld_dev_scale = s_in;
    c.p.in_n = a * b * n;
    c.p.mid_n = ws_extent(p, 0);
    c.p.out_n = ws_extent(p, 1);
    c.p.discard = st == kF32 && p->tiles[sid] < 2;
    c.nslot = p->tiles[sid] % 2 == 0 ? 3 : 2;
    c.fwd = 1;
    // x items: 16 real t columns of one wall row, a rows; y items: 8 complex columns of one kx, b rows
    // no L2 promotion: a wider fetch would pull in the next chunks' columns, whose
    // items come hundreds of tickets later (evicted by then, read twice)
    if (!encode_3d(&c.map1, H, rb, (unsigned long long)(b * n), a, 1, b * n * rb, a * b * n * rb, 16,
                   (unsigned)std::min<long long>(a, 256), false) ||
        !encode_3d(&c.map2, b0, cb, n, b, hx, n * cb, b * n * cb, 8, (unsigned)std::min<long long>(b, 256), false))
      return fail(NLOS_ERR_CUDA, "fk xy-forward: tensor map encoding failed");
    NLOS_CU(cudaMemsetAsync(sync, 0, sync_bytes, s), "fk chain counters");
    NLOS_CU(launch_fk_chain(c, st, s), "fk xy-forward");
    NLOS_MARK(p, s, sid++);
  } else {
  // FK1: x forward (real input, scaled by t/(n-1), zero-padded to Lx, kx in [0, Lx/2])
  l = axis(st, (int)Lx, 1, H, b0, b * n, 0, b * n, 0, b * n, (int)a, (int)hx, 0, g2a, p->tw[(int)Lx], p->tiles[sid]);
  // tiles [0, n): direct loads, two real columns per complex transform;
  // [n, 2n): TMA staging, one real column per transform; [2n, 3n): TMA
  // staging of column pairs (n column widths)
  const int nicx = axis_ic_count((int)Lx);
  l.load_mode = (l.tile < nicx || l.tile >= 2 * nicx) ? kLoadRealPair : kLoadReal;
  l.p.t_len = part == 1 ? 0 : (int)n;
  l.p.t_scale = ramp;
  l.p.ld_dev_scale = s_in;
  l.err = err;
  attach_tmap(l);
  set_extents(l, a * b * n, ws_extent(p, 0));
  NLOS_CU(launch_axis_fft(l, s), "fk x-forward");
  NLOS_MARK(p, s, sid++);
  // FK1: y forward (zero-padded to Ly)
  l = axis(st, (int)Ly, hx, b0, b1, n, b * n, n, Ly * n, n, (int)b, (int)Ly, 0, g2b, p->tw[(int)Ly], p->tiles[sid]);
  l.err = err;
  attach_tmap(l);
  set_extents(l, ws_extent(p, 0), ws_extent(p, 1));
  NLOS_CU(launch_axis_fft(l, s), "fk y-forward");
  NLOS_MARK(p, s, sid++);
  }
  if (part == 1) return NLOS_OK;
  // FK3: t forward + Stolt + inverse along z for both Hermitian partners
  FkZParams z{};
  z.G = b1;
  z.psi = b2;
  z.tw = p->tw[(int)Lt];
  z.tw32 = p->tw32.count((int)Lt) ? p->tw32[(int)Lt] : nullptr;
  z.ax = p->ax;
  z.ay = p->ay;
  z.a_pad = (int)Lx;
  z.b_pad = (int)Ly;
  z.n = (int)n;
  z.L = (int)Lt;
  z.pad = (int)pf;
  z.npencils = hx * Ly;
  z.ld_scale = g2n;
  z.st_scale = g2n;
  z.t_ramp = part == 2 ? ramp : 0.0f;
  z.G_n = ws_extent(p, 1);
  z.psi_n = ws_extent(p, 2);
  z.err = err;
  if (p->zlast) {
    // FK3 without its inverses: the resampled spectra of both partners
    NLOS_CU(launch_fk_stolt(z, st, p->tiles[sid], s), "fk stolt stage");
    NLOS_MARK(p, s, sid++);
    // FK4: y inverse (keep y < b) then x inverse (keep x < a), complex, into
    // the second buffer (the forward spectrum is no longer needed)
    FkChainLaunch c{};
    c.p = ch;
    c.p.in = b2;
    c.p.mid = b0;
    c.p.out = b1;
    c.p.s1 = g2b;
    c.p.s2 = g2a;
    c.p.in_n = ws_extent(p, 2);
    c.p.mid_n = ws_extent(p, 0);
    c.p.out_n = std::min<long long>(ws_extent(p, 1), a * b * n);
    c.p.discard = st == kF32 && p->tiles[sid] < 2;
    c.nslot = p->tiles[sid] % 2 == 0 ? 3 : 2;
    c.fwd = 0;
    c.store_mode = kStoreCpx;   // the storage type
    const unsigned box = (unsigned)std::min<long long>(Lx, 256);
    if (!encode_3d(&c.map1, b2, cb, n, Ly, Lx, n * cb, Ly * n * cb, 8, box, false) ||
        !encode_3d(&c.map2, b0, cb, n, Lx, b, b * n * cb, n * cb, 8, box, false))
      return fail(NLOS_ERR_CUDA, "fk yx-inverse: tensor map encoding failed");
    NLOS_CU(cudaMemsetAsync(sync, 0, sync_bytes, s), "fk chain counters");
    NLOS_CU(launch_fk_chain(c, st, s), "fk yx-inverse");
    NLOS_MARK(p, s, sid++);
    // FK5: z inverse of the a x b kept pencils, |psi|^2 (or psi) with the normalisation
    // (the pass scales applied before this last transform now include the x inverse's)
    const double gz = gprod * g2a;
    FkZInvParams zi{};
    zi.in = b1;
    zi.out = vol;
    zi.tw = p->tw[(int)Lt];
    zi.tw32 = p->tw32[(int)Lt];
    zi.L = (int)Lt;
    zi.n = (int)n;
    zi.npencils = a * b;
    zi.scale = (float)(cpx ? 1.0 / (N * gz) : 1.0 / (N * N * gz * gz));
    zi.dev_scale = cpx ? inv_s : inv_s2;
    zi.complex_out = cpx ? 1 : 0;
    zi.in_n = std::min<long long>(ws_extent(p, 1), a * b * n);
    zi.out_n = a * b * n;
    zi.err = err;
    NLOS_CU(launch_fk_zinv(zi, st, p->tiles[sid], s), "fk z-inverse");
    NLOS_MARK(p, s, sid++);
    return NLOS_OK;
  }
  NLOS_CU(launch_fk_zstage(z, st, p->tiles[sid], s), "fk stolt stage");
  NLOS_MARK(p, s, sid++);
  if (p->fused) {
    // FK4 fused: y inverse (keep y < b) then x inverse (keep x < a) with |psi|^2
    FkChainLaunch c{};
    c.p = ch;
    c.p.in = b2;
    c.p.mid = b0;
    c.p.out = vol;
    c.p.s1 = g2b;
    c.p.s2 = fscale;
    c.p.st_dev_scale = cpx ? inv_s : inv_s2;
    c.p.in_n = ws_extent(p, 2);
    c.p.mid_n = ws_extent(p, 0);
    c.p.out_n = a * b * n;
    c.p.discard = st == kF32 && p->tiles[sid] < 2;
    c.nslot = p->tiles[sid] % 2 == 0 ? 3 : 2;
    c.fwd = 0;
    c.store_mode = cpx ? kStoreCpx32 : kStoreAbs2;
    // y items: 8 complex columns of one kx, Ly rows; x items: 8 complex columns of one wall row y, Lx rows
    const unsigned box = (unsigned)std::min<long long>(Lx, 256);
    if (!encode_3d(&c.map1, b2, cb, n, Ly, Lx, n * cb, Ly * n * cb, 8, box, false) ||
        !encode_3d(&c.map2, b0, cb, n, Lx, b, b * n * cb, n * cb, 8, box, false))
      return fail(NLOS_ERR_CUDA, "fk yx-inverse: tensor map encoding failed");
    NLOS_CU(cudaMemsetAsync(sync, 0, sync_bytes, s), "fk chain counters");
    NLOS_CU(launch_fk_chain(c, st, s), "fk yx-inverse");
    NLOS_MARK(p, s, sid++);
    return NLOS_OK;
  }
  // FK4: y inverse (keep y < b)
  l = axis(st, (int)Ly, Lx, b2, b0, n, Ly * n, n, b * n, n, (int)Ly, (int)b, 1, g2b, p->tw[(int)Ly], p->tiles[sid]);
  l.err = err;
  attach_tmap(l);
  set_extents(l, ws_extent(p, 2), ws_extent(p, 0));
  NLOS_CU(launch_axis_fft(l, s), "fk y-inverse");
  NLOS_MARK(p, s, sid++);
  // FK4: x inverse (keep x < a), |psi|^2 with the 1/(Lx Ly Lt) normalisation
  l = axis(st, (int)Lx, 1, b0, vol, b * n, 0, b * n, 0, b * n, (int)Lx, (int)a, 1, fscale, p->tw[(int)Lx], p->tiles[sid]);
  l.store_mode = cpx ? kStoreCpx32 : kStoreAbs2;
  l.p.st_dev_scale = cpx ? inv_s : inv_s2;
  l.err = err;
  attach_tmap(l);
  set_extents(l, ws_extent(p, 0), a * b * n);
  NLOS_CU(launch_axis_fft(l, s), "fk x-inverse");
  NLOS_MARK(p, s, sid++);
  return NLOS_OK;
}

// H: the transient; or, when P_in is given (float32 plans only), the band
// transform is skipped and P_in is the compact phasor field [x][y][F]; or,
// when G0 is given (float32 plans only), the band and the lateral forward
// transforms come from the shared spectrum G0 [Lx/2 + 1][Ly][n] (the x then y
// forward transforms of the transient, taken once for both experts).
nlos_status_t run_pf(nlos_plan_s* p, const void* H, const void* P_in, void* vol, char* ws, cudaStream_t s,
                     const void* G0) {
  const int st = p->storage;
  const long long a = p->a, b = p->b, n = p->n, F = p->F, D = p->D;
  void* b0 = ws + p->off[0];
  void* b1 = ws + p->off[1];
  void* b2 = ws + p->off[2];
  float* scal = reinterpret_cast<float*>(ws + p->off_scal);
  int* err = reinterpret_cast<int*>(ws + p->off_scal + kErrOffset);
  const float* s_in = nullptr;
  const float* inv_s = nullptr;
  int sid = 0;
  NLOS_MARK(p, s, -1);
  if (st != kF32 && !P_in && !G0) {
    NLOS_CU(launch_volume_scale(H, a * b * n, (int)n, 0.0f, st, kVolumeTarget,
                                reinterpret_cast<float*>(ws + p->off_part), kScalePartials, scal, s),
            "volume scale");
    NLOS_MARK(p, s, sid++);
    s_in = scal;
    inv_s = scal + 1;
  }
  const long long Nu = p->Lx, Nv = p->Ly, Lt = p->Lt;
  const float gn = pass_scale(st, (int)Lt), g2a = pass_scale(st, (int)Nu), g2b = pass_scale(st, (int)Nv);
  // depth-sum output scale: undoes the stored kernel's scale and, for 16-bit
  // storage, divides by 16 so sums over the band stay inside the half range
  const float c3 = st == kF32 ? 1.0f : (float)(1.0 / (16.0 * p->kr_scale));
  const double c3_data = st == kF32 ? 1.0 : 1.0 / 16.0;      // c3 * kr_scale
  // PF1: temporal band transform with w(f)
  PfBandParams bp{};
  bp.H = H;
  bp.P = b0;
  bp.tw = p->tw[(int)Lt];
  bp.w = p->w;
  bp.n = (int)n;
  bp.L = (int)Lt;
  bp.k_lo = p->k_lo;
  bp.F = (int)F;
  bp.npencils = a * b;
  bp.ld_scale = 1.0f;
  bp.ld_dev_scale = s_in;
  bp.st_scale = gn;
  bp.H_n = a * b * n;
  bp.P_n = ws_extent(p, 0);
  bp.err = err;
  // the float32 tensor-core depth sum scales the phasors by a bound taken from
  // their largest component: the band transform records it as it stores them
  unsigned* amax = reinterpret_cast<unsigned*>(ws + p->off_scal + kAmaxOffset);
  const bool f16x3 = p->Bu && p->kind_u == kUmmaF16x3;
  if (f16x3 && !P_in) {
    NLOS_CU(cudaMemsetAsync(amax, 0, sizeof(unsigned), s), "phasor bound clear");
    bp.amax = amax;
  }
  const void* P = P_in ? P_in : b0;
  AxisLaunch l{};
  if (G0) {
    // PF1 + PF2 from the shared spectrum: its lateral transforms are already
    // taken (the y and x forward stages record no time of their own)
    PfSpecParams sp{};
    sp.G = static_cast<const float2*>(G0);
    sp.Phat = static_cast<float2*>(b2);
    sp.tw = p->tw[(int)Lt];
    sp.w = p->w;
    sp.n = (int)n;
    sp.L = (int)Lt;
    sp.k_lo = p->k_lo;
    sp.F = (int)F;
    sp.Lx = (int)Nu;
    sp.Ly = (int)Nv;
    sp.amax = bp.amax;
    sp.G_n = (Nu / 2 + 1) * Nv * n;
    sp.Phat_n = ws_extent(p, 2);
    sp.err = err;
    NLOS_CU(launch_pf_band_spectrum(sp, s), "pf band from shared spectrum");
    NLOS_MARK(p, s, sid++);
    sid += 2;
  } else {
  if (!P_in) NLOS_CU(launch_pf_band(bp, st, s), "pf band transform");
  NLOS_MARK(p, s, sid++);
  // PF2: top-left padding and 2D forward transform (y then x) of every band slice
  l = axis(st, (int)Nv, a, P, b1, F, b * F, F, Nv * F, F, (int)b, (int)Nv, 0, g2b, p->tw[(int)Nv], p->tiles[sid]);
  l.err = err;
  attach_tmap(l);
  set_extents(l, P_in ? a * b * F : ws_extent(p, 0), ws_extent(p, 1));
  NLOS_CU(launch_axis_fft(l, s), "pf y-forward");
  NLOS_MARK(p, s, sid++);
  l = axis(st, (int)Nu, 1, b1, b2, Nv * F, 0, Nv * F, 0, Nv * F, (int)a, (int)Nu, 0, g2a, p->tw[(int)Nu], p->tiles[sid]);
  l.err = err;
  attach_tmap(l);
  set_extents(l, ws_extent(p, 1), ws_extent(p, 2));
  NLOS_CU(launch_axis_fft(l, s), "pf x-forward");
  NLOS_MARK(p, s, sid++);
  }
  if (p->d.method == NLOS_PHASOR_DENSE) {
    // PF3, dense kernel: C = sum_f Phat * Khat (Alg. 3), every pixel written
    PfDenseParams dp{static_cast<const float2*>(b2), p->Kd, static_cast<float2*>(b1), Nu * Nv, (int)F, (int)D};
    NLOS_CU(launch_pf_dense(dp, s), "pf dense depth sum");
  } else {
    // PF3: depth sum (pixels beyond the cutoff stay zero); f16 and float32
    // plans run it on the tensor cores (f16 operands / three products of f16 parts)
    // unless the stage's launch shape asks for the FFMA form
    // rows the depth sum does not store: pixels beyond the cutoff, and the
    // rows of tiles whose frequency sum is split (their parts are added)
    const size_t row_bytes = complex_bytes(st) * D;
    if (p->Bu && p->tiles[sid] != 1) {
      PfUmmaParams up{};
      up.Phat = b2;
      up.B = p->Bu;
      up.C = b1;
      up.tile_i01 = p->tu_i01;
      up.tile_pix = p->tu_pix;
      up.tile_alpha = p->tu_alpha;
      up.tile_acut = p->tu_acut;
      up.ntiles = p->ntiles_u;
      up.F = (int)F;
      up.D = (int)D;
      up.Db = p->Db_u;
      up.nblk = p->nblk_u;
      up.KC = p->KC_u;
      up.kind = p->kind_u;
      up.scale = p->kind_u == kUmmaF16 ? c3 : (float)(c3_data / p->bu_scale);
      if (p->kind_u == kUmmaF16x3) {
        // bound on |Phat|: the 2D transforms sum a x b phasors of modulus
        // <= sqrt(2) max|component| (times the passes' scales); phasors the
        // caller supplied get their maximum here
        if (P_in) {
          NLOS_CU(cudaMemsetAsync(amax, 0, sizeof(unsigned), s), "phasor bound clear");
          NLOS_CU(launch_absmax(static_cast<const float*>(P), 2 * a * b * F, amax, s), "phasor bound");
        }
        // (phasors taken from the shared spectrum had their own maximum recorded)
        int e2 = 0;
        frexp(G0 ? 1.5 : 1.5 * (double)a * b * g2a * g2b, &e2);
        up.amax = amax;
        up.abound_exp = e2;
      }
      up.err = err;
      up.Phat_n = ws_extent(p, 2);
      up.C_n = ws_extent(p, 1);
      // launch shape 0: persistent warp-specialised schedule; 2: one CTA per tile
      const bool ws_sched = p->tiles[sid] != 2;
      const int t0 = ws_sched ? pf_umma_first_split_tile(up) : up.ntiles;
      NLOS_CU(launch_clear_rows2(b1, p->clr_pix, p->nclr, p->tu_pix + (size_t)t0 * kUmmaTile,
                                 (long long)(up.ntiles - t0) * kUmmaTile, row_bytes, s),
              "pf clear");
      NLOS_CU(launch_pf_umma(up, ws_sched, s), "pf depth sum (tensor cores)");
    } else {
    NLOS_CU(launch_clear_rows(b1, p->clr_pix, p->nclr, row_bytes, s), "pf clear");
    PfDepthParams dp{};
    dp.Phat = b2;
    dp.K = p->Kr;
    dp.C = b1;
    dp.chunk_i01 = p->ch_i01;
    dp.chunk_pix = p->ch_pix;
    dp.chunk_alpha = p->ch_alpha;
    dp.chunk_acut = p->ch_acut;
    dp.nchunks = p->nchunks;
    dp.F = (int)F;
    dp.D = (int)D;
    dp.scale = c3;
    NLOS_CU(launch_pf_depth(dp, st, p->kr_storage, s), "pf depth sum");
    }
  }
  NLOS_MARK(p, s, sid++);
  // PF4: 2D inverse transform per depth (y then x), crop, |.| with 1/(4ab)
  l = axis(st, (int)Nv, Nu, b1, b0, D, Nv * D, D, b * D, D, (int)Nv, (int)b, 1, g2b, p->tw[(int)Nv], p->tiles[sid]);
  l.err = err;
  attach_tmap(l);
  set_extents(l, ws_extent(p, 1), ws_extent(p, 0));
  NLOS_CU(launch_axis_fft(l, s), "pf y-inverse");
  NLOS_MARK(p, s, sid++);
  // scales the data carries into this last pass (it applies none of its own)
  const double gprod = (double)gn * g2b * g2a * c3_data * g2b;
  const float fscale = (float)(1.0 / ((double)Nu * Nv * gprod));
  l = axis(st, (int)Nu, 1, b0, vol, b * D, 0, b * D, 0, b * D, (int)Nu, (int)a, 1, fscale, p->tw[(int)Nu], p->tiles[sid]);
  l.store_mode = p->d.output == NLOS_OUT_COMPLEX ? kStoreCpx32 : kStoreAbs;
  l.p.st_dev_scale = inv_s;
  l.err = err;
  attach_tmap(l);
  set_extents(l, ws_extent(p, 0), a * b * D);
  NLOS_CU(launch_axis_fft(l, s), "pf x-inverse");
  NLOS_MARK(p, s, sid++);
  return NLOS_OK;
}

nlos_status_t run_plan(nlos_plan_s* p, const void* H, void* vol, void* ws, cudaStream_t s) {
  char* w = static_cast<char*>(ws);
  // errors left pending by earlier, unrelated runtime calls of this thread
  // (the runtime is shared with the host application) must not be reported
  // against this sequence's launches
  cudaGetLastError();
  return p->d.method == NLOS_FK ? run_fk(p, H, vol, w, s, 0) : run_pf(p, H, nullptr, vol, w, s, nullptr);
}

// Dense method (Alg. 3): Khat[kx][ky][f][d] = DFT2 of the spatial kernel on
// the signed padded grid, built once per plan (float64 phase, float32 FFTs
// along y then x through the axis kernels).
nlos_status_t build_dense(nlos_plan_s* p, const std::vector<double>& kappa, const std::vector<double>& depth,
                          int sig_s, int sig_t, double dx, double dy) {
  const int Nu = p->Lx, Nv = p->Ly;
  const long long FD = (long long)p->F * p->D;
  const size_t bytes = sizeof(float2) * (size_t)Nu * Nv * FD;
  nlos_status_t st;
  if ((st = ensure_twiddles(p, Nu)) != NLOS_OK) return st;
  if ((st = ensure_twiddles(p, Nv)) != NLOS_OK) return st;
  void* Kd = nullptr;
  if ((st = dalloc(p, &Kd, bytes, "dense kernel")) != NLOS_OK) return st;
  double *dk = nullptr, *ddep = nullptr;
  float2* T = nullptr;
  cudaError_t e = cudaMalloc(&dk, sizeof(double) * p->F);
  if (e == cudaSuccess) e = cudaMalloc(&ddep, sizeof(double) * p->D);
  if (e == cudaSuccess) e = cudaMalloc(&T, bytes);
  if (e == cudaSuccess) e = cudaMemcpy(dk, kappa.data(), sizeof(double) * p->F, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(ddep, depth.data(), sizeof(double) * p->D, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) {
    DenseGenParams g{dk, ddep, Nu, Nv, p->F, p->D, dx, dy, (double)sig_s, (double)sig_t, p->d.delta_m,
                     static_cast<float2*>(Kd)};
    e = launch_dense_gen(g, 0);    // spatial kernel into Kd, then y (Kd -> T) and x (T -> Kd)
  }
  if (e == cudaSuccess) {
    AxisLaunch l = axis(kF32, Nv, Nu, Kd, T, FD, Nv * FD, FD, Nv * FD, FD, Nv, Nv, 0, 1.0f, p->tw[Nv], 0);
    e = launch_axis_fft(l, 0);
  }
  if (e == cudaSuccess) {
    AxisLaunch l = axis(kF32, Nu, 1, T, Kd, (long long)Nv * FD, 0, (long long)Nv * FD, 0, (long long)Nv * FD, Nu, Nu, 0,
                        1.0f, p->tw[Nu], 0);
    e = launch_axis_fft(l, 0);
  }
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (dk) cudaFree(dk);
  if (ddep) cudaFree(ddep);
  if (T) cudaFree(T);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return cuda_fail(e, "dense kernel build");
  }
  p->Kd = static_cast<float2*>(Kd);
  return NLOS_OK;
}

std::mutex g_pool_mu;
cudaStream_t g_streams[kBatchStreams];
cudaEvent_t g_fork = nullptr;
cudaEvent_t g_join[kBatchStreams];
bool g_pool_ready = false;

nlos_status_t ensure_pool() {
  std::lock_guard<std::mutex> lk(g_pool_mu);
  if (g_pool_ready) return NLOS_OK;
  NLOS_CU(cudaEventCreateWithFlags(&g_fork, cudaEventDisableTiming), "batch pool");
  for (int i = 0; i < kBatchStreams; ++i) {
    NLOS_CU(cudaStreamCreateWithFlags(&g_streams[i], cudaStreamNonBlocking), "batch pool");
    NLOS_CU(cudaEventCreateWithFlags(&g_join[i], cudaEventDisableTiming), "batch pool");
  }
  g_pool_ready = true;
  return NLOS_OK;
}

nlos_status_t validate(const nlos_plan_desc_t* d) {
  if (!d) return fail(NLOS_ERR_INVALID_ARG, "desc is NULL");
  if (d->method != NLOS_FK && d->method != NLOS_PHASOR_RSD && d->method != NLOS_PHASOR_DENSE)
    return fail(NLOS_ERR_INVALID_ARG, "unknown method %d", d->method);
  if (d->method == NLOS_PHASOR_DENSE && d->storage != NLOS_F32)
    return fail(NLOS_ERR_UNSUPPORTED, "the dense phasor-field method stores float32 only");
  if (d->storage != NLOS_F32 && d->storage != NLOS_F16 && d->storage != NLOS_BF16)
    return fail(NLOS_ERR_INVALID_ARG, "unknown storage %d", d->storage);
  if (d->nx <= 0 || d->ny <= 0 || d->nt <= 0) return fail(NLOS_ERR_INVALID_ARG, "sizes must be positive");
  if (!(d->bin_width_s > 0) || !(d->wall_w_m > 0) || !(d->wall_h_m > 0))
    return fail(NLOS_ERR_INVALID_ARG, "bin width and wall extent must be > 0");
  if (d->pad_factor != 2 && d->pad_factor != 1) return fail(NLOS_ERR_INVALID_ARG, "pad_factor must be 1 or 2");
  if (d->output != NLOS_OUT_MAGNITUDE && d->output != NLOS_OUT_COMPLEX)
    return fail(NLOS_ERR_INVALID_ARG, "unknown output %d", d->output);
  if (d->pad_factor == 1 && d->method != NLOS_FK)
    return fail(NLOS_ERR_UNSUPPORTED, "the unpadded variant exists for f-k only");
  if (d->pad_factor == 1 && (d->nx < 16 || d->ny < 16))
    return fail(NLOS_ERR_UNSUPPORTED, "unpadded f-k needs nx, ny >= 16");
  if (d->pad_factor == 1 && (!is_pow2(d->nx) || !is_pow2(d->ny) || !is_pow2(d->nt)))
    return fail(NLOS_ERR_UNSUPPORTED, "unpadded f-k needs power-of-two sizes");
  if (d->nx < 8 || d->ny < 8 || d->nx > 1024 || d->ny > 1024)
    return fail(NLOS_ERR_UNSUPPORTED, "nx, ny must be in [8, 1024]");
  if (d->nt < 16 || d->nt > 4096) return fail(NLOS_ERR_UNSUPPORTED, "nt must be in [16, 4096]");
  if (d->method != NLOS_FK) {
    if (d->n_depths < 1 || d->n_depths > 8192) return fail(NLOS_ERR_INVALID_ARG, "n_depths must be in [1, 8192]");
    if (!(d->depth_min_m > 0) || d->depth_max_m < d->depth_min_m)
      return fail(NLOS_ERR_INVALID_ARG, "depth range must satisfy 0 < min <= max");
    if (d->wavelength_m < 0 || d->cycles < 0) return fail(NLOS_ERR_INVALID_ARG, "wavelength/cycles must be >= 0");
    const bool conf = d->sigma_s == 0 && d->sigma_t == 0;
    if (!conf && !(d->sigma_s >= 1 && d->sigma_t >= 0)) return fail(NLOS_ERR_INVALID_ARG, "bad modality pair");
  }
  return NLOS_OK;
}

void destroy_pipe(HostPipe* hp) {
  if (!hp) return;
  for (int k = 0; k < kPipeSlots; ++k) {
    if (hp->in_ready[k]) cudaEventDestroy(hp->in_ready[k]);
    if (hp->done[k]) cudaEventDestroy(hp->done[k]);
    if (hp->out_free[k]) cudaEventDestroy(hp->out_free[k]);
  }
  if (hp->start) cudaEventDestroy(hp->start);
  if (hp->h2d) cudaStreamDestroy(hp->h2d);
  if (hp->comp) cudaStreamDestroy(hp->comp);
  if (hp->d2h) cudaStreamDestroy(hp->d2h);
  delete hp;
}

nlos_status_t ensure_pipe(nlos_plan_s* p, size_t ib, size_t ob) {
  if (p->pipe) return NLOS_OK;
  HostPipe* hp = new HostPipe();
  cudaError_t e = cudaSuccess;
  for (int k = 0; k < kPipeSlots && e == cudaSuccess; ++k) {
    e = cudaEventCreateWithFlags(&hp->in_ready[k], cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&hp->done[k], cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&hp->out_free[k], cudaEventDisableTiming);
  }
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&hp->start, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&hp->h2d, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&hp->comp, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&hp->d2h, cudaStreamNonBlocking);
  if (e != cudaSuccess) {
    destroy_pipe(hp);
    cudaGetLastError();
    return cuda_fail(e, "host pipeline streams");
  }
  nlos_status_t st = NLOS_OK;
  for (int k = 0; k < kPipeSlots && st == NLOS_OK; ++k) {
    st = dalloc(p, &hp->d_in[k], ib, "host pipeline staging");
    if (st == NLOS_OK) st = dalloc(p, &hp->d_out[k], ob, "host pipeline staging");
  }
  if (st != NLOS_OK) {
    destroy_pipe(hp);
    return st;
  }
  p->pipe = hp;
  return NLOS_OK;
}

}  // namespace

extern "C" {

void nlos_plan_desc_default(nlos_plan_desc_t* d) {
  if (!d) return;
  memset(d, 0, sizeof *d);
  d->method = NLOS_FK;
  d->storage = NLOS_F32;
  d->pad_factor = 2;
  d->cycles = 5.0;
}

nlos_status_t nlos_plan_create(const nlos_plan_desc_t* desc, nlos_plan_t* out) {
  return nlos_plan_create_ex(desc, 0, out);
}

nlos_status_t nlos_plan_create_ex(const nlos_plan_desc_t* desc, int flags, nlos_plan_t* out) {
  g_err.clear();
  if (!out) return fail(NLOS_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  nlos_status_t st = validate(desc);
  if (st != NLOS_OK) return st;
  nlos_plan_s* p = new nlos_plan_s();
  p->d = *desc;
  p->a = desc->nx;
  p->b = desc->ny;
  p->n = desc->nt;
  {
    // transform lengths: f-k pads every axis to the next power of two >= 2x
    // (exactly 2x for power-of-two sizes) or keeps it (pad_factor 1); phasor
    // fields pad x and y the same way and transform t at the next power of
    // two >= nt
    const bool fk = desc->method == NLOS_FK;
    const int pad = fk ? desc->pad_factor : 2;
    p->Lx = pad == 1 ? p->a : pow2_at_least(2 * p->a);
    p->Ly = pad == 1 ? p->b : pow2_at_least(2 * p->b);
    p->Lt = fk ? (pad == 1 ? p->n : pow2_at_least(2 * p->n)) : pow2_at_least(p->n);
  }
  p->storage = desc->storage;
  p->fused = desc->method == NLOS_FK && !(flags & NLOS_PLAN_SEPARATE_AXES) &&
             fk_chain_eligible(p->a, p->b, p->n, p->Lx, p->Ly, desc->pad_factor);
  // plans with fused lateral stages and L = 2n take the inverse temporal
  // transform last, on the kept pencils
  p->zlast = p->fused && p->Lt == 2 * p->n;
  if (p->storage != kF32) p->stage_names.push_back("volume_scale");
  const char* fk_names[] = {"fk_x_forward", "fk_y_forward", "fk_stolt_z", "fk_y_inverse", "fk_x_inverse"};
  const char* fk_fused_names[] = {"fk_xy_forward", "fk_stolt_z", "fk_yx_inverse"};
  const char* fk_zlast_names[] = {"fk_xy_forward", "fk_stolt", "fk_yx_inverse", "fk_z_inverse"};
  const char* pf_names[] = {"pf_band", "pf_y_forward", "pf_x_forward", "pf_depth_sum", "pf_y_inverse",
                            "pf_x_inverse"};
  if (desc->method == NLOS_FK && p->zlast) for (const char* nm : fk_zlast_names) p->stage_names.push_back(nm);
  else if (desc->method == NLOS_FK && p->fused) for (const char* nm : fk_fused_names) p->stage_names.push_back(nm);
  else if (desc->method == NLOS_FK) for (const char* nm : fk_names) p->stage_names.push_back(nm);
  else for (const char* nm : pf_names) p->stage_names.push_back(nm);
  for (const std::string& nm : p->stage_names) {
    const bool xs = nm.find("_x_") != std::string::npos, ys = nm.find("_y_") != std::string::npos;
    const bool umma = nm == "pf_depth_sum" && desc->method == NLOS_PHASOR_RSD &&
                      (desc->storage == NLOS_F16 || desc->storage == NLOS_F32);
    const bool chain = nm == "fk_xy_forward" || nm == "fk_yx_inverse";
    const bool zsplit = nm == "fk_stolt" || nm == "fk_z_inverse";
    p->stage_kind.push_back(nm == "fk_x_forward" ? 3 : xs || ys ? 1 : nm == "fk_stolt_z" ? 2 : umma ? 4 : chain ? 5
                            : zsplit ? 6 : 0);
    p->stage_len.push_back(xs ? p->Lx : ys ? p->Ly : (nm == "fk_stolt_z" || zsplit) ? p->Lt : 0);
  }
  // default launch shapes: TMA-staged axis transforms (each falls back to
  // direct loads where the layout does not allow TMA); the autotuner may
  // choose others
  p->tiles.assign(p->stage_names.size(), 0);
  for (size_t i = 0; i < p->tiles.size(); ++i) {
    if (p->stage_kind[i] == 1 || p->stage_kind[i] == 3) p->tiles[i] = axis_ic_count(p->stage_len[i]);
    if (p->stage_kind[i] == 2) p->tiles[i] = fk_tile_default(p->stage_len[i]);
    if (p->stage_kind[i] == 5) p->tiles[i] = 1;   // fused lateral pair: two slots, intermediate dropped from L2
  }
  st = desc->method == NLOS_FK ? build_fk(p) : build_pf(p);
  // every stage buffer lies inside [0, ws_bytes): the regions are laid out in
  // order and the scalar area and partials close the workspace. Callers that
  // supply scratch (nlos_reconstruct_ws, the fixed array of
  // nlos_reconstruct_noalloc) size it by ws_bytes alone.
  if (st == NLOS_OK && !(p->off[0] <= p->off[1] && p->off[1] <= p->off[2] && p->off[2] <= p->off_scal &&
                         p->off_scal + 256 <= p->off_part && p->off_part < p->off_sync && p->off_sync < p->ws_bytes))
    st = fail(NLOS_ERR_UNSUPPORTED, "internal: workspace layout out of order");
  const bool own_ws = !(flags & NLOS_PLAN_NO_WORKSPACE);
  if (st == NLOS_OK && own_ws) st = dalloc(p, &p->ws, p->ws_bytes, "workspace");
  if (st == NLOS_OK && own_ws) {
    cudaError_t e = cudaMemset(p->ws, 0, p->ws_bytes);
    if (e != cudaSuccess) st = cuda_fail(e, "workspace clear");
  }
  if (st != NLOS_OK) {
    for (void* v : p->allocs) cudaFree(v);
    delete p;
    return st;
  }
  *out = p;
  return NLOS_OK;
}

nlos_status_t nlos_plan_query(nlos_plan_t p, size_t out_shape[3], size_t* workspace_bytes, size_t* input_bytes,
                              size_t* output_bytes) {
  if (!p) return fail(NLOS_ERR_INVALID_ARG, "plan is NULL");
  if (out_shape) {
    out_shape[0] = p->a;
    out_shape[1] = p->b;
    out_shape[2] = p->nz;
  }
  if (workspace_bytes) *workspace_bytes = p->ws_bytes;
  if (input_bytes) *input_bytes = (size_t)p->a * p->b * p->n * real_bytes(p->storage);
  if (output_bytes)
    *output_bytes = (size_t)p->a * p->b * p->nz * (p->d.output == NLOS_OUT_COMPLEX ? sizeof(float2) : sizeof(float));
  return NLOS_OK;
}

nlos_status_t nlos_reconstruct_ws(nlos_plan_t p, const void* transient, void* volume, void* workspace,
                                  size_t workspace_bytes, void* stream) {
  if (!p) return fail(NLOS_ERR_INVALID_ARG, "plan is NULL");
  if (!transient || !volume) return fail(NLOS_ERR_INVALID_ARG, "transient/volume is NULL");
  if (!workspace || workspace_bytes < p->ws_bytes)
    return fail(NLOS_ERR_INVALID_ARG, "workspace too small (%zu < %zu)", workspace_bytes, p->ws_bytes);
  if (reinterpret_cast<uintptr_t>(workspace) & 255) return fail(NLOS_ERR_INVALID_ARG, "workspace not 256-byte aligned");
  return run_plan(p, transient, volume, workspace, static_cast<cudaStream_t>(stream));
}

nlos_status_t nlos_reconstruct(nlos_plan_t p, const void* transient, void* volume, void* stream) {
  if (!p) return fail(NLOS_ERR_INVALID_ARG, "plan is NULL");
  if (!p->ws) return fail(NLOS_ERR_INVALID_ARG, "plan was created without a workspace; use nlos_reconstruct_ws");
  return nlos_reconstruct_ws(p, transient, volume, p->ws, p->ws_bytes, stream);
}

nlos_status_t nlos_plan_band(nlos_plan_t p, int* k_lo, int* n_freqs) {
  if (!p) return fail(NLOS_ERR_INVALID_ARG, "plan is NULL");
  if (p->d.method == NLOS_FK) return fail(NLOS_ERR_INVALID_ARG, "not a phasor-field plan");
  if (k_lo) *k_lo = p->k_lo;
  if (n_freqs) *n_freqs = p->F;
  return NLOS_OK;
}

nlos_status_t nlos_bin_phasors(nlos_plan_t p, const uint32_t* pixel, const uint32_t* ticks, long long count,
                               uint32_t t0_ticks, uint32_t ticks_per_bin, int flags, void* phasors,
                               void* stream) {
  if (!p) return fail(NLOS_ERR_INVALID_ARG, "plan is NULL");
  if (p->d.method == NLOS_FK) return fail(NLOS_ERR_INVALID_ARG, "not a phasor-field plan");
  if (!phasors || count < 0 || (count > 0 && (!pixel || !ticks)) || ticks_per_bin == 0 || (flags & ~7) ||
      (flags & NLOS_BIN_DIRECT && flags & NLOS_BIN_VIA_HISTOGRAM))
    return fail(NLOS_ERR_INVALID_ARG, "bad binning arguments");
  const bool accumulate = flags & NLOS_BIN_ACCUMULATE;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaGetLastError();
  // route: per-photon phasors (cost ~ photons x F) or a histogram in the
  // workspace plus the band transform (cost ~ grid size)
  const long long cells = (long long)p->a * p->b * p->n;
  const size_t hbytes = sizeof(float) * (size_t)cells;
  const bool room = p->ws && hbytes <= p->off_scal;
  if (flags & NLOS_BIN_VIA_HISTOGRAM && !room)
    return fail(NLOS_ERR_INVALID_ARG, "the histogram route needs the plan's workspace");
  const bool hist = room && !(flags & NLOS_BIN_DIRECT) &&
                    ((flags & NLOS_BIN_VIA_HISTOGRAM) || (double)count * p->F > 2.0 * (double)cells);
  if (hist) {
    float* Hs = static_cast<float*>(p->ws);
    NLOS_CU(cudaMemsetAsync(Hs, 0, hbytes, s), "histogram clear");
    NLOS_CU(launch_bin_transient(pixel, ticks, count, (uint32_t)((long long)p->a * p->b), (uint32_t)p->n, t0_ticks,
                                 ticks_per_bin, Hs, s),
            "photon histogram");
    PfBandParams bp{};
    bp.H = Hs;
    bp.P = phasors;
    bp.tw = p->tw[p->Lt];
    bp.w = p->w;
    bp.n = p->n;
    bp.L = p->Lt;
    bp.k_lo = p->k_lo;
    bp.F = p->F;
    bp.npencils = (long long)p->a * p->b;
    bp.ld_scale = 1.0f;
    bp.st_scale = 1.0f;
    bp.accumulate = accumulate ? 1 : 0;
    NLOS_CU(launch_pf_band(bp, kF32, s), "phasors from histogram");
    return NLOS_OK;
  }
  if (!accumulate) NLOS_CU(cudaMemsetAsync(phasors, 0, sizeof(float2) * (size_t)p->a * p->b * p->F, s), "phasor clear");
  if (count == 0) return NLOS_OK;
  PhasorBinParams q{};
  q.pixel = pixel;
  q.ticks = ticks;
  q.count = count;
  q.npix = (uint32_t)((long long)p->a * p->b);
  q.nt = p->n;
  q.n = p->Lt;
  q.t0 = t0_ticks;
  q.tpb = ticks_per_bin;
  q.phase = p->phase;
  q.w = p->w;
  q.k_lo = p->k_lo;
  q.F = p->F;
  q.P = static_cast<float2*>(phasors);
  q.err = p->ws ? reinterpret_cast<int*>(static_cast<char*>(p->ws) + p->off_scal + kErrOffset) : nullptr;
  NLOS_CU(launch_bin_phasors(q, s), "phasor binning");
  return NLOS_OK;
}

nlos_status_t nlos_reconstruct_phasors(nlos_plan_t p, const void* phasors, void* volume, void* stream) {
  if (!p) return fail(NLOS_ERR_INVALID_ARG, "plan is NULL");
  if (p->d.method == NLOS_FK) return fail(NLOS_ERR_INVALID_ARG, "not a phasor-field plan");
  if (p->storage != kF32) return fail(NLOS_ERR_UNSUPPORTED, "phasor input needs a float32 plan");
  if (!phasors || !volume) return fail(NLOS_ERR_INVALID_ARG, "phasors/volume is NULL");
  if (!p->ws) return fail(NLOS_ERR_INVALID_ARG, "plan was created without a workspace");
  cudaGetLastError();
  return run_pf(p, nullptr, phasors, volume, static_cast<char*>(p->ws), static_cast<cudaStream_t>(stream), nullptr);
}


nlos_status_t nlos_reconstruct_moe(nlos_plan_t fk, nlos_plan_t pf, const void* transient, void* volume_fk,
                                   void* volume_pf, void* stream, void* stream2) {
  if (!fk || !pf) return fail(NLOS_ERR_INVALID_ARG, "plan is NULL");
  if (!transient || !volume_fk || !volume_pf) return fail(NLOS_ERR_INVALID_ARG, "transient/volume is NULL");
  if (fk->d.method != NLOS_FK || pf->d.method == NLOS_FK)
    return fail(NLOS_ERR_INVALID_ARG, "needs an f-k plan and a phasor-field plan");
  if (!fk->ws || !pf->ws) return fail(NLOS_ERR_INVALID_ARG, "both plans need their own workspace");
  if (fk->storage != kF32 || pf->storage != kF32)
    return fail(NLOS_ERR_UNSUPPORTED, "the shared spectrum needs float32 plans");
  if (fk->a != pf->a || fk->b != pf->b || fk->n != pf->n || fk->Lx != pf->Lx || fk->Ly != pf->Ly)
    return fail(NLOS_ERR_INVALID_ARG, "plans differ in grid (%dx%dx%d vs %dx%dx%d) or lateral padding", fk->a, fk->b,
                fk->n, pf->a, pf->b, pf->n);
  cudaStream_t s = static_cast<cudaStream_t>(stream), s2 = static_cast<cudaStream_t>(stream2);
  const bool two = s2 != s;
  if (two)
    for (cudaEvent_t& e : fk->moe_ev)
      if (!e) NLOS_CU(cudaEventCreateWithFlags(&e, cudaEventDisableTiming), "mixture-of-experts event");
  cudaGetLastError();
  char* wf = static_cast<char*>(fk->ws);
  // the shared spectrum lives in the f-k plan's second buffer, which the
  // f-k temporal stage only reads and the phasor branch only reads
  const void* G0 = wf + fk->off[1];
  nlos_status_t st = run_fk(fk, transient, volume_fk, wf, s, 1);
  if (st != NLOS_OK) return st;
  if (two) {
    NLOS_CU(cudaEventRecord(fk->moe_ev[0], s), "mixture-of-experts order");
    NLOS_CU(cudaStreamWaitEvent(s2, fk->moe_ev[0], 0), "mixture-of-experts order");
  }
  st = run_pf(pf, nullptr, nullptr, volume_pf, static_cast<char*>(pf->ws), s2, G0);
  if (st != NLOS_OK) return st;
  st = run_fk(fk, transient, volume_fk, wf, s, 2);
  if (st != NLOS_OK) return st;
  if (two) {
    // join: the next call's spectrum must not overwrite what the phasor branch still reads
    NLOS_CU(cudaEventRecord(fk->moe_ev[1], s2), "mixture-of-experts order");
    NLOS_CU(cudaStreamWaitEvent(s, fk->moe_ev[1], 0), "mixture-of-experts order");
  }
  return NLOS_OK;
}

nlos_status_t nlos_reconstruct_host_many(nlos_plan_t p, const void* const* transients_host, void* const* volumes_host,
                                         int n, void* stream) {
  if (!p) return fail(NLOS_ERR_INVALID_ARG, "plan is NULL");
  if (n < 0 || (n > 0 && (!transients_host || !volumes_host))) return fail(NLOS_ERR_INVALID_ARG, "bad host arrays");
  if (!p->ws) return fail(NLOS_ERR_INVALID_ARG, "plan was created without a workspace");
  for (int i = 0; i < n; ++i)
    if (!transients_host[i] || !volumes_host[i]) return fail(NLOS_ERR_INVALID_ARG, "host buffer %d is NULL", i);
  if (n == 0) return NLOS_OK;
  size_t ib = 0, ob = 0;
  nlos_plan_query(p, nullptr, nullptr, &ib, &ob);
  nlos_status_t st = ensure_pipe(p, ib, ob);
  if (st != NLOS_OK) return st;
  HostPipe* hp = p->pipe;
  cudaGetLastError();
  // everything runs after the work already queued on the caller's stream
  NLOS_CU(cudaEventRecord(hp->start, static_cast<cudaStream_t>(stream)), "host pipeline order");
  NLOS_CU(cudaStreamWaitEvent(hp->h2d, hp->start, 0), "host pipeline order");
  NLOS_CU(cudaStreamWaitEvent(hp->comp, hp->start, 0), "host pipeline order");
  NLOS_CU(cudaStreamWaitEvent(hp->d2h, hp->start, 0), "host pipeline order");
  for (int i = 0; i < n; ++i) {
    const int k = i % kPipeSlots;
    if (i >= kPipeSlots) NLOS_CU(cudaStreamWaitEvent(hp->h2d, hp->done[k], 0), "host pipeline order");
    NLOS_CU(cudaMemcpyAsync(hp->d_in[k], transients_host[i], ib, cudaMemcpyHostToDevice, hp->h2d), "host->device copy");
    NLOS_CU(cudaEventRecord(hp->in_ready[k], hp->h2d), "host pipeline order");
    NLOS_CU(cudaStreamWaitEvent(hp->comp, hp->in_ready[k], 0), "host pipeline order");
    if (i >= kPipeSlots) NLOS_CU(cudaStreamWaitEvent(hp->comp, hp->out_free[k], 0), "host pipeline order");
    st = run_plan(p, hp->d_in[k], hp->d_out[k], p->ws, hp->comp);
    if (st != NLOS_OK) {
      cudaStreamSynchronize(hp->comp);
      cudaStreamSynchronize(hp->h2d);
      cudaStreamSynchronize(hp->d2h);
      return st;
    }
    NLOS_CU(cudaEventRecord(hp->done[k], hp->comp), "host pipeline order");
    NLOS_CU(cudaStreamWaitEvent(hp->d2h, hp->done[k], 0), "host pipeline order");
    NLOS_CU(cudaMemcpyAsync(volumes_host[i], hp->d_out[k], ob, cudaMemcpyDeviceToHost, hp->d2h), "device->host copy");
    NLOS_CU(cudaEventRecord(hp->out_free[k], hp->d2h), "host pipeline order");
  }
  NLOS_CU(cudaStreamSynchronize(hp->d2h), "host pipeline sync");
  NLOS_CU(cudaStreamSynchronize(hp->comp), "host pipeline sync");
  NLOS_CU(cudaStreamSynchronize(hp->h2d), "host pipeline sync");
  return NLOS_OK;
}

nlos_status_t nlos_reconstruct_host(nlos_plan_t p, const void* th, void* vh, void* stream) {
  if (!p) return fail(NLOS_ERR_INVALID_ARG, "plan is NULL");
  if (!th || !vh) return fail(NLOS_ERR_INVALID_ARG, "host buffer is NULL");
  if (!p->ws) return fail(NLOS_ERR_INVALID_ARG, "plan was created without a workspace");
  size_t ib = 0, ob = 0;
  nlos_plan_query(p, nullptr, nullptr, &ib, &ob);
  nlos_status_t st;
  if (!p->d_in && (st = dalloc(p, &p->d_in, ib, "host staging")) != NLOS_OK) return st;
  if (!p->d_out && (st = dalloc(p, &p->d_out, ob, "host staging")) != NLOS_OK) return st;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  NLOS_CU(cudaMemcpyAsync(p->d_in, th, ib, cudaMemcpyHostToDevice, s), "host->device copy");
  st = run_plan(p, p->d_in, p->d_out, p->ws, s);
  if (st != NLOS_OK) return st;
  NLOS_CU(cudaMemcpyAsync(vh, p->d_out, ob, cudaMemcpyDeviceToHost, s), "device->host copy");
  NLOS_CU(cudaStreamSynchronize(s), "host call sync");
  return NLOS_OK;
}

nlos_status_t nlos_reconstruct_batch(const nlos_plan_t* plans, const void* const* transients, void* const* volumes,
                                     void* const* workspaces, int n, void* stream) {
  if (n < 0 || (n > 0 && (!plans || !transients || !volumes))) return fail(NLOS_ERR_INVALID_ARG, "bad batch arrays");
  if (n == 0) return NLOS_OK;
  for (int i = 0; i < n; ++i) {
    if (!plans[i] || !transients[i] || !volumes[i]) return fail(NLOS_ERR_INVALID_ARG, "batch item %d is NULL", i);
    if (!workspaces && !plans[i]->ws)
      return fail(NLOS_ERR_INVALID_ARG, "batch item %d: plan has no workspace and none was given", i);
    if (!workspaces)
      for (int j = 0; j < i; ++j)
        if (plans[j] == plans[i]) return fail(NLOS_ERR_INVALID_ARG, "plan repeated in batch without workspaces");
    if (workspaces && (!workspaces[i] || (reinterpret_cast<uintptr_t>(workspaces[i]) & 255)))
      return fail(NLOS_ERR_INVALID_ARG, "batch workspace %d is NULL or misaligned", i);
  }
  nlos_status_t st = ensure_pool();
  if (st != NLOS_OK) return st;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int used = std::min(n, kBatchStreams);
  NLOS_CU(cudaEventRecord(g_fork, s), "batch fork");
  for (int k = 0; k < used; ++k) NLOS_CU(cudaStreamWaitEvent(g_streams[k], g_fork, 0), "batch fork");
  for (int i = 0; i < n; ++i) {
    void* ws = workspaces ? workspaces[i] : plans[i]->ws;
    st = run_plan(plans[i], transients[i], volumes[i], ws, g_streams[i % kBatchStreams]);
    if (st != NLOS_OK) return st;
  }
  for (int k = 0; k < used; ++k) {
    NLOS_CU(cudaEventRecord(g_join[k], g_streams[k]), "batch join");
    NLOS_CU(cudaStreamWaitEvent(s, g_join[k], 0), "batch join");
  }
  return NLOS_OK;
}

// ---------------------------------------------------------------------------
// autotuner: coordinate descent over each stage's tile variants, timing the
// whole sequence with CUDA events; results cached per plan shape (and in a
// JSON file named by NLOS_AUTOTUNE_CACHE, if set)
// ---------------------------------------------------------------------------
}  // extern "C"

namespace {
std::mutex g_tune_mu;
std::map<std::string, std::vector<int>> g_tune_cache;
bool g_tune_loaded = false;

std::string tune_key(const nlos_plan_s* p) {
  char buf[256];
  snprintf(buf, sizeof buf, "m%d_s%d_%dx%dx%d_F%d_D%d", p->d.method, p->storage, p->a, p->b, p->n, p->F, p->D);
  return buf;
}

void tune_cache_load() {
  if (g_tune_loaded) return;
  g_tune_loaded = true;
  const char* path = getenv("NLOS_AUTOTUNE_CACHE");
  if (!path) return;
  FILE* f = fopen(path, "r");
  if (!f) return;
  std::string txt;
  char buf[4096];
  size_t k;
  while ((k = fread(buf, 1, sizeof buf, f)) > 0) txt.append(buf, k);
  fclose(f);
  // flat JSON object: {"key": [v, v, ...], ...}
  size_t i = 0;
  while ((i = txt.find('"', i)) != std::string::npos) {
    const size_t e = txt.find('"', i + 1);
    if (e == std::string::npos) break;
    const std::string key = txt.substr(i + 1, e - i - 1);
    const size_t lb = txt.find('[', e), rb = txt.find(']', e);
    if (lb == std::string::npos || rb == std::string::npos || rb < lb) break;
    std::vector<int> v;
    const char* c = txt.c_str() + lb + 1;
    while (c < txt.c_str() + rb) {
      char* endp = nullptr;
      const long x = strtol(c, &endp, 10);
      if (endp == c) { ++c; continue; }
      v.push_back((int)x);
      c = endp;
    }
    g_tune_cache[key] = v;
    i = rb + 1;
  }
}

void tune_cache_save() {
  const char* path = getenv("NLOS_AUTOTUNE_CACHE");
  if (!path) return;
  FILE* f = fopen(path, "w");
  if (!f) return;
  fprintf(f, "{\n");
  size_t n = 0;
  for (const auto& kv : g_tune_cache) {
    fprintf(f, "  \"%s\": [", kv.first.c_str());
    for (size_t j = 0; j < kv.second.size(); ++j) fprintf(f, "%s%d", j ? ", " : "", kv.second[j]);
    fprintf(f, "]%s\n", ++n < g_tune_cache.size() ? "," : "");
  }
  fprintf(f, "}\n");
  fclose(f);
}

int stage_variants(const nlos_plan_s* p, size_t i) {
  if (p->stage_kind[i] == 1) return axis_tile_count(p->stage_len[i]);
  if (p->stage_kind[i] == 2) return fk_tile_count(p->stage_len[i]);
  if (p->stage_kind[i] == 3) return 3 * axis_ic_count(p->stage_len[i]);
  if (p->stage_kind[i] == 4) return 3;   // tensor cores (persistent), FFMA, tensor cores (CTA per tile)
  // fused lateral pair: {3, 2} slots per CTA x {intermediate dropped from L2 after use, kept}
  if (p->stage_kind[i] == 5) return 4;
  // temporal stages of the split inverse: radix-16 / radix-32 passes x two pencils-per-CTA counts
  if (p->stage_kind[i] == 6) return 4;
  return 1;
}
}  // namespace

extern "C" {

nlos_status_t nlos_plan_autotune(nlos_plan_t p, void* stream) {
  if (!p) return fail(NLOS_ERR_INVALID_ARG, "plan is NULL");
  if (p->prof_on) return fail(NLOS_ERR_INVALID_ARG, "disable stage tracing before autotuning");
  const std::string key = tune_key(p);
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    tune_cache_load();
    auto it = g_tune_cache.find(key);
    if (it != g_tune_cache.end() && it->second.size() == p->tiles.size()) {
      p->tiles = it->second;
      p->tuned = true;
      return NLOS_OK;
    }
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  size_t ib = 0, ob = 0;
  nlos_plan_query(p, nullptr, nullptr, &ib, &ob);
  void *din = nullptr, *dout = nullptr, *tws = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e = cudaMalloc(&din, ib);
  if (e == cudaSuccess) e = cudaMalloc(&dout, ob);
  if (e == cudaSuccess && !p->ws) e = cudaMalloc(&tws, p->ws_bytes);
  void* ws = p->ws ? p->ws : tws;
  if (e == cudaSuccess) e = cudaMemsetAsync(din, 0, ib, s);
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  nlos_status_t st = e == cudaSuccess ? NLOS_OK : cuda_fail(e, "autotune buffers");
  auto time_seq = [&](float* ms) -> nlos_status_t {
    nlos_status_t r = run_plan(p, din, dout, ws, s);
    if (r != NLOS_OK) return r;
    NLOS_CU(cudaEventRecord(e0, s), "autotune timing");
    for (int k = 0; k < 3; ++k) {
      r = run_plan(p, din, dout, ws, s);
      if (r != NLOS_OK) return r;
    }
    NLOS_CU(cudaEventRecord(e1, s), "autotune timing");
    NLOS_CU(cudaEventSynchronize(e1), "autotune timing");
    NLOS_CU(cudaEventElapsedTime(ms, e0, e1), "autotune timing");
    return NLOS_OK;
  };
  for (size_t i = 0; st == NLOS_OK && i < p->tiles.size(); ++i) {
    const int nv = stage_variants(p, i);
    if (nv < 2) continue;
    int best = p->tiles[i];
    float best_ms = 1e30f;
    for (int v = 0; v < nv && st == NLOS_OK; ++v) {
      p->tiles[i] = v;
      float ms = 0.f;
      st = time_seq(&ms);
      if (st == NLOS_OK && ms < best_ms) {
        best_ms = ms;
        best = v;
      }
    }
    p->tiles[i] = best;
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaStreamSynchronize(s);
  if (din) cudaFree(din);
  if (dout) cudaFree(dout);
  if (tws) cudaFree(tws);
  if (st != NLOS_OK) return st;
  p->tuned = true;
  std::lock_guard<std::mutex> lk(g_tune_mu);
  g_tune_cache[key] = p->tiles;
  tune_cache_save();
  return NLOS_OK;
}

nlos_status_t nlos_plan_get_tiles(nlos_plan_t p, int* tiles, int capacity, int* n_stages) {
  if (!p) return fail(NLOS_ERR_INVALID_ARG, "plan is NULL");
  if (n_stages) *n_stages = (int)p->tiles.size();
  for (int i = 0; tiles && i < capacity && i < (int)p->tiles.size(); ++i) tiles[i] = p->tiles[i];
  return NLOS_OK;
}

nlos_status_t nlos_plan_set_tiles(nlos_plan_t p, const int* tiles, int n) {
  if (!p || !tiles || n != (int)p->tiles.size()) return fail(NLOS_ERR_INVALID_ARG, "bad tile vector");
  for (int i = 0; i < n; ++i)
    if (tiles[i] < 0 || tiles[i] >= stage_variants(p, i)) return fail(NLOS_ERR_INVALID_ARG, "tile %d out of range", i);
  for (int i = 0; i < n; ++i) p->tiles[i] = tiles[i];
  return NLOS_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// graph batches: many captures recorded once into a CUDA graph, items
// spread over side streams (longest first, onto the least-loaded stream) so
// independent captures overlap; one workspace per side stream
// ---------------------------------------------------------------------------
struct nlos_batch_s {
  int n = 0;
  std::vector<void*> ws;
  std::vector<cudaStream_t> side;
  std::vector<cudaEvent_t> join;
  cudaEvent_t fork = nullptr;
  cudaStream_t cap = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  std::vector<int> stream_of;
};

namespace {
void batch_free(nlos_batch_s* b) {
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  for (cudaEvent_t e : b->join) cudaEventDestroy(e);
  if (b->fork) cudaEventDestroy(b->fork);
  for (cudaStream_t t : b->side) cudaStreamDestroy(t);
  if (b->cap) cudaStreamDestroy(b->cap);
  for (void* w : b->ws) cudaFree(w);
  delete b;
}
}  // namespace

extern "C" {

nlos_status_t nlos_batch_create(const nlos_plan_t* plans, const void* const* transients, void* const* volumes, int n,
                                int max_streams, nlos_batch_t* out) {
  if (!out) return fail(NLOS_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (n <= 0 || !plans || !transients || !volumes) return fail(NLOS_ERR_INVALID_ARG, "bad batch arrays");
  for (int i = 0; i < n; ++i) {
    if (!plans[i] || !transients[i] || !volumes[i]) return fail(NLOS_ERR_INVALID_ARG, "batch item %d is NULL", i);
    if (plans[i]->prof_on) return fail(NLOS_ERR_INVALID_ARG, "disable stage tracing before recording a batch");
  }
  const int ns = std::max(1, std::min(n, max_streams > 0 ? max_streams : kBatchStreams));
  nlos_batch_s* b = new nlos_batch_s();
  b->n = n;
  // longest-processing-time-first assignment by workspace size (a proxy for the padded volume)
  std::vector<int> order(n);
  for (int i = 0; i < n; ++i) order[i] = i;
  std::stable_sort(order.begin(), order.end(), [&](int u, int v) { return plans[u]->ws_bytes > plans[v]->ws_bytes; });
  std::vector<double> load(ns, 0.0);
  std::vector<size_t> need(ns, 0);
  b->stream_of.assign(n, 0);
  for (int i : order) {
    const int k = (int)(std::min_element(load.begin(), load.end()) - load.begin());
    b->stream_of[i] = k;
    load[k] += (double)plans[i]->ws_bytes;
    need[k] = std::max(need[k], plans[i]->ws_bytes);
  }
  cudaError_t e = cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming);
  for (int k = 0; k < ns && e == cudaSuccess; ++k) {
    cudaStream_t t;
    cudaEvent_t ev;
    void* w = nullptr;
    e = cudaStreamCreateWithFlags(&t, cudaStreamNonBlocking);
    if (e != cudaSuccess) break;
    b->side.push_back(t);
    e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
    if (e != cudaSuccess) break;
    b->join.push_back(ev);
    e = cudaMalloc(&w, std::max<size_t>(need[k], 256));
    if (e != cudaSuccess) break;
    b->ws.push_back(w);
  }
  if (e != cudaSuccess) {
    nlos_status_t r = cuda_fail(e, "batch resources");
    batch_free(b);
    return r;
  }
  // one eager pass loads every kernel and sets attributes outside the capture
  nlos_status_t st = NLOS_OK;
  for (int i = 0; i < n && st == NLOS_OK; ++i)
    st = run_plan(plans[i], transients[i], volumes[i], b->ws[b->stream_of[i]], b->cap);
  if (st == NLOS_OK) {
    e = cudaStreamSynchronize(b->cap);
    if (e != cudaSuccess) st = cuda_fail(e, "batch warm-up");
  }
  if (st == NLOS_OK) {
    e = cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) st = cuda_fail(e, "batch capture");
  }
  if (st == NLOS_OK) {
    bool ok = cudaEventRecord(b->fork, b->cap) == cudaSuccess;
    for (int k = 0; ok && k < ns; ++k) ok = cudaStreamWaitEvent(b->side[k], b->fork, 0) == cudaSuccess;
    for (int i = 0; ok && i < n; ++i)
      ok = run_plan(plans[i], transients[i], volumes[i], b->ws[b->stream_of[i]], b->side[b->stream_of[i]]) == NLOS_OK;
    for (int k = 0; ok && k < ns; ++k) {
      ok = cudaEventRecord(b->join[k], b->side[k]) == cudaSuccess;
      if (ok) ok = cudaStreamWaitEvent(b->cap, b->join[k], 0) == cudaSuccess;
    }
    e = cudaStreamEndCapture(b->cap, &b->graph);
    if (!ok || e != cudaSuccess) st = fail(NLOS_ERR_CUDA, "batch capture failed: %s", cudaGetErrorString(cudaGetLastError()));
  }
  if (st == NLOS_OK) {
    e = cudaGraphInstantiate(&b->exec, b->graph, 0);
    if (e != cudaSuccess) st = cuda_fail(e, "batch graph instantiate");
  }
  if (st != NLOS_OK) {
    batch_free(b);
    return st;
  }
  *out = b;
  return NLOS_OK;
}

nlos_status_t nlos_batch_launch(nlos_batch_t b, void* stream) {
  if (!b) return fail(NLOS_ERR_INVALID_ARG, "batch is NULL");
  NLOS_CU(cudaGraphLaunch(b->exec, static_cast<cudaStream_t>(stream)), "batch launch");
  return NLOS_OK;
}

nlos_status_t nlos_batch_destroy(nlos_batch_t b) {
  if (!b) return fail(NLOS_ERR_INVALID_ARG, "batch is NULL");
  cudaDeviceSynchronize();
  batch_free(b);
  return NLOS_OK;
}

nlos_status_t nlos_workspace_check(nlos_plan_t p, const void* workspace, int* code) {
  if (!p) return fail(NLOS_ERR_INVALID_ARG, "plan is NULL");
  const char* ws = static_cast<const char*>(workspace ? workspace : p->ws);
  if (!ws) return fail(NLOS_ERR_INVALID_ARG, "no workspace");
  int v = 0;
  NLOS_CU(cudaMemcpy(&v, ws + p->off_scal + kErrOffset, sizeof v, cudaMemcpyDeviceToHost), "error word read");
  if (v != 0) NLOS_CU(cudaMemset(const_cast<char*>(ws) + p->off_scal + kErrOffset, 0, sizeof v), "error word reset");
  if (code) *code = v;
  if (v == kDevErrTmaTimeout) return fail(NLOS_ERR_TIMEOUT, "a staged-load wait ran out of its iteration limit");
  if (v == kDevErrChainTimeout) return fail(NLOS_ERR_TIMEOUT, "a fused stage's chunk wait ran out of its iteration limit");
  if (v == kDevErrBounds) return fail(NLOS_ERR_CUDA, "bounds-checked build: an index fell outside its buffer");
  if (v != 0) return fail(NLOS_ERR_CUDA, "device error word %d", v);
  return NLOS_OK;
}

nlos_status_t nlos_plan_set_profiling(nlos_plan_t p, int enable) {
  if (!p) return fail(NLOS_ERR_INVALID_ARG, "plan is NULL");
  p->prof_on = enable != 0;
  return NLOS_OK;
}

nlos_status_t nlos_plan_stage_times(nlos_plan_t p, double* times_ms, int capacity, int* n_stages,
                                    long long* calls) {
  if (!p) return fail(NLOS_ERR_INVALID_ARG, "plan is NULL");
  const int ns = (int)p->stage_names.size();
  if (n_stages) *n_stages = ns;
  long long nc = 0;
  for (size_t i = 0; i < p->prof_used; ++i) {
    NLOS_CU(cudaEventSynchronize(p->prof_pool[i]), "profiling read");
    const int stg = p->prof_stage[i];
    if (stg < 0) {
      ++nc;
      continue;
    }
    if (i == 0) continue;
    float ms = 0.f;
    NLOS_CU(cudaEventElapsedTime(&ms, p->prof_pool[i - 1], p->prof_pool[i]), "profiling read");
    if (times_ms && stg < capacity) times_ms[stg] += ms;
  }
  if (calls) *calls = nc;
  p->prof_used = 0;
  p->prof_stage.clear();
  return NLOS_OK;
}

const char* nlos_plan_stage_name(nlos_plan_t p, int i) {
  if (!p || i < 0 || i >= (int)p->stage_names.size()) return nullptr;
  return p->stage_names[i].c_str();
}

nlos_status_t nlos_plan_memory(nlos_plan_t p, size_t* resident_bytes) {
  if (!p || !resident_bytes) return fail(NLOS_ERR_INVALID_ARG, "plan and resident_bytes must be non-NULL");
  *resident_bytes = p->resident;
  return NLOS_OK;
}

nlos_status_t nlos_plan_destroy(nlos_plan_t p) {
  if (!p) return fail(NLOS_ERR_INVALID_ARG, "plan is NULL");
  cudaDeviceSynchronize();
  destroy_pipe(p->pipe);
  for (cudaEvent_t e : p->prof_pool) cudaEventDestroy(e);
  for (cudaEvent_t e : p->moe_ev)
    if (e) cudaEventDestroy(e);
  for (void* v : p->allocs) cudaFree(v);
  delete p;
  return NLOS_OK;
}

void nlos_debug_fail_allocation(int k) { g_fail_alloc.store(k > 0 ? k : 0); }

const char* nlos_last_error(void) { return g_err.c_str(); }

#ifdef NLOS_BOUNDS_CHECK
const char* nlos_version(void) { return "nlos-gb300 0.2 (sm_103a, bounds-checked)"; }
#else
const char* nlos_version(void) { return "nlos-gb300 0.2 (sm_103a)"; }
#endif

}  // extern "C"

// Narrow accessors for entry points compiled in other files of the library.
namespace nlos {
size_t plan_workspace_bytes(const nlos_plan_s* p) { return p->ws_bytes; }
size_t plan_resident_bytes(const nlos_plan_s* p) { return p->resident; }
bool plan_profiling(const nlos_plan_s* p) { return p->prof_on; }
nlos_status_t plan_run(nlos_plan_s* p, const void* H, void* vol, void* ws, cudaStream_t s) {
  return run_plan(p, H, vol, ws, s);
}
nlos_status_t set_error(nlos_status_t st, const char* msg) { return fail(st, "%s", msg); }
const nlos_plan_desc_t* plan_desc(const nlos_plan_s* p) { return &p->d; }
}  // namespace nlos
