/*
 * nlos.h - C ABI of the GB300 wave-based NLOS reconstruction library
 * (confocal f-k migration and radial phasor-field RSD reconstruction).
 *
 * Conventions shared by every entry point
 *   - Transient input H is [x][y][t] (t fastest, "index-major" temporal bins,
 *     Sec. 4.1/4.2), nx * ny * nt elements of the plan's storage type:
 *     float32 (NLOS_F32), IEEE half (NLOS_F16) or bfloat16 (NLOS_BF16).
 *   - Output volume is float32 [x][y][z] (z fastest), nx * ny * nz elements:
 *       f-k:     nz = nt, voxel (i, j, k) = |Psi|^2 at depth k * c * dt / 2
 *                (Eq. 2), wall sample (i, j);
 *       phasor:  nz = n_depths, |I| on depth plane d_min + k (d_max - d_min)/(D-1).
 *   - Device pointers are caller-owned device memory; the library never frees
 *     or retains them after the call's work completes. Calls are asynchronous
 *     on `stream` (a cudaStream_t passed as void*, NULL = legacy default
 *     stream) unless stated otherwise; inputs are never modified.
 *   - A plan owns its constant tables and one default workspace. Two calls
 *     that use the same workspace must not overlap on the device; use
 *     nlos_reconstruct_ws with distinct workspaces for concurrent calls.
 *   - No exception crosses the ABI. Every call returns nlos_status_t; on
 *     failure nlos_last_error() (per thread) describes it. Invalid arguments
 *     are rejected before any device work is enqueued.
 *   - Every step runs on the GPU in this library's kernels; there is no CPU
 *     fallback.
 */
#ifndef NLOS_H_
#define NLOS_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* NLOS_FK: f-k migration (Alg. 1/2). NLOS_PHASOR_RSD: symmetry-aware radial
 * phasor-field reconstruction (Alg. 4). NLOS_PHASOR_DENSE: phasor fields with
 * the dense Fourier-domain propagation kernel (Alg. 3): per plan, every
 * (frequency, depth) kernel is stored over the padded grid (4 nx ny F D
 * complex float32 values; float32 storage only); it reproduces the direct
 * Rayleigh-Sommerfeld sum of Eq. 3 on the wall grid. */
typedef enum { NLOS_FK = 0, NLOS_PHASOR_RSD = 1, NLOS_PHASOR_DENSE = 2 } nlos_method_t;
typedef enum { NLOS_F32 = 0, NLOS_F16 = 1, NLOS_BF16 = 2 } nlos_storage_t;
typedef enum { NLOS_OUT_MAGNITUDE = 0, NLOS_OUT_COMPLEX = 1 } nlos_output_t;
typedef enum {
  NLOS_OK = 0,
  NLOS_ERR_INVALID_ARG = 1,
  NLOS_ERR_OUT_OF_MEMORY = 2,
  NLOS_ERR_CUDA = 3,
  NLOS_ERR_UNSUPPORTED = 4,
  NLOS_ERR_TIMEOUT = 5
} nlos_status_t;

typedef struct nlos_plan_s* nlos_plan_t;
typedef struct nlos_batch_s* nlos_batch_t;
typedef struct nlos_server_s* nlos_server_t;

/*
 * Capture and method description (problem statement of Sec. 3: confocal
 * transient H(x_s, x_s, t) sampled on an nx x ny wall grid over a
 * wall_w_m x wall_h_m relay wall, nt bins of bin_width_s).
 *   nx, ny        scan grid in [8, 1024] (any size: padded axes run at the
 *                 smallest power of two >= 2x the size)
 *   nt            time bins in [16, 4096] (the f-k time axis padded like x, y;
 *                 the phasor band transform runs at the next power of two >= nt)
 *   bin_width_s   time-bin width dt (> 0)
 *   wall_w_m/h_m  scanned wall extent along x / y (> 0); wall samples are cell centres
 *   method        nlos_method_t
 *   storage       nlos_storage_t of the input and of stored intermediates;
 *                 reduced precision uses a per-volume scale, arithmetic is float32
 *                 (the phasor depth sum runs on tensor cores: f16 operands for
 *                 16-bit storage; for float32 storage every operand split into
 *                 two f16 parts, three exact products per term, float32 sums)
 *   pad_factor    2: zero padding x2 on every axis (Sec. 4.2); 1: unpadded f-k
 *                 (Sec. 4.2's Pad x1 variant; nx, ny >= 16, powers of two);
 *                 other values INVALID_ARG
 *   output        NLOS_OUT_MAGNITUDE: float32 volume, |Psi|^2 for f-k (Alg. 1)
 *                 and |I| for phasor fields (Alg. 4); NLOS_OUT_COMPLEX: the
 *                 complex field itself (Psi, or I) as interleaved float32
 *                 (re, im) pairs, twice the bytes, the input of the coherence
 *                 merge of Eqs. 8-9
 * Phasor-field only (Sec. 4.3, Eqs. 4-7):
 *   wavelength_m  virtual wavelength (0 -> 4 * wall_w_m / nx)
 *   cycles        Gaussian virtual-wave width in periods (0 -> 5)
 *   n_depths, depth_min_m, depth_max_m   D reconstruction planes, d_min..d_max
 *   sigma_s, sigma_t   modality pair (0,0 -> confocal (2,0); (1,1) non-confocal)
 *   delta_m       calibration path offset Delta (Eq. 4)
 */
typedef struct {
  int nx, ny, nt;
  double bin_width_s;
  double wall_w_m, wall_h_m;
  int method;
  int storage;
  int pad_factor;
  double wavelength_m;
  double cycles;
  int n_depths;
  double depth_min_m, depth_max_m;
  int sigma_s, sigma_t;
  double delta_m;
  int output;
} nlos_plan_desc_t;

/* Fill *desc with defaults (f-k, float32, pad 2, cycles 5, confocal). */
void nlos_plan_desc_default(nlos_plan_desc_t* desc);

/*
 * Build a plan: validates the description, generates the float64 tables
 * (FFT twiddles, Stolt coordinate constants; for phasor fields the
 * virtual-wave band, the radial kernel K_r(rho, f, d) of Eq. 6 and the
 * pixel-to-radius chunks of the supplementary lookup), uploads them, and
 * allocates the default workspace. Synchronous. *out receives an opaque
 * handle owned by the caller until nlos_plan_destroy.
 * Errors: INVALID_ARG (null pointer, sizes, extents <= 0, empty band),
 * UNSUPPORTED (sizes outside the ranges above, unpadded phasor fields,
 * unpadded f-k of non-power-of-two sizes, 16-bit dense phasor fields),
 * OUT_OF_MEMORY, CUDA.
 */
nlos_status_t nlos_plan_create(const nlos_plan_desc_t* desc, nlos_plan_t* out);

/* nlos_plan_create with flags. NLOS_PLAN_NO_WORKSPACE: do not allocate the
 * default workspace (the plan is then used only through nlos_reconstruct_ws,
 * batches or a server, which provide their own). */
#define NLOS_PLAN_NO_WORKSPACE 1
/* NLOS_PLAN_SEPARATE_AXES: run the f-k lateral transforms as four separate
 * passes (x forward, y forward, y inverse, x inverse) even where the fused
 * pairs apply (zero-padded f-k with Lx = Ly <= 1024 and nt a multiple of 16:
 * x then y forward in one launch, y then x inverse in another, each pair's
 * intermediate kept in L2). Same arithmetic; for comparison and testing. */
#define NLOS_PLAN_SEPARATE_AXES 2
nlos_status_t nlos_plan_create_ex(const nlos_plan_desc_t* desc, int flags, nlos_plan_t* out);

/*
 * Shape and byte counts of a plan: out_shape = {nx, ny, nz}; workspace_bytes
 * is the size nlos_reconstruct_ws needs; input/output_bytes are the sizes of
 * one transient and one volume. Any output pointer may be NULL.
 */
nlos_status_t nlos_plan_query(nlos_plan_t plan, size_t out_shape[3], size_t* workspace_bytes,
                              size_t* input_bytes, size_t* output_bytes);

/*
 * Reconstruct one capture (f-k: Alg. 1/2 with Eq. 2; phasor: Alg. 4) from the
 * device transient into the device volume, using the plan's workspace.
 * Asynchronous on stream.
 */
nlos_status_t nlos_reconstruct(nlos_plan_t plan, const void* transient, void* volume, void* stream);

/*
 * Same as nlos_reconstruct with a caller-owned device workspace of at least
 * workspace_bytes (from nlos_plan_query), 256-byte aligned. Lets several
 * reconstructions of one plan run concurrently on different streams.
 */
nlos_status_t nlos_reconstruct_ws(nlos_plan_t plan, const void* transient, void* volume, void* workspace,
                                  size_t workspace_bytes, void* stream);

/*
 * End-to-end call on HOST buffers: copies the transient host->device, runs
 * nlos_reconstruct, copies the volume device->host and waits for completion
 * (synchronous). Host buffers may be pageable or pinned; device staging
 * buffers are owned by the plan.
 */
nlos_status_t nlos_reconstruct_host(nlos_plan_t plan, const void* transient_host, void* volume_host,
                                    void* stream);

/*
 * Reconstruct n captures from host memory into host memory, pipelined: while
 * capture i is reconstructed, capture i+1 is copied in and capture i-1
 * copied out, on library-owned streams and three device staging slots per
 * plan (allocated on first use, kept until nlos_plan_destroy). The work is
 * ordered after what is already queued on `stream`; the call returns when
 * every volume is in host memory. Host buffers should be page-locked for the
 * copies to overlap. transients_host / volumes_host are host arrays of n
 * host pointers (input_bytes / output_bytes each, from nlos_plan_query).
 * Uses the plan's own workspace: no other call may use the plan meanwhile.
 * Errors: INVALID_ARG (NULL plan or pointers, n < 0, plan without
 * workspace), OUT_OF_MEMORY (staging), CUDA.
 */
nlos_status_t nlos_reconstruct_host_many(nlos_plan_t plan, const void* const* transients_host,
                                         void* const* volumes_host, int n, void* stream);

/*
 * Reconstruct n captures with one launch sequence each, forked over the
 * library's internal streams so that small captures overlap on the device and
 * joined back to `stream`. plans[i] describes capture i;
 * workspaces[i] (each at least that plan's workspace_bytes) must be distinct;
 * pass NULL for workspaces to use each plan's default workspace (then every
 * plan may appear only once). Asynchronous on stream; may be captured into a
 * CUDA graph.
 */
nlos_status_t nlos_reconstruct_batch(const nlos_plan_t* plans, const void* const* transients,
                                     void* const* volumes, void* const* workspaces, int n, void* stream);

/*
 * Reconstruct like nlos_reconstruct, but allocate nothing: the scratch comes
 * from a fixed 32 MiB array in device memory that the library holds on every
 * GPU it is loaded on, instead of the plan's workspace. (The paper has no
 * counterpart; this serves callers that cannot call cudaMalloc at
 * reconstruction time: real-time loops, where an allocation may synchronise
 * the device and stall a frame, and applications that give this library a
 * fixed share of device memory and manage the rest in their own pool.) The
 * plan must already exist. The first call on each device also looks the
 * array's address up with cudaGetSymbolAddress (a synchronous runtime call;
 * later calls on that device reuse it). Errors: INVALID_ARG if the plan's workspace_bytes exceed 32 MiB,
 * if an argument is NULL, or if stage tracing is enabled on the plan; CUDA if
 * the lookup fails. All calls share the array, which keeps the previous
 * call's contents: calls that overlap on the GPU race and must be serialised
 * by the caller. A bounded wait that gives up inside the call is not
 * observable here (its error word lives in the array, which
 * nlos_workspace_check does not read). Asynchronous on stream.
 */
nlos_status_t nlos_reconstruct_noalloc(nlos_plan_t plan, const void* transient, void* volume, void* stream);

/*
 * Autotune the plan's launch shapes: for every stage with more than one
 * kernel variant (column tiles and TMA staging of the x/y transforms, pencils
 * per CTA of the f-k temporal stage, the phasor depth sum's persistent
 * tensor-core, one-CTA-per-tile tensor-core and FP32-FMA forms) time the
 * whole reconstruction with each variant on a
 * scratch input (coordinate descent, CUDA events on `stream`) and keep the
 * fastest. Results are cached per plan shape for the process and, when the
 * environment variable NLOS_AUTOTUNE_CACHE names a file, in that JSON file
 * (read on first use, rewritten after tuning). Synchronous; allocates a
 * scratch transient and volume for the duration of the call. Variants
 * differ in numerics only by rounding (every one within the storage type's
 * tolerance of the float64 method). Errors: INVALID_ARG (NULL plan, tracing enabled),
 * OUT_OF_MEMORY, CUDA.
 */
nlos_status_t nlos_plan_autotune(nlos_plan_t plan, void* stream);

/* Current variant index of each stage (tiles[i], i < min(capacity, *n_stages)). */
nlos_status_t nlos_plan_get_tiles(nlos_plan_t plan, int* tiles, int capacity, int* n_stages);

/* Set every stage's variant explicitly (n must equal the stage count; each index in range). */
nlos_status_t nlos_plan_set_tiles(nlos_plan_t plan, const int* tiles, int n);

/*
 * Record a batch of n reconstructions into one CUDA graph (the batching of
 * Sec. 4.1's graph replay, extended to many captures of uneven size): item i
 * reconstructs transients[i] into volumes[i] (caller-owned device buffers,
 * fixed for the batch's life) with plans[i]. Items are assigned longest
 * first to the least-loaded of up to max_streams side streams (0 -> 8) that
 * fork from and join to the launching stream inside the graph, so independent
 * captures overlap on the device; each side stream owns one workspace sized
 * for its largest item (owned by the batch). Creation runs the batch once
 * eagerly (loading kernels) and then records it; synchronous.
 * Errors: INVALID_ARG (NULL arrays/items, tracing enabled), OUT_OF_MEMORY, CUDA.
 */
nlos_status_t nlos_batch_create(const nlos_plan_t* plans, const void* const* transients, void* const* volumes,
                                int n, int max_streams, nlos_batch_t* out);

/* Launch the recorded graph on stream (asynchronous); reads the batch's inputs, writes its outputs. */
nlos_status_t nlos_batch_launch(nlos_batch_t batch, void* stream);

/* Release the graph, its streams and workspaces (synchronises the device). */
nlos_status_t nlos_batch_destroy(nlos_batch_t batch);

/*
 * Continuous-batching server (Sec. 4.1's producer-consumer front end, served
 * from many clients). Requests of any description are queued by any thread
 * and served by one scheduler thread: plans are created and autotuned
 * (nlos_plan_autotune, whose process-wide cache serves repeats) once per
 * distinct description and stay resident; memory_budget_bytes covers the resident
 * plans (tables, radial kernels, tensor-core operand stores, dense kernels)
 * and the workspaces of running requests, and idle plans (no request queued
 * or running) are evicted least recently used first when a new plan or an
 * admission needs the room; a request is admitted in arrival order as soon
 * as one of n_slots streams is free and its workspace (the padded volume's
 * footprint) fits; admitted requests are launched outside the queue's lock
 * and overlap on the device, at stream priorities ranked by age (the oldest
 * running request highest), and each signals its completion through a host
 * function on its stream. Workspaces come from the stream-ordered
 * allocator. Each result equals that of a standalone nlos_reconstruct with
 * the same description.
 * Errors: INVALID_ARG (budget 0, slots outside [1, 64]), CUDA.
 */
nlos_status_t nlos_server_create(size_t memory_budget_bytes, int n_slots, nlos_server_t* out);

/* Create (and keep) the plan for desc ahead of the first request. Synchronous. */
nlos_status_t nlos_server_preload(nlos_server_t server, const nlos_plan_desc_t* desc);

/*
 * Queue one request: transient/volume are caller-owned device buffers (input
 * ready when this is called, output valid once nlos_server_wait returns).
 * Creates the plan if the description is new (synchronous, stalls the
 * device; may wait for running requests to release plans it can evict).
 * *ticket identifies the request. Errors: INVALID_ARG (NULL arguments,
 * invalid description), OUT_OF_MEMORY (the plan and its workspace exceed the
 * whole budget), UNSUPPORTED, CUDA.
 */
nlos_status_t nlos_server_submit(nlos_server_t server, const nlos_plan_desc_t* desc, const void* transient,
                                 void* volume, uint64_t* ticket);

/*
 * Block until the request finished (or timeout_s elapsed, <= 0: one hour);
 * returns its latency (submission to observed completion) and forgets the
 * ticket. Errors: INVALID_ARG (unknown ticket), TIMEOUT, CUDA.
 */
nlos_status_t nlos_server_wait(nlos_server_t server, uint64_t ticket, double timeout_s, double* latency_ms);

/* Latency percentiles and throughput of the completed requests (optionally reset). */
nlos_status_t nlos_server_stats(nlos_server_t server, double* p50_ms, double* p99_ms, double* volumes_per_s,
                                unsigned long long* completed, int reset);

/*
 * Device memory the server accounts against its budget: the resident plans'
 * tables and kernels (*plan_bytes), the workspaces of the requests on the
 * device (*workspace_bytes), and how many idle plans it has evicted to make
 * room (*evictions). Any pointer may be NULL. Errors: INVALID_ARG.
 */
nlos_status_t nlos_server_memory(nlos_server_t server, size_t* plan_bytes, size_t* workspace_bytes,
                                 unsigned long long* evictions);

/* Finish queued work, stop the scheduler, release plans and streams. */
nlos_status_t nlos_server_destroy(nlos_server_t server);

/*
 * Read and clear the device error word of a workspace (NULL: the plan's
 * default one). Kernels that stage tiles with TMA wait on barriers with an
 * iteration limit; a wait that runs out records a timeout there and the
 * kernel returns instead of hanging (code 1; code 2 for the chunk counters
 * of the fused f-k stages). In the bounds-checked build (compiled with
 * NLOS_BOUNDS_CHECK; nlos_version says so) every global access of the
 * transform, Stolt, band, depth-sum and binning kernels checks its index
 * against its buffer's extent, and one outside records code 3 and is
 * skipped. Synchronous.
 * Returns OK (code 0), TIMEOUT (codes 1, 2) or CUDA (code 3 or a failed read).
 */
nlos_status_t nlos_workspace_check(nlos_plan_t plan, const void* workspace, int* code);

/*
 * Self-test of the bounds checks: one thread checks an index one past the end
 * of a small buffer (without accessing it) and one inside. *code is 3 in the
 * bounds-checked build (the check recorded the index) and 0 in the normal
 * build (checks compile away). Synchronous. Errors: INVALID_ARG,
 * OUT_OF_MEMORY, CUDA.
 */
nlos_status_t nlos_selftest_bounds(int* code);

/*
 * Self-test of that bounded wait: one CTA waits at most `limit` polls on a
 * barrier that nothing arrives on. Returns TIMEOUT with *code = 1 when the
 * wait gave up as it should (the context stays usable). Synchronous.
 */
nlos_status_t nlos_selftest_bounded_wait(int limit, int* code);

/*
 * Stage tracing. While enabled, every reconstruction with this plan records a
 * CUDA event before its first stage and after each stage, on the call's
 * stream (use one stream per plan while profiling).
 */
nlos_status_t nlos_plan_set_profiling(nlos_plan_t plan, int enable);

/*
 * Wait for the recorded events, add each stage's elapsed milliseconds into
 * times_ms[0 .. min(capacity, *n_stages)), return the stage count and the
 * number of profiled calls, and clear the record. Synchronous.
 */
nlos_status_t nlos_plan_stage_times(nlos_plan_t plan, double* times_ms, int capacity, int* n_stages,
                                    long long* calls);

/* Name of stage i of the plan's sequence (NULL if out of range). */
const char* nlos_plan_stage_name(nlos_plan_t plan, int stage);

/*
 * Photon binning (Sec. 4.1). A SPAD stream is `count` photon records given as
 * two device arrays: pixel[i], the wall index x * ny + y of the point the
 * photon was detected at, and ticks[i], its time of flight in integer clock
 * ticks. The record's bin is (ticks - t0_ticks) / ticks_per_bin (integer
 * division); records with ticks < t0_ticks, bin >= nt or pixel >= nx * ny are
 * dropped. With accumulate == 0 the output is cleared first, otherwise the
 * photons are added to it (streaming several batches into one frame).
 * Asynchronous on stream; allocates nothing. Errors: INVALID_ARG (NULL
 * output, NULL records with count > 0, count < 0, ticks_per_bin == 0).
 *
 * nlos_bin_transient: transient[x][y][t] (float32, nx * ny * nt) += 1 per
 *   kept photon: the histogram H consumed by nlos_reconstruct. Counts are
 *   exact up to 2^24 per bin.
 */
nlos_status_t nlos_bin_transient(const uint32_t* pixel, const uint32_t* ticks, long long count, int nx, int ny,
                                 int nt, uint32_t t0_ticks, uint32_t ticks_per_bin, int accumulate,
                                 float* transient, void* stream);

/*
 * nlos_bin_phasors: photons of a phasor-field plan's grid (nx, ny, nt)
 *   accumulated into its compact phasor field: phasors[x][y][f]
 *   (interleaved float32 complex, nx * ny * F values, F from nlos_plan_band)
 *   += w(f) exp(-2 pi i k_f b / nt) for a photon in bin b, with k_f = k_lo + f
 *   the band bins and w(f) the virtual-wave weights of the plan (Sec. 3.1);
 *   i.e. w(f) times the temporal DFT of the binned histogram at the band bins.
 *   Two routes give these phasors: per photon (one warp per 32 records,
 *   lanes over frequencies, vector atomics; cost ~ photons x F), or through
 *   an atomic histogram in the plan's workspace and a temporal FFT per wall
 *   point (cost ~ nx ny nt). By default the second is taken when
 *   photons x F > 2 nx ny nt and the plan has a workspace; the histogram
 *   route uses the plan's workspace like nlos_reconstruct.
 *   flags: NLOS_BIN_ACCUMULATE adds to `phasors` instead of overwriting them;
 *   NLOS_BIN_DIRECT / NLOS_BIN_VIA_HISTOGRAM force a route.
 *   Errors: as above, and INVALID_ARG for a plan that is not phasor-field,
 *   unknown or contradictory flags, or the histogram route forced on a plan
 *   without workspace.
 */
#define NLOS_BIN_ACCUMULATE 1
#define NLOS_BIN_DIRECT 2
#define NLOS_BIN_VIA_HISTOGRAM 4
nlos_status_t nlos_bin_phasors(nlos_plan_t plan, const uint32_t* pixel, const uint32_t* ticks, long long count,
                               uint32_t t0_ticks, uint32_t ticks_per_bin, int flags, void* phasors,
                               void* stream);

/* Band of a phasor-field plan: first DFT bin k_lo and count F of the band
 * frequencies (either pointer may be NULL). INVALID_ARG for f-k plans. */
nlos_status_t nlos_plan_band(nlos_plan_t plan, int* k_lo, int* n_freqs);

/*
 * Reconstruct from a compact phasor field (Alg. 4 from its spatial
 * transforms on; the band transform of the transient is skipped): phasors
 * as written by nlos_bin_phasors, device, [x][y][F] complex float32. Uses the
 * plan's workspace; asynchronous on stream. Errors: INVALID_ARG (NULL
 * pointers, f-k plan, plan without workspace), UNSUPPORTED (16-bit storage
 * plans: the phasor input is float32).
 */
nlos_status_t nlos_reconstruct_phasors(nlos_plan_t plan, const void* phasors, void* volume, void* stream);

/*
 * nlos_reconstruct_moe: both experts of the mixture (Sec. 4.4) from one
 * transient, with the lateral forward transform shared. The x then y forward
 * transform of the transient is taken once (the f-k forward spectrum, before
 * f-k's t/(n-1) ramp); the f-k branch applies the ramp as its temporal stage
 * reads that spectrum (the ramp commutes with the lateral transforms), and
 * the phasor-field branch takes each stored pencil's temporal DFT, keeps its
 * band and writes the Hermitian partner (-kx, -ky) from the mirrored bins
 * (Sec. 3.1 band transform, Eq. 6 propagation input). Results equal those of
 * nlos_reconstruct on each plan up to rounding.
 *   fk_plan: NLOS_FK; pf_plan: NLOS_PHASOR_RSD or NLOS_PHASOR_DENSE; both
 *   float32 storage, created with their own workspace, for the same grid
 *   (nx, ny, nt) and the same padded lateral lengths (the same pad_factor).
 *   transient: device float32 [nx][ny][nt]; volume_fk, volume_pf: device,
 *   each plan's output layout. The spectrum is written into the f-k plan's
 *   workspace, the phasor branch's intermediates into its own.
 *   stream: the f-k branch and the shared transform run here. stream2: the
 *   phasor branch; it waits for the shared spectrum, and stream waits for the
 *   phasor branch before the call's last work is done, so everything the call
 *   wrote is complete once `stream` reaches it. stream2 == stream runs the
 *   two branches one after the other. Two plan events are created on the
 *   first two-stream call.
 * Asynchronous. Errors: INVALID_ARG (NULL pointers, wrong methods, no
 * workspace, grids or paddings that differ), UNSUPPORTED (16-bit storage),
 * CUDA (launch). The plans' workspaces must not be in use elsewhere meanwhile.
 */
nlos_status_t nlos_reconstruct_moe(nlos_plan_t fk_plan, nlos_plan_t pf_plan, const void* transient, void* volume_fk,
                                   void* volume_pf, void* stream, void* stream2);

/*
 * Post-processing of reconstructed volumes. All pointers are device memory
 * owned by the caller; volumes are [nx][ny][nz] with depth innermost; every
 * call is asynchronous on stream and allocates nothing. Errors: INVALID_ARG
 * (NULL pointers, non-positive sizes, N_w outside [1, 16]), CUDA (launch).
 *
 * nlos_max_image: the display reduction of Alg. 1 / Sec. 4.2,
 *   image[x][y] = max_z volume[x][y][z] (its square root if take_sqrt, which
 *   turns an f-k |Psi|^2 volume into an |Psi| image). image is float32 [nx][ny].
 */
nlos_status_t nlos_max_image(const float* volume, int nx, int ny, int nz, int take_sqrt, float* image, void* stream);

/*
 * nlos_moe_mix: the mixture of experts of Eq. 10 (Sec. 4.4) on two float32
 * images of `count` pixels: both are divided by their own maximum, mixed as
 * f = f_fk * (f_rsd + eps)^beta, and the result divided by its maximum.
 * One thread block; out may alias neither input.
 */
nlos_status_t nlos_moe_mix(const float* img_fk, const float* img_rsd, long long count, float beta, float eps,
                           float* out, void* stream);

/*
 * nlos_coherence_merge: the coherence factor of Eq. 8 and the merged
 * magnitude of Eq. 9 over a window of N_w = nw complex volumes (interleaved
 * float32 (re, im), `count` voxels each; frames[] is a host array of nw device
 * pointers, e.g. NLOS_OUT_COMPLEX reconstructions):
 *   C = |sum_j f_j| / (eps + sum_j |f_j|),  merged = C |sum_j f_j| / N_w.
 * coherence may be NULL; eps must be > 0.
 */
nlos_status_t nlos_coherence_merge(const void* const* frames, int nw, long long count, float eps, float* merged,
                                   float* coherence, void* stream);

/*
 * nlos_dda: depth-dependent averaging of the last N_w = nw float32 volumes
 * (Sec. 4.4; the paper does not fix the weights). frames[0] is the newest
 * frame; plane z averages the newest N(z) = min(N_w, 1 + floor(N_w z / nz))
 * frames, so near planes keep their temporal detail and far, weak planes are
 * averaged over the whole window. frames[] is a host array of device pointers
 * to [nxy][nz] volumes.
 */
nlos_status_t nlos_dda(const float* const* frames, int nw, long long nxy, int nz, float* out, void* stream);

/* Tensor-core self-check (tcgen05 on sm_103a): one CTA computes
 * D = A B^T for fixed small-integer A (128 x 64) and B (n_cols x 64) with
 * f16 MMAs into tensor memory and writes D (128 x n_cols float32, row-major)
 * to the device buffer out; the caller compares it with the exact product.
 * *code receives the device error word (non-zero: the MMA completion wait
 * gave up, NLOS_ERR_TIMEOUT). Synchronous. n_cols: multiple of 16 in [16, 256]. */
nlos_status_t nlos_selftest_umma(int n_cols, float* out, int* code);

/* FP32 FMA throughput probe (the denominator of the rooflines of FMA-bound
 * kernels): launches `blocks` CTAs of 256 threads on `stream`, each thread
 * running 8 independent chains of x <- x * params[0] + params[1] (starting
 * near params[2]) for 16 * iters steps. params: device, 3 floats; sink:
 * device, blocks * 256 floats, written only in a case that cannot occur.
 * *flops receives the flops the launch executes; the caller times it.
 * Asynchronous; INVALID_ARG on NULL pointers or non-positive counts. */
nlos_status_t nlos_ffma_rate_launch(const float* params, float* sink, int blocks, int iters, double* flops,
                                    void* stream);

/* Testing hook for the failure path (fault injection on the host): the k-th
 * device allocation that plan creation or host staging makes from now on
 * (k >= 1) fails as if the device were out of memory, and the call returns
 * NLOS_ERR_OUT_OF_MEMORY after releasing what it had allocated; k = 0
 * disables. Process-wide; not for production use. */
void nlos_debug_fail_allocation(int k);

/*
 * Device memory the plan holds (its tables, twiddles, radial or dense kernel,
 * tensor-core operand stores and, unless created with
 * NLOS_PLAN_NO_WORKSPACE, its workspace; host-call staging once used).
 * Errors: INVALID_ARG.
 */
nlos_status_t nlos_plan_memory(nlos_plan_t plan, size_t* resident_bytes);

/* Release the plan's tables, workspace and staging buffers (synchronises the device). */
nlos_status_t nlos_plan_destroy(nlos_plan_t plan);

/* Description of the calling thread's most recent failure ("" if none). */
const char* nlos_last_error(void);

/* Library version string. */
const char* nlos_version(void);

#ifdef __cplusplus
}
#endif

#endif /* NLOS_H_ */
