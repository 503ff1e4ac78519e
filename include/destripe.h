/*
 * destripe.h -- C ABI of the GB300 destriper.
 *
 * Maximum-likelihood destriping of polarimeter / radiometer timelines
 * (Zonca, Williams, Meinhold & Lubin 2013, "Destriping Cosmic Microwave
 * Background Polarimeter data", Sect. 3).  The data model is
 *
 *     y = A_p m + F~ a + w                       (Eqs. destmodel and noise)
 *
 * with A_p the pointing-and-rotation operator (one pixel per sample, rows
 * w_o(t) per output kind), F~ the baseline matrix (each of the n_b baselines of
 * an output repeated over its L samples) and w white noise.  The baselines solve
 *
 *     [F~^T Z F~] a = F~^T Z y,   Z = V - V A_p M^-1 A_p^T V   (destriping equation)
 *
 * where V holds the 0/1 sample weights and M_p = sum_t v w w^T is the per-pixel
 * normal matrix (h_p times the identity for a q+u polarimeter, Sect. 3).
 *
 * Conventions shared by every call:
 *  - All d_* arguments are DEVICE pointers on the current CUDA device.  The
 *    caller owns them; a plan keeps the pointing pointers passed to
 *    destripe_plan (pixels are copied, cos/sin are referenced) until
 *    destripe_destroy, and keeps no other caller pointer past a call.
 *  - Arrays are dense and contiguous.  Timelines are output-major
 *    [n_outputs][n_samples]; baselines are output-major
 *    [n_outputs][n_baselines]; maps are component-major [n_comp][n_pix] with
 *    components (I), (Q, U) or (I, Q, U) -- I when any output carries I, Q and U
 *    when any output carries polarisation.  d_cos2psi and d_sin2psi must be
 *    16-byte aligned.
 *  - Work is enqueued on desc->stream (a cudaStream_t; NULL = legacy default
 *    stream).  Calls return once the work is enqueued, except destripe_plan,
 *    destripe_solve and destripe_run_host, which synchronise the stream because
 *    they return host-side results.
 *  - Errors are reported as ds_status codes only; nothing aborts or throws
 *    across the ABI.  destripe_strerror gives a static message.
 *  - A plan is not thread-safe; distinct plans are independent.
 *  - Precision: DS_PREC_FP64 computes every step in float64 and takes float64
 *    timelines y.  DS_PREC_MIXED takes float32 timelines y; the per-sample work
 *    of the CG iterations (expand, bin, rescan, baseline sums) runs in float32;
 *    the right-hand side, the residual refreshes that keep the iteration honest
 *    and the maps read their operands as double-float pairs (two float32, about
 *    48 significant bits) and sum in compensated float32 (Sum2 / Dot2 of Ogita,
 *    Rump and Oishi) flushed to float64 accumulators; pixel matrices, their
 *    inverses and rcond cut, pixel solves and the CG vectors and scalars are
 *    float64.
 */
#ifndef DESTRIPE_H
#define DESTRIPE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ds_plan_s* ds_plan_t;

typedef enum {
  DS_OK = 0,
  DS_EINVAL = 1,    /* bad descriptor or argument (sizes, kinds, alignment, NULL) */
  DS_ENOMEM = 2,    /* device allocation failed */
  DS_ECUDA = 3,     /* a CUDA runtime call failed */
  DS_ENOCONV = 4,   /* CG reached max_iter; the best iterate is still written */
  DS_ETIMEOUT = 5,  /* reserved: a bounded device wait gave up (no call waits on the device) */
  DS_ENAN = 6,      /* non-finite value met in the data or the iteration */
  DS_EPIX = 7,      /* a pixel index outside [0, 12 nside^2) */
  DS_ESTATE = 8     /* call not valid for this plan (e.g. precision mismatch) */
} ds_status;

/* Output kinds and their rows w_o(t), c = cos 2psi, s = sin 2psi (Sect. 3). */
typedef enum {
  DS_KIND_I = 0,   /* (1)            on I                  */
  DS_KIND_Q = 1,   /* ( c, s)        on (Q, U): q channel   */
  DS_KIND_U = 2,   /* (-s, c)        on (Q, U): u channel   */
  DS_KIND_IQU = 3  /* (1, c, s)      on (I, Q, U): radiometer */
} ds_kind;

typedef enum { DS_PREC_FP64 = 0, DS_PREC_MIXED = 1 } ds_prec;

#define DS_MAX_OUTPUTS 4

typedef struct {
  int64_t n_samples;              /* n_t >= 1, < 2^31 */
  int32_t nside;                  /* HEALPix resolution, power of two, 1..8192 */
  int32_t n_outputs;              /* 1..DS_MAX_OUTPUTS outputs sharing the pointing */
  int32_t kinds[DS_MAX_OUTPUTS];  /* ds_kind of each output */
  int64_t baseline_len;           /* L >= 1 samples per baseline; the last one may be short */
  int32_t precision;              /* ds_prec */
  int32_t reserved;               /* must be 0 */
  double rcond_min;               /* pixel cut on lambda_min/lambda_max of M_p; <= 0 means 1e-3 */
  void* stream;                   /* cudaStream_t */
} ds_desc;

typedef struct {
  int64_t n_samples;
  int64_t n_baselines;   /* per output: ceil(n_t / L) */
  int64_t n_unknowns;    /* n_outputs * n_baselines */
  int64_t n_pix;         /* 12 nside^2 */
  int64_t n_good_pix;    /* pixels kept by the cut */
  int64_t n_valid;       /* samples with weight 1 after flags and the cut */
  int32_t n_outputs;
  int32_t n_comp;        /* 1, 2 or 3 */
  int64_t device_bytes;  /* bytes the plan holds on the device */
  int32_t layout;        /* form of the float32 operator in use (tune key "layout") */
  int32_t bin_order;     /* run-length operator: 1 = binning over the pixel-major copy
                            (built by the first solve or operator application) */
  int64_t n_runs;        /* run-length records held, time-ordered or tiled (0 if none) */
} ds_info;

/* Build a plan: hits, per-pixel normal matrices M_p, their inverses and the
 * rcond cut (Sect. 3: hitmap h = P^T P and the QU / IQU weighting).
 *   d_pix      int32 [n_t]  HEALPix RING pixel of each sample (copied)
 *   d_cos2psi  float [n_t]  cos 2psi (referenced until destroy; 16-B aligned)
 *   d_sin2psi  float [n_t]  sin 2psi (referenced until destroy; 16-B aligned)
 *   d_valid    uint8 [n_t]  1 = good sample, 0 = flagged; NULL = all good.  A flag
 *                           applies to every output of the sample.
 * Samples on cut pixels get weight 0 in every later call.  Returns DS_EPIX if a
 * valid sample has a pixel outside the map.  Synchronises desc->stream. */
ds_status destripe_plan(const ds_desc* desc, const int32_t* d_pix, const float* d_cos2psi,
                        const float* d_sin2psi, const uint8_t* d_valid, ds_plan_t* out);

/* Sizes and state of a plan (Sect. 3: the numbers of samples, baselines and
 * map pixels that fix the shapes of F~, P and the maps; the pixels kept by the
 * cut and the weight-1 samples).  info: host struct, filled on DS_OK; no device
 * work. */
ds_status destripe_plan_info(ds_plan_t plan, ds_info* info);

/* Binned map m = M^-1 sum_t sum_o v w_o(t) (y_o(t) - a_o[t / L]) (Eqs. mapQ/mapU
 * with the general pixel weight), 0 on cut pixels.
 *   d_y    [n_o][n_t] float64 (FP64 plan) or float32 (MIXED plan)
 *   d_a    float64 [n_o][n_b] baselines to subtract, or NULL for none
 *   d_map  float64 [n_c][n_pix] output
 *   d_hits int32 [n_pix] output (valid samples per pixel, before the cut), or NULL
 *   d_mask uint8 [n_pix] output (1 = pixel kept), or NULL
 * Always accumulated in float64. */
ds_status destripe_bin(ds_plan_t plan, const void* d_y, const double* d_a, double* d_map,
                       int32_t* d_hits, uint8_t* d_mask);

/* Left-hand operator of the destriping equation, d_Ax = F~^T Z F~ d_x
 * (Sect. 3: expand, bin, per-pixel solve, rescan, per-baseline sum).
 *   d_x, d_Ax  float64 [n_o][n_b]; must not alias.
 * Uses the plan's precision for the per-sample work. */
ds_status destripe_apply_A(ds_plan_t plan, const double* d_x, double* d_Ax);

/* Right-hand side of the destriping equation (Sect. 3), d_b = F~^T Z y: bin y,
 * solve each pixel, rescan the map and sum y minus the rescan per baseline.
 *   d_y  timelines as for destripe_bin;  d_b  float64 [n_o][n_b] output
 * Float64 accumulation (compensated float32 sums flushed to float64 in MIXED
 * plans).  Asynchronous on the plan's stream. */
ds_status destripe_rhs(ds_plan_t plan, const void* d_y, double* d_b);

/* Solve the destriping equation by conjugate gradient (Sect. 3 names CG; the
 * operator is symmetric positive semi-definite).
 *   d_y        timelines as for destripe_bin
 *   d_a        float64 [n_o][n_b]: in = starting guess if warm_start, out = baselines,
 *              gauge-fixed (outputs carrying I get zero mean over baselines with data;
 *              baselines without data are 0)
 *   tol        stop when ||b - A a|| / ||b|| < tol (recursive residual, confirmed by a
 *              float64 residual in MIXED mode).  For outputs carrying I, b's component
 *              along the null mode (rounding only, b lying in the range of A) is
 *              removed first, so that a right-hand side of rounding size (a noiseless
 *              sky) converges to null baselines
 *   max_iter   iteration cap (<= 0 means 10000)
 *   iters, rel_resid  host outputs (may be NULL): iterations run and the float64
 *              relative residual at exit
 * Returns DS_ENOCONV (with the best iterate written) if max_iter is reached.
 * Synchronises desc->stream. */
ds_status destripe_solve(ds_plan_t plan, const void* d_y, double* d_a, double tol,
                         int32_t max_iter, int32_t warm_start, int32_t* iters,
                         double* rel_resid);

/* Destriped map m(y - F~ a) plus hits and mask (the outputs of Sect. 4). */
ds_status destripe_map(ds_plan_t plan, const void* d_y, const double* d_a, double* d_map,
                       int32_t* d_hits, uint8_t* d_mask);

/* Remove the I null mode from d_a in place (see destripe_solve).  The paper's
 * polarimeter case (q, u outputs, Sect. 3) has no such mode; outputs that carry I
 * leave a common offset of all their baselines undetermined (the I map absorbs
 * it), fixed here by a zero mean over the baselines with data; baselines without
 * data are set to 0.  d_a float64 [n_o][n_b]; asynchronous on the plan's stream. */
ds_status destripe_gauge(ds_plan_t plan, double* d_a);

void destripe_destroy(ds_plan_t plan);

const char* destripe_strerror(ds_status status);

/* Whole job from HOST buffers: copy the pointing and timelines to the device,
 * plan, solve, build the destriped map, copy a, the map, hits and mask back.
 * Host arrays may be pageable or pinned.  h_valid may be NULL.  Outputs
 * h_a [n_o][n_b], h_map [n_c][n_pix], h_hits [n_pix], h_mask [n_pix] may each
 * be NULL to skip the copy.  h_y is float64 for FP64, float32 for MIXED.
 * Synchronises desc->stream. */
ds_status destripe_run_host(const ds_desc* desc, const int32_t* h_pix, const float* h_cos2psi,
                            const float* h_sin2psi, const uint8_t* h_valid, const void* h_y,
                            double tol, int32_t max_iter, double* h_a, double* h_map,
                            int32_t* h_hits, uint8_t* h_mask, int32_t* iters,
                            double* rel_resid);

/* White-noise gap filling (Sect. 2, data description: flagged and missing samples
 * are replaced by Gaussian white noise with the mean and standard deviation of the
 * good samples of each day), in place, so that the destriper can run on a
 * timeline of constant sampling with every sample valid.
 *   desc       n_samples, n_outputs, precision (type of y) and stream are used
 *   d_valid    uint8 [n_t], 1 = good sample, 0 = flagged (required)
 *   block_len  samples per day (>= 1; the last block may be shorter)
 *   seed       key of the random draws
 *   d_y        [n_o][n_t] float64 (DS_PREC_FP64) or float32 (DS_PREC_MIXED), in/out:
 *              each flagged sample of output o in day d becomes
 *              mean + std * z (population statistics of the good samples of that
 *              output and day; 0 when the day has none), z standard normal from
 *              Philox4x32-10 (Salmon et al. 2011) with counter (t mod 2^32,
 *              t div 2^32, o, 0) and key (seed mod 2^32, seed div 2^32), Box-Muller of
 *              its first two words u0, u1: sqrt(-2 ln u0') cos(2 pi u1'), u' =
 *              (u + 1/2) 2^-32.  Good samples are not written.
 * Asynchronous on desc->stream; allocates a small table of day statistics. */
ds_status destripe_gapfill(const ds_desc* desc, const uint8_t* d_valid, int64_t block_len,
                           uint64_t seed, void* d_y);

/* Amplitude spectra of the timelines y (d_a NULL) or of the baseline-removed
 * y - F~ a (Sect. 6, frequency domain), per output.  The timeline is cut into
 * floor(n_t / seg_len) segments of seg_len samples (the tail is dropped); the
 * one-sided power spectral density P_k = 2 |X_k|^2 / (f_samp seg_len), averaged
 * over segments (k = 0 and k = seg_len / 2 not doubled), gives the amplitude
 * sqrt(P_k), averaged over n_bins bins of linearly growing length: with
 * K = seg_len / 2, bin j (0-based) holds k = e_j + 1 .. e_{j+1},
 * e_j = floor(K j (j + 1) / (n_bins (n_bins + 1))).  Samples are used as given
 * (fill gaps first, destripe_gapfill).
 *   d_y      timelines as for destripe_bin;  d_a  float64 [n_o][n_b] or NULL
 *   seg_len  2 .. n_t;  n_bins >= 1 with n_bins (n_bins + 1) / 2 <= seg_len / 2
 *   f_samp   sampling rate (Hz)
 *   d_freq   float64 [n_bins] mean frequency of each bin, or NULL
 *   d_amp    float64 [n_o][n_bins] mean amplitude (units of y per sqrt(Hz))
 * Uses cuFFT; takes its work buffers from the plan's memory pool.  Synchronises
 * the plan's stream. */
ds_status destripe_spectrum(ds_plan_t plan, const void* d_y, const double* d_a, int64_t seg_len,
                            int32_t n_bins, double f_samp, double* d_freq, double* d_amp);

/* Pointing of an analytic ground scan, computed on the device (Sect. 5, scanning
 * strategy: a spin about the vertical axis at fixed elevation, the sky turning with
 * the Earth; Sect. 3: the parallactic angle psi orients the polarimeter; HEALPix
 * RING pixels as cited in Sect. 3).  For sample k = first_sample + i:
 *   t = k (1 / f_samp), az = az0 + 2 pi t / spin_period, lst = lst0 + 2 pi t / sidereal_day,
 *   sin dec = sin el sin lat + cos el cos lat cos az,
 *   H = atan2(-sin az cos el, sin el cos lat - cos el sin lat cos az), RA = lst - H mod 2 pi,
 *   psi = atan2(sin H, tan lat cos dec - sin dec cos H) + 2 pi t / pol_rotation_period
 * (no modulator term when pol_rotation_period is 0); d_pix[i] = RING pixel of
 * (pi/2 - dec, RA) at nside, d_cos2psi[i] / d_sin2psi[i] = cos 2psi / sin 2psi rounded
 * to float32.  Each step is one float64 operation in this order (no fused
 * multiply-adds), so that the output is reproducible bit for bit.
 *   d_pix int32 [n], d_cos2psi / d_sin2psi float [n]: device outputs (caller-owned)
 * Asynchronous on stream.  Runs on the float64 pipe: on GB300 it is slower than
 * copying precomputed pointing from the host, and it serves plan-time generation
 * of simulated scans. */
typedef struct {
  double f_samp;               /* Hz */
  double spin_period;          /* s per azimuth revolution */
  double elevation_deg;
  double latitude_deg;
  double az0;                  /* rad, azimuth at t = 0 (north through east) */
  double lst0;                 /* rad, local sidereal time at t = 0 */
  double sidereal_day;         /* s */
  double pol_rotation_period;  /* s; 0 = no modulator */
} ds_scan;

ds_status destripe_scan_pointing(const ds_scan* scan, int64_t first_sample, int64_t n_samples,
                                 int32_t nside, int32_t* d_pix, float* d_cos2psi,
                                 float* d_sin2psi, void* stream);

/* Kernel timing and launch counts of a plan (no counterpart in the paper; it
 * exists to measure the kernels against the HBM roofline).  While profiling is
 * enabled, the captured CG graph records CUDA events around the binning and
 * rescan kernels of every iteration; destripe_solve accumulates their elapsed
 * times over the iterations that actually ran.  Launch counting is always on.
 *   enable  1 = enable and reset the counters, 0 = disable, -1 = leave as is
 *   out     may be NULL; filled with the counters since the last reset */
typedef struct {
  int64_t kernel_launches;  /* kernels this plan launched (graph nodes counted per replay) */
  int64_t graph_launches;   /* replays of the captured CG graph */
  int64_t iterations;       /* CG iterations that ran */
  int64_t timed_iterations; /* iterations with event timings (profiling enabled) */
  double bin_ms;            /* sum over timed iterations: binning kernel of A p */
  double rescan_ms;         /* sum: rescan + per-baseline-sum kernel of A p */
  double solve_ms;          /* sum: per-pixel solve kernel of A p */
  double iteration_ms;      /* sum: whole iteration, first kernel start to last kernel end */
} ds_profile;

ds_status destripe_profile(ds_plan_t plan, int32_t enable, ds_profile* out);

/* Tuning knobs of a plan (no counterpart in the paper; used by the autotuner).
 * Keys and values:
 *   "reliable_delta"  in (0, 1): MIXED plans recompute the residual in float64 each time
 *                     ||r|| has dropped by this factor since the last recomputation
 *                     (default 1e-5)
 *   "refresh_max"     MIXED plans: recompute the residual in float64 at least every this
 *                     many iterations, whatever the drop (default 50)
 *   "drift_ratio"     MIXED plans: when a recomputed ||r||^2 exceeds this many times the
 *                     recursive one, the float32 operator cannot follow the problem and
 *                     the solve continues with the accurate operator (default 1e4)
 *   "accurate_start"  MIXED plans: 1 = iterate with the accurate operator from the start
 *                     (small ill-conditioned problems converge in several times fewer
 *                     iterations with it)
 *   "stall_iters"     stop a solve, with DS_ENOCONV and its best iterate, when its residual
 *                     has not dropped 10x within this many iterations: an ill-posed
 *                     system has reached its floor (default 2000; 0 = never)
 *   "bin_mode"        MIXED plans: 1 = float32 pixel sums with one vector atomic per run
 *                     (default), 0 = float64 pixel sums with scalar atomics
 *   "graph_iters"     1..64 CG iterations per captured graph replay; 0 (default) = 16,
 *                     halved down to 4 while a replay would hold more than about 4 ms
 *                     of work (estimated at 2 ns per sample and output)
 *   "accurate_df"     MIXED plans: 1 = the accurate passes (right-hand side, maps,
 *                     float64 residual refreshes) use double-float operands and
 *                     compensated float32 sums on the float32 pipes with float64
 *                     accumulators (default), 0 = float64
 *   "blocks_per_sm"   1..32 resident-block target of the streaming kernels (default 16)
 *   "layout"          MIXED plans: 0 = the float32 operator reads the time-ordered pixel
 *                     indices; 2 = run-length records: per run of consecutive samples on
 *                     one pixel within a baseline, (pixel, count, sum cos 2psi, sum
 *                     sin 2psi) and the baseline (20 bytes per run; built by
 *                     destripe_plan, and used by default, when there are at most 0.6 runs
 *                     per sample; built on request otherwise); 1 = a chunk-local index (per chunk of
 *                     consecutive samples: the sorted distinct pixels and a 16-bit rank per
 *                     sample), bins into shared memory and stages the chunk's map in
 *                     shared memory.  The index is built on the plan's stream when first
 *                     requested (6 bytes per sample of device memory; synchronises);
 *                     3 = time-tiled, pixel-sorted run records (runs of at most 255
 *                     samples; 32 bytes per run of device memory, built on request,
 *                     synchronises): the binning reads the runs sorted by pixel within
 *                     long tiles ("bin_tile_samples"), each lane summing consecutive
 *                     runs of one pixel in registers with about one vector reduction per
 *                     pixel and tile; the rescan reads them sorted within tiles of a few
 *                     hours whose baseline sums stay in shared memory
 *   "bin_tile_samples"  layout 3: samples per long tile of the binning (default 2^26,
 *                     about two weeks at 50 Hz); set before the layout is built, else
 *                     DS_ESTATE
 *   "chunk"           MIXED plans: rebuild the chunk-local index with this many samples
 *                     per chunk (2048, 4096, 8192 or 16384; synchronises)
 *   "rescan_dedup"    MIXED plans: 1 = the float32 rescan reads the map once per run of
 *                     equal pixels within a thread's 4 samples (default), 0 = once per sample
 *   "samples_per_thread"  MIXED plans: 4 (default) or 8 consecutive samples per thread in
 *                     the float32 operator (8: two 16-byte loads per stream per thread)
 *   "bin_order"       MIXED plans with run-length records: 1 = the binning passes read a
 *                     pixel-major copy of the records (24 more bytes per run, built on the
 *                     plan's stream by the first destripe_solve or destripe_apply_A, or
 *                     here) with one warp per pixel and one plain store of its sums, no
 *                     atomic updates (default); 0 = they read the records in time order
 *                     with one reduction per run.
 *   "rescan_samples"  MIXED plans with run-length records: 1 = the rescans read the
 *                     time-ordered samples (12 bytes per sample) instead of the records
 *                     (20 bytes per run); chosen when the records are requested above
 *                     0.6 runs per sample
 *   "precond"         preconditioner of the CG (no counterpart in the paper, which uses
 *                     unpreconditioned Krylov solvers): 0 = none (default below 2^23
 *                     samples, where the coarse space's build of a few ms does not pay
 *                     and D^-1 alone saves no iterations); 1 = D^-1, the valid samples of
 *                     each baseline; 2 = two-level (default from 2^23 samples): D^-1 plus a
 *                     coarse correction R E^+ R^T on a space of large-scale sky modes
 *                     (cells of the sphere, "coarse_nside"), E = R^T A R built once per
 *                     plan at its first solve (from the pixel-major run records, made
 *                     for the purpose when the plan has none; synchronises).  Where
 *                     baselines sweep more than two cells for over a fifth of the valid
 *                     samples (long baselines) the coarse space is not built and the
 *                     plan iterates plain CG (D^-1 alone is nearly a scalar there).  A solve that breaks down or stalls with the
 *                     coarse correction (a nearly singular system whose slow modes
 *                     the iteration's arithmetic cannot resolve) continues from its
 *                     best iterate with D^-1 alone, which the plan keeps afterwards.
 *                     The solution is the same; the iterations are fewer where short
 *                     baselines leave slow sky-like modes
 *   "coarse_nside"    two-level preconditioner: 12 coarse_nside^2 cells (power of two,
 *                     1..64, default 8; at most the map's nside); a change rebuilds E
 *   "rescan_rounds"   MIXED plans: rounds of 32 work items (runs, or 4-sample groups)
 *                     per warp chunk in the rescans that keep per-lane baseline sums
 *                     across rounds and flush them across the warp only where a baseline
 *                     ends: 0 = chosen from the problem size and the grid (default, up to
 *                     16), 1..16 = fixed (1: a flush after every round)
 * Returns DS_EINVAL for an unknown key or value, DS_ESTATE when the plan cannot
 * use the value.  Takes effect at the next call. */
ds_status destripe_tune(ds_plan_t plan, const char* key, double value);

/* ---- Batched and served solves ---------------------------------------------------
 * (No counterpart in the paper, which destripes one dataset at a time.)  A batch
 * advances many independent problems through CG together: every kernel of an
 * iteration is one launch over the tiles of all problems still running, and a
 * fixed number of iterations is captured in one CUDA graph that stays valid while
 * problems are added and retired (continuous batching).  Only DS_PREC_MIXED plans
 * with the default precision knobs can join, and all problems of a batch must
 * have the same number of map components.  Each problem's iteration is the
 * single-problem one (same arithmetic, same float64 residual refreshes and
 * stopping rule), so its result does not depend on the rest of the batch beyond
 * float32 summation order.  Work is enqueued on the batch's stream; plans stay
 * owned by the caller and must outlive their slot.
 *
 * destripe_batch_create: room for max_slots (1..4096) problems.
 * destripe_batch_add:    computes the problem's right-hand side and CG start
 *     (d_a0: float64 [n_o][n_b] starting guess or NULL) and gives it a slot.
 *     DS_ESTATE if the batch is full, the plan is already in it, or it cannot join;
 *     DS_ENAN if the timelines hold a non-finite value on a valid sample (the problem
 *     does not join).  Waits on the batch's stream for the problem's start.
 * destripe_batch_step:   runs CG iterations for every running problem, at least
 *     min_iters unless all have stopped; *n_running = problems not yet stopped.
 *     Synchronises the stream.
 * destripe_batch_slot_status: done flag, iterations, float64 relative residual of a
 *     slot as of the last step.
 * destripe_batch_retire: gauge-fixes the slot's baselines, copies them to d_a (may be
 *     NULL), frees the slot; returns the problem's solve status (DS_OK, DS_ENOCONV, ...).
 * destripe_batch_tune:   launch shape of the batched kernels: "tile_samples" (samples per
 *     work tile of the per-sample passes, 4096..2^24, default 16384), "tile_pixels"
 *     (pixels per tile of the pixel solve, default 16384), "tile_unknowns" (unknowns
 *     per tile of the CG vector kernels, default 4096), "blocks_per_sm" (1..32,
 *     default 8).  Re-captures the iteration graph at the next step.
 * destripe_batch_autotune: picks the launch shape for the problems in the batch
 *     (no counterpart in the paper).  Coordinate descent over blocks_per_sm
 *     {4, 8, 16}, tile_samples {8192 .. 65536}, tile_pixels {4096, 16384, 65536} and
 *     tile_unknowns {2048, 4096, 16384}, starting from the shape in force: each trial
 *     replays the iteration graph once (8 real CG iterations of every running
 *     problem), times it with CUDA events and scores sample-iterations per second; a
 *     candidate must beat the best by 2%.  At most max_trials timed replays (<= 0: 12).
 *     The chosen shape stays in force; *out (may be NULL) reports it.  Problems that
 *     converge during tuning stop as in destripe_batch_step.  Synchronises the stream.
 * destripe_batch_info:   slots in use and kernels launched so far. */
typedef struct ds_batch_s* ds_batch_t;

ds_status destripe_batch_create(int32_t max_slots, void* stream, ds_batch_t* out);
ds_status destripe_batch_add(ds_batch_t batch, ds_plan_t plan, const void* d_y,
                             const double* d_a0, double tol, int32_t max_iter, int32_t* slot);
ds_status destripe_batch_step(ds_batch_t batch, int32_t min_iters, int32_t* n_running);
ds_status destripe_batch_slot_status(ds_batch_t batch, int32_t slot, int32_t* done,
                                     int32_t* iters, double* rel_resid);
ds_status destripe_batch_retire(ds_batch_t batch, int32_t slot, double* d_a, int32_t* iters,
                                double* rel_resid);
ds_status destripe_batch_tune(ds_batch_t batch, const char* key, double value);

typedef struct {
  int32_t tile_samples;   /* chosen launch shape */
  int32_t tile_pixels;
  int32_t tile_unknowns;
  int32_t blocks_per_sm;
  int32_t trials;         /* timed graph replays */
  int32_t pad;
  double rate;            /* sample-iterations per second of the chosen shape */
  double rate_initial;    /* ... of the shape in force before the call */
} ds_batch_tuning;

ds_status destripe_batch_autotune(ds_batch_t batch, int32_t max_trials, ds_batch_tuning* out);
ds_status destripe_batch_info(ds_batch_t batch, int32_t* n_slots_used, int64_t* kernel_launches);
void destripe_batch_destroy(ds_batch_t batch);

/* ---- Time-sharded solves ----------------------------------------------------------
 * Sect. 4 distributes the data over processes by time (Epetra maps over the
 * samples and baselines) and exchanges pixel-domain quantities once per operator
 * application (Export / Import).  Here each rank (one process per GPU) holds a
 * contiguous time slice of the timeline that starts on a baseline boundary, with
 * its pointing, its data and its slice of the baselines, and the library calls the
 * caller's all-reduce at every exchange point:
 *   - the plan's hits (int32 [n_pix]) and pixel matrices (float64 [n_pix][n_m],
 *     n_m = 1, 3 or 6), before the rcond cut, so that every rank cuts alike;
 *   - the pixel sums of every operator application, right-hand side and map,
 *     between the binning and the per-pixel solve (float32 [n_pix][4] in the float32
 *     iteration, float64 [n_pix][4] otherwise);
 *   - the CG scalars (dot products; the gauge's sum and count), float64.
 * allreduce(d_buf, count, dtype, stream, user) must replace the count values at
 * d_buf (device memory of this rank) by their sum over all ranks, ordered after the
 * work enqueued on stream (a cudaStream_t) and before the work enqueued after the
 * call returns (an NCCL all-reduce enqueued on stream does both; a host-side
 * all-reduce synchronises stream first).  It returns 0 on success; any other value
 * ends the library call with DS_ECUDA.  Every rank must make the same sequence of
 * calls.  A sharded plan works with destripe_rhs, destripe_apply_A (this rank's
 * rows), destripe_bin / destripe_map (the global map on every rank) and
 * destripe_solve_sharded; destripe_solve, the preconditioner and batches refuse
 * it (DS_ESTATE). */
typedef enum { DS_DT_F64 = 0, DS_DT_F32 = 1, DS_DT_I32 = 2 } ds_dtype;
typedef int32_t (*ds_allreduce_fn)(void* d_buf, int64_t count, int32_t dtype, void* stream,
                                   void* user);
typedef struct {
  ds_allreduce_fn allreduce;  /* required */
  void* user;                 /* passed through */
} ds_exchange;

/* A plan on this rank's slice (desc->n_samples: the slice's samples; the slice
 * starts on a baseline boundary of the global timeline, so that every rank's
 * baselines are whole, the last one possibly short on the last rank).  Arguments
 * as for destripe_plan; the exchange is called for the hits and pixel matrices.
 * Synchronises desc->stream. */
ds_status destripe_plan_sharded(const ds_desc* desc, const ds_exchange* ex, const int32_t* d_pix,
                                const float* d_cos2psi, const float* d_sin2psi,
                                const uint8_t* d_valid, ds_plan_t* out);

/* CG on the sharded destriping equation (no counterpart beyond Sect. 4's
 * distributed Krylov solver: every rank holds its slice of the vectors; dot
 * products and the pixel sums are exchanged).  Arguments as for destripe_solve,
 * with d_a this rank's slice [n_o][n_b_local].  The iteration runs from the host
 * (no captured graph): the operator in the plan's precision, and in MIXED plans the
 * float64 residual refreshes of destripe_solve; the gauge uses the global mean.
 * Synchronises the plan's stream. */
ds_status destripe_solve_sharded(ds_plan_t plan, const void* d_y, double* d_a, double tol,
                                 int32_t max_iter, int32_t warm_start, int32_t* iters,
                                 double* rel_resid);

/* Binned map without any device allocation (no counterpart in the paper: it
 * serves callers that cannot allocate device memory when they need a map, such
 * as processes whose device memory is owned by another allocator and loops that
 * forbid allocation after start-up).  Same result as destripe_plan followed by
 * destripe_bin(plan, d_y, NULL, ...), from the pointing and data directly.
 *   desc        as for destripe_plan (desc->baseline_len is not used)
 *   d_pix, d_cos2psi, d_sin2psi, d_valid   pointing as for destripe_plan (cos and sin
 *               16-byte aligned); hits, pixel matrices, cut and inverses are those a
 *               plan of the same descriptor computes
 *   d_y         [n_o][n_t] float64 (DS_PREC_FP64) or float32 (DS_PREC_MIXED)
 *   d_map       float64 [n_c][n_pix] output; d_hits, d_mask optional outputs
 * Intermediate sums live in one fixed device array declared by the library
 * (4.2 MB, held by every GPU that loads the library until exit); maps of more
 * than DS_NOALLOC_MAX_PIX pixels (nside > 64) return DS_EINVAL.  Every call
 * reuses that array (it clears what must start at zero), so calls that overlap
 * on the GPU race and must be serialised by the caller.  The first call on a
 * device looks up the array's address on that device; make it before any stream
 * capture.  Calls no allocation routine.  Accumulates in float64; returns
 * DS_EPIX for a valid sample with a pixel outside the map.  Synchronises
 * desc->stream. */
#define DS_NOALLOC_MAX_PIX 49152

ds_status destripe_bin_noalloc(const ds_desc* desc, const int32_t* d_pix,
                               const float* d_cos2psi, const float* d_sin2psi,
                               const uint8_t* d_valid, const void* d_y, double* d_map,
                               int32_t* d_hits, uint8_t* d_mask);

#ifdef __cplusplus
}
#endif

#endif /* DESTRIPE_H */
