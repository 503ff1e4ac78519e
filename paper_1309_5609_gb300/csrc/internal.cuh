// Internal declarations of the destriper library (not part of the C ABI).
//
// Device data of a plan (all dense, 256-byte aligned allocations):
//   pix      int32 [n_t]      pixel of each sample, or -1 when the sample is
//                             flagged or falls on a cut pixel (weight v = 0)
//   c, s     float [n_t]      caller's cos 2psi / sin 2psi (referenced)
//   hits     int32 [n_pix]    valid samples per pixel before the cut
//   mask     uint8 [n_pix]    1 = pixel kept
//   minv     f64 [n_pix][NM]  packed symmetric M_p^-1 (NM = 1, 3, 6), 0 if cut
//   bins     f64 [n_pix][4]   pixel sums, kept at zero between uses
//   map32    f32 [n_pix][4]   map in the mixed-precision iteration
//   map64    f64 [n_pix][4]   map in float64 passes
//   xdf      f32x2 [n_u]      mixed plans: the baselines of an accurate pass as
//                             double-float pairs (split once per pass)
//   nvalid   int32 [n_b]      valid samples per baseline (gauge)
//   lid      uint16 [n_pad]   mixed plans: chunk-local pixel rank of each sample
//   upix     int32 [n_pad]    mixed plans: sorted distinct pixels of each chunk
//   ucnt     int32 [chunks]   mixed plans: distinct pixels per chunk
//   CG vectors f64 [n_u]      x, r, p, q, b, t (n_u = n_o * n_b)
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/destripe.h"

namespace ds {

// Kind sets with their rows known at compile time; GEN* take kinds at run time.
enum KindSet {
  KS_QU = 0, KS_IQU3 = 1, KS_IQU1 = 2, KS_I = 3, KS_GEN1 = 4, KS_GEN2 = 5, KS_GEN3 = 6,
  KS_QU12 = 7  // one or two outputs, each q or u (components Q, U): lone q / u, and mixes of them
};

struct KindsArg {
  int n_o;
  int kind[DS_MAX_OUTPUTS];
};

// Gate of a kernel inside the CG graph: it does nothing once *done != 0; when
// need is given, unless *need != 0; when skip is given, if *skip != 0.
struct Gate {
  const int* done;
  const int* need;
  const int* skip = nullptr;
};

__device__ __forceinline__ bool gate_closed(const Gate& g) {
  if (g.done != nullptr && *(volatile const int*)g.done) return true;
  if (g.need != nullptr && *(volatile const int*)g.need == 0) return true;
  if (g.skip != nullptr && *(volatile const int*)g.skip != 0) return true;
  return false;
}

// Baseline of a thread's sample position as it strides through the timeline by
// a fixed step: b = t / L and the offset r = t - b L, advanced by additions
// instead of a 64-bit division per step.
struct BaselineCursor {
  int64_t b, r, dq, dr;
  __device__ __forceinline__ BaselineCursor(int64_t t, int64_t step, int64_t L)
      : b(t / L), r(t - (t / L) * L), dq(step / L), dr(step - (step / L) * L) {}
  __device__ __forceinline__ void advance(int64_t L) {
    b += dq;
    r += dr;
    if (r >= L) {
      r -= L;
      b += 1;
    }
  }
  // first sample of the next baseline
  __device__ __forceinline__ int64_t next_start(int64_t t, int64_t L) const { return t + (L - r); }
};

// One run of consecutive samples on one pixel within a baseline (runs.cu):
// its samples' count and sums of cos 2psi and sin 2psi.
struct RunRec {
  int pix;
  float n, c, s;
};

// Device-resident CG state (float64 scalars and control words).
struct CgState {
  double rr;         // ||r||^2 of the current residual
  double rr_old;     // ||r||^2 before the last update (for beta)
  double pq;         // p . A p
  double alpha;
  double bb;         // ||b||^2
  double rr_anchor;  // ||r||^2 at the last float64 residual
  double tol2;       // tol^2 * bb
  double delta2;     // reliable-update trigger ratio (squared)
  double rr_true;    // float64 ||b - A x||^2 at the last check
  int iter;
  int max_iter;
  int done;
  int need;          // run the float64 residual this iteration
  int status;        // 0 ok, 1 converged, 2 max_iter, 3 breakdown, 4 non-finite
  int mixed;         // 1: recursive residual is confirmed in float64
  int n_reliable;    // float64 residual updates done
  int last_refresh;  // iteration of the last float64 residual
  int refresh_max;   // refresh at least every refresh_max iterations (stagnation guard)
  int accurate;      // 1: the float32 operator could not follow; iterate with the accurate one
  int improved;      // the last float64 residual is the best so far: keep x
  int accurate_start;  // 1: iterate with the accurate operator from the start
  int pad1;
  double rr_best;    // smallest float64 ||b - A x||^2 seen (mixed plans keep that x)
  double drift2;     // ||r_true||^2 / ||r_recursive||^2 above which the accurate operator takes over
  double rr_progress;  // the residual at the last 10x improvement
  int progress_iter;   // ... and its iteration
  int stall_iters;     // stop when no 10x improvement for this many iterations (0 = never)
  // preconditioned CG (z = the preconditioned residual)
  int precond;         // 0: none (z = r); 1: D^-1; 2: D^-1 + coarse correction
  int pad2;
  double rz;           // r . z of the current residual
  double rz_old;       // ... before the last update (for beta)
  double rdr;          // r . D^-1 r (the coarse part is added by the coarse kernel)
};

enum ErrBits { ERR_PIX = 1, ERR_NAN = 2 };

constexpr int kPcSlots = 2;  // coarse cells kept per baseline by the two-level preconditioner
constexpr size_t kPcRestrictSmemMax = 160 * 1024;  // float32 R^T r sums per block (40960 columns)
constexpr int64_t kPcMinSamples = int64_t(1) << 23;  // the two-level default from this many samples

struct Plan {
  ds_desc desc;
  cudaStream_t stream;
  cudaStream_t cap_stream;  // private stream used only to capture graphs
  int device;
  int num_sms;
  int n_o, n_c, nm;
  int kindset;
  KindsArg kinds;
  int has_I_outputs;
  int64_t n_t, npix, L, n_b, n_u;
  int64_t n_good, n_valid;
  const float* c;
  const float* s;
  int32_t* pix;
  int32_t* hits;
  uint8_t* mask;
  double* minv;
  double* bins;
  float* bins32;      // float32 pixel sums [n_pix][4] for the mixed operator (vector atomics)
  float* map32;
  float* maplo;       // low parts of the double-float map [n_pix][4] (mixed plans)
  float2* xdf;        // baselines split into double-float pairs [n_u] (mixed plans)
  float* x32;         // baselines of the float32 operator, rounded once per apply [n_u]
  double* map64;
  int32_t* nvalid;
  double *x, *r, *p, *q, *b, *t;
  double* x_best;     // mixed plans: iterate with the smallest float64 residual
  double* red;        // reduction partials [red_len]
  int red_len;
  unsigned* counters; // last-block tickets [8]
  CgState* state;     // device
  CgState* h_state;   // pinned host mirror
  int32_t* err;       // device error word
  int32_t* h_err;     // pinned
  double* scal;       // device scratch scalars [8]
  double* h_scal;     // pinned [8]
  int64_t device_bytes;
  // captured iteration graphs: [0] float32 operator, [1] accurate operator
  cudaGraphExec_t graph_exec;
  cudaGraphExec_t graph_exec_acc;
  int graph_iters;
  int graph_profiled;       // graph holds event nodes
  // profiling
  int profiling;
  cudaEvent_t* ev;          // [graph_iters][5] when profiled
  int64_t launches;         // kernel launches (host-side count)
  int64_t graph_launches;
  int64_t iterations;
  int64_t timed_iterations;
  double t_bin, t_rescan, t_solve, t_iter;
  // tuning knobs (destripe_tune)
  double reliable_delta;    // float64 residual after every 1/delta drop of ||r||
  int bin_mode;             // mixed binning: 0 = float64 atomics, 1 = float32 vector atomics
  int graph_iters_cfg;      // CG iterations per captured graph
  int blocks_per_sm;        // streaming-kernel blocks per SM
  int accurate_df;          // mixed plans: accurate passes in compensated float32 (1) or float64 (0)
  int refresh_max;          // mixed plans: float64 residual at least every this many iterations
  double drift_ratio;       // mixed plans: squared true / recursive residual ratio of the switch
  int accurate_start;       // mixed plans: 1 = accurate operator from the first iteration
  int stall_iters;          // stop a solve whose residual has not dropped 10x in this many iterations
  int layout;               // mixed operator: 0 = time-ordered pixels, 1 = chunk-local index,
                            // 2 = run-length records, 3 = time-tiled pixel-sorted records
  int rescan_dedup;         // float32 rescan: reuse the map value of a repeated pixel
  int rescan_rounds;        // rounds per warp chunk of the carried-sum rescans (0: automatic)
  int samples_per_thread;   // float32 operator: 4 or 8 consecutive samples per thread
  // chunk-local pixel index (chunked.cu)
  uint16_t* lid;
  int32_t* upix;
  int32_t* ucnt;
  int ck_C;                 // samples per chunk
  int64_t ck_nchunks;
  int ck_umax;              // most distinct pixels in one chunk
  int ck_ustride;           // shared-array stride (>= ck_umax)
  int ck_threads;           // threads per block of the chunked passes
  int ck_bin_blocks;        // resident blocks per SM (occupancy)
  int ck_rescan_blocks;
  // run-length records (runs.cu), built on request
  RunRec* rl_rec;
  int32_t* rl_b;
  int64_t rl_n;
  int64_t* rl_tiles;        // runs per construction tile, between count and fill
  float4* rl_df;            // per run: (sum cos 2psi, sum sin 2psi) as double-float pairs
  // pixel-major copy of the runs (runs_pm.cu): the runs of pixel p are
  // pm_off[p] .. pm_off[p + 1] - 1, in no particular order
  uint32_t* pm_off;         // [n_pix + 1]
  float4* pm_rec;           // per run: (count, sum cos, sum sin, baseline as int bits)
  float2* pm_lo;            // per run: low parts of the double-float sums (the record holds the high)
  float4* x4;               // [n_b] float32 baselines of every output, per baseline
  float4* xd4;              // [2][n_b] split baselines: hi parts, then lo parts
  int bin_order;            // run-length plans: 1 = bin pixel-major (default), 0 = in time order
  int pm_pending;           // the copy is being built on the side stream: unusable until pm_join
  // time-tiled, pixel-sorted run records (tiles.cu; layout 3)
  int4* tl_rec;             // [runs] (pixel, n << 24 | baseline in tile, sum cos, sum sin)
  int64_t* tl_off;          // [tiles + 1] first record of each tile
  int64_t tl_tiles;         // tiles of tl_tb consecutive baselines
  int64_t tl_tb;
  int tl_bin_blocks;        // resident blocks per SM of the two passes
  int tl_rescan_blocks;
  int4* tl2_rec;            // the same records sorted by pixel within long tiles (binning)
  int64_t* tl2_off;         // [tiles + 1]
  int64_t* tl2_chunk;       // [tiles + 1] first warp chunk of each long tile
  int64_t tl2_tiles, tl2_tb, tl2_chunks;
  uint32_t* tl2_end;        // [tiles][ranks] end of each pixel rank's records in a long tile
  int64_t tl2_nkeys;        // pixel ranks (observed pixels)
  int64_t tl_bin_samples;   // samples per long tile (tune key "bin_tile_samples")
  int tl_pending;           // layout 3 chosen by the plan, records not built yet (tl_ensure)
  int64_t tl_runs;          // records of each tiled copy
  float4* tl_x4;            // [n_b] float32 baselines of every output, per baseline
  unsigned* tl_mmax;        // largest |m| of the operator's map (float bits): the rescan's scale
  int rescan_samples;       // run-length plans: the rescans read the time-ordered samples (dense
                            // runs: a record per run costs more than 12 bytes per sample)
  // preconditioner of the CG (precond.cu): 0 none, 1 D^-1 (valid samples per
  // baseline), 2 two-level (D^-1 plus a coarse space of large-scale sky modes)
  int precond;
  int pc_nside;             // the coarse space has 12 pc_nside^2 cells
  int pc_built;             // coarse space and E^+ built for this plan
  int pc_fallback;          // a solve broke down with the coarse correction: D^-1 alone
  int pc_probed;            // the probe of long baselines ran (and found enough kept samples)
  int pc_n;                 // coarse columns (kept cells x n_c)
  int pc_cells;             // kept cells
  float4* pc_slot;          // [n_b][kPcSlots] per slot: x = kept-cell number (int bits, -1 =
                            // none); y, z, w = the cell's share of the baseline's valid
                            // samples and their cos 2psi, sin 2psi sums over the valid count
  double* pc_einv;          // [pc_n][pc_n] generalised inverse of E = R^T A R
  double* pc_u;             // [pc_n] R^T r, kept at zero between uses
  float* pc_c;              // [pc_n] coarse correction E^+ R^T r, rounded to float32
  // time-sharded plans (shard.cu): the caller's all-reduce over the ranks, called
  // at every exchange point (plan matrices, pixel sums, CG scalars); its first
  // failure is kept in shard_err and ends the call in progress
  ds_allreduce_fn shard_allreduce;
  void* shard_user;
  mutable int shard_err;
  cudaStream_t side_stream; // builds the pixel-major copy beside the first right-hand side
  cudaEvent_t side_ev[2];   // records ready (plan stream) / copy built (side stream)
};

// api.cu: device memory of a plan from the library's stream-ordered pool;
// counted in device_bytes when count is set
cudaError_t plan_alloc(Plan& P, void** ptr, size_t bytes, bool count);
// the same, ordered on another stream of the plan
cudaError_t plan_alloc_on(Plan& P, cudaStream_t st, void** ptr, size_t bytes, bool count);

// runs.cu
ds_status rl_count(Plan& P, int64_t* d_total);
// with_df: also the double-float run sums of the accurate run passes and the
// pixel-major copy (the tiled records do without them)
ds_status rl_fill(Plan& P, int64_t n_runs, bool with_df = true);
ds_status rl_build(Plan& P, bool with_df = true);
ds_status pm_build(Plan& P, cudaStream_t st);
// builds the pixel-major copy on the plan's stream before its first use if the
// plan bins from it
ds_status pm_ensure(Plan& P);
// the same on the plan's side stream, overlapping what the plan's stream does
// next; pm_join makes the plan's stream wait for it
ds_status pm_begin(Plan& P, bool* started);
ds_status pm_join(Plan& P, bool started);
void pm_release(Plan& P, cudaStream_t st);
void rl_release(Plan& P, cudaStream_t st);
// runs_pm.cu: the binning pass over the pixel-major copy (one warp per pixel, no atomics)
bool pm_ready(const Plan& P);
void launch_bin_pm(const Plan& P, cudaStream_t st, Gate g);
void launch_bin_pm_df(const Plan& P, cudaStream_t st, Gate g);
constexpr double kRunsPerSampleMax = 0.6;  // plans build run records at or below this ratio
bool rl_ready(const Plan& P);
// tiles.cu: time-tiled, pixel-sorted run records (layout 3)
ds_status tl_build(Plan& P);
bool tl_ready(const Plan& P);
void launch_pack_tl(const Plan& P, cudaStream_t st, const double* x, Gate g);
ds_status tl_ensure(Plan& P);
void launch_bin_tl(const Plan& P, cudaStream_t st, Gate g);
void launch_rescan_tl(const Plan& P, cudaStream_t st, double* out, Gate g);
void launch_bin_rl(const Plan& P, cudaStream_t st, Gate g);
void launch_rescan_rl(const Plan& P, cudaStream_t st, double* out, Gate g);
bool rl_df_ready(const Plan& P);
void launch_bin_rl_df(const Plan& P, cudaStream_t st, Gate g);
void launch_rescan_rl_df(const Plan& P, cudaStream_t st, double* out, Gate g);

// chunked.cu
constexpr int kChunkMin = 2048, kChunkMax = 16384;
int ck_default_chunk(int64_t n_t, int num_sms);
cudaError_t ck_build(Plan& P, int C, unsigned long long* umax);
cudaError_t ck_finish(Plan& P, int64_t umax);
bool ck_ready(const Plan& P);
void launch_bin_ck(const Plan& P, cudaStream_t st, const double* x, Gate g);
void launch_rescan_ck(const Plan& P, cudaStream_t st, const double* x, double* out, Gate g);

// kernels launched by one CG iteration (for the launch counter)
int kernels_per_iteration(const Plan& P, bool accurate);

// ---- launch helpers ---------------------------------------------------------
int stream_grid(const Plan& P, int64_t work_items, int block, int per_sm);

// apply.cu: per-sample passes and the pixel solve
void launch_bin_x(const Plan& P, cudaStream_t st, bool fp64, const double* x, Gate g);
void launch_bin_y(const Plan& P, cudaStream_t st, const void* y, const double* a, Gate g);
void launch_pixel_solve(const Plan& P, cudaStream_t st, bool fp64, double* out_map, Gate g);
void launch_rescan_x(const Plan& P, cudaStream_t st, bool fp64, const double* x, double* out, Gate g);
void launch_rescan_y(const Plan& P, cudaStream_t st, const void* y, double* out, Gate g);
// apply_df.cu: accurate passes of mixed plans (double-float operands, compensated sums)
// rounds of 32 work items per warp chunk of the carried-sum rescans over n_units items
int rescan_rounds(const Plan& P, int64_t n_units, int grid);
void launch_split_df(const Plan& P, cudaStream_t st, const double* x, Gate g);
void launch_bin_df(const Plan& P, cudaStream_t st, const double* x, const float* y, Gate g);
void launch_pixel_solve_df(const Plan& P, cudaStream_t st, double* out_map, Gate g);
void launch_rescan_df(const Plan& P, cudaStream_t st, const double* x, const float* y,
                      double* out, Gate g);
// full operator pieces
void enqueue_apply(const Plan& P, cudaStream_t st, bool fp64, const double* x, double* out, Gate g,
                   cudaEvent_t* ev = nullptr);
void enqueue_rhs(const Plan& P, cudaStream_t st, const void* y, double* out, Gate g);
void enqueue_map(const Plan& P, cudaStream_t st, const void* y, const double* a, double* out_map);

// plan.cu
ds_status plan_build(Plan& P, const int32_t* d_pix, const uint8_t* d_valid);
// hits and M_p of the samples (M packed [n_pix][NM], both accumulated: zero them
// first); df: compensated float32 sums of the mixed plans
void launch_plan_matrices(int kindset, bool df, int grid, cudaStream_t st, const int32_t* pix,
                          const float* c, const float* s, const uint8_t* valid, int32_t* hits,
                          double* mm, int64_t n_t, int64_t npix, KindsArg kk, int32_t* err);
// rcond cut and M_p^-1 in place, mask, kept-pixel count (accumulated into n_good)
void launch_pixel_invert(int n_c, int grid, cudaStream_t st, double* mm, const int32_t* hits,
                         uint8_t* mask, int64_t npix, double rcond_min,
                         unsigned long long* n_good);
// api.cu: kernel specialisation of a set of output kinds
int kindset_of(const int* kinds, int n_o, int n_c);

// shard.cu: the caller's all-reduce (sum) of count values at d_buf, ordered on st;
// a no-op for plans that are not sharded
void shard_exchange(const Plan& P, cudaStream_t st, void* d_buf, int64_t count, int32_t dtype);
// api.cu: a plan on the given pointing, sharded when ex is not NULL
ds_status plan_create(const ds_desc* desc, const ds_exchange* ex, const int32_t* d_pix,
                      const float* d_cos2psi, const float* d_sin2psi, const uint8_t* d_valid,
                      ds_plan_t* out);

// precond.cu: coarse space and coarse matrix of the two-level preconditioner
__host__ __device__ int coarse_cell(int64_t p, int64_t nside, int64_t nc);
ds_status pc_build(Plan& P, bool* made_runs, bool* made_pm);
// builds the coarse space, first making (and afterwards freeing) the run records
// and their pixel-major copy when the plan's operator does not keep them
ds_status pc_prepare(Plan& P);
ds_status pc_probe(Plan& P);
bool pc_restrict_fits(const Plan& P, int n);
int pc_mode(const Plan& P);
void pc_free(Plan& P, cudaStream_t st);
bool pc_ready(const Plan& P);
// cg.cu: the preconditioner's kernels of one CG step (restrict, coarse solve,
// new direction), gated by the CG state
void enqueue_precond_direction(const Plan& P, cudaStream_t st);

}  // namespace ds

#define DS_CUDA_TRY(expr)                                   \
  do {                                                      \
    cudaError_t e_ = (expr);                                \
    if (e_ != cudaSuccess) {                                \
      return (e_ == cudaErrorMemoryAllocation) ? DS_ENOMEM : DS_ECUDA; \
    }                                                       \
  } while (0)
