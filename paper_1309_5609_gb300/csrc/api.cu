// C ABI entry points (include/destripe.h).
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <new>
#include <mutex>
#include <string>

#include "internal.cuh"

namespace ds {
void enqueue_dot(const Plan& P, cudaStream_t st, const double* a, const double* b, int64_t n,
                 double* out);
void enqueue_gauge(const Plan& P, cudaStream_t st, double* a);
void enqueue_iteration(const Plan& P, cudaStream_t st, cudaEvent_t* ev, bool accurate);
void enqueue_cg_setup(const Plan& P, cudaStream_t st, double tol, int max_iter, double delta,
                      int warm, bool precond);
}  // namespace ds

using namespace ds;

namespace {

constexpr int kGraphItersMax = 64;     // upper bound of CG iterations per captured graph

int n_comp_of(const int* kinds, int n_o, int* has_i_out) {
  bool I = false, P = false;
  int hi = 0;
  for (int o = 0; o < n_o; ++o) {
    if (kinds[o] == DS_KIND_I || kinds[o] == DS_KIND_IQU) { I = true; hi = 1; }
    if (kinds[o] == DS_KIND_Q || kinds[o] == DS_KIND_U || kinds[o] == DS_KIND_IQU) P = true;
  }
  *has_i_out = hi;
  return (I && P) ? 3 : (P ? 2 : 1);
}

}  // namespace

int ds::kindset_of(const int* k, int n_o, int n_c) {
  if (n_o == 2 && k[0] == DS_KIND_Q && k[1] == DS_KIND_U) return KS_QU;
  if (n_o == 3 && k[0] == DS_KIND_I && k[1] == DS_KIND_Q && k[2] == DS_KIND_U) return KS_IQU3;
  if (n_o == 1 && k[0] == DS_KIND_IQU) return KS_IQU1;
  if (n_o == 1 && k[0] == DS_KIND_I) return KS_I;
  if (n_c == 2 && n_o <= 2) return KS_QU12;  // q and u outputs only, at most two
  return n_c == 1 ? KS_GEN1 : (n_c == 2 ? KS_GEN2 : KS_GEN3);
}

namespace {

// Plan memory comes from one stream-ordered pool per device, owned by the library:
// freeing a plan needs no device-wide synchronisation (cudaFree has one), and a
// plan built after another reuses its memory without a trip to the driver (mapping
// a tiled plan's 80 GB anew costs about 0.1 s).  Up to half of the device's memory
// of freed plan memory stays in the pool.
constexpr int kMaxDevices = 64;
std::mutex g_pool_mutex;
cudaMemPool_t g_pools[kMaxDevices] = {};

cudaError_t plan_pool(int device, cudaMemPool_t* out) {
  if (device < 0 || device >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_pool_mutex);
  if (g_pools[device] == nullptr) {
    cudaMemPoolProps props = {};
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = device;
    cudaMemPool_t pool = nullptr;
    cudaError_t e = cudaMemPoolCreate(&pool, &props);
    if (e != cudaSuccess) return e;
    size_t free_b = 0, total_b = 0;
    int cur = 0;
    uint64_t keep = uint64_t(8) << 30;
    if (cudaGetDevice(&cur) == cudaSuccess && cur == device &&
        cudaMemGetInfo(&free_b, &total_b) == cudaSuccess)
      keep = (uint64_t)total_b / 2;
    e = cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
    if (e != cudaSuccess) {
      cudaMemPoolDestroy(pool);
      return e;
    }
    g_pools[device] = pool;
  }
  *out = g_pools[device];
  return cudaSuccess;
}

}  // namespace

cudaError_t ds::plan_alloc_on(Plan& P, cudaStream_t st, void** ptr, size_t bytes, bool count) {
  if (count) P.device_bytes += (int64_t)bytes;
  cudaMemPool_t pool = nullptr;
  const cudaError_t e = plan_pool(P.device, &pool);
  if (e != cudaSuccess) return e;
  return cudaMallocFromPoolAsync(ptr, bytes, pool, st);
}

cudaError_t ds::plan_alloc(Plan& P, void** ptr, size_t bytes, bool count) {
  return plan_alloc_on(P, P.stream, ptr, bytes, count);
}

namespace {

template <typename T>
cudaError_t dalloc(Plan& P, T** ptr, int64_t count) {
  const size_t bytes = sizeof(T) * (size_t)(count > 0 ? count : 1);
  P.device_bytes += (int64_t)bytes;
  cudaMemPool_t pool = nullptr;
  const cudaError_t e = plan_pool(P.device, &pool);
  if (e != cudaSuccess) return e;
  return cudaMallocFromPoolAsync(reinterpret_cast<void**>(ptr), bytes, pool, P.stream);
}

void plan_free(Plan* P) {
  if (P == nullptr) return;
  if (P->side_stream) cudaStreamSynchronize(P->side_stream);  // a copy still being built
  if (P->graph_exec) cudaGraphExecDestroy(P->graph_exec);
  if (P->graph_exec_acc) cudaGraphExecDestroy(P->graph_exec_acc);
  if (P->ev) {
    for (int i = 0; i < kGraphItersMax * 5; ++i) cudaEventDestroy(P->ev[i]);
    delete[] P->ev;
  }
  void* dev[] = {P->tl_rec, P->tl_off, P->tl2_rec, P->tl2_off, P->tl2_chunk, P->tl2_end, P->tl_x4, P->tl_mmax, P->pc_slot, P->pc_einv, P->pc_u, P->pc_c, P->pm_off, P->pm_rec, P->pm_lo, P->x4, P->xd4, P->rl_df, P->rl_tiles, P->rl_rec, P->rl_b, P->x32, P->xdf, P->lid, P->upix, P->ucnt, P->pix, P->hits, P->mask, P->minv, P->bins, P->bins32, P->map32, P->maplo, P->map64, P->nvalid,
                 P->x,   P->r,    P->p,    P->q,    P->b,    P->t,     P->x_best, P->red,   P->counters,
                 P->state, P->err, P->scal};
  // the plan's own stream is the last user of its memory (batches retire a
  // problem, synchronising their stream, before its plan may be destroyed)
  for (void* d : dev)
    if (d) cudaFreeAsync(d, P->stream);
  if (P->h_state) cudaFreeHost(P->h_state);
  if (P->h_err) cudaFreeHost(P->h_err);
  if (P->h_scal) cudaFreeHost(P->h_scal);
  if (P->cap_stream) cudaStreamDestroy(P->cap_stream);
  if (P->side_stream) cudaStreamDestroy(P->side_stream);
  for (cudaEvent_t e : P->side_ev)
    if (e) cudaEventDestroy(e);
  delete P;
}

ds_status check_desc(const ds_desc* d) {
  if (d == nullptr) return DS_EINVAL;
  if (d->n_samples < 1 || d->n_samples >= (int64_t(1) << 31)) return DS_EINVAL;
  if (d->nside < 1 || d->nside > 8192 || (d->nside & (d->nside - 1)) != 0) return DS_EINVAL;
  if (d->n_outputs < 1 || d->n_outputs > DS_MAX_OUTPUTS) return DS_EINVAL;
  for (int o = 0; o < d->n_outputs; ++o)
    if (d->kinds[o] < DS_KIND_I || d->kinds[o] > DS_KIND_IQU) return DS_EINVAL;
  if (d->baseline_len < 1 || d->baseline_len > d->n_samples * 1 + (int64_t(1) << 30)) return DS_EINVAL;
  if (d->precision != DS_PREC_FP64 && d->precision != DS_PREC_MIXED) return DS_EINVAL;
  if (d->reserved != 0) return DS_EINVAL;
  return DS_OK;
}

ds_status launch_status() {
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? DS_OK : DS_ECUDA;
}

// Drops a non-sticky error left by an earlier, already-reported runtime call so
// that launch_status() only sees this call's launches.
void clear_stale_error() { (void)cudaGetLastError(); }

ds_status capture_iterations(Plan& P, bool accurate, cudaEvent_t* ev, cudaGraphExec_t* out) {
  cudaGraph_t graph = nullptr;
  DS_CUDA_TRY(cudaStreamBeginCapture(P.cap_stream, cudaStreamCaptureModeThreadLocal));
  for (int k = 0; k < P.graph_iters; ++k)
    enqueue_iteration(P, P.cap_stream, ev ? ev + 5 * k : nullptr, accurate);
  cudaError_t e = cudaStreamEndCapture(P.cap_stream, &graph);
  if (e != cudaSuccess) return DS_ECUDA;
  e = cudaGraphInstantiate(out, graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) {
    *out = nullptr;
    return DS_ECUDA;
  }
  // upload now, off the plan's stream: the first replay then starts at once
  if (cudaGraphUpload(*out, P.cap_stream) != cudaSuccess) return DS_ECUDA;
  return DS_OK;
}

// CG iterations per graph replay: 16, halved (down to 4) while a replay would hold
// more than about 4 ms of work, estimated at 2 ns per sample and output.  Long
// replays hide the host's wait between them; short ones instantiate faster and
// run fewer gated iterations after convergence.
int graph_iters_for(const Plan& P) {
  if (P.graph_iters_cfg > 0) return P.graph_iters_cfg;
  const double est_ms = 2e-9 * (double)P.n_t * (double)P.desc.n_outputs;
  int gi = 16;
  while (gi > 4 && gi * est_ms > 4.0) gi /= 2;
  return gi;
}

ds_status build_graph(Plan& P) {
  const int gi = graph_iters_for(P);
  if (P.graph_exec && P.graph_profiled == P.profiling && P.graph_iters == gi) return DS_OK;
  if (P.graph_exec) {
    cudaGraphExecDestroy(P.graph_exec);
    P.graph_exec = nullptr;
  }
  if (P.graph_exec_acc) {
    cudaGraphExecDestroy(P.graph_exec_acc);
    P.graph_exec_acc = nullptr;
  }
  if (P.profiling && P.ev == nullptr) {
    P.ev = new (std::nothrow) cudaEvent_t[kGraphItersMax * 5];
    if (P.ev == nullptr) return DS_ENOMEM;
    for (int i = 0; i < kGraphItersMax * 5; ++i) DS_CUDA_TRY(cudaEventCreate(&P.ev[i]));
  }
  P.graph_iters = gi;
  // the accurate-operator graph is captured when a problem first needs it
  ds_status s = capture_iterations(P, false, P.profiling ? P.ev : nullptr, &P.graph_exec);
  if (s != DS_OK) return s;
  P.graph_profiled = P.profiling;
  return DS_OK;
}

// Adds the event timings of the first n_ran iterations of the last graph replay.
void collect_times(Plan& P, int n_ran) {
  if (!P.graph_profiled || P.ev == nullptr) return;
  for (int k = 0; k < n_ran && k < P.graph_iters; ++k) {
    cudaEvent_t* e = P.ev + 5 * k;
    float t01 = 0.f, t12 = 0.f, t23 = 0.f, t04 = 0.f;
    if (cudaEventElapsedTime(&t01, e[0], e[1]) != cudaSuccess ||
        cudaEventElapsedTime(&t12, e[1], e[2]) != cudaSuccess ||
        cudaEventElapsedTime(&t23, e[2], e[3]) != cudaSuccess ||
        cudaEventElapsedTime(&t04, e[0], e[4]) != cudaSuccess) {
      clear_stale_error();
      return;
    }
    P.t_bin += t01;
    P.t_solve += t12;
    P.t_rescan += t23;
    P.t_iter += t04;
    P.timed_iterations += 1;
  }
}

// Allocates (once) and builds the chunk-local pixel index for chunk length C
// (mixed plans, on request: the default operator reads the time-ordered pixels).
ds_status chunk_index(Plan& P, int C) {
  clear_stale_error();
  cudaError_t e = cudaSuccess;
  if (P.lid == nullptr) {
    const int64_t n_pad = (P.n_t + kChunkMax - 1) / kChunkMax * kChunkMax;
    if (e == cudaSuccess) e = dalloc(P, &P.lid, n_pad);
    if (e == cudaSuccess) e = dalloc(P, &P.upix, n_pad);
    if (e == cudaSuccess) e = dalloc(P, &P.ucnt, (P.n_t + kChunkMin - 1) / kChunkMin);
    if (e != cudaSuccess) {
      for (void* d : {(void*)P.lid, (void*)P.upix, (void*)P.ucnt})
        if (d) cudaFreeAsync(d, P.stream);
      P.lid = nullptr;
      P.upix = nullptr;
      P.ucnt = nullptr;
      return e == cudaErrorMemoryAllocation ? DS_ENOMEM : DS_ECUDA;
    }
  }
  unsigned long long* umax = reinterpret_cast<unsigned long long*>(P.scal) + 2;
  DS_CUDA_TRY(cudaMemsetAsync(umax, 0, sizeof(unsigned long long), P.stream));
  DS_CUDA_TRY(ck_build(P, C, umax));
  DS_CUDA_TRY(cudaMemcpyAsync(P.h_scal + 2, umax, sizeof(unsigned long long),
                              cudaMemcpyDeviceToHost, P.stream));
  DS_CUDA_TRY(cudaStreamSynchronize(P.stream));
  unsigned long long hu = 0;
  std::memcpy(&hu, P.h_scal + 2, sizeof(hu));
  DS_CUDA_TRY(ck_finish(P, (int64_t)hu));
  P.launches += 1;
  return DS_OK;
}

}  // namespace

extern "C" {

const char* destripe_strerror(ds_status s) {
  switch (s) {
    case DS_OK: return "ok";
    case DS_EINVAL: return "invalid argument";
    case DS_ENOMEM: return "device allocation failed";
    case DS_ECUDA: return "CUDA runtime error";
    case DS_ENOCONV: return "conjugate gradient did not converge within max_iter";
    case DS_ETIMEOUT: return "bounded device wait timed out";
    case DS_ENAN: return "non-finite value in data or iteration";
    case DS_EPIX: return "pixel index outside the map";
    case DS_ESTATE: return "call not valid for this plan";
  }
  return "unknown status";
}

ds_status destripe_plan(const ds_desc* desc, const int32_t* d_pix, const float* d_cos2psi,
                        const float* d_sin2psi, const uint8_t* d_valid, ds_plan_t* out) {
  return plan_create(desc, nullptr, d_pix, d_cos2psi, d_sin2psi, d_valid, out);
}

}  // extern "C"

ds_status ds::plan_create(const ds_desc* desc, const ds_exchange* ex, const int32_t* d_pix,
                          const float* d_cos2psi, const float* d_sin2psi,
                          const uint8_t* d_valid, ds_plan_t* out) {
  if (out == nullptr) return DS_EINVAL;
  *out = nullptr;
  ds_status s = check_desc(desc);
  if (s != DS_OK) return s;
  if (d_pix == nullptr || d_cos2psi == nullptr || d_sin2psi == nullptr) return DS_EINVAL;
  if (ex != nullptr && ex->allreduce == nullptr) return DS_EINVAL;
  if ((reinterpret_cast<uintptr_t>(d_cos2psi) & 15) || (reinterpret_cast<uintptr_t>(d_sin2psi) & 15))
    return DS_EINVAL;
  Plan* P = new (std::nothrow) Plan();
  if (P == nullptr) return DS_ENOMEM;
  std::memset(static_cast<void*>(P), 0, sizeof(Plan));
  P->desc = *desc;
  if (!(P->desc.rcond_min > 0.0)) P->desc.rcond_min = 1e-3;
  P->stream = static_cast<cudaStream_t>(desc->stream);
  P->n_o = desc->n_outputs;
  P->kinds.n_o = desc->n_outputs;
  for (int o = 0; o < DS_MAX_OUTPUTS; ++o) P->kinds.kind[o] = o < desc->n_outputs ? desc->kinds[o] : 0;
  P->n_c = n_comp_of(desc->kinds, desc->n_outputs, &P->has_I_outputs);
  P->nm = P->n_c * (P->n_c + 1) / 2;
  P->kindset = kindset_of(desc->kinds, desc->n_outputs, P->n_c);
  P->n_t = desc->n_samples;
  P->L = desc->baseline_len;
  P->n_b = (P->n_t + P->L - 1) / P->L;
  P->n_u = P->n_b * P->n_o;
  P->npix = int64_t(12) * desc->nside * desc->nside;
  P->c = d_cos2psi;
  P->s = d_sin2psi;
  if (cudaGetDevice(&P->device) != cudaSuccess ||
      cudaDeviceGetAttribute(&P->num_sms, cudaDevAttrMultiProcessorCount, P->device) != cudaSuccess) {
    plan_free(P);
    return DS_ECUDA;
  }
  P->red_len = 2 * P->num_sms * 8 + 64;
  P->reliable_delta = 1e-5;
  P->bin_mode = P->desc.precision == DS_PREC_MIXED ? 1 : 0;
  P->graph_iters_cfg = 0;  // from the problem's size
  P->blocks_per_sm = 16;
  P->accurate_df = 1;
  P->refresh_max = 50;
  P->drift_ratio = 1e4;
  P->accurate_start = 0;
  P->stall_iters = 2000;
  P->layout = 0;
  P->rescan_dedup = 1;
  P->rescan_rounds = 0;
  P->bin_order = 1;
  P->samples_per_thread = 4;
  // the coarse space costs a few ms to build (one sweep launch per coarse column),
  // and D^-1 alone (about a scalar where baselines hold equal counts) saves no
  // iterations: small problems iterate plain CG, with one kernel less per iteration
  P->precond = desc->n_samples >= kPcMinSamples ? 2 : 0;
  P->pc_nside = 8;
  P->tl_bin_samples = int64_t(1) << 26;
  if (ex != nullptr) {
    P->shard_allreduce = ex->allreduce;
    P->shard_user = ex->user;
    P->precond = 1;  // the coarse matrix would need every rank's pixel terms
  }
  cudaError_t e = cudaSuccess;
#define DS_ALLOC(ptr, n) \
  if (e == cudaSuccess) e = dalloc(*P, &P->ptr, (n));
  DS_ALLOC(pix, P->n_t);
  DS_ALLOC(hits, P->npix);
  DS_ALLOC(mask, P->npix);
  DS_ALLOC(minv, P->npix * P->nm);
  DS_ALLOC(bins, P->npix * 4);
  if (P->desc.precision == DS_PREC_MIXED) DS_ALLOC(bins32, P->npix * 4);
  if (P->desc.precision == DS_PREC_MIXED) DS_ALLOC(maplo, P->npix * 4);
  if (P->desc.precision == DS_PREC_MIXED) DS_ALLOC(xdf, P->n_u);
  if (P->desc.precision == DS_PREC_MIXED) DS_ALLOC(x32, P->n_u);
  DS_ALLOC(map32, P->npix * 4);
  DS_ALLOC(map64, P->npix * 4);
  DS_ALLOC(nvalid, P->n_b);
  DS_ALLOC(x, P->n_u);
  DS_ALLOC(r, P->n_u);
  DS_ALLOC(p, P->n_u);
  DS_ALLOC(q, P->n_u);
  DS_ALLOC(b, P->n_u);
  DS_ALLOC(t, P->n_u);
  if (P->desc.precision == DS_PREC_MIXED) DS_ALLOC(x_best, P->n_u);

  DS_ALLOC(red, P->red_len);
  DS_ALLOC(counters, 8);
  DS_ALLOC(state, 1);
  DS_ALLOC(err, 1);
  DS_ALLOC(scal, 8);
#undef DS_ALLOC
  if (e == cudaSuccess) e = cudaMallocHost(reinterpret_cast<void**>(&P->h_state), sizeof(CgState));
  if (e == cudaSuccess) e = cudaMallocHost(reinterpret_cast<void**>(&P->h_err), sizeof(int32_t));
  if (e == cudaSuccess) e = cudaMallocHost(reinterpret_cast<void**>(&P->h_scal), sizeof(double) * 8);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&P->cap_stream, cudaStreamNonBlocking);
  if (e != cudaSuccess) {
    plan_free(P);
    return e == cudaErrorMemoryAllocation ? DS_ENOMEM : DS_ECUDA;
  }
  cudaStream_t st = P->stream;
  e = cudaMemsetAsync(P->bins, 0, sizeof(double) * P->npix * 4, st);
  if (e == cudaSuccess && P->bins32) e = cudaMemsetAsync(P->bins32, 0, sizeof(float) * P->npix * 4, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(P->counters, 0, sizeof(unsigned) * 8, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(P->state, 0, sizeof(CgState), st);
  if (e == cudaSuccess) e = cudaMemsetAsync(P->x, 0, sizeof(double) * P->n_u, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(P->map32, 0, sizeof(float) * P->npix * 4, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(P->map64, 0, sizeof(double) * P->npix * 4, st);
  // cut pixels keep a zero map from here on (the batched pixel solves skip them)
  if (e == cudaSuccess && P->maplo) e = cudaMemsetAsync(P->maplo, 0, sizeof(float) * P->npix * 4, st);
  if (e != cudaSuccess) {
    plan_free(P);
    return DS_ECUDA;
  }
  s = plan_build(*P, d_pix, d_valid);
  P->launches += 3;
  if (s != DS_OK) {
    cudaStreamSynchronize(st);
    plan_free(P);
    return s;
  }
  *out = reinterpret_cast<ds_plan_t>(P);
  return DS_OK;
}

extern "C" {

ds_status destripe_plan_info(ds_plan_t plan, ds_info* info) {
  if (plan == nullptr || info == nullptr) return DS_EINVAL;
  const Plan& P = *reinterpret_cast<Plan*>(plan);
  info->n_samples = P.n_t;
  info->n_baselines = P.n_b;
  info->n_unknowns = P.n_u;
  info->n_pix = P.npix;
  info->n_good_pix = P.n_good;
  info->n_valid = P.n_valid;
  info->n_outputs = P.n_o;
  info->n_comp = P.n_c;
  info->device_bytes = P.device_bytes;
  info->layout = P.layout;
  info->bin_order = (P.layout == 2 && P.bin_order == 1 && P.rl_rec != nullptr) ? 1 : 0;
  info->n_runs = P.rl_rec != nullptr ? P.rl_n : (P.tl_rec != nullptr ? P.tl_runs : 0);
  return DS_OK;
}

void destripe_destroy(ds_plan_t plan) {
  if (plan == nullptr) return;
  Plan* P = reinterpret_cast<Plan*>(plan);
  cudaStreamSynchronize(P->stream);
  plan_free(P);
}

ds_status destripe_apply_A(ds_plan_t plan, const double* d_x, double* d_Ax) {
  if (plan == nullptr || d_x == nullptr || d_Ax == nullptr || d_x == d_Ax) return DS_EINVAL;
  Plan& P = *reinterpret_cast<Plan*>(plan);
  clear_stale_error();
  ds_status sp = tl_ensure(P);
  if (sp == DS_OK) sp = pm_ensure(P);
  if (sp != DS_OK) return sp;
  DS_CUDA_TRY(cudaMemsetAsync(d_Ax, 0, sizeof(double) * P.n_u, P.stream));
  enqueue_apply(P, P.stream, P.desc.precision == DS_PREC_FP64, d_x, d_Ax, Gate{nullptr, nullptr});
  P.launches += 3;
  return launch_status();
}

ds_status destripe_rhs(ds_plan_t plan, const void* d_y, double* d_b) {
  if (plan == nullptr || d_y == nullptr || d_b == nullptr) return DS_EINVAL;
  Plan& P = *reinterpret_cast<Plan*>(plan);
  clear_stale_error();
  DS_CUDA_TRY(cudaMemsetAsync(d_b, 0, sizeof(double) * P.n_u, P.stream));
  enqueue_rhs(P, P.stream, d_y, d_b, Gate{nullptr, nullptr});
  P.launches += 3;
  return launch_status();
}

static ds_status map_common(ds_plan_t plan, const void* d_y, const double* d_a, double* d_map,
                            int32_t* d_hits, uint8_t* d_mask) {
  if (plan == nullptr || d_y == nullptr || d_map == nullptr) return DS_EINVAL;
  Plan& P = *reinterpret_cast<Plan*>(plan);
  clear_stale_error();
  enqueue_map(P, P.stream, d_y, d_a, d_map);
  P.launches += 2;
  if (d_hits)
    DS_CUDA_TRY(cudaMemcpyAsync(d_hits, P.hits, sizeof(int32_t) * P.npix, cudaMemcpyDeviceToDevice, P.stream));
  if (d_mask)
    DS_CUDA_TRY(cudaMemcpyAsync(d_mask, P.mask, P.npix, cudaMemcpyDeviceToDevice, P.stream));
  return launch_status();
}

ds_status destripe_bin(ds_plan_t plan, const void* d_y, const double* d_a, double* d_map,
                       int32_t* d_hits, uint8_t* d_mask) {
  return map_common(plan, d_y, d_a, d_map, d_hits, d_mask);
}

ds_status destripe_map(ds_plan_t plan, const void* d_y, const double* d_a, double* d_map,
                       int32_t* d_hits, uint8_t* d_mask) {
  if (d_a == nullptr) return DS_EINVAL;
  return map_common(plan, d_y, d_a, d_map, d_hits, d_mask);
}

ds_status destripe_gauge(ds_plan_t plan, double* d_a) {
  if (plan == nullptr || d_a == nullptr) return DS_EINVAL;
  Plan& P = *reinterpret_cast<Plan*>(plan);
  clear_stale_error();
  enqueue_gauge(P, P.stream, d_a);
  P.launches += 2;
  return launch_status();
}

ds_status destripe_solve(ds_plan_t plan, const void* d_y, double* d_a, double tol,
                         int32_t max_iter, int32_t warm_start, int32_t* iters, double* rel_resid) {
  if (plan == nullptr || d_y == nullptr || d_a == nullptr) return DS_EINVAL;
  if (!(tol >= 0.0) || !std::isfinite(tol)) return DS_EINVAL;
  Plan& P = *reinterpret_cast<Plan*>(plan);
  if (P.shard_allreduce != nullptr) return DS_ESTATE;  // destripe_solve_sharded
  if (max_iter <= 0) max_iter = 10000;
  clear_stale_error();
  cudaStream_t st = P.stream;
  if (warm_start)
    DS_CUDA_TRY(cudaMemcpyAsync(P.x, d_a, sizeof(double) * P.n_u, cudaMemcpyDeviceToDevice, st));
  DS_CUDA_TRY(cudaMemsetAsync(P.b, 0, sizeof(double) * P.n_u, st));
  // a first solve builds the tiled records the plan chose, and the pixel-major copy
  // beside its right-hand side
  const ds_status stl = tl_ensure(P);
  if (stl != DS_OK) return stl;
  // the probe of long baselines waits for its result, so it comes before the
  // right-hand side is queued
  const ds_status spr = pc_probe(P);
  if (spr != DS_OK) return spr;
  bool pm_started = false;
  const ds_status sp = pm_begin(P, &pm_started);
  if (sp != DS_OK) return sp;
  enqueue_rhs(P, st, d_y, P.b, Gate{nullptr, nullptr});
  // b lies in the range of A up to rounding: its component along A's null vector
  // (one offset on every I-carrying baseline) is rounding alone, which CG cannot
  // reduce and which would grow the iterate along that vector.  Removed here, so
  // that a right-hand side of rounding size (a noiseless sky) is solved like any
  // other.
  if (P.has_I_outputs) {
    enqueue_gauge(P, st, P.b);
    P.launches += 2;
  }
  ds_status s = pm_join(P, pm_started);
  if (s != DS_OK) return s;
  // the two-level preconditioner's coarse space, built once per plan
  if (P.precond == 2 && !P.pc_built) {
    s = pc_prepare(P);
    if (s != DS_OK) return s;
  }
  enqueue_cg_setup(P, st, tol, max_iter, P.reliable_delta, warm_start ? 1 : 0, true);
  P.launches += 3 + 3 + (warm_start ? 3 : 0) + (pc_mode(P) ? 3 : 0);
  s = launch_status();
  if (s != DS_OK) return s;
  s = build_graph(P);
  if (s != DS_OK) return s;
  const int max_launches = max_iter / P.graph_iters + 4;
  bool done = false;
  int iter_before = 0;
  bool accurate = P.accurate_start != 0 && P.desc.precision == DS_PREC_MIXED;
  for (int k = 0; k < max_launches && !done; ++k) {
    // a mixed problem that the float32 operator cannot follow continues with the
    // accurate one (the switch is decided on the device at a float64 refresh)
    if (accurate && P.graph_exec_acc == nullptr && P.desc.precision == DS_PREC_MIXED) {
      const ds_status sa = capture_iterations(P, true, nullptr, &P.graph_exec_acc);
      if (sa != DS_OK) return sa;
    }
    const bool acc_now = accurate && P.graph_exec_acc != nullptr;
    DS_CUDA_TRY(cudaGraphLaunch(acc_now ? P.graph_exec_acc : P.graph_exec, st));
    DS_CUDA_TRY(cudaMemcpyAsync(P.h_state, P.state, sizeof(CgState), cudaMemcpyDeviceToHost, st));
    DS_CUDA_TRY(cudaStreamSynchronize(st));
    done = P.h_state->done != 0;
    accurate = P.h_state->accurate != 0;
    P.graph_launches += 1;
    P.launches += (int64_t)P.graph_iters * kernels_per_iteration(P, acc_now);
    const int ran = P.h_state->iter - iter_before;
    iter_before = P.h_state->iter;
    P.iterations += ran;
    if (!acc_now) collect_times(P, ran);  // events live in the float32 graph only
  }
  DS_CUDA_TRY(cudaMemcpyAsync(P.h_state, P.state, sizeof(CgState), cudaMemcpyDeviceToHost, st));
  DS_CUDA_TRY(cudaMemcpyAsync(P.h_err, P.err, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
  DS_CUDA_TRY(cudaStreamSynchronize(st));
  const CgState H = *P.h_state;
  // Mixed plans that did not converge return the iterate with the smallest
  // float64 residual seen (a float32 operator can drift on ill-posed problems).
  const bool use_best = P.x_best != nullptr && H.status != 1 && !(H.rr_true <= H.rr_best);
  double* result = use_best ? P.x_best : P.x;
  // The coarse correction boosts the slow sky-like modes.  Where A is nearly
  // singular along them, the iteration's arithmetic cannot resolve them and CG
  // breaks down (no curvature, non-finite values) or stalls.  Such a solve goes on
  // without the coarse correction from its best iterate, and the plan keeps D^-1
  // alone from then on.
  const bool broke = (H.status == 3 && !(H.rr_true <= H.tol2)) || H.status == 4 || H.status == 5;
  if (broke && pc_ready(P) && std::isfinite(H.bb) && H.iter < max_iter) {
    P.pc_fallback = 1;
    for (cudaGraphExec_t* gx : {&P.graph_exec, &P.graph_exec_acc})
      if (*gx) {
        cudaGraphExecDestroy(*gx);
        *gx = nullptr;
      }
    const bool from_zero = !use_best && H.status == 4;  // float64 plan with non-finite x
    if (from_zero) DS_CUDA_TRY(cudaMemsetAsync(d_a, 0, sizeof(double) * P.n_u, st));
    else DS_CUDA_TRY(cudaMemcpyAsync(d_a, result, sizeof(double) * P.n_u, cudaMemcpyDeviceToDevice, st));
    int32_t it2 = 0;
    const ds_status s2 = destripe_solve(plan, d_y, d_a, tol, max_iter - H.iter, 1, &it2, rel_resid);
    if (iters) *iters = H.iter + it2;
    return s2;
  }
  enqueue_gauge(P, st, result);
  P.launches += 2;
  DS_CUDA_TRY(cudaMemcpyAsync(d_a, result, sizeof(double) * P.n_u, cudaMemcpyDeviceToDevice, st));
  DS_CUDA_TRY(cudaStreamSynchronize(st));
  const double rr_out = use_best ? H.rr_best : H.rr_true;
  if (iters) *iters = H.iter;
  if (rel_resid) *rel_resid = H.bb > 0.0 ? std::sqrt(rr_out / H.bb) : 0.0;
  if (!std::isfinite(H.bb)) return DS_ENAN;
  if (!done) return DS_ENOCONV;
  switch (H.status) {
    case 1: return DS_OK;
    case 2: return DS_ENOCONV;
    case 3: return H.rr_true <= H.tol2 ? DS_OK : DS_ENOCONV;
    case 5: return DS_ENOCONV;  // stalled: no 10x residual drop in stall_iters iterations
    default: return P.x_best != nullptr ? DS_ENOCONV : DS_ENAN;
  }
}

ds_status destripe_profile(ds_plan_t plan, int32_t enable, ds_profile* out) {
  if (plan == nullptr) return DS_EINVAL;
  Plan& P = *reinterpret_cast<Plan*>(plan);
  if (enable == 1 || enable == 0) {
    P.profiling = enable;
    if (enable == 1) {
      P.launches = 0;
      P.graph_launches = 0;
      P.iterations = 0;
      P.timed_iterations = 0;
      P.t_bin = P.t_rescan = P.t_solve = P.t_iter = 0.0;
    }
  }
  if (out) {
    out->kernel_launches = P.launches;
    out->graph_launches = P.graph_launches;
    out->iterations = P.iterations;
    out->timed_iterations = P.timed_iterations;
    out->bin_ms = P.t_bin;
    out->rescan_ms = P.t_rescan;
    out->solve_ms = P.t_solve;
    out->iteration_ms = P.t_iter;
  }
  return DS_OK;
}

ds_status destripe_tune(ds_plan_t plan, const char* key, double value) {
  if (plan == nullptr || key == nullptr) return DS_EINVAL;
  Plan& P = *reinterpret_cast<Plan*>(plan);
  const std::string k(key);
  if (k == "reliable_delta") {
    if (!(value > 0.0 && value < 1.0)) return DS_EINVAL;
    P.reliable_delta = value;
  } else if (k == "bin_mode") {
    if (value != 0.0 && value != 1.0) return DS_EINVAL;
    if (value == 1.0 && P.bins32 == nullptr) return DS_ESTATE;
    P.bin_mode = (int)value;
  } else if (k == "graph_iters") {
    if (!(value >= 0.0 && value <= kGraphItersMax) || value != std::floor(value)) return DS_EINVAL;
    P.graph_iters_cfg = (int)value;
  } else if (k == "accurate_df") {
    if (value != 0.0 && value != 1.0) return DS_EINVAL;
    if (value == 1.0 && P.maplo == nullptr) return DS_ESTATE;
    P.accurate_df = (int)value;
  } else if (k == "refresh_max") {
    if (!(value >= 1.0 && value <= 1e6)) return DS_EINVAL;
    P.refresh_max = (int)value;
  } else if (k == "layout") {
    if (value != 0.0 && value != 1.0 && value != 2.0 && value != 3.0) return DS_EINVAL;
    if (value != 0.0 && P.desc.precision != DS_PREC_MIXED) return DS_ESTATE;
    P.tl_pending = 0;  // an explicit choice replaces the plan's own
    if (value == 1.0 && P.lid == nullptr) {
      const ds_status s = chunk_index(P, ck_default_chunk(P.n_t, P.num_sms));
      if (s != DS_OK) return s;
    }
    if (value == 2.0 && P.rl_rec != nullptr && P.rl_df == nullptr) {
      cudaStreamSynchronize(P.stream);
      rl_release(P, P.stream);  // runs kept for tiles lack the accurate passes' sums
    }
    if (value == 2.0 && P.rl_rec == nullptr) {
      clear_stale_error();
      const ds_status s = rl_build(P);
      if (s != DS_OK) return s;
      // records asked for above the automatic density: the rescans keep the samples
      P.rescan_samples = (double)P.rl_n > kRunsPerSampleMax * (double)P.n_t ? 1 : 0;
    }
    if (value == 3.0 && P.tl_rec == nullptr) {
      clear_stale_error();
      ds_status s = P.rl_rec == nullptr ? rl_build(P) : DS_OK;
      if (s == DS_OK) s = tl_build(P);
      if (s == DS_OK && cudaStreamSynchronize(P.stream) != cudaSuccess) s = DS_ECUDA;
      if (s != DS_OK) return s;
    }
    P.layout = (int)value;
  } else if (k == "chunk") {
    const int C = (int)value;
    if ((double)C != value || C < kChunkMin || C > kChunkMax || (C & (C - 1)) != 0) return DS_EINVAL;
    if (P.desc.precision != DS_PREC_MIXED) return DS_ESTATE;
    const ds_status s = chunk_index(P, C);
    if (s != DS_OK) return s;
  } else if (k == "drift_ratio") {
    if (!(value > 1.0 && value < 1e30)) return DS_EINVAL;
    P.drift_ratio = value;
  } else if (k == "stall_iters") {
    if (!(value >= 0.0 && value <= 1e9)) return DS_EINVAL;
    P.stall_iters = (int)value;
  } else if (k == "accurate_start") {
    if (value != 0.0 && value != 1.0) return DS_EINVAL;
    if (value == 1.0 && P.desc.precision != DS_PREC_MIXED) return DS_ESTATE;
    P.accurate_start = (int)value;
  } else if (k == "samples_per_thread") {
    if (value != 4.0 && value != 8.0) return DS_EINVAL;
    P.samples_per_thread = (int)value;
  } else if (k == "rescan_dedup") {
    if (value != 0.0 && value != 1.0) return DS_EINVAL;
    P.rescan_dedup = (int)value;
  } else if (k == "bin_order") {
    if (value != 0.0 && value != 1.0) return DS_EINVAL;
    if (P.desc.precision != DS_PREC_MIXED) return DS_ESTATE;
    if (value == 1.0 && P.pm_rec == nullptr && P.rl_rec != nullptr) {
      clear_stale_error();
      ds_status s = pm_build(P, P.stream);
      if (s == DS_OK && cudaStreamSynchronize(P.stream) != cudaSuccess) s = DS_ECUDA;
      if (s != DS_OK) return s;
    }
    P.bin_order = (int)value;
  } else if (k == "rescan_rounds") {
    if (!(value >= 0.0 && value <= 16.0) || (double)(int)value != value) return DS_EINVAL;
    P.rescan_rounds = (int)value;
  } else if (k == "rescan_samples") {
    if (value != 0.0 && value != 1.0) return DS_EINVAL;
    P.rescan_samples = (int)value;
  } else if (k == "precond") {
    if (value != 0.0 && value != 1.0 && value != 2.0) return DS_EINVAL;
    if (value == 2.0 && P.shard_allreduce != nullptr) return DS_ESTATE;
    P.precond = (int)value;
  } else if (k == "coarse_nside") {
    const int nc = (int)value;
    if ((double)nc != value || nc < 1 || nc > 64 || (nc & (nc - 1)) != 0) return DS_EINVAL;
    if (nc != P.pc_nside) {
      cudaStreamSynchronize(P.stream);
      pc_free(P, P.stream);
      P.pc_nside = nc;
    }
  } else if (k == "bin_tile_samples") {
    if (!(value >= 1.0 && value <= 1e15) || (double)(int64_t)value != value) return DS_EINVAL;
    if (P.tl_rec != nullptr) return DS_ESTATE;  // the long tiles are already built
    P.tl_bin_samples = (int64_t)value;
  } else if (k == "blocks_per_sm") {
    if (!(value >= 1.0 && value <= 32.0)) return DS_EINVAL;
    P.blocks_per_sm = (int)value;
  } else {
    return DS_EINVAL;
  }
  // the captured graphs bake in launch shapes and kernel choices: rebuild them
  if (P.graph_exec) {
    cudaGraphExecDestroy(P.graph_exec);
    P.graph_exec = nullptr;
  }
  if (P.graph_exec_acc) {
    cudaGraphExecDestroy(P.graph_exec_acc);
    P.graph_exec_acc = nullptr;
  }
  return DS_OK;
}

ds_status destripe_run_host(const ds_desc* desc, const int32_t* h_pix, const float* h_c,
                            const float* h_s, const uint8_t* h_valid, const void* h_y,
                            double tol, int32_t max_iter, double* h_a, double* h_map,
                            int32_t* h_hits, uint8_t* h_mask, int32_t* iters,
                            double* rel_resid) {
  ds_status s = check_desc(desc);
  if (s != DS_OK) return s;
  if (!h_pix || !h_c || !h_s || !h_y) return DS_EINVAL;
  cudaStream_t st = static_cast<cudaStream_t>(desc->stream);
  const int64_t n_t = desc->n_samples, n_o = desc->n_outputs;
  const int64_t n_b = (n_t + desc->baseline_len - 1) / desc->baseline_len;
  int has_i;
  const int64_t n_c = n_comp_of(desc->kinds, desc->n_outputs, &has_i);
  const int64_t npix = int64_t(12) * desc->nside * desc->nside;
  const size_t ysz = desc->precision == DS_PREC_FP64 ? sizeof(double) : sizeof(float);
  int32_t* d_pix = nullptr;
  float *d_c = nullptr, *d_s = nullptr;
  uint8_t *d_valid = nullptr, *d_mask = nullptr;
  void* d_y = nullptr;
  double *d_a = nullptr, *d_map = nullptr;
  int32_t* d_hits = nullptr;
  ds_plan_t plan = nullptr;
  // device buffers come from the library's pool (reused across calls)
  int device = 0;
  cudaMemPool_t pool = nullptr;
  cudaError_t e = cudaGetDevice(&device);
  if (e == cudaSuccess) e = plan_pool(device, &pool);
  auto dmalloc = [&](void** ptr, size_t bytes) { return cudaMallocFromPoolAsync(ptr, bytes, pool, st); };
  if (e == cudaSuccess) e = dmalloc(reinterpret_cast<void**>(&d_pix), sizeof(int32_t) * n_t);
  if (e == cudaSuccess) e = dmalloc(reinterpret_cast<void**>(&d_c), sizeof(float) * n_t);
  if (e == cudaSuccess) e = dmalloc(reinterpret_cast<void**>(&d_s), sizeof(float) * n_t);
  if (e == cudaSuccess && h_valid) e = dmalloc(reinterpret_cast<void**>(&d_valid), n_t);
  if (e == cudaSuccess) e = dmalloc(&d_y, ysz * n_t * n_o);
  if (e == cudaSuccess) e = dmalloc(reinterpret_cast<void**>(&d_a), sizeof(double) * n_b * n_o);
  if (e == cudaSuccess) e = dmalloc(reinterpret_cast<void**>(&d_map), sizeof(double) * n_c * npix);
  if (e == cudaSuccess) e = dmalloc(reinterpret_cast<void**>(&d_hits), sizeof(int32_t) * npix);
  if (e == cudaSuccess) e = dmalloc(reinterpret_cast<void**>(&d_mask), npix);
  if (e == cudaSuccess) e = cudaMemcpyAsync(d_pix, h_pix, sizeof(int32_t) * n_t, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(d_c, h_c, sizeof(float) * n_t, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(d_s, h_s, sizeof(float) * n_t, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess && h_valid) e = cudaMemcpyAsync(d_valid, h_valid, n_t, cudaMemcpyHostToDevice, st);
  // the timelines travel on a second stream while the plan (pointing only) is built
  cudaStream_t st_y = nullptr;
  cudaEvent_t ev_alloc = nullptr, ev_y = nullptr;
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&st_y, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ev_alloc, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ev_y, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventRecord(ev_alloc, st);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(st_y, ev_alloc, 0);
  if (e == cudaSuccess) e = cudaMemcpyAsync(d_y, h_y, ysz * n_t * n_o, cudaMemcpyHostToDevice, st_y);
  if (e == cudaSuccess) e = cudaEventRecord(ev_y, st_y);
  if (e != cudaSuccess) s = (e == cudaErrorMemoryAllocation) ? DS_ENOMEM : DS_ECUDA;
  if (s == DS_OK) s = destripe_plan(desc, d_pix, d_c, d_s, d_valid, &plan);
  // the work of the first solve that reads only the pointing (the tiled records, a
  // coarse space that needs no pixel-major copy) also runs while the timelines travel
  if (s == DS_OK) {
    Plan& P = *reinterpret_cast<Plan*>(plan);
    s = tl_ensure(P);
    if (s == DS_OK) s = pc_probe(P);
    if (s == DS_OK && P.precond == 2 && !P.pc_built && P.layout == 3 && P.tl2_end != nullptr)
      s = pc_prepare(P);
  }
  if (ev_y != nullptr && cudaStreamWaitEvent(st, ev_y, 0) != cudaSuccess && s == DS_OK) s = DS_ECUDA;
  ds_status solve_s = DS_OK;
  if (s == DS_OK) {
    solve_s = destripe_solve(plan, d_y, d_a, tol, max_iter, 0, iters, rel_resid);
    if (solve_s != DS_OK && solve_s != DS_ENOCONV) s = solve_s;
  }
  if (s == DS_OK && h_map) s = destripe_map(plan, d_y, d_a, d_map, d_hits, d_mask);
  if (s == DS_OK && h_a) s = cudaMemcpyAsync(h_a, d_a, sizeof(double) * n_b * n_o, cudaMemcpyDeviceToHost, st) == cudaSuccess ? DS_OK : DS_ECUDA;
  if (s == DS_OK && h_map) s = cudaMemcpyAsync(h_map, d_map, sizeof(double) * n_c * npix, cudaMemcpyDeviceToHost, st) == cudaSuccess ? DS_OK : DS_ECUDA;
  if (s == DS_OK && h_hits && h_map) s = cudaMemcpyAsync(h_hits, d_hits, sizeof(int32_t) * npix, cudaMemcpyDeviceToHost, st) == cudaSuccess ? DS_OK : DS_ECUDA;
  if (s == DS_OK && h_mask && h_map) s = cudaMemcpyAsync(h_mask, d_mask, npix, cudaMemcpyDeviceToHost, st) == cudaSuccess ? DS_OK : DS_ECUDA;
  if (cudaStreamSynchronize(st) != cudaSuccess && s == DS_OK) s = DS_ECUDA;
  if (st_y != nullptr) {
    cudaStreamSynchronize(st_y);  // the timeline copy has ended even on an early error
    cudaStreamDestroy(st_y);
  }
  if (ev_alloc) cudaEventDestroy(ev_alloc);
  if (ev_y) cudaEventDestroy(ev_y);
  if (plan) destripe_destroy(plan);
  void* bufs[] = {d_pix, d_c, d_s, d_valid, d_y, d_a, d_map, d_hits, d_mask};
  for (void* b : bufs)
    if (b) cudaFreeAsync(b, st);
  cudaStreamSynchronize(st);
  if (s == DS_OK && solve_s == DS_ENOCONV) s = DS_ENOCONV;
  return s;
}

}  // extern "C"
