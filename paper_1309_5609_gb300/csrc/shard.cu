// Time-sharded solves: one problem over several processes (one per GPU), each
// holding a contiguous time slice (Sect. 4: the Epetra maps distribute samples and
// baselines by time; the pixel-domain quantities are exchanged once per operator
// application).  The exchange itself is the caller's all-reduce (ds_exchange),
// called by the plan build (hits, pixel matrices), by every binning pass before
// its pixel solve (apply.cu) and by the CG below (dot products, gauge sums).
//
// The CG runs from the host: every scalar is reduced over the ranks before the
// next step needs it, so that no rank's kernels ever wait on another rank.
#include <cmath>

#include "internal.cuh"

namespace ds {

void enqueue_dot(const Plan& P, cudaStream_t st, const double* a, const double* b, int64_t n,
                 double* out);

void shard_exchange(const Plan& P, cudaStream_t st, void* d_buf, int64_t count, int32_t dtype) {
  if (P.shard_allreduce == nullptr || P.shard_err) return;
  if (P.shard_allreduce(d_buf, count, dtype, static_cast<void*>(st), P.shard_user) != 0)
    P.shard_err = 1;
}

namespace {

constexpr int kBlock = 256;

__global__ void __launch_bounds__(kBlock) k_sh_update(double* __restrict__ x,
                                                      double* __restrict__ r,
                                                      const double* __restrict__ p,
                                                      const double* __restrict__ q, double alpha,
                                                      int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    x[i] = fma(alpha, p[i], x[i]);
    r[i] = fma(-alpha, q[i], r[i]);
  }
}

// r = b - t, t = 0
__global__ void __launch_bounds__(kBlock) k_sh_residual(double* __restrict__ r,
                                                        const double* __restrict__ b,
                                                        double* __restrict__ t, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    r[i] = b[i] - t[i];
    t[i] = 0.0;
  }
}

// p = r + beta p, q = 0
__global__ void __launch_bounds__(kBlock) k_sh_direction(double* __restrict__ p,
                                                         const double* __restrict__ r,
                                                         double* __restrict__ q, double beta,
                                                         int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    p[i] = fma(beta, p[i], r[i]);
    q[i] = 0.0;
  }
}

// sums[0] += this rank's baselines of I-carrying outputs with data, sums[1] += their count
__global__ void __launch_bounds__(kBlock) k_sh_gauge_sums(const double* __restrict__ a,
                                                          const int32_t* __restrict__ nvalid,
                                                          int64_t n_b, KindsArg kk,
                                                          double* __restrict__ sums) {
  double s = 0.0, c = 0.0;
  for (int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; b < n_b;
       b += (int64_t)gridDim.x * blockDim.x) {
    if (nvalid[b] <= 0) continue;
    for (int o = 0; o < kk.n_o; ++o)
      if (kk.kind[o] == DS_KIND_I || kk.kind[o] == DS_KIND_IQU) {
        s += a[o * n_b + b];
        c += 1.0;
      }
  }
  for (int d = 16; d > 0; d >>= 1) {
    s += __shfl_down_sync(0xffffffffu, s, d);
    c += __shfl_down_sync(0xffffffffu, c, d);
  }
  if ((threadIdx.x & 31) == 0 && c > 0.0) {
    atomicAdd(sums, s);
    atomicAdd(sums + 1, c);
  }
}

__global__ void __launch_bounds__(kBlock) k_sh_gauge_apply(double* __restrict__ a,
                                                           const int32_t* __restrict__ nvalid,
                                                           int64_t n_b, KindsArg kk,
                                                           const double* __restrict__ sums) {
  const double mean = sums[1] > 0.0 ? sums[0] / sums[1] : 0.0;
  for (int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; b < n_b;
       b += (int64_t)gridDim.x * blockDim.x) {
    const bool has = nvalid[b] > 0;
    for (int o = 0; o < kk.n_o; ++o) {
      double v = a[o * n_b + b];
      if (!has) v = 0.0;
      else if (kk.kind[o] == DS_KIND_I || kk.kind[o] == DS_KIND_IQU) v -= mean;
      a[o * n_b + b] = v;
    }
  }
}

int vgrid(const Plan& P, int64_t n) { return stream_grid(P, n, kBlock, 8); }

// Dot product over all ranks: this rank's share (deterministic block partials),
// then the exchange, then to the host.
ds_status global_dot(Plan& P, const double* a, const double* b, int64_t n, double* out) {
  cudaStream_t st = P.stream;
  enqueue_dot(P, st, a, b, n, P.scal + 6);
  shard_exchange(P, st, P.scal + 6, 1, DS_DT_F64);
  if (P.shard_err) return DS_ECUDA;
  DS_CUDA_TRY(cudaMemcpyAsync(P.h_scal + 6, P.scal + 6, sizeof(double), cudaMemcpyDeviceToHost, st));
  DS_CUDA_TRY(cudaStreamSynchronize(st));
  *out = P.h_scal[6];
  return DS_OK;
}

}  // namespace

}  // namespace ds

using namespace ds;

extern "C" {

ds_status destripe_plan_sharded(const ds_desc* desc, const ds_exchange* ex, const int32_t* d_pix,
                                const float* d_cos2psi, const float* d_sin2psi,
                                const uint8_t* d_valid, ds_plan_t* out) {
  if (ex == nullptr || ex->allreduce == nullptr) return DS_EINVAL;
  const ds_status s = plan_create(desc, ex, d_pix, d_cos2psi, d_sin2psi, d_valid, out);
  if (s == DS_OK) reinterpret_cast<Plan*>(*out)->precond = 0;
  return s;
}

ds_status destripe_solve_sharded(ds_plan_t plan, const void* d_y, double* d_a, double tol,
                                 int32_t max_iter, int32_t warm_start, int32_t* iters,
                                 double* rel_resid) {
  if (plan == nullptr || d_y == nullptr || d_a == nullptr) return DS_EINVAL;
  if (!(tol >= 0.0) || !std::isfinite(tol)) return DS_EINVAL;
  Plan& P = *reinterpret_cast<Plan*>(plan);
  if (P.shard_allreduce == nullptr) return DS_ESTATE;
  if (max_iter <= 0) max_iter = 10000;
  (void)cudaGetLastError();
  P.shard_err = 0;
  cudaStream_t st = P.stream;
  const int64_t n = P.n_u;
  const bool mixed = P.desc.precision == DS_PREC_MIXED;
  const int g = vgrid(P, n);
  const Gate open{nullptr, nullptr};
  ds_status s = pm_ensure(P);
  if (s != DS_OK) return s;
  // b = F~^T Z y (pixel sums exchanged inside)
  DS_CUDA_TRY(cudaMemsetAsync(P.b, 0, sizeof(double) * n, st));
  enqueue_rhs(P, st, d_y, P.b, open);
  // x0, r0 = b - A x0
  DS_CUDA_TRY(cudaMemsetAsync(P.t, 0, sizeof(double) * n, st));
  if (warm_start) {
    DS_CUDA_TRY(cudaMemcpyAsync(P.x, d_a, sizeof(double) * n, cudaMemcpyDeviceToDevice, st));
    enqueue_apply(P, st, true, P.x, P.t, open);
  } else {
    DS_CUDA_TRY(cudaMemsetAsync(P.x, 0, sizeof(double) * n, st));
  }
  k_sh_residual<<<g, kBlock, 0, st>>>(P.r, P.b, P.t, n);
  DS_CUDA_TRY(cudaMemcpyAsync(P.p, P.r, sizeof(double) * n, cudaMemcpyDeviceToDevice, st));
  DS_CUDA_TRY(cudaMemsetAsync(P.q, 0, sizeof(double) * n, st));
  DS_CUDA_TRY(cudaGetLastError());
  double bb = 0.0, rr = 0.0;
  if ((s = global_dot(P, P.b, P.b, n, &bb)) != DS_OK) return s;
  if ((s = global_dot(P, P.r, P.r, n, &rr)) != DS_OK) return s;
  if (!std::isfinite(bb) || !std::isfinite(rr)) return DS_ENAN;
  const double tol2 = tol * tol * bb;
  const double delta2 = P.reliable_delta * P.reliable_delta;
  double rr_anchor = rr;
  int it = 0, last_refresh = 0;
  bool converged = rr <= tol2, failed = false;
  while (!converged && it < max_iter) {
    ++it;
    enqueue_apply(P, st, !mixed, P.p, P.q, open);
    double pq = 0.0;
    if ((s = global_dot(P, P.p, P.q, n, &pq)) != DS_OK) return s;
    if (!std::isfinite(pq)) return DS_ENAN;
    if (!(pq > 0.0)) {  // no curvature left along p
      failed = true;
      break;
    }
    const double alpha = rr / pq;
    k_sh_update<<<g, kBlock, 0, st>>>(P.x, P.r, P.p, P.q, alpha, n);
    double rr_new = 0.0;
    if ((s = global_dot(P, P.r, P.r, n, &rr_new)) != DS_OK) return s;
    if (!std::isfinite(rr_new)) return DS_ENAN;
    // float32 iterations: the residual is recomputed in the accurate arithmetic
    // whenever it has dropped by the refresh ratio, claims convergence, or has gone
    // refresh_max iterations without a refresh
    if (mixed && (rr_new <= tol2 || rr_new < delta2 * rr_anchor ||
                  it - last_refresh >= P.refresh_max || it == max_iter)) {
      enqueue_apply(P, st, true, P.x, P.t, open);
      k_sh_residual<<<g, kBlock, 0, st>>>(P.r, P.b, P.t, n);
      if ((s = global_dot(P, P.r, P.r, n, &rr_new)) != DS_OK) return s;
      rr_anchor = rr_new;
      last_refresh = it;
    }
    if (rr_new <= tol2) converged = true;
    const double beta = rr_new / rr;
    rr = rr_new;
    if (!converged) k_sh_direction<<<g, kBlock, 0, st>>>(P.p, P.r, P.q, beta, n);
    if (P.shard_err) return DS_ECUDA;
  }
  // gauge with the mean over every rank's baselines
  DS_CUDA_TRY(cudaMemsetAsync(P.scal + 4, 0, sizeof(double) * 2, st));
  k_sh_gauge_sums<<<vgrid(P, P.n_b), kBlock, 0, st>>>(P.x, P.nvalid, P.n_b, P.kinds, P.scal + 4);
  shard_exchange(P, st, P.scal + 4, 2, DS_DT_F64);
  k_sh_gauge_apply<<<vgrid(P, P.n_b), kBlock, 0, st>>>(P.x, P.nvalid, P.n_b, P.kinds, P.scal + 4);
  DS_CUDA_TRY(cudaMemcpyAsync(d_a, P.x, sizeof(double) * n, cudaMemcpyDeviceToDevice, st));
  DS_CUDA_TRY(cudaGetLastError());
  DS_CUDA_TRY(cudaStreamSynchronize(st));
  if (P.shard_err) return DS_ECUDA;
  P.iterations += it;
  if (iters) *iters = it;
  if (rel_resid) *rel_resid = bb > 0.0 ? std::sqrt(rr / bb) : 0.0;
  if (converged) return DS_OK;
  return failed && rr <= tol2 ? DS_OK : DS_ENOCONV;
}

}  // extern "C"
