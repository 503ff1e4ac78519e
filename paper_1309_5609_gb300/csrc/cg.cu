// Conjugate gradient on the destriping equation (Sect. 3 names CG; the operator
// F~^T Z F~ is symmetric positive semi-definite), with every scalar kept on the
// device so that iterations run back to back inside one captured CUDA graph.
//
// Dot products are deterministic: each block writes its partial sum, and the
// last block to finish (ticket counter) adds the partials in block order.
//
// In mixed precision the per-sample operator runs in float32.  Whenever the
// recursive residual has dropped by a set factor since the last float64 check,
// or claims convergence, the residual is recomputed as b - A x with the float64
// operator and CG continues from it ("reliable updates").
#include <cmath>

#include "cg_state.cuh"
#include "df.cuh"
#include "internal.cuh"
#include "rows.cuh"

namespace ds {

namespace {

constexpr int kBlock = 256;

__device__ __forceinline__ double block_sum(double v) {
  __shared__ double sm[32];
  for (int d = 16; d > 0; d >>= 1) v += __shfl_down_sync(0xffffffffu, v, d);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) sm[wid] = v;
  __syncthreads();
  v = 0.0;
  if (wid == 0) {
    v = lane < (int)(blockDim.x >> 5) ? sm[lane] : 0.0;
    for (int d = 16; d > 0; d >>= 1) v += __shfl_down_sync(0xffffffffu, v, d);
  }
  __syncthreads();
  return v;  // valid in thread 0
}

// Writes this block's partial; returns true in exactly one thread of the last
// block, with *total = sum of all partials in block order.
__device__ bool finish_sum(double partial, double* __restrict__ red, unsigned* __restrict__ ticket,
                           double* total) {
  __shared__ bool last;
  const double bs = block_sum(partial);
  if (threadIdx.x == 0) {
    red[blockIdx.x] = bs;
    __threadfence();
    const unsigned t = atomicAdd(ticket, 1u);
    last = (t == gridDim.x - 1);
  }
  __syncthreads();
  if (!last) return false;
  __threadfence();
  double v = 0.0;
  // fixed order: thread i adds partials i, i + blockDim, ... then a block sum
  for (unsigned i = threadIdx.x; i < gridDim.x; i += blockDim.x) v += ((volatile double*)red)[i];
  v = block_sum(v);
  if (threadIdx.x == 0) {
    *ticket = 0u;
    *total = v;
    return true;
  }
  return false;
}

// The same, returning true in every thread of the last block, with *total (the
// sum of all partials in block order) valid in all of them.
__device__ bool finish_sum_block(double partial, double* __restrict__ red,
                                 unsigned* __restrict__ ticket, double* total) {
  __shared__ bool last;
  __shared__ double s_tot;
  const double bs = block_sum(partial);
  if (threadIdx.x == 0) {
    red[blockIdx.x] = bs;
    __threadfence();
    const unsigned t = atomicAdd(ticket, 1u);
    last = (t == gridDim.x - 1);
  }
  __syncthreads();
  if (!last) return false;
  __threadfence();
  double v = 0.0;
  for (unsigned i = threadIdx.x; i < gridDim.x; i += blockDim.x) v += ((volatile double*)red)[i];
  v = block_sum(v);
  if (threadIdx.x == 0) {
    *ticket = 0u;
    s_tot = v;
  }
  __syncthreads();
  *total = s_tot;
  return true;
}

// The vector kernels below read pairs of elements with one 16-byte load (the
// vectors are 256-byte aligned allocations); with odd n, thread 0 of block 0 also
// takes the last element.  Every thread's share is fixed, so sums stay
// deterministic.
__device__ __forceinline__ int64_t gtid() { return (int64_t)blockIdx.x * blockDim.x + threadIdx.x; }
__device__ __forceinline__ int64_t gstride() { return (int64_t)gridDim.x * blockDim.x; }

__global__ void __launch_bounds__(kBlock) k_dot(const double* __restrict__ a,
                                                const double* __restrict__ b, int64_t n,
                                                double* __restrict__ red, unsigned* ticket,
                                                double* __restrict__ out, Gate g) {
  if (gate_closed(g)) return;
  const double2* a2 = reinterpret_cast<const double2*>(a);
  const double2* b2 = reinterpret_cast<const double2*>(b);
  double acc = 0.0;
  for (int64_t i = gtid(); i < (n >> 1); i += gstride()) {
    const double2 u = a2[i], v = b2[i];
    acc = fma(u.x, v.x, acc);
    acc = fma(u.y, v.y, acc);
  }
  if ((n & 1) && gtid() == 0) acc = fma(a[n - 1], b[n - 1], acc);
  double tot;
  if (finish_sum(acc, red, ticket, &tot)) *out = tot;
}

// CG start: x = x0 or 0; r = b - t (t = A x0, or 0); p = r; rr = r.r.
__global__ void __launch_bounds__(kBlock) k_cg_start(double* __restrict__ x, double* __restrict__ r,
                                                     double* __restrict__ p, double* __restrict__ q,
                                                     const double* __restrict__ b,
                                                     double* __restrict__ t, int warm, int64_t n,
                                                     double* __restrict__ red, unsigned* ticket,
                                                     CgState* st, double* __restrict__ x_best) {
  double acc = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double ri = warm ? b[i] - t[i] : b[i];
    if (!warm) x[i] = 0.0;
    if (x_best != nullptr) x_best[i] = warm ? x[i] : 0.0;
    r[i] = ri;
    p[i] = ri;
    q[i] = 0.0;
    t[i] = 0.0;
    acc += ri * ri;
  }
  double tot;
  if (finish_sum(acc, red, ticket, &tot)) {
    st->rr = tot;
    st->rr_old = tot;
    st->rr_anchor = tot;
    st->rr_true = tot;
    st->iter = 0;
    st->need = 0;
    st->n_reliable = 0;
    st->last_refresh = 0;
    st->accurate = st->accurate_start;
    st->improved = 0;
    st->rr_best = tot;
    st->rr_progress = tot;
    st->progress_iter = 0;
    st->status = 0;
    st->done = 0;
    if (!isfinite(tot) || !isfinite(st->bb)) {
      st->status = 4;
      st->done = 1;
    } else if (tot <= st->tol2) {
      st->status = 1;
      st->done = 1;
    }
  }
}

// pq = p . q ; alpha = rr / pq
__global__ void __launch_bounds__(kBlock) k_cg_alpha(const double* __restrict__ p,
                                                     const double* __restrict__ q, int64_t n,
                                                     double* __restrict__ red, unsigned* ticket,
                                                     CgState* st) {
  if (st->done) return;
  const double2* p2 = reinterpret_cast<const double2*>(p);
  const double2* q2 = reinterpret_cast<const double2*>(q);
  double acc = 0.0;
  for (int64_t i = gtid(); i < (n >> 1); i += gstride()) {
    const double2 u = p2[i], v = q2[i];
    acc = fma(u.x, v.x, acc);
    acc = fma(u.y, v.y, acc);
  }
  if ((n & 1) && gtid() == 0) acc = fma(p[n - 1], q[n - 1], acc);
  double tot;
  if (finish_sum(acc, red, ticket, &tot)) {
    st->pq = tot;
    st->improved = 0;
    if (!isfinite(tot)) {
      st->status = 4;
      st->done = 1;
    } else if (!(tot > 0.0)) {
      st->status = 3;  // breakdown: the direction carries no curvature
      st->done = 1;
    } else {
      st->alpha = (st->precond ? st->rz : st->rr) / tot;
      if (!isfinite(st->alpha)) {
        st->status = 4;
        st->done = 1;
      }
    }
  }
}

// x += alpha p ; r -= alpha q ; rr_new = r.r ; convergence / reliable-update test
__global__ void __launch_bounds__(kBlock) k_cg_update(double* __restrict__ x,
                                                      double* __restrict__ r,
                                                      const double* __restrict__ p,
                                                      const double* __restrict__ q, int64_t n,
                                                      double* __restrict__ red, unsigned* ticket,
                                                      CgState* st) {
  if (st->done) return;
  const double alpha = st->alpha;
  double2* x2 = reinterpret_cast<double2*>(x);
  double2* r2 = reinterpret_cast<double2*>(r);
  const double2* p2 = reinterpret_cast<const double2*>(p);
  const double2* q2 = reinterpret_cast<const double2*>(q);
  double acc = 0.0;
  for (int64_t i = gtid(); i < (n >> 1); i += gstride()) {
    double2 xv = x2[i], rv = r2[i];
    const double2 pv = p2[i], qv = q2[i];
    xv.x = fma(alpha, pv.x, xv.x);
    xv.y = fma(alpha, pv.y, xv.y);
    rv.x = fma(-alpha, qv.x, rv.x);
    rv.y = fma(-alpha, qv.y, rv.y);
    x2[i] = xv;
    r2[i] = rv;
    acc = fma(rv.x, rv.x, acc);
    acc = fma(rv.y, rv.y, acc);
  }
  if ((n & 1) && gtid() == 0) {
    x[n - 1] = fma(alpha, p[n - 1], x[n - 1]);
    const double ri = fma(-alpha, q[n - 1], r[n - 1]);
    r[n - 1] = ri;
    acc = fma(ri, ri, acc);
  }
  double tot;
  if (finish_sum(acc, red, ticket, &tot)) {
    st->rr_old = st->rr;
    st->rr = tot;
    st->iter += 1;
    if (!isfinite(tot)) {
      st->status = 4;
      st->done = 1;
      return;
    }
    const bool conv = tot <= st->tol2;
    if (st->mixed) {
      // refresh when the recursive residual has dropped enough, claims convergence,
      // has gone refresh_max iterations without a refresh (a float32 operator can
      // stall it), or the iteration budget is spent
      if (conv || tot < st->delta2 * st->rr_anchor || st->iter >= st->max_iter ||
          st->iter - st->last_refresh >= st->refresh_max)
        st->need = 1;
    } else {
      st->rr_true = tot;
      track_progress(st, tot);
      if (conv) {
        st->status = CG_CONVERGED;
        st->done = 1;
      } else if (st->iter >= st->max_iter) {
        st->status = CG_MAX_ITER;
        st->done = 1;
      } else if (stalled(st)) {
        st->status = CG_STALLED;
        st->done = 1;
      }
    }
  }
}

// Reliable update: r = b - t (t = A x in float64); clears t.
__global__ void __launch_bounds__(kBlock) k_cg_reliable(double* __restrict__ r,
                                                        const double* __restrict__ b,
                                                        double* __restrict__ t, int64_t n,
                                                        double* __restrict__ red, unsigned* ticket,
                                                        CgState* st) {
  if (st->done || !st->need) return;
  double2* r2 = reinterpret_cast<double2*>(r);
  double2* t2 = reinterpret_cast<double2*>(t);
  const double2* b2 = reinterpret_cast<const double2*>(b);
  double acc = 0.0;
  for (int64_t i = gtid(); i < (n >> 1); i += gstride()) {
    const double2 bv = b2[i], tv = t2[i];
    const double2 rv = make_double2(bv.x - tv.x, bv.y - tv.y);
    r2[i] = rv;
    t2[i] = make_double2(0.0, 0.0);
    acc = fma(rv.x, rv.x, acc);
    acc = fma(rv.y, rv.y, acc);
  }
  if ((n & 1) && gtid() == 0) {
    const double ri = b[n - 1] - t[n - 1];
    r[n - 1] = ri;
    t[n - 1] = 0.0;
    acc = fma(ri, ri, acc);
  }
  double tot;
  if (finish_sum(acc, red, ticket, &tot)) {
    after_refresh(st, tot);
  }
}

// x_best = x after a float64 residual that improved on every earlier one
__global__ void __launch_bounds__(kBlock) k_cg_keep_best(const double* __restrict__ x,
                                                         double* __restrict__ x_best, int64_t n,
                                                         const CgState* st) {
  if (!st->improved) return;
  const double2* a2 = reinterpret_cast<const double2*>(x);
  double2* b2 = reinterpret_cast<double2*>(x_best);
  for (int64_t i = gtid(); i < (n >> 1); i += gstride()) b2[i] = a2[i];
  if ((n & 1) && gtid() == 0) x_best[n - 1] = x[n - 1];
}

// p = r + beta p ; q = 0
__global__ void __launch_bounds__(kBlock) k_cg_direction(double* __restrict__ p,
                                                         const double* __restrict__ r,
                                                         double* __restrict__ q, int64_t n,
                                                         const CgState* st) {
  if (st->done) return;
  const double beta = st->rr / st->rr_old;
  double2* p2 = reinterpret_cast<double2*>(p);
  double2* q2 = reinterpret_cast<double2*>(q);
  const double2* r2 = reinterpret_cast<const double2*>(r);
  for (int64_t i = gtid(); i < (n >> 1); i += gstride()) {
    const double2 rv = r2[i];
    double2 pv = p2[i];
    pv.x = fma(beta, pv.x, rv.x);
    pv.y = fma(beta, pv.y, rv.y);
    p2[i] = pv;
    q2[i] = make_double2(0.0, 0.0);
  }
  if ((n & 1) && gtid() == 0) {
    p[n - 1] = fma(beta, p[n - 1], r[n - 1]);
    q[n - 1] = 0.0;
  }
}

// ---- preconditioned directions (precond.cu builds the coarse space) ----------------
// z = D^-1 r (+ R E^+ R^T r), rz = r . z, p = z + beta p.  D^-1 is the float32
// reciprocal of the valid samples of the unknown's baseline (0 without any), the
// same in every kernel.  The coarse part runs in float32 (R is stored in float32;
// the residual enters R^T r rounded to float32, the correction R c is summed in
// float32 and added to the float64 D^-1 r): GB300's float64 pipe is narrow, and
// the float64 work of these kernels is kept to the few operations that feed r . z.

__device__ __forceinline__ double pc_dinv(int nv) {
  return nv > 0 ? f64_of_f32(__frcp_rn((float)nv)) : 0.0;
}

// Sums of the NC values over each segment of lanes with equal consecutive keys,
// left in the segment's first lane (keys need not be sorted: a key that comes
// back later in the warp starts a new segment).
template <int NC>
__device__ __forceinline__ void seg_sum_to_head(int key, float (&val)[NC]) {
  const unsigned full = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  const int next = __shfl_down_sync(full, key, 1);
  bool stop = lane == 31 || next != key;  // the segment ends within [lane, lane + w)
#pragma unroll
  for (int w = 1; w < 32; w <<= 1) {
    const bool s2 = __shfl_down_sync(full, stop, w);
#pragma unroll
    for (int c = 0; c < NC; ++c) {
      const float v2 = __shfl_down_sync(full, val[c], w);
      if (!stop) val[c] += v2;
    }
    if (!stop) stop = s2;
  }
}

// u += R^T r (float32 sums per block in shared memory, where the warps' segment
// heads add with native float atomics; one float64 flush per block) and
// r . D^-1 r; mode 1 (no coarse space): rz = r . D^-1 r.  One thread per
// baseline: its outputs' residuals meet the slot's moments in registers.  R and
// the residual enter in float32 already, so the block's float32 sums lose nothing
// the coarse correction keeps.
template <int KS>
__global__ void __launch_bounds__(kBlock) k_pc_restrict(const double* __restrict__ r,
                                                        const int32_t* __restrict__ nvalid,
                                                        const float4* __restrict__ slot,
                                                        int64_t n_b, KindsArg kk, int n,
                                                        double* __restrict__ u,
                                                        double* __restrict__ red, unsigned* ticket,
                                                        CgState* st) {
  if (st->done) return;
  using K = KSet<KS>;
  constexpr int NC = K::NC, NO = K::NO;
  const int n_o = K::n_o(kk);
  extern __shared__ float s_u[];
  for (int i = threadIdx.x; i < n; i += blockDim.x) s_u[i] = 0.f;
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  double acc = 0.0;
  for (int64_t bb = (int64_t)blockIdx.x * blockDim.x + threadIdx.x - lane; bb < n_b;
       bb += stride) {
    const int64_t b = bb + lane;
    const bool in = b < n_b;
    const double dinv = in ? pc_dinv(nvalid[b]) : 0.0;
    float rf[NO];
#pragma unroll
    for (int o = 0; o < NO; ++o) {
      const double ri = (in && o < n_o) ? r[(int64_t)o * n_b + b] : 0.0;
      acc = fma(ri * dinv, ri, acc);
      rf[o] = __double2float_rn(ri);
    }
    if (n > 0) {
#pragma unroll
      for (int s = 0; s < kPcSlots; ++s) {
        const float4 m = in ? slot[b * kPcSlots + s] : make_float4(__int_as_float(-1), 0.f, 0.f, 0.f);
        const int key = __float_as_int(m.x);
        float v[NC];
#pragma unroll
        for (int c = 0; c < NC; ++c) v[c] = 0.f;
#pragma unroll
        for (int o = 0; o < NO; ++o) {
          if (o >= n_o) continue;
          float w[NC];
          row_moments<NC>(K::kind(o, kk), m.y, m.z, m.w, w);
#pragma unroll
          for (int c = 0; c < NC; ++c) v[c] = fmaf(w[c], rf[o], v[c]);
        }
        seg_sum_to_head<NC>(key, v);
        const int kprev = __shfl_up_sync(0xffffffffu, key, 1);
        if (key >= 0 && (lane == 0 || kprev != key)) {
#pragma unroll
          for (int c = 0; c < NC; ++c) atomicAdd(s_u + key * NC + c, v[c]);
        }
      }
    }
  }
  __syncthreads();
  for (int j = threadIdx.x; j < n; j += blockDim.x)
    if (s_u[j] != 0.f) atomicAdd(u + j, f64_of_f32(s_u[j]));
  double tot;
  if (finish_sum(acc, red, ticket, &tot)) {
    if (n > 0) {
      st->rdr = tot;
    } else {
      st->rz_old = st->rz;
      st->rz = tot;
    }
  }
}

// c = E^+ u (one warp per row; also rounded to float32 for the direction kernel),
// rz = r . D^-1 r + u . c; the last block clears u.
__global__ void __launch_bounds__(kBlock) k_pc_coarse(const double* __restrict__ einv,
                                                      double* __restrict__ u,
                                                      float* __restrict__ c, int n,
                                                      double* __restrict__ red, unsigned* ticket,
                                                      CgState* st) {
  if (st->done) return;
  const unsigned full = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  double acc = 0.0;
  for (int64_t row = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); row < n;
       row += warps) {
    const double* e = einv + row * n;
    double s = 0.0;
    for (int j = lane; j < n; j += 32) s = fma(e[j], u[j], s);
    for (int d = 16; d > 0; d >>= 1) s += __shfl_xor_sync(full, s, d);
    if (lane == 0) {
      c[row] = __double2float_rn(s);
      acc = fma(s, u[row], acc);
    }
  }
  double tot;
  if (finish_sum_block(acc, red, ticket, &tot)) {
    if (threadIdx.x == 0) {
      st->rz_old = st->rz;
      st->rz = st->rdr + tot;
    }
    for (int j = threadIdx.x; j < n; j += blockDim.x) u[j] = 0.0;
  }
}

// p = D^-1 r + R c + beta p (beta = 0 at the start); q = 0.  One thread per
// baseline and all its outputs.
template <int KS>
__global__ void __launch_bounds__(kBlock) k_pc_direction(double* __restrict__ p,
                                                         const double* __restrict__ r,
                                                         double* __restrict__ q,
                                                         const int32_t* __restrict__ nvalid,
                                                         const float4* __restrict__ slot,
                                                         const float* __restrict__ c,
                                                         int64_t n_b, KindsArg kk, int n,
                                                         const CgState* st) {
  if (st->done) return;
  using K = KSet<KS>;
  constexpr int NC = K::NC, NO = K::NO;
  const int n_o = K::n_o(kk);
  const double beta = st->iter == 0 ? 0.0 : st->rz / st->rz_old;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; b < n_b; b += stride) {
    const double dinv = pc_dinv(nvalid[b]);
    float4 m[kPcSlots];
    float cv[kPcSlots][NC];
#pragma unroll
    for (int s = 0; s < kPcSlots; ++s) {
      m[s] = n > 0 ? slot[b * kPcSlots + s] : make_float4(__int_as_float(-1), 0.f, 0.f, 0.f);
      const int k = __float_as_int(m[s].x);
#pragma unroll
      for (int cc = 0; cc < NC; ++cc) cv[s][cc] = k >= 0 ? __ldg(c + k * NC + cc) : 0.f;
    }
#pragma unroll
    for (int o = 0; o < NO; ++o) {
      if (o >= n_o) continue;
      const int64_t i = (int64_t)o * n_b + b;
      double z = dinv * r[i];
      if (n > 0) {
        float zc = 0.f;
#pragma unroll
        for (int s = 0; s < kPcSlots; ++s) {
          float w[NC];
          row_moments<NC>(K::kind(o, kk), m[s].y, m[s].z, m[s].w, w);
#pragma unroll
          for (int cc = 0; cc < NC; ++cc) zc = fmaf(w[cc], cv[s][cc], zc);
        }
        z += f64_of_f32(zc);
      }
      p[i] = fma(beta, p[i], z);
      q[i] = 0.0;
    }
  }
}

// Gauge: mean over (I-carrying outputs, baselines with data) -> scal[0..1]
__global__ void __launch_bounds__(kBlock) k_gauge_sum(const double* __restrict__ a,
                                                      const int32_t* __restrict__ nvalid,
                                                      int64_t n_b, KindsArg kk,
                                                      double* __restrict__ red, unsigned* ticket,
                                                      double* __restrict__ out) {
  double s = 0.0, c = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n_b;
       i += (int64_t)gridDim.x * blockDim.x) {
    if (nvalid[i] > 0) {
      for (int o = 0; o < kk.n_o; ++o)
        if (kk.kind[o] == DS_KIND_I || kk.kind[o] == DS_KIND_IQU) {
          s += a[o * n_b + i];
          c += 1.0;
        }
    }
  }
  double tot;
  if (finish_sum(s, red, ticket, &tot)) out[0] = tot;
  __syncthreads();
  if (finish_sum(c, red + gridDim.x, ticket + 1, &tot)) out[1] = tot;
}

__global__ void __launch_bounds__(kBlock) k_gauge_apply(double* __restrict__ a,
                                                        const int32_t* __restrict__ nvalid,
                                                        int64_t n_b, KindsArg kk,
                                                        const double* __restrict__ sums) {
  const double mean = sums[1] > 0.0 ? sums[0] / sums[1] : 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n_b;
       i += (int64_t)gridDim.x * blockDim.x) {
    const bool has = nvalid[i] > 0;
    for (int o = 0; o < kk.n_o; ++o) {
      double v = a[o * n_b + i];
      if (!has) v = 0.0;
      else if (kk.kind[o] == DS_KIND_I || kk.kind[o] == DS_KIND_IQU) v -= mean;
      a[o * n_b + i] = v;
    }
  }
}

__global__ void k_set_state(CgState* st, double tol, int max_iter, int mixed, double delta,
                            int refresh_max, double drift2, int accurate_start,
                            int stall_iters, int precond) {
  st->tol2 = tol * tol * st->bb;
  st->precond = precond;
  st->rz = 0.0;
  st->rz_old = 0.0;
  st->rdr = 0.0;
  st->stall_iters = stall_iters;
  st->drift2 = drift2;
  st->accurate_start = mixed ? accurate_start : 0;
  st->max_iter = max_iter;
  st->refresh_max = refresh_max;
  st->mixed = mixed;
  st->delta2 = delta * delta;
  st->done = 0;
  st->need = 0;
}

}  // namespace

static int vec_grid(const Plan& P, int64_t n) { return stream_grid(P, (n + 1) / 2, kBlock, 8); }

void enqueue_dot(const Plan& P, cudaStream_t st, const double* a, const double* b, int64_t n,
                 double* out) {
  k_dot<<<vec_grid(P, n), kBlock, 0, st>>>(a, b, n, P.red, P.counters, out, Gate{nullptr, nullptr});
}

void enqueue_gauge(const Plan& P, cudaStream_t st, double* a) {
  k_gauge_sum<<<vec_grid(P, P.n_b), kBlock, 0, st>>>(a, P.nvalid, P.n_b, P.kinds, P.red,
                                                      P.counters + 2, P.scal + 4);
  k_gauge_apply<<<vec_grid(P, P.n_b), kBlock, 0, st>>>(a, P.nvalid, P.n_b, P.kinds, P.scal + 4);
}

void enqueue_precond_direction(const Plan& P, cudaStream_t st) {
  const bool coarse = pc_ready(P);
  const int n = coarse ? P.pc_n : 0;
  const int vg = vec_grid(P, P.n_b);
  with_kindset(P.kindset, [&](auto ksc) {
    constexpr int KS = decltype(ksc)::value;
    k_pc_restrict<KS><<<vg, kBlock, sizeof(float) * n, st>>>(
        P.r, P.nvalid, P.pc_slot, P.n_b, P.kinds, n, P.pc_u, P.red, P.counters + 4, P.state);
    if (coarse)
      k_pc_coarse<<<stream_grid(P, (int64_t)n * 32, kBlock, 8), kBlock, 0, st>>>(
          P.pc_einv, P.pc_u, P.pc_c, n, P.red, P.counters + 5, P.state);
    k_pc_direction<KS><<<vg, kBlock, 0, st>>>(P.p, P.r, P.q, P.nvalid, P.pc_slot, P.pc_c, P.n_b,
                                             P.kinds, n, P.state);
  });
}

// Shared memory of the restriction kernel for n coarse columns (above 48 KB it
// needs the opt-in); false when n columns do not fit a block.
bool pc_restrict_fits(const Plan& P, int n) {
  const size_t bytes = sizeof(float) * (size_t)n;
  if (bytes > kPcRestrictSmemMax) return false;
  bool ok = true;
  with_kindset(P.kindset, [&](auto ksc) {
    constexpr int KS = decltype(ksc)::value;
    if (cudaFuncSetAttribute(k_pc_restrict<KS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)(bytes > 0 ? bytes : 1)) != cudaSuccess)
      ok = false;
  });
  return ok;
}

// accurate: the iteration applies the operator in the accurate arithmetic
int kernels_per_iteration(const Plan& P, bool accurate) {
  const int pc = pc_mode(P);  // extra kernels of the direction
  if (P.desc.precision != DS_PREC_MIXED) return 6 + pc;
  const bool df = P.accurate_df && P.maplo != nullptr;  // + the baseline split kernel
  const bool f32 = P.x32 != nullptr && !accurate && P.layout != 1;
  // pixel-major binning packs the baselines per baseline first (one kernel per bin)
  const bool pm = P.layout == 2 && pm_ready(P);
  const int packs = (pm && P.n_o > 1) ? (df ? 1 : 0) + (accurate ? (df ? 1 : 0) : (f32 ? 1 : 0)) : 0;
  return 11 + (df ? 1 : 0) + (df && accurate ? 1 : 0) + (f32 ? 1 : 0) + packs + pc;
}

// One CG iteration (gated by state->done), used both directly and under capture.
// accurate: apply the operator in the accurate arithmetic (a mixed problem that
// the float32 operator could not follow).  ev (optional): 5 events; the first
// four bracket the operator kernels, the fifth marks the end of the iteration.
void enqueue_iteration(const Plan& P, cudaStream_t st, cudaEvent_t* ev, bool accurate) {
  const bool mixed = P.desc.precision == DS_PREC_MIXED;
  const int vg = vec_grid(P, P.n_u);
  if (mixed) {
    Gate g{&P.state->done, nullptr};
    enqueue_apply(P, st, accurate, P.p, P.q, g, ev);
  } else {
    Gate g{&P.state->done, nullptr};
    enqueue_apply(P, st, true, P.p, P.q, g, ev);
  }
  k_cg_alpha<<<vg, kBlock, 0, st>>>(P.p, P.q, P.n_u, P.red, P.counters, P.state);
  k_cg_update<<<vg, kBlock, 0, st>>>(P.x, P.r, P.p, P.q, P.n_u, P.red, P.counters, P.state);
  if (mixed) {
    Gate gr{&P.state->done, &P.state->need};
    enqueue_apply(P, st, true, P.x, P.t, gr);
    k_cg_reliable<<<vg, kBlock, 0, st>>>(P.r, P.b, P.t, P.n_u, P.red, P.counters, P.state);
    k_cg_keep_best<<<vg, kBlock, 0, st>>>(P.x, P.x_best, P.n_u, P.state);
  }
  if (pc_mode(P))
    enqueue_precond_direction(P, st);
  else
    k_cg_direction<<<vg, kBlock, 0, st>>>(P.p, P.r, P.q, P.n_u, P.state);
  if (ev) cudaEventRecordWithFlags(ev[4], st, cudaEventRecordExternal);
}

void enqueue_cg_setup(const Plan& P, cudaStream_t st, double tol, int max_iter, double delta,
                      int warm, bool precond) {
  const bool mixed = P.desc.precision == DS_PREC_MIXED;
  // bb = b . b
  enqueue_dot(P, st, P.b, P.b, P.n_u, &P.state->bb);
  k_set_state<<<1, 1, 0, st>>>(P.state, tol, max_iter, mixed ? 1 : 0, delta, P.refresh_max,
                               P.drift_ratio, P.accurate_start, P.stall_iters,
                               precond && pc_mode(P) ? 1 : 0);
  if (warm) {
    cudaMemsetAsync(P.t, 0, sizeof(double) * P.n_u, st);
    enqueue_apply(P, st, true, P.x, P.t, Gate{nullptr, nullptr});
  }
  k_cg_start<<<vec_grid(P, P.n_u), kBlock, 0, st>>>(P.x, P.r, P.p, P.q, P.b, P.t, warm, P.n_u,
                                                     P.red, P.counters, P.state, P.x_best);
  if (precond && pc_mode(P)) enqueue_precond_direction(P, st);  // the first direction z_0
}

}  // namespace ds
