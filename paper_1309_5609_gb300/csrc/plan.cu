// Plan construction: hits h = P^T P, per-pixel normal matrices M_p, their
// inverses and the rcond cut, and the per-sample weights that every later pass
// uses (Sect. 3: hitmap, Eqs. mapQ/mapU and the QU / IQU weighting).
#include <cmath>
#include <cstring>
#include <type_traits>

#include "df.cuh"
#include "internal.cuh"
#include "pixmat.cuh"
#include "rows.cuh"

namespace ds {

namespace {

constexpr int kBlock = 256;

// 4-sample groups per thread in k_plan_accum_df: longer stretches per thread end
// fewer runs of equal pixels early (each run end: one float64 atomic add per
// nonzero matrix entry, the pass's bound).
constexpr int kAccumGroups = 4;

// Packed index of the upper triangle of a symmetric NC x NC matrix.
template <int NC>
__device__ __forceinline__ constexpr int sym_index(int i, int j) {
  if (i > j) { int t = i; i = j; j = t; }
  return i * NC - i * (i - 1) / 2 + (j - i);
}

// Entries that are exactly zero (structurally, e.g. I x Q for separate I and q
// outputs, or the q+u cross term c s - s c) cost no atomic.
template <int NC>
__device__ __forceinline__ void flush_m(int32_t* __restrict__ hits, double* __restrict__ mm, int p,
                                        int h, const double (&acc)[NC * (NC + 1) / 2]) {
  constexpr int NM = NC * (NC + 1) / 2;
  atomicAdd(hits + p, h);
#pragma unroll
  for (int j = 0; j < NM; ++j)
    if (acc[j] != 0.0) atomicAdd(mm + (int64_t)p * NM + j, acc[j]);
}

template <int NC>
__device__ __forceinline__ void flush_m_ds(int32_t* __restrict__ hits, double* __restrict__ mm,
                                           int p, int h, const dsum (&acc)[NC * (NC + 1) / 2]) {
  constexpr int NM = NC * (NC + 1) / 2;
  atomicAdd(hits + p, h);
#pragma unroll
  for (int j = 0; j < NM; ++j)
    if (ds_nonzero(acc[j])) atomicAdd(mm + (int64_t)p * NM + j, ds_to_double(acc[j]));
}

// Same as k_plan_accum with the run sums of w w^T as compensated float32 sums:
// the entries are products of float32 numbers, exact as (product, error) pairs,
// so float64 is only needed for the atomic adds.  Used by mixed-precision plans.
template <int KS>
__global__ void __launch_bounds__(256) k_plan_accum_df(const int32_t* __restrict__ pix,
                                                       const float* __restrict__ cc,
                                                       const float* __restrict__ ss,
                                                       const uint8_t* __restrict__ valid,
                                                       int32_t* __restrict__ hits,
                                                       double* __restrict__ mm, int64_t n_t,
                                                       int64_t npix, KindsArg kk,
                                                       int32_t* __restrict__ err) {
  using K = KSet<KS>;
  constexpr int NC = K::NC, NO = K::NO, NM = NC * (NC + 1) / 2;
  const int n_o = K::n_o(kk);
  const int64_t nvec = (n_t + 3) >> 2;
  const int64_t n_units = (nvec + kAccumGroups - 1) / kAccumGroups;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  // cos / sin are 16-byte aligned (checked when the plan is made); the pixels may not be
  const bool pix4 = (reinterpret_cast<uintptr_t>(pix) & 15) == 0;
  for (int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; u < n_units; u += stride) {
    dsum acc[NM];
#pragma unroll
    for (int j = 0; j < NM; ++j) acc[j] = ds_zero();
    int cur = -1, h = 0;
    for (int gi = 0; gi < kAccumGroups; ++gi) {
      const int64_t v = u * kAccumGroups + gi;
      if (v >= nvec) break;
      const int64_t t0 = v << 2;
      int p[4];
      float c[4], s[4];
      if (t0 + 4 <= n_t) {
        if (pix4) {
          const int4 pp = __ldcs(reinterpret_cast<const int4*>(pix) + v);
          p[0] = pp.x; p[1] = pp.y; p[2] = pp.z; p[3] = pp.w;
        } else {
#pragma unroll
          for (int k = 0; k < 4; ++k) p[k] = pix[t0 + k];
        }
        const float4 c4 = __ldcs(reinterpret_cast<const float4*>(cc) + v);
        const float4 s4 = __ldcs(reinterpret_cast<const float4*>(ss) + v);
        c[0] = c4.x; c[1] = c4.y; c[2] = c4.z; c[3] = c4.w;
        s[0] = s4.x; s[1] = s4.y; s[2] = s4.z; s[3] = s4.w;
      } else {
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          const bool in = t0 + k < n_t;
          p[k] = in ? pix[t0 + k] : -1;
          c[k] = in ? cc[t0 + k] : 0.f;
          s[k] = in ? ss[t0 + k] : 0.f;
        }
      }
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const int64_t t = t0 + k;
        if (t >= n_t) break;
        if (valid != nullptr && valid[t] == 0) continue;
        if (p[k] < 0 || p[k] >= npix) {
          atomicOr(err, ERR_PIX);
          continue;
        }
        if (p[k] != cur) {
          if (cur >= 0) flush_m_ds<NC>(hits, mm, cur, h, acc);
          cur = p[k];
          h = 0;
#pragma unroll
          for (int j = 0; j < NM; ++j) acc[j] = ds_zero();
        }
        h += 1;
#pragma unroll
        for (int o = 0; o < NO; ++o) {
          if (o < n_o) {
            float row[NC];
#pragma unroll
            for (int j = 0; j < NC; ++j) row[j] = 0.f;
            row_bin<NC, float>(K::kind(o, kk), c[k], s[k], 1.0f, row);
#pragma unroll
            for (int i = 0; i < NC; ++i)
#pragma unroll
              for (int j = i; j < NC; ++j) {
                if (row[i] != 0.f && row[j] != 0.f) ds_add_prod(acc[sym_index<NC>(i, j)], row[i], row[j]);
              }
          }
        }
      }
#pragma unroll
      for (int j = 0; j < NM; ++j) ds_norm(acc[j]);
    }
    if (cur >= 0) flush_m_ds<NC>(hits, mm, cur, h, acc);
  }
}

// hits[p] += 1 and M_p += sum_o w_o w_o^T for every valid sample (float64).
template <int KS>
__global__ void __launch_bounds__(kBlock) k_plan_accum(const int32_t* __restrict__ pix,
                                                       const float* __restrict__ cc,
                                                       const float* __restrict__ ss,
                                                       const uint8_t* __restrict__ valid,
                                                       int32_t* __restrict__ hits,
                                                       double* __restrict__ mm, int64_t n_t,
                                                       int64_t npix, KindsArg kk,
                                                       int32_t* __restrict__ err) {
  using K = KSet<KS>;
  constexpr int NC = K::NC, NO = K::NO, NM = NC * (NC + 1) / 2;
  const int n_o = K::n_o(kk);
  const int64_t nvec = (n_t + 3) >> 2;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < nvec; v += stride) {
    const int64_t t0 = v << 2;
    double acc[NM];
#pragma unroll
    for (int j = 0; j < NM; ++j) acc[j] = 0.0;
    int cur = -1, h = 0;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const int64_t t = t0 + k;
      if (t >= n_t) break;
      if (valid != nullptr && valid[t] == 0) continue;
      const int p = pix[t];
      if (p < 0 || p >= npix) {
        atomicOr(err, ERR_PIX);
        continue;
      }
      const double c = cc[t], s = ss[t];
      double w[NM];
#pragma unroll
      for (int j = 0; j < NM; ++j) w[j] = 0.0;
#pragma unroll
      for (int o = 0; o < NO; ++o) {
        if (o < n_o) {
          double row[NC];
#pragma unroll
          for (int j = 0; j < NC; ++j) row[j] = 0.0;
          row_bin<NC, double>(K::kind(o, kk), c, s, 1.0, row);
#pragma unroll
          for (int i = 0; i < NC; ++i)
#pragma unroll
            for (int j = i; j < NC; ++j) w[sym_index<NC>(i, j)] += row[i] * row[j];
        }
      }
      if (p != cur) {
        if (cur >= 0) flush_m<NC>(hits, mm, cur, h, acc);
        cur = p;
        h = 1;
#pragma unroll
        for (int j = 0; j < NM; ++j) acc[j] = w[j];
      } else {
        h += 1;
#pragma unroll
        for (int j = 0; j < NM; ++j) acc[j] += w[j];
      }
    }
    if (cur >= 0) flush_m<NC>(hits, mm, cur, h, acc);
  }
}

// Per pixel: rcond cut and M_p^-1 (in place over M), mask, good-pixel count.
template <int NC>
__global__ void __launch_bounds__(kBlock) k_pixel_invert(double* __restrict__ mm,
                                                         const int32_t* __restrict__ hits,
                                                         uint8_t* __restrict__ mask,
                                                         int64_t npix, double rcond_min,
                                                         unsigned long long* __restrict__ n_good) {
  constexpr int NM = NC * (NC + 1) / 2;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  unsigned long long good = 0;
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < npix; p += stride) {
    double a[NM], inv[NM];
#pragma unroll
    for (int j = 0; j < NM; ++j) a[j] = mm[p * NM + j];
    bool keep = false;
    if (hits[p] > 0) {
      const double rc = rcond_of<NC>(a);
      keep = rc >= rcond_min;
    }
    if (keep) {
      sym_inverse<NC>(a, inv);
      good += 1;
    } else {
#pragma unroll
      for (int j = 0; j < NM; ++j) inv[j] = 0.0;
    }
#pragma unroll
    for (int j = 0; j < NM; ++j) mm[p * NM + j] = inv[j];
    mask[p] = keep ? 1 : 0;
  }
  for (int d = 16; d > 0; d >>= 1) good += __shfl_down_sync(0xffffffffu, good, d);
  if ((threadIdx.x & 31) == 0 && good) atomicAdd(n_good, good);
}

// Effective pixel of each sample (-1 when flagged or on a cut pixel) and the
// number of weight-1 samples per baseline.
__global__ void __launch_bounds__(kBlock) k_plan_weights(const int32_t* __restrict__ pix_in,
                                                         const uint8_t* __restrict__ valid,
                                                         const uint8_t* __restrict__ mask,
                                                         int32_t* __restrict__ pix_out,
                                                         int32_t* __restrict__ nvalid,
                                                         int64_t n_t, int64_t npix, int64_t L,
                                                         unsigned long long* __restrict__ n_valid) {
  const unsigned full = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  const int64_t nvec = (n_t + 3) >> 2;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  unsigned long long total = 0;
  for (int64_t vb = (int64_t)blockIdx.x * blockDim.x + threadIdx.x - lane; vb < nvec;
       vb += stride) {
    const int64_t v = vb + lane;
    int key = -1, cnt = 0;
    if (v < nvec) {
      const int64_t t0 = v << 2;
      int64_t b = t0 / L, bend = (b + 1) * L;
      key = (int)b;
      for (int k = 0; k < 4; ++k) {
        const int64_t t = t0 + k;
        if (t >= n_t) break;
        if (t >= bend) {
          if (cnt) atomicAdd(nvalid + b, cnt);
          total += cnt;
          cnt = 0;
          b += 1;
          bend += L;
          key = (int)b;
        }
        const int p = pix_in[t];
        const bool ok = (valid == nullptr || valid[t] != 0) && p >= 0 && p < npix && mask[p];
        pix_out[t] = ok ? p : -1;
        cnt += ok ? 1 : 0;
      }
    }
    total += cnt;
    for (int d = 1; d < 32; d <<= 1) {
      const int k2 = __shfl_down_sync(full, key, d);
      const int c2 = __shfl_down_sync(full, cnt, d);
      if (lane + d < 32 && k2 == key) cnt += c2;
    }
    const int kp = __shfl_up_sync(full, key, 1);
    if (key >= 0 && (lane == 0 || kp != key) && cnt) atomicAdd(nvalid + key, cnt);
  }
  for (int d = 16; d > 0; d >>= 1) total += __shfl_down_sync(full, total, d);
  if (lane == 0 && total) atomicAdd(n_valid, total);
}

}  // namespace

void launch_plan_matrices(int kindset, bool df, int grid, cudaStream_t st, const int32_t* pix,
                          const float* c, const float* s, const uint8_t* valid, int32_t* hits,
                          double* mm, int64_t n_t, int64_t npix, KindsArg kk, int32_t* err) {
  with_kindset(kindset, [&](auto ksc) {
    constexpr int KS = decltype(ksc)::value;
    if (df)
      k_plan_accum_df<KS><<<grid, kBlock, 0, st>>>(pix, c, s, valid, hits, mm, n_t, npix, kk, err);
    else
      k_plan_accum<KS><<<grid, kBlock, 0, st>>>(pix, c, s, valid, hits, mm, n_t, npix, kk, err);
  });
}

void launch_pixel_invert(int n_c, int grid, cudaStream_t st, double* mm, const int32_t* hits,
                         uint8_t* mask, int64_t npix, double rcond_min,
                         unsigned long long* n_good) {
  if (n_c == 1)
    k_pixel_invert<1><<<grid, kBlock, 0, st>>>(mm, hits, mask, npix, rcond_min, n_good);
  else if (n_c == 2)
    k_pixel_invert<2><<<grid, kBlock, 0, st>>>(mm, hits, mask, npix, rcond_min, n_good);
  else
    k_pixel_invert<3><<<grid, kBlock, 0, st>>>(mm, hits, mask, npix, rcond_min, n_good);
}

ds_status plan_build(Plan& P, const int32_t* d_pix, const uint8_t* d_valid) {
  cudaStream_t st = P.stream;
  const int nm = P.nm;
  DS_CUDA_TRY(cudaMemsetAsync(P.hits, 0, sizeof(int32_t) * P.npix, st));
  DS_CUDA_TRY(cudaMemsetAsync(P.minv, 0, sizeof(double) * P.npix * nm, st));
  DS_CUDA_TRY(cudaMemsetAsync(P.nvalid, 0, sizeof(int32_t) * P.n_b, st));
  DS_CUDA_TRY(cudaMemsetAsync(P.err, 0, sizeof(int32_t), st));
  DS_CUDA_TRY(cudaMemsetAsync(P.scal, 0, sizeof(double) * 8, st));
  const int grid = stream_grid(P, (P.n_t + 3) / 4, kBlock, 8);
  launch_plan_matrices(P.kindset, P.desc.precision == DS_PREC_MIXED && P.accurate_df, grid, st,
                       d_pix, P.c, P.s, d_valid, P.hits, P.minv, P.n_t, P.npix, P.kinds, P.err);
  DS_CUDA_TRY(cudaGetLastError());
  // a sharded plan cuts on the hits and matrices of all ranks
  shard_exchange(P, st, P.hits, P.npix, DS_DT_I32);
  shard_exchange(P, st, P.minv, P.npix * nm, DS_DT_F64);
  if (P.shard_err) return DS_ECUDA;
  unsigned long long* counts = reinterpret_cast<unsigned long long*>(P.scal);
  const int pgrid = stream_grid(P, P.npix, kBlock, 8);
  launch_pixel_invert(P.n_c, pgrid, st, P.minv, P.hits, P.mask, P.npix, P.desc.rcond_min, counts);
  DS_CUDA_TRY(cudaGetLastError());
  k_plan_weights<<<grid, kBlock, 0, st>>>(d_pix, d_valid, P.mask, P.pix, P.nvalid, P.n_t, P.npix,
                                          P.L, counts + 1);
  DS_CUDA_TRY(cudaGetLastError());
  // mixed plans: count the run-length records of the float32 operator (counts + 2)
  const bool runs = P.desc.precision == DS_PREC_MIXED && P.x32 != nullptr;
  if (runs) {
    const ds_status s = rl_count(P, reinterpret_cast<int64_t*>(counts + 2));
    if (s != DS_OK) return s;
  }
  DS_CUDA_TRY(cudaMemcpyAsync(P.h_scal, P.scal, sizeof(double) * 3, cudaMemcpyDeviceToHost, st));
  DS_CUDA_TRY(cudaMemcpyAsync(P.h_err, P.err, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
  DS_CUDA_TRY(cudaStreamSynchronize(st));
  unsigned long long hc[3];
  std::memcpy(hc, P.h_scal, sizeof(hc));
  P.n_good = (int64_t)hc[0];
  P.n_valid = (int64_t)hc[1];
  if (*P.h_err & ERR_PIX) return DS_EPIX;
  // the records pay when runs are long enough; with short runs, long problems
  // (a tile of the binning or more) sort their runs by pixel within time tiles,
  // and the others keep the time-ordered passes
  if (runs) {
    const int64_t n_runs = (int64_t)hc[2];
    if ((double)n_runs <= kRunsPerSampleMax * (double)P.n_t) {
      const ds_status s = rl_fill(P, n_runs);
      if (s != DS_OK) return s;
      P.layout = 2;
    } else if (P.n_t >= P.tl_bin_samples && P.shard_allreduce == nullptr) {
      // built by the first single-problem solve or operator application (tl_ensure):
      // batched problems run their own kernels and never pay for it
      cudaFreeAsync(P.rl_tiles, st);
      P.rl_tiles = nullptr;
      P.layout = 3;
      P.tl_pending = 1;
    } else {
      cudaFreeAsync(P.rl_tiles, st);
      P.rl_tiles = nullptr;
    }
  }
  return DS_OK;
}

}  // namespace ds
