// Run-length form of the float32 operator.
//
// Within a baseline the expanded baselines F~ x are constant, so the samples of
// a run of consecutive samples on one pixel enter the binning only through
//   n = number of samples,  C = sum cos 2psi,  S = sum sin 2psi
// and every row of Sect. 3 is linear in (1, cos 2psi, sin 2psi):
//   I: n z   q: (C z, S z)   u: (-S z, C z)   iqu: (n z, C z, S z)
// and the same run contributes to the per-baseline sum of the rescan
//   n z_o - (row_o summed over the run) . m_p.
// At plan time (runs_build.cu) each run becomes one 16-byte record (pixel, n, C,
// S) plus its baseline index; the per-iteration passes here stream 20 bytes per
// run instead of 12 bytes per sample (an exact reformulation: only float32
// rounding order changes).  Runs are cut at baseline ends and at samples of
// weight 0.
#include "df.cuh"
#include "internal.cuh"
#include "rows.cuh"
#include "runs.cuh"
#include "stream_common.cuh"
#include "stream_df.cuh"

namespace ds {

namespace {

constexpr int kBlock = 256;

template <int KS>
__global__ void __launch_bounds__(kBlock) k_rl_bin(const RunRec* __restrict__ rec,
                                                   const int32_t* __restrict__ rb, int64_t n_runs,
                                                   const float* __restrict__ x,
                                                   float* __restrict__ bins, int64_t n_b,
                                                   KindsArg kk, Gate g) {
  if (gate_closed(g)) return;
  using K = KSet<KS>;
  constexpr int NC = K::NC, NO = K::NO;
  const int n_o = K::n_o(kk);
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n_runs; i += stride) {
    const RunRec r = load_run(rec, i);
    const int64_t b = __ldcs(rb + i);
    float acc[NC];
#pragma unroll
    for (int j = 0; j < NC; ++j) acc[j] = 0.f;
#pragma unroll
    for (int o = 0; o < NO; ++o)
      if (o < n_o) run_bin<NC>(K::kind(o, kk), r.n, r.c, r.s, __ldg(x + o * n_b + b), acc);
    flush_bins<NC, float>(bins, r.pix, acc);
  }
}

// out[o][b] += n x[o][b] - (run sums) . m over the runs of baseline b, in float32
// partial sums flushed to float64.  Each warp walks a chunk of `rounds` x 32
// consecutive runs, one per lane per round; a lane keeps the sum of its current
// baseline across rounds with the total count of its samples (whose term,
// count x x[o][b], joins the sum at the flush), and the warp flushes all lanes'
// sums together (a segmented sum over the lanes: shuffles, which share the
// load/store pipe with the map gathers) only when some lane's next run lies in
// another baseline or some lane runs out of runs, and at the chunk's end.
template <int KS>
__global__ void __launch_bounds__(kBlock) k_rl_rescan(const RunRec* __restrict__ rec,
                                                      const int32_t* __restrict__ rb,
                                                      int64_t n_runs, const float* __restrict__ x,
                                                      const float* __restrict__ map,
                                                      double* __restrict__ out, int64_t n_b,
                                                      KindsArg kk, int rounds, Gate g) {
  if (gate_closed(g)) return;
  using K = KSet<KS>;
  constexpr int NC = K::NC, NO = K::NO;
  const int n_o = K::n_o(kk);
  const unsigned full = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  const int64_t span = (int64_t)rounds * 32;
  const int64_t n_chunks = (n_runs + span - 1) / span;
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t ch = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); ch < n_chunks;
       ch += warps) {
    int key = -1;     // baseline of the lane's open sums (-1: none)
    float cnt = 0.f;  // samples in them
    float acc[NO];
#pragma unroll
    for (int o = 0; o < NO; ++o) acc[o] = 0.f;
    for (int k = 0; k < rounds; ++k) {
      const int64_t i = ch * span + (int64_t)k * 32 + lane;
      const bool active = i < n_runs;
      if (!__any_sync(full, active)) break;
      const int b = active ? __ldcs(rb + i) : -1;
      if (__any_sync(full, !active || (key >= 0 && b != key))) {
        if (key >= 0 && cnt != 0.f) {
#pragma unroll
          for (int o = 0; o < NO; ++o)
            if (o < n_o) acc[o] = fmaf(cnt, __ldg(x + o * n_b + key), acc[o]);
        }
        warp_segment_flush<NO, float>(key, acc, n_o, out, n_b);
        key = -1;
        cnt = 0.f;
#pragma unroll
        for (int o = 0; o < NO; ++o) acc[o] = 0.f;
      }
      if (!active) continue;
      key = b;
      const RunRec r = load_run(rec, i);
      float m[NC];
      load_map<NC, float>(map, r.pix, m);
      cnt += r.n;
#pragma unroll
      for (int o = 0; o < NO; ++o)
        if (o < n_o) acc[o] -= run_dot<NC>(K::kind(o, kk), r.n, r.c, r.s, m);
    }
    if (key >= 0 && cnt != 0.f) {
#pragma unroll
      for (int o = 0; o < NO; ++o)
        if (o < n_o) acc[o] = fmaf(cnt, __ldg(x + o * n_b + key), acc[o]);
    }
    warp_segment_flush<NO, float>(key, acc, n_o, out, n_b);
  }
}

// ---- accurate operator over runs (passes over baselines: F~ x, no timelines) ----
// Compensated sums throughout: the run sums C, S are exact double-float pairs,
// the baselines come split (xdf), the map as (map_hi, map_lo).

// acc -= (w_kind-run sums) . m
template <int NC>
__device__ __forceinline__ void run_sub_dot_ds(int kind, float n, df C, df S, const df (&m)[NC],
                                               dsum& acc) {
  using F = Frame<NC>;
  if (kind == DS_KIND_I) {
    if constexpr (F::I >= 0) ds_add_prod(acc, m[F::I], -n);
  } else if (kind == DS_KIND_Q) {
    if constexpr (F::Q >= 0) {
      ds_add_prod(acc, C, df_neg(m[F::Q]));
      ds_add_prod(acc, S, df_neg(m[F::U]));
    }
  } else if (kind == DS_KIND_U) {
    if constexpr (F::Q >= 0) {
      ds_add_prod(acc, C, df_neg(m[F::U]));
      ds_add_prod(acc, S, m[F::Q]);
    }
  } else {
    if constexpr (F::I >= 0 && F::Q >= 0) {
      ds_add_prod(acc, m[F::I], -n);
      ds_add_prod(acc, C, df_neg(m[F::Q]));
      ds_add_prod(acc, S, df_neg(m[F::U]));
    }
  }
}

template <int KS>
__global__ void __launch_bounds__(kBlock) k_rl_bin_df(const RunRec* __restrict__ rec,
                                                      const float4* __restrict__ rdf,
                                                      const int32_t* __restrict__ rb,
                                                      int64_t n_runs, const float2* __restrict__ x,
                                                      double* __restrict__ bins, int64_t n_b,
                                                      KindsArg kk, Gate g) {
  if (gate_closed(g)) return;
  using K = KSet<KS>;
  constexpr int NC = K::NC, NO = K::NO;
  const int n_o = K::n_o(kk);
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n_runs; i += stride) {
    const RunRec r = load_run(rec, i);
    const float4 cs = __ldcs(rdf + i);
    const df C{cs.x, cs.y}, S{cs.z, cs.w};
    const int64_t b = __ldcs(rb + i);
    dsum acc[NC];
#pragma unroll
    for (int j = 0; j < NC; ++j) acc[j] = ds_zero();
#pragma unroll
    for (int o = 0; o < NO; ++o)
      if (o < n_o) {
        const float2 z2 = __ldg(x + o * n_b + b);
        run_bin_ds<NC>(K::kind(o, kk), r.n, C, S, df{z2.x, z2.y}, acc);
      }
    flush_bins_ds<NC>(bins, r.pix, acc);
  }
}

// out[o][b] += n x[o][b] - (run sums) . m over the runs of baseline b.  Each warp
// walks a chunk of `rounds` x 32 consecutive runs, one per lane per round; a lane
// keeps the sums of its current baseline across rounds with the total count of
// their samples (whose term, count x x[o][b], joins the sums at the flush), and the
// warp flushes all lanes' sums together only when some lane's next run lies in
// another baseline or some lane runs out of runs, and at the chunk's end.
template <int KS>
__global__ void __launch_bounds__(kBlock) k_rl_rescan_df(const RunRec* __restrict__ rec,
                                                         const float4* __restrict__ rdf,
                                                         const int32_t* __restrict__ rb,
                                                         int64_t n_runs,
                                                         const float2* __restrict__ x,
                                                         const float* __restrict__ map_hi,
                                                         const float* __restrict__ map_lo,
                                                         double* __restrict__ out, int64_t n_b,
                                                         KindsArg kk, int rounds, Gate g) {
  if (gate_closed(g)) return;
  using K = KSet<KS>;
  constexpr int NC = K::NC, NO = K::NO;
  const int n_o = K::n_o(kk);
  const unsigned full = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  const int64_t span = (int64_t)rounds * 32;
  const int64_t n_chunks = (n_runs + span - 1) / span;
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t ch = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); ch < n_chunks;
       ch += warps) {
    int key = -1;     // baseline of the lane's open sums (-1: none)
    float cnt = 0.f;  // samples in them
    dsum acc[NO];
#pragma unroll
    for (int o = 0; o < NO; ++o) acc[o] = ds_zero();
    for (int k = 0; k < rounds; ++k) {
      const int64_t i = ch * span + (int64_t)k * 32 + lane;
      const bool active = i < n_runs;
      if (!__any_sync(full, active)) break;
      const int b = active ? __ldcs(rb + i) : -1;
      if (__any_sync(full, !active || (key >= 0 && b != key))) {
        if (key >= 0 && cnt != 0.f) {
#pragma unroll
          for (int o = 0; o < NO; ++o)
            if (o < n_o) ds_add_prod(acc[o], df_ldg(x, o * n_b + key), cnt);
        }
        warp_segment_flush_ds<NO>(key, acc, n_o, out, n_b);
        key = -1;
        cnt = 0.f;
#pragma unroll
        for (int o = 0; o < NO; ++o) acc[o] = ds_zero();
      }
      if (!active) continue;
      key = b;
      const RunRec r = load_run(rec, i);
      const float4 cs = __ldcs(rdf + i);
      const df C{cs.x, cs.y}, S{cs.z, cs.w};
      const float4 h = __ldg(reinterpret_cast<const float4*>(map_hi) + r.pix);
      const float4 l = __ldg(reinterpret_cast<const float4*>(map_lo) + r.pix);
      const float hh[4] = {h.x, h.y, h.z, h.w}, ll[4] = {l.x, l.y, l.z, l.w};
      df m[NC];
#pragma unroll
      for (int j = 0; j < NC; ++j) m[j] = df{hh[j], ll[j]};
      cnt += r.n;
#pragma unroll
      for (int o = 0; o < NO; ++o)
        if (o < n_o) {
          run_sub_dot_ds<NC>(K::kind(o, kk), r.n, C, S, m, acc[o]);
          ds_norm(acc[o]);
        }
    }
    if (key >= 0 && cnt != 0.f) {
#pragma unroll
      for (int o = 0; o < NO; ++o)
        if (o < n_o) ds_add_prod(acc[o], df_ldg(x, o * n_b + key), cnt);
    }
    warp_segment_flush_ds<NO>(key, acc, n_o, out, n_b);
  }
}

}  // namespace

bool rl_ready(const Plan& P) { return P.layout == 2 && P.rl_rec != nullptr && P.x32 != nullptr; }

void launch_bin_rl(const Plan& P, cudaStream_t st, Gate g) {
  if (pm_ready(P)) {
    launch_bin_pm(P, st, g);
    return;
  }
  const int grid = stream_grid(P, P.rl_n, kBlock, P.blocks_per_sm);
  with_kindset(P.kindset, [&](auto ksc) {
    constexpr int KS = decltype(ksc)::value;
    k_rl_bin<KS><<<grid, kBlock, 0, st>>>(P.rl_rec, P.rl_b, P.rl_n, P.x32, P.bins32, P.n_b,
                                          P.kinds, g);
  });
}

void launch_rescan_rl(const Plan& P, cudaStream_t st, double* out, Gate g) {
  const int grid = stream_grid(P, P.rl_n, kBlock, P.blocks_per_sm);
  const int rounds = rescan_rounds(P, P.rl_n, grid);
  with_kindset(P.kindset, [&](auto ksc) {
    constexpr int KS = decltype(ksc)::value;
    k_rl_rescan<KS><<<grid, kBlock, 0, st>>>(P.rl_rec, P.rl_b, P.rl_n, P.x32, P.map32, out,
                                             P.n_b, P.kinds, rounds, g);
  });
}

}  // namespace ds

namespace ds {

bool rl_df_ready(const Plan& P) { return P.layout == 2 && P.rl_df != nullptr && P.xdf != nullptr; }

// x must have been split into P.xdf (launch_split_df)
void launch_bin_rl_df(const Plan& P, cudaStream_t st, Gate g) {
  if (pm_ready(P)) {
    launch_bin_pm_df(P, st, g);
    return;
  }
  const int grid = stream_grid(P, P.rl_n, kBlock, P.blocks_per_sm);
  with_kindset(P.kindset, [&](auto ksc) {
    constexpr int KS = decltype(ksc)::value;
    k_rl_bin_df<KS><<<grid, kBlock, 0, st>>>(P.rl_rec, P.rl_df, P.rl_b, P.rl_n, P.xdf, P.bins,
                                             P.n_b, P.kinds, g);
  });
}

void launch_rescan_rl_df(const Plan& P, cudaStream_t st, double* out, Gate g) {
  const int grid = stream_grid(P, P.rl_n, kBlock, P.blocks_per_sm);
  const int rounds = rescan_rounds(P, P.rl_n, grid);
  with_kindset(P.kindset, [&](auto ksc) {
    constexpr int KS = decltype(ksc)::value;
    k_rl_rescan_df<KS><<<grid, kBlock, 0, st>>>(P.rl_rec, P.rl_df, P.rl_b, P.rl_n, P.xdf,
                                                P.map32, P.maplo, out, P.n_b, P.kinds, rounds, g);
  });
}

}  // namespace ds
