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

template <int KS>
__global__ void __launch_bounds__(kBlock) k_rl_rescan(const RunRec* __restrict__ rec,
                                                      const int32_t* __restrict__ rb,
                                                      int64_t n_runs, const float* __restrict__ x,
                                                      const float* __restrict__ map,
                                                      double* __restrict__ out, int64_t n_b,
                                                      KindsArg kk, Gate g) {
  if (gate_closed(g)) return;
  using K = KSet<KS>;
  constexpr int NC = K::NC, NO = K::NO;
  const int n_o = K::n_o(kk);
  const int lane = threadIdx.x & 31;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t ib = (int64_t)blockIdx.x * blockDim.x + threadIdx.x - lane; ib < n_runs;
       ib += stride) {
    const int64_t i = ib + lane;
    int key = -1;
    float acc[NO];
#pragma unroll
    for (int o = 0; o < NO; ++o) acc[o] = 0.f;
    if (i < n_runs) {
      const RunRec r = load_run(rec, i);
      const int b = __ldcs(rb + i);
      float m[NC];
      load_map<NC, float>(map, r.pix, m);
      key = b;
#pragma unroll
      for (int o = 0; o < NO; ++o)
        if (o < n_o) {
          const float z = __ldg(x + o * n_b + b);
          acc[o] = fmaf(r.n, z, -run_dot<NC>(K::kind(o, kk), r.n, r.c, r.s, m));
        }
    }
    warp_segment_flush<NO, float>(key, acc, n_o, out, n_b);
  }
}

// ---- accurate operator over runs (passes over baselines: F~ x, no timelines) ----
// Double-float throughout: the run sums C, S are exact double-float pairs, the
// baselines come split (xdf), the map as (map_hi, map_lo).

template <int NC>
__device__ __forceinline__ void run_bin_df(int kind, float n, df C, df S, df z, df (&acc)[NC]) {
  using F = Frame<NC>;
  if (kind == DS_KIND_I) {
    if constexpr (F::I >= 0) acc[F::I] = df_add(acc[F::I], df_mul_f(z, n));
  } else if (kind == DS_KIND_Q) {
    if constexpr (F::Q >= 0) {
      acc[F::Q] = df_add(acc[F::Q], df_mul(z, C));
      acc[F::U] = df_add(acc[F::U], df_mul(z, S));
    }
  } else if (kind == DS_KIND_U) {
    if constexpr (F::Q >= 0) {
      acc[F::Q] = df_sub(acc[F::Q], df_mul(z, S));
      acc[F::U] = df_add(acc[F::U], df_mul(z, C));
    }
  } else {
    if constexpr (F::I >= 0 && F::Q >= 0) {
      acc[F::I] = df_add(acc[F::I], df_mul_f(z, n));
      acc[F::Q] = df_add(acc[F::Q], df_mul(z, C));
      acc[F::U] = df_add(acc[F::U], df_mul(z, S));
    }
  }
}

template <int NC>
__device__ __forceinline__ df run_dot_df(int kind, float n, df C, df S, const df (&m)[NC]) {
  using F = Frame<NC>;
  if (kind == DS_KIND_I) {
    if constexpr (F::I >= 0) return df_mul_f(m[F::I], n);
  } else if (kind == DS_KIND_Q) {
    if constexpr (F::Q >= 0) return df_add(df_mul(C, m[F::Q]), df_mul(S, m[F::U]));
  } else if (kind == DS_KIND_U) {
    if constexpr (F::Q >= 0) return df_sub(df_mul(C, m[F::U]), df_mul(S, m[F::Q]));
  } else {
    if constexpr (F::I >= 0 && F::Q >= 0)
      return df_add(df_mul_f(m[F::I], n), df_add(df_mul(C, m[F::Q]), df_mul(S, m[F::U])));
  }
  return df{0.f, 0.f};
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
    df acc[NC];
#pragma unroll
    for (int j = 0; j < NC; ++j) acc[j] = df{0.f, 0.f};
#pragma unroll
    for (int o = 0; o < NO; ++o)
      if (o < n_o) {
        const float2 z2 = __ldg(x + o * n_b + b);
        run_bin_df<NC>(K::kind(o, kk), r.n, C, S, df{z2.x, z2.y}, acc);
      }
    flush_bins_df<NC>(bins, r.pix, acc);
  }
}

template <int KS>
__global__ void __launch_bounds__(kBlock) k_rl_rescan_df(const RunRec* __restrict__ rec,
                                                         const float4* __restrict__ rdf,
                                                         const int32_t* __restrict__ rb,
                                                         int64_t n_runs,
                                                         const float2* __restrict__ x,
                                                         const float* __restrict__ map_hi,
                                                         const float* __restrict__ map_lo,
                                                         double* __restrict__ out, int64_t n_b,
                                                         KindsArg kk, Gate g) {
  if (gate_closed(g)) return;
  using K = KSet<KS>;
  constexpr int NC = K::NC, NO = K::NO;
  const int n_o = K::n_o(kk);
  const int lane = threadIdx.x & 31;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t ib = (int64_t)blockIdx.x * blockDim.x + threadIdx.x - lane; ib < n_runs;
       ib += stride) {
    const int64_t i = ib + lane;
    int key = -1;
    df acc[NO];
#pragma unroll
    for (int o = 0; o < NO; ++o) acc[o] = df{0.f, 0.f};
    if (i < n_runs) {
      const RunRec r = load_run(rec, i);
      const float4 cs = __ldcs(rdf + i);
      const df C{cs.x, cs.y}, S{cs.z, cs.w};
      const int b = __ldcs(rb + i);
      const float4 h = __ldg(reinterpret_cast<const float4*>(map_hi) + r.pix);
      const float4 l = __ldg(reinterpret_cast<const float4*>(map_lo) + r.pix);
      const float hh[4] = {h.x, h.y, h.z, h.w}, ll[4] = {l.x, l.y, l.z, l.w};
      df m[NC];
#pragma unroll
      for (int j = 0; j < NC; ++j) m[j] = df{hh[j], ll[j]};
      key = b;
#pragma unroll
      for (int o = 0; o < NO; ++o)
        if (o < n_o) {
          const float2 z2 = __ldg(x + o * n_b + b);
          acc[o] = df_sub(df_mul_f(df{z2.x, z2.y}, r.n), run_dot_df<NC>(K::kind(o, kk), r.n, C, S, m));
        }
    }
    warp_segment_flush_df<NO>(key, acc, n_o, out, n_b);
  }
}

}  // namespace

bool rl_ready(const Plan& P) { return P.layout == 2 && P.rl_rec != nullptr && P.x32 != nullptr; }

void launch_bin_rl(const Plan& P, cudaStream_t st, Gate g) {
  const int grid = stream_grid(P, P.rl_n, kBlock, P.blocks_per_sm);
  with_kindset(P.kindset, [&](auto ksc) {
    constexpr int KS = decltype(ksc)::value;
    k_rl_bin<KS><<<grid, kBlock, 0, st>>>(P.rl_rec, P.rl_b, P.rl_n, P.x32, P.bins32, P.n_b,
                                          P.kinds, g);
  });
}

void launch_rescan_rl(const Plan& P, cudaStream_t st, double* out, Gate g) {
  const int grid = stream_grid(P, P.rl_n, kBlock, P.blocks_per_sm);
  with_kindset(P.kindset, [&](auto ksc) {
    constexpr int KS = decltype(ksc)::value;
    k_rl_rescan<KS><<<grid, kBlock, 0, st>>>(P.rl_rec, P.rl_b, P.rl_n, P.x32, P.map32, out,
                                             P.n_b, P.kinds, g);
  });
}

}  // namespace ds

namespace ds {

bool rl_df_ready(const Plan& P) { return P.layout == 2 && P.rl_df != nullptr && P.xdf != nullptr; }

// x must have been split into P.xdf (launch_split_df)
void launch_bin_rl_df(const Plan& P, cudaStream_t st, Gate g) {
  const int grid = stream_grid(P, P.rl_n, kBlock, P.blocks_per_sm);
  with_kindset(P.kindset, [&](auto ksc) {
    constexpr int KS = decltype(ksc)::value;
    k_rl_bin_df<KS><<<grid, kBlock, 0, st>>>(P.rl_rec, P.rl_df, P.rl_b, P.rl_n, P.xdf, P.bins,
                                             P.n_b, P.kinds, g);
  });
}

void launch_rescan_rl_df(const Plan& P, cudaStream_t st, double* out, Gate g) {
  const int grid = stream_grid(P, P.rl_n, kBlock, P.blocks_per_sm);
  with_kindset(P.kindset, [&](auto ksc) {
    constexpr int KS = decltype(ksc)::value;
    k_rl_rescan_df<KS><<<grid, kBlock, 0, st>>>(P.rl_rec, P.rl_df, P.rl_b, P.rl_n, P.xdf,
                                                P.map32, P.maplo, out, P.n_b, P.kinds, g);
  });
}

}  // namespace ds
