// Binning over the pixel-major copy of the run records (built by runs_build.cu):
// the pixel sums P^T V F~ x of the operator (Sect. 3) with one warp per pixel.
// The warp walks the pixel's runs (32 per round, each a 16-byte record), gathers
// the baselines of every output of the run's baseline with one 16-byte load
// (packed per baseline once per pass), sums the run contributions in registers
// and writes the pixel's sums with one plain store: no atomic update at all,
// where the time-ordered binning issues one vector reduction per run.  The
// accurate variant sums in compensated float32 (df.cuh) and stores float64.
// The pixel solve that follows reads the sums exactly as after the other forms.
#include "df.cuh"
#include "internal.cuh"
#include "rows.cuh"
#include "runs.cuh"

namespace ds {

namespace {

constexpr int kBlock = 256;

// x4[b] = (x[0][b], .., x[n_o - 1][b]) from the float32 baselines [n_o][n_b]
__global__ void __launch_bounds__(kBlock) k_pm_pack_x(const float* __restrict__ x32,
                                                      float4* __restrict__ x4, int64_t n_b,
                                                      int n_o, Gate g) {
  if (gate_closed(g)) return;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; b < n_b; b += stride) {
    float v[4] = {0.f, 0.f, 0.f, 0.f};
    for (int o = 0; o < n_o; ++o) v[o] = x32[o * n_b + b];
    x4[b] = make_float4(v[0], v[1], v[2], v[3]);
  }
}

// xd4[b] = hi parts, xd4[n_b + b] = lo parts of the split baselines [n_o][n_b]
__global__ void __launch_bounds__(kBlock) k_pm_pack_xdf(const float2* __restrict__ xdf,
                                                        float4* __restrict__ xd4, int64_t n_b,
                                                        int n_o, Gate g) {
  if (gate_closed(g)) return;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; b < n_b; b += stride) {
    float h[4] = {0.f, 0.f, 0.f, 0.f}, l[4] = {0.f, 0.f, 0.f, 0.f};
    for (int o = 0; o < n_o; ++o) {
      const float2 v = xdf[o * n_b + b];
      h[o] = v.x;
      l[o] = v.y;
    }
    xd4[b] = make_float4(h[0], h[1], h[2], h[3]);
    xd4[n_b + b] = make_float4(l[0], l[1], l[2], l[3]);
  }
}

__device__ __forceinline__ float f4_at(const float4& v, int i) {
  return i == 0 ? v.x : (i == 1 ? v.y : (i == 2 ? v.z : v.w));
}

// Baselines of run record r: all outputs' packed per baseline (x4), or, with one
// output, the float32 baselines themselves (4 bytes a gather instead of 16).
template <bool ONE>
__device__ __forceinline__ float4 pm_baselines(const void* __restrict__ xb, const float4& r) {
  const int b = __float_as_int(r.w);
  if constexpr (ONE) {
    return make_float4(__ldg(static_cast<const float*>(xb) + b), 0.f, 0.f, 0.f);
  } else {
    return __ldg(static_cast<const float4*>(xb) + b);
  }
}

// bins[p] = sum over the runs of p of (row sums) x[o][b], float32.  Each lane
// takes two runs per step with both loads issued first.
template <int KS, bool ONE>
__global__ void __launch_bounds__(kBlock) k_pm_bin(const uint32_t* __restrict__ off,
                                                   const float4* __restrict__ rec,
                                                   const void* __restrict__ xb,
                                                   float* __restrict__ bins, int64_t npix,
                                                   KindsArg kk, Gate g) {
  if (gate_closed(g)) return;
  using K = KSet<KS>;
  constexpr int NC = K::NC, NO = K::NO;
  const int n_o = K::n_o(kk);
  const unsigned full = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  const float4 zero = make_float4(0.f, 0.f, 0.f, 0.f);
  for (int64_t p = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); p < npix;
       p += warps) {
    const uint32_t beg = __ldg(off + p), end = __ldg(off + p + 1);
    float acc[NC];
#pragma unroll
    for (int j = 0; j < NC; ++j) acc[j] = 0.f;
    for (uint32_t i = beg + lane; i < end; i += 64) {
      const bool two = i + 32 < end;
      const float4 r0 = __ldcs(rec + i);
      const float4 r1 = two ? __ldcs(rec + i + 32) : zero;
      const float4 z0 = pm_baselines<ONE>(xb, r0);
      const float4 z1 = two ? pm_baselines<ONE>(xb, r1) : zero;
#pragma unroll
      for (int o = 0; o < NO; ++o)
        if (o < n_o) run_bin<NC>(K::kind(o, kk), r0.x, r0.y, r0.z, f4_at(z0, o), acc);
      if (two) {
#pragma unroll
        for (int o = 0; o < NO; ++o)
          if (o < n_o) run_bin<NC>(K::kind(o, kk), r1.x, r1.y, r1.z, f4_at(z1, o), acc);
      }
    }
#pragma unroll
    for (int d = 16; d > 0; d >>= 1)
#pragma unroll
      for (int j = 0; j < NC; ++j) acc[j] += __shfl_xor_sync(full, acc[j], d);
    if (lane == 0) {
      float v[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
      for (int j = 0; j < NC; ++j) v[j] = acc[j];
      reinterpret_cast<float4*>(bins)[p] = make_float4(v[0], v[1], v[2], v[3]);
    }
  }
}

// The accurate variant: double-float run sums (high parts from the record, low
// parts beside it) and baselines, compensated sums (renormalised every step),
// float64 pixel sums.  Baselines: hi parts xd4[b], lo parts xd4[n_b + b]; with one
// output (ONE), the split pairs xdf[b] themselves.
template <int KS, bool ONE>
__global__ void __launch_bounds__(kBlock) k_pm_bin_df(const uint32_t* __restrict__ off,
                                                      const float4* __restrict__ rec,
                                                      const float2* __restrict__ lo,
                                                      const float4* __restrict__ xd4,
                                                      const float2* __restrict__ xdf,
                                                      double* __restrict__ bins, int64_t npix,
                                                      int64_t n_b, KindsArg kk, Gate g) {
  if (gate_closed(g)) return;
  using K = KSet<KS>;
  constexpr int NC = K::NC, NO = K::NO;
  const int n_o = K::n_o(kk);
  const unsigned full = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t p = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); p < npix;
       p += warps) {
    const uint32_t beg = __ldg(off + p), end = __ldg(off + p + 1);
    dsum acc[NC];
#pragma unroll
    for (int j = 0; j < NC; ++j) acc[j] = ds_zero();
    for (uint32_t i = beg + lane; i < end; i += 32) {
      const float4 r = __ldcs(rec + i);
      const float2 l = __ldcs(lo + i);
      const int b = __float_as_int(r.w);
      float4 zh, zl;
      if constexpr (ONE) {
        const float2 z = __ldg(xdf + b);
        zh = make_float4(z.x, 0.f, 0.f, 0.f);
        zl = make_float4(z.y, 0.f, 0.f, 0.f);
      } else {
        zh = __ldg(xd4 + b);
        zl = __ldg(xd4 + n_b + b);
      }
#pragma unroll
      for (int o = 0; o < NO; ++o)
        if (o < n_o)
          run_bin_ds<NC>(K::kind(o, kk), r.x, df{r.y, l.x}, df{r.z, l.y},
                         df{f4_at(zh, o), f4_at(zl, o)}, acc);
#pragma unroll
      for (int j = 0; j < NC; ++j) ds_norm(acc[j]);
    }
#pragma unroll
    for (int d = 16; d > 0; d >>= 1)
#pragma unroll
      for (int j = 0; j < NC; ++j) {
        const df o2 = df{__shfl_xor_sync(full, acc[j].hi, d), __shfl_xor_sync(full, acc[j].lo, d)};
        ds_add(acc[j], o2);
      }
    if (lane == 0) {
      double v[4] = {0.0, 0.0, 0.0, 0.0};
#pragma unroll
      for (int j = 0; j < NC; ++j) v[j] = ds_to_double(acc[j]);
      double2* dst = reinterpret_cast<double2*>(bins) + 2 * p;
      dst[0] = make_double2(v[0], v[1]);
      dst[1] = make_double2(v[2], v[3]);
    }
  }
}

}  // namespace

bool pm_ready(const Plan& P) {
  return P.bin_order == 1 && P.pm_rec != nullptr && !P.pm_pending;
}

// P.x32 holds the float32 baselines of this pass (k_to_f32)
void launch_bin_pm(const Plan& P, cudaStream_t st, Gate g) {
  const bool one = P.n_o == 1;
  if (!one)
    k_pm_pack_x<<<stream_grid(P, P.n_b, kBlock, 8), kBlock, 0, st>>>(P.x32, P.x4, P.n_b, P.n_o, g);
  const int grid = stream_grid(P, P.npix * 32, kBlock, P.blocks_per_sm);
  with_kindset(P.kindset, [&](auto ksc) {
    constexpr int KS = decltype(ksc)::value;
    if (one)
      k_pm_bin<KS, true><<<grid, kBlock, 0, st>>>(P.pm_off, P.pm_rec, P.x32, P.bins32, P.npix,
                                                  P.kinds, g);
    else
      k_pm_bin<KS, false><<<grid, kBlock, 0, st>>>(P.pm_off, P.pm_rec, P.x4, P.bins32, P.npix,
                                                   P.kinds, g);
  });
}

// P.xdf holds the split baselines of this pass (launch_split_df)
void launch_bin_pm_df(const Plan& P, cudaStream_t st, Gate g) {
  const bool one = P.n_o == 1;
  if (!one)
    k_pm_pack_xdf<<<stream_grid(P, P.n_b, kBlock, 8), kBlock, 0, st>>>(P.xdf, P.xd4, P.n_b,
                                                                       P.n_o, g);
  const int grid = stream_grid(P, P.npix * 32, kBlock, P.blocks_per_sm);
  with_kindset(P.kindset, [&](auto ksc) {
    constexpr int KS = decltype(ksc)::value;
    if (one)
      k_pm_bin_df<KS, true><<<grid, kBlock, 0, st>>>(P.pm_off, P.pm_rec, P.pm_lo, P.xd4, P.xdf,
                                                     P.bins, P.npix, P.n_b, P.kinds, g);
    else
      k_pm_bin_df<KS, false><<<grid, kBlock, 0, st>>>(P.pm_off, P.pm_rec, P.pm_lo, P.xd4, P.xdf,
                                                      P.bins, P.npix, P.n_b, P.kinds, g);
  });
}

}  // namespace ds
