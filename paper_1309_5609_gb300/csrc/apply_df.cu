// Accurate passes of mixed-precision plans in compensated float32 arithmetic
// (df.cuh): the right-hand side F~^T Z y, the maps M^-1 A_p^T V (y - F~ a) and
// the float64 residual refreshes b - F~^T Z F~ x of the CG iteration (Sect. 3).
//
// Per sample everything is float32: cos 2psi, sin 2psi and float32 data are
// exact float32 numbers, so their products are exact as (product, error) pairs,
// and the sums are the compensated (hi, lo) sums of df.cuh.  float64 appears only
// once per run of equal pixels (the atomic add into the float64 pixel sums), once
// per flushed baseline sum, per baseline (splitting x) and per pixel (the pixel
// solve).  The binning pass takes 4 consecutive samples per thread; the rescan
// walks chunks of consecutive samples per warp.
#include <type_traits>

#include "df.cuh"
#include "internal.cuh"
#include "rows.cuh"
#include "stream_df.cuh"

namespace ds {

namespace {

constexpr int kBlock = 256;

// Resident blocks per SM requested for the double-float streaming passes: their
// register count limits occupancy.  3 caps them at 85 registers (from 80-100):
// measured 16% faster right-hand side on the B-Machine-like workload; 4 (64
// registers) spills and gains nothing more.
constexpr int kDfMinBlocks = 3;

// x[i] -> (hi, lo) with hi = x rounded to float32, lo = the rest rounded to float32
__global__ void __launch_bounds__(kBlock) k_split_df(const double* __restrict__ x,
                                                     float2* __restrict__ xs, int64_t n, Gate g) {
  if (gate_closed(g)) return;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const df d = df_from_double(x[i]);
    xs[i] = make_float2(d.hi, d.lo);
  }
}

// y[o][4v .. 4v + 3] of every output: one 16-byte load per output when the rows
// are 16-byte aligned (n_t a multiple of 4) and the 4 samples are in range
template <int NO>
__device__ __forceinline__ void load_y4(const float* __restrict__ y, int n_o, int64_t n_t,
                                        int64_t v, float (&yv)[NO][4]) {
  const int64_t t0 = v << 2;
  const bool vec = ((n_t & 3) == 0) && t0 + 4 <= n_t;
#pragma unroll
  for (int o = 0; o < NO; ++o) {
    if (o >= n_o) {
#pragma unroll
      for (int k = 0; k < 4; ++k) yv[o][k] = 0.f;
    } else if (vec) {
      const float4 q = __ldcs(reinterpret_cast<const float4*>(y + (int64_t)o * n_t) + v);
      yv[o][0] = q.x; yv[o][1] = q.y; yv[o][2] = q.z; yv[o][3] = q.w;
    } else {
#pragma unroll
      for (int k = 0; k < 4; ++k) yv[o][k] = t0 + k < n_t ? y[(int64_t)o * n_t + t0 + k] : 0.f;
    }
  }
}

// bins[p] += sum_o w_o(t) z_o(t), z = x[o][t/L] (ZY false) or y[o][t] - a[o][t/L] (ZY true);
// the baselines come split into double-float pairs (xs, NULL for none).  A lane
// takes 4 consecutive samples, a warp 128; each run of equal pixels is one
// compensated sum per component and ends in one float64 atomic add per component
// (the pass's bound).  A run that crosses from one lane's samples into the next
// lane's is handed on instead of flushed twice: each lane keeps its first and last
// run open, a segmented shuffle scan over the lanes carries every last run into
// the next lane while that lane's first run has the same pixel (through lanes
// whose samples are all on that pixel), and the lane where the run ends flushes it.
template <int KS, bool ZY>
__global__ void __launch_bounds__(kBlock, kDfMinBlocks) k_bin_df(const int32_t* __restrict__ pix,
                                                   const float* __restrict__ cc,
                                                   const float* __restrict__ ss,
                                                   const float2* __restrict__ x,
                                                   const float* __restrict__ y,
                                                   double* __restrict__ bins, int64_t n_t,
                                                   int64_t L, int64_t n_b, KindsArg kk, Gate g) {
  if (gate_closed(g)) return;
  using K = KSet<KS>;
  constexpr int NC = K::NC, NO = K::NO;
  const int n_o = K::n_o(kk);
  const bool hasx = x != nullptr;
  const unsigned full = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  const unsigned upto = lane == 31 ? full : (2u << lane) - 1u;
  const int64_t nvec = (n_t + 3) >> 2;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int64_t v0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  BaselineCursor bc(v0 << 2, stride << 2, L);
  for (int64_t vb = v0 - lane; vb < nvec; vb += stride, bc.advance(L)) {
    const int64_t v = vb + lane;
    int head_p = -1, cur = -1, nruns = 0;
    dsum head[NC], acc[NC];
#pragma unroll
    for (int j = 0; j < NC; ++j) head[j] = acc[j] = ds_zero();
    if (v < nvec) {
      int p[4];
      float c[4], s[4];
      load4_df(pix, cc, ss, v, n_t, p, c, s);
      float yv[NO][4];
      if constexpr (ZY) load_y4<NO>(y, n_o, n_t, v, yv);
      const int64_t t0 = v << 2;
      int64_t b = bc.b;
      int64_t bend = bc.next_start(t0, L);
      df zb[NO];
#pragma unroll
      for (int o = 0; o < NO; ++o)
        zb[o] = (o < n_o && hasx) ? df_ldg(x, o * n_b + b) : df{0.f, 0.f};
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const int64_t t = t0 + k;
        if (t >= n_t) break;
        if (t >= bend) {
          b += 1;
          bend += L;
#pragma unroll
          for (int o = 0; o < NO; ++o)
            zb[o] = (o < n_o && hasx) ? df_ldg(x, o * n_b + b) : df{0.f, 0.f};
        }
        if (p[k] < 0) continue;
        if (p[k] != cur) {
          if (cur >= 0) {
            if (nruns == 1) {  // the lane's first run stays open for the hand-off
              head_p = cur;
#pragma unroll
              for (int j = 0; j < NC; ++j) head[j] = acc[j];
            } else {
              flush_bins_ds<NC>(bins, cur, acc);
            }
          }
          cur = p[k];
          nruns += 1;
#pragma unroll
          for (int j = 0; j < NC; ++j) acc[j] = ds_zero();
        }
#pragma unroll
        for (int o = 0; o < NO; ++o) {
          if (o < n_o) {
            if constexpr (ZY) {
              if (hasx) {
                // z = y - a exactly as an unnormalised pair
                const df e = two_sum(yv[o][k], -zb[o].hi);
                row_bin_ds<NC>(K::kind(o, kk), c[k], s[k], df{e.hi, __fsub_rn(e.lo, zb[o].lo)}, acc);
              } else {
                row_bin_ds<NC>(K::kind(o, kk), c[k], s[k], yv[o][k], acc);
              }
            } else {
              row_bin_ds<NC>(K::kind(o, kk), c[k], s[k], zb[o], acc);
            }
          }
        }
      }
#pragma unroll
      for (int j = 0; j < NC; ++j) ds_norm(acc[j]);
    }
    // acc is the lane's last run (pixel cur); with a single run it is also the first
    const bool single = nruns == 1;
    if (single) head_p = cur;
    const int prev_tail = __shfl_up_sync(full, cur, 1);
    const bool link = lane > 0 && head_p >= 0 && head_p == prev_tail;  // takes the previous lane's run
    const bool through = single && link;
    // out = the last run's sums including what flows in through single-run lanes
    const unsigned starts = __ballot_sync(full, !through);  // lane 0 always starts a segment
    const int seg0 = 31 - __clz(starts & upto);
    const unsigned reach = __reduce_max_sync(full, (unsigned)(lane - seg0));
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      if ((unsigned)d > reach) break;
#pragma unroll
      for (int j = 0; j < NC; ++j) {
        const df o2 = df{__shfl_up_sync(full, acc[j].hi, d), __shfl_up_sync(full, acc[j].lo, d)};
        if (lane - d >= seg0) ds_add(acc[j], o2);
      }
    }
    dsum in[NC];
#pragma unroll
    for (int j = 0; j < NC; ++j) {
      const df o2 = df{__shfl_up_sync(full, acc[j].hi, 1), __shfl_up_sync(full, acc[j].lo, 1)};
      in[j] = dsum{o2.hi, o2.lo};
    }
    const bool next_link = __shfl_down_sync(full, link, 1) && lane < 31;
    if (!single && head_p >= 0) {
      if (link) {
#pragma unroll
        for (int j = 0; j < NC; ++j) ds_add(head[j], ds_pair(in[j]));
      }
      flush_bins_ds<NC>(bins, head_p, head);
    }
    if (cur >= 0 && !next_link) flush_bins_ds<NC>(bins, cur, acc);
  }
}

// m_p = M_p^-1 s_p in float64; the map is stored as a double-float pair
// (map_hi, map_lo) of float4 rows; optionally also component-major float64.
template <int NC>
__global__ void __launch_bounds__(kBlock) k_pixel_solve_df(double* __restrict__ bins,
                                                           const double* __restrict__ minv,
                                                           const uint8_t* __restrict__ mask,
                                                           float* __restrict__ map_hi,
                                                           float* __restrict__ map_lo,
                                                           double* __restrict__ out_map,
                                                           int64_t npix, Gate g) {
  if (gate_closed(g)) return;
  constexpr int NM = NC * (NC + 1) / 2;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < npix; p += stride) {
    double s[NC], m[NC];
    const double2 s01 = reinterpret_cast<const double2*>(bins)[2 * p];
    s[0] = s01.x;
    if constexpr (NC > 1) s[1] = s01.y;
    if constexpr (NC > 2) s[2] = bins[4 * p + 2];
    reinterpret_cast<double2*>(bins)[2 * p] = make_double2(0.0, 0.0);
    if constexpr (NC > 2) bins[4 * p + 2] = 0.0;
    if (mask[p]) {
      double mi[NM];
#pragma unroll
      for (int j = 0; j < NM; ++j) mi[j] = minv[p * NM + j];
      sym_mul<NC>(mi, s, m);
    } else {
#pragma unroll
      for (int j = 0; j < NC; ++j) m[j] = 0.0;
    }
    float hi[4] = {0.f, 0.f, 0.f, 0.f}, lo[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
    for (int j = 0; j < NC; ++j) {
      const df d = df_from_double(m[j]);
      hi[j] = d.hi;
      lo[j] = d.lo;
    }
    reinterpret_cast<float4*>(map_hi)[p] = make_float4(hi[0], hi[1], hi[2], hi[3]);
    reinterpret_cast<float4*>(map_lo)[p] = make_float4(lo[0], lo[1], lo[2], lo[3]);
    if (out_map != nullptr) {
#pragma unroll
      for (int j = 0; j < NC; ++j) out_map[(int64_t)j * npix + p] = m[j];
    }
  }
}

// out[o][b] += sum_{t in b} v (z_o(t) - w_o(t) . m_p(t)), z = x[o][b] (ZY false) or
// y[o][t] - x[o][b] (ZY true), in compensated sums.  Each warp walks a chunk of
// `rounds` x 128 consecutive samples, 4 per lane per round.  A lane keeps the sums
// of its current baseline across rounds together with the count of their samples
// (whose baseline term, count x x[o][b], joins the sums when they are flushed).
// The warp flushes every lane's sums at once (a segmented sum over the lanes)
// only when some lane's next samples start another baseline or some lane runs
// out of samples; a lane whose four samples cross a baseline end flushes its own
// sums there; the chunk's end flushes the rest.
template <int KS, bool ZY>
__global__ void __launch_bounds__(kBlock, kDfMinBlocks) k_rescan_df(const int32_t* __restrict__ pix,
                                                      const float* __restrict__ cc,
                                                      const float* __restrict__ ss,
                                                      const float2* __restrict__ x,
                                                      const float* __restrict__ y,
                                                      const float* __restrict__ map_hi,
                                                      const float* __restrict__ map_lo,
                                                      double* __restrict__ out, int64_t n_t,
                                                      int64_t L, int64_t n_b, KindsArg kk,
                                                      int rounds, Gate g) {
  if (gate_closed(g)) return;
  using K = KSet<KS>;
  constexpr int NC = K::NC, NO = K::NO;
  const int n_o = K::n_o(kk);
  const bool hasx = x != nullptr;
  const unsigned full = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  const int64_t nvec = (n_t + 3) >> 2;
  const int64_t span = (int64_t)rounds * 32;
  const int64_t n_chunks = (nvec + span - 1) / span;
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t ch = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); ch < n_chunks;
       ch += warps) {
    int key = -1;     // baseline of the lane's open sums (-1: none)
    float cnt = 0.f;  // their valid samples
    dsum acc[NO];
#pragma unroll
    for (int o = 0; o < NO; ++o) acc[o] = ds_zero();
    // the baseline term of the open sums: -cnt x (ZY) or +cnt x
    auto fold = [&]() {
      if (hasx && key >= 0 && cnt != 0.f) {
#pragma unroll
        for (int o = 0; o < NO; ++o)
          if (o < n_o) ds_add_prod(acc[o], df_ldg(x, o * n_b + key), ZY ? -cnt : cnt);
      }
    };
    auto reset = [&]() {
      key = -1;
      cnt = 0.f;
#pragma unroll
      for (int o = 0; o < NO; ++o) acc[o] = ds_zero();
    };
    BaselineCursor bc((ch * span + lane) << 2, 128, L);
    for (int r = 0; r < rounds; ++r, bc.advance(L)) {
      const int64_t v = ch * span + (int64_t)r * 32 + lane;
      const bool active = v < nvec;
      if (!__any_sync(full, active)) break;
      const int bf = (int)bc.b;  // baseline of the lane's first sample this round
      if (__any_sync(full, !active || (key >= 0 && bf != key))) {
        fold();
        warp_segment_flush_ds<NO>(key, acc, n_o, out, n_b);
        reset();
      }
      if (!active) continue;
      if (key < 0) key = bf;
      int p[4];
      float c[4], s[4];
      load4_df(pix, cc, ss, v, n_t, p, c, s);
      df m[NC] = {};  // the map pair, gathered once per run of equal pixels
      int mp = -1;
      float yv[NO][4];
      if constexpr (ZY) load_y4<NO>(y, n_o, n_t, v, yv);
      const int64_t t0 = v << 2;
      int64_t bend = bc.next_start(t0, L);
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const int64_t t = t0 + k;
        if (t >= n_t) break;
        if (t >= bend) {
          fold();
#pragma unroll
          for (int o = 0; o < NO; ++o)
            if (o < n_o && ds_nonzero(acc[o]))
              atomicAdd(out + (int64_t)o * n_b + key, ds_to_double(acc[o]));
          const int next = key + 1;
          reset();
          key = next;
          bend += L;
        }
        if (p[k] < 0) continue;
        if (p[k] != mp) {
          mp = p[k];
          const float4 h = __ldg(reinterpret_cast<const float4*>(map_hi) + mp);
          const float4 l = __ldg(reinterpret_cast<const float4*>(map_lo) + mp);
          const float hh[4] = {h.x, h.y, h.z, h.w}, ll[4] = {l.x, l.y, l.z, l.w};
#pragma unroll
          for (int j = 0; j < NC; ++j) m[j] = df{hh[j], ll[j]};
        }
        cnt += 1.f;
#pragma unroll
        for (int o = 0; o < NO; ++o) {
          if (o < n_o) {
            if constexpr (ZY) ds_add(acc[o], yv[o][k]);
            row_sub_dot_ds<NC>(K::kind(o, kk), c[k], s[k], m, acc[o]);
          }
        }
      }
#pragma unroll
      for (int o = 0; o < NO; ++o) ds_norm(acc[o]);
    }
    fold();
    warp_segment_flush_ds<NO>(key, acc, n_o, out, n_b);
  }
}

}  // namespace

// ---- launchers (mixed-precision plans only: y is float32) --------------------------

// Long chunks amortise the warp flushes of the carried-sum rescans; at least four
// chunks per warp of the grid keep the warps evenly loaded.
int rescan_rounds(const Plan& P, int64_t n_units, int grid) {
  if (P.rescan_rounds > 0) return P.rescan_rounds;
  const int64_t warps = (int64_t)grid * (kBlock / 32);
  const int64_t r = n_units / (32 * warps * 4);
  return (int)(r < 1 ? 1 : (r > 16 ? 16 : r));
}

// Splits the baselines of an accurate pass into P.xdf (once per pass: the
// per-sample kernels then read float32 pairs and do no float64 work per sample).
void launch_split_df(const Plan& P, cudaStream_t st, const double* x, Gate g) {
  k_split_df<<<stream_grid(P, P.n_u, kBlock, 8), kBlock, 0, st>>>(x, P.xdf, P.n_u, g);
}

// x: baselines already split by launch_split_df (then P.xdf is read), or NULL
void launch_bin_df(const Plan& P, cudaStream_t st, const double* x, const float* y, Gate g) {
  const int grid = stream_grid(P, (P.n_t + 3) / 4, kBlock, P.blocks_per_sm);
  const float2* xs = x != nullptr ? P.xdf : nullptr;
  with_kindset(P.kindset, [&](auto ksc) {
    constexpr int KS = decltype(ksc)::value;
    if (y != nullptr)
      k_bin_df<KS, true><<<grid, kBlock, 0, st>>>(P.pix, P.c, P.s, xs, y, P.bins, P.n_t, P.L,
                                                   P.n_b, P.kinds, g);
    else
      k_bin_df<KS, false><<<grid, kBlock, 0, st>>>(P.pix, P.c, P.s, xs, nullptr, P.bins, P.n_t,
                                                    P.L, P.n_b, P.kinds, g);
  });
}

void launch_pixel_solve_df(const Plan& P, cudaStream_t st, double* out_map, Gate g) {
  const int grid = stream_grid(P, P.npix, kBlock, 8);
  if (P.n_c == 1)
    k_pixel_solve_df<1><<<grid, kBlock, 0, st>>>(P.bins, P.minv, P.mask, P.map32, P.maplo,
                                                  out_map, P.npix, g);
  else if (P.n_c == 2)
    k_pixel_solve_df<2><<<grid, kBlock, 0, st>>>(P.bins, P.minv, P.mask, P.map32, P.maplo,
                                                  out_map, P.npix, g);
  else
    k_pixel_solve_df<3><<<grid, kBlock, 0, st>>>(P.bins, P.minv, P.mask, P.map32, P.maplo,
                                                  out_map, P.npix, g);
}

void launch_rescan_df(const Plan& P, cudaStream_t st, const double* x, const float* y,
                      double* out, Gate g) {
  const int grid = stream_grid(P, (P.n_t + 3) / 4, kBlock, P.blocks_per_sm);
  const int rounds = rescan_rounds(P, (P.n_t + 3) / 4, grid);
  const float2* xs = x != nullptr ? P.xdf : nullptr;
  with_kindset(P.kindset, [&](auto ksc) {
    constexpr int KS = decltype(ksc)::value;
    if (y != nullptr)
      k_rescan_df<KS, true><<<grid, kBlock, 0, st>>>(P.pix, P.c, P.s, xs, y, P.map32, P.maplo,
                                                      out, P.n_t, P.L, P.n_b, P.kinds, rounds, g);
    else
      k_rescan_df<KS, false><<<grid, kBlock, 0, st>>>(P.pix, P.c, P.s, xs, nullptr, P.map32,
                                                       P.maplo, out, P.n_t, P.L, P.n_b, P.kinds,
                                                       rounds, g);
  });
}

}  // namespace ds
