// Per-sample passes of the destriping operator and the per-pixel solve
// (Sect. 3: F~ expands baselines to the timeline, P~^T R^T bins into pixel sums,
// M^-1 weights them into a map, R P~ rescans the map, F~^T sums per baseline).
//
// Work split: every thread owns 4 consecutive samples and reads them with one
// 16-byte load per stream (pixel, cos 2psi, sin 2psi); a warp covers 128
// consecutive samples.  Consecutive samples often share a pixel, so binning
// aggregates runs of equal pixels in registers before each atomic add into the
// float64 pixel sums.  Per-baseline sums are reduced across the warp by a
// segmented shuffle scan on the baseline index and added with one atomic per
// warp segment.
#include <type_traits>

#include "internal.cuh"
#include "rows.cuh"
#include "stream_common.cuh"

namespace ds {

namespace {

constexpr int kBlock = 256;

// ---- binning: bins[p] += sum_o w_o(t) z_o(t) over samples with v = 1 ----------
// ZY = false: z_o(t) = x[o][t / L]          (F~ x, the operator)
// ZY = true : z_o(t) = y[o][t] - a[o][t/L]  (data minus baselines; a may be NULL)
template <int KS, typename T, bool ZY, typename YT, typename BT, typename XT = double>
__global__ void __launch_bounds__(kBlock) k_bin(const int32_t* __restrict__ pix,
                                                const float* __restrict__ cc,
                                                const float* __restrict__ ss,
                                                const XT* __restrict__ x,
                                                const YT* __restrict__ y,
                                                BT* __restrict__ bins, int64_t n_t, int64_t L,
                                                int64_t n_b, KindsArg kk, Gate g) {
  if (gate_closed(g)) return;
  using K = KSet<KS>;
  constexpr int NC = K::NC, NO = K::NO;
  const int n_o = K::n_o(kk);
  const int64_t nvec = (n_t + 3) >> 2;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < nvec; v += stride) {
    int p[4];
    float c[4], s[4];
    load4(pix, cc, ss, v, n_t, p, c, s);
    const int64_t t0 = v << 2;
    int64_t b = t0 / L;
    int64_t bend = (b + 1) * L;
    T zb[NO];
#pragma unroll
    for (int o = 0; o < NO; ++o)
      zb[o] = (o < n_o && x != nullptr) ? (T)__ldg(x + o * n_b + b) : T(0);
    T acc[NC];
#pragma unroll
    for (int j = 0; j < NC; ++j) acc[j] = T(0);
    int cur = -1;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const int64_t t = t0 + k;
      if (t >= n_t) break;
      if (t >= bend) {
        b += 1;
        bend += L;
#pragma unroll
        for (int o = 0; o < NO; ++o)
          zb[o] = (o < n_o && x != nullptr) ? (T)__ldg(x + o * n_b + b) : T(0);
      }
      if (p[k] < 0) continue;
      T w[NC];
#pragma unroll
      for (int j = 0; j < NC; ++j) w[j] = T(0);
#pragma unroll
      for (int o = 0; o < NO; ++o) {
        if (o < n_o) {
          T z = zb[o];
          if constexpr (ZY) z = (T)y[(int64_t)o * n_t + t] - z;
          row_bin<NC, T>(K::kind(o, kk), (T)c[k], (T)s[k], z, w);
        }
      }
      if (p[k] != cur) {
        if (cur >= 0) flush_bins<NC, T>(bins, cur, acc);
        cur = p[k];
#pragma unroll
        for (int j = 0; j < NC; ++j) acc[j] = w[j];
      } else {
#pragma unroll
        for (int j = 0; j < NC; ++j) acc[j] += w[j];
      }
    }
    if (cur >= 0) flush_bins<NC, T>(bins, cur, acc);
  }
}

// ---- float32 operator, 8 samples per thread ------------------------------------
// The same passes as k_bin / k_rescan (float32 arithmetic, float32 baselines and
// map, float32 pixel sums) with two 16-byte loads per stream per thread, so that
// twice the bytes are in flight per resident warp.

// Samples 8 u .. 8 u + 7; past n_t: pixel -1.
__device__ __forceinline__ void load8(const int32_t* __restrict__ pix,
                                      const float* __restrict__ cc,
                                      const float* __restrict__ ss, int64_t u, int64_t n_t,
                                      int (&p)[8], float (&c)[8], float (&s)[8]) {
  const int64_t t0 = u << 3;
  if (t0 + 8 <= n_t) {
    const int4 p0 = ld_stream(reinterpret_cast<const int4*>(pix) + 2 * u);
    const int4 p1 = ld_stream(reinterpret_cast<const int4*>(pix) + 2 * u + 1);
    const float4 c0 = ld_stream(reinterpret_cast<const float4*>(cc) + 2 * u);
    const float4 c1 = ld_stream(reinterpret_cast<const float4*>(cc) + 2 * u + 1);
    const float4 s0 = ld_stream(reinterpret_cast<const float4*>(ss) + 2 * u);
    const float4 s1 = ld_stream(reinterpret_cast<const float4*>(ss) + 2 * u + 1);
    p[0] = p0.x; p[1] = p0.y; p[2] = p0.z; p[3] = p0.w;
    p[4] = p1.x; p[5] = p1.y; p[6] = p1.z; p[7] = p1.w;
    c[0] = c0.x; c[1] = c0.y; c[2] = c0.z; c[3] = c0.w;
    c[4] = c1.x; c[5] = c1.y; c[6] = c1.z; c[7] = c1.w;
    s[0] = s0.x; s[1] = s0.y; s[2] = s0.z; s[3] = s0.w;
    s[4] = s1.x; s[5] = s1.y; s[6] = s1.z; s[7] = s1.w;
  } else {
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      const bool in = t0 + k < n_t;
      p[k] = in ? pix[t0 + k] : -1;
      c[k] = in ? cc[t0 + k] : 0.f;
      s[k] = in ? ss[t0 + k] : 0.f;
    }
  }
}

template <int KS>
__global__ void __launch_bounds__(kBlock) k_bin8(const int32_t* __restrict__ pix,
                                                 const float* __restrict__ cc,
                                                 const float* __restrict__ ss,
                                                 const float* __restrict__ x,
                                                 float* __restrict__ bins, int64_t n_t, int64_t L,
                                                 int64_t n_b, KindsArg kk, Gate g) {
  if (gate_closed(g)) return;
  using K = KSet<KS>;
  constexpr int NC = K::NC, NO = K::NO;
  const int n_o = K::n_o(kk);
  const int64_t n8 = (n_t + 7) >> 3;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; u < n8; u += stride) {
    int p[8];
    float c[8], s[8];
    load8(pix, cc, ss, u, n_t, p, c, s);
    const int64_t t0 = u << 3;
    int64_t b = t0 / L;
    int64_t bend = (b + 1) * L;
    float zb[NO];
#pragma unroll
    for (int o = 0; o < NO; ++o) zb[o] = o < n_o ? __ldg(x + o * n_b + b) : 0.f;
    float acc[NC];
#pragma unroll
    for (int j = 0; j < NC; ++j) acc[j] = 0.f;
    int cur = -1;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      const int64_t t = t0 + k;
      if (t >= n_t) break;
      if (t >= bend) {
        b += 1;
        bend += L;
#pragma unroll
        for (int o = 0; o < NO; ++o) zb[o] = o < n_o ? __ldg(x + o * n_b + b) : 0.f;
      }
      if (p[k] < 0) continue;
      float w[NC];
#pragma unroll
      for (int j = 0; j < NC; ++j) w[j] = 0.f;
#pragma unroll
      for (int o = 0; o < NO; ++o)
        if (o < n_o) row_bin<NC, float>(K::kind(o, kk), c[k], s[k], zb[o], w);
      if (p[k] != cur) {
        if (cur >= 0) flush_bins<NC, float>(bins, cur, acc);
        cur = p[k];
#pragma unroll
        for (int j = 0; j < NC; ++j) acc[j] = w[j];
      } else {
#pragma unroll
        for (int j = 0; j < NC; ++j) acc[j] += w[j];
      }
    }
    if (cur >= 0) flush_bins<NC, float>(bins, cur, acc);
  }
}

template <int KS>
__global__ void __launch_bounds__(kBlock) k_rescan8(const int32_t* __restrict__ pix,
                                                    const float* __restrict__ cc,
                                                    const float* __restrict__ ss,
                                                    const float* __restrict__ x,
                                                    const float* __restrict__ map,
                                                    double* __restrict__ out, int64_t n_t,
                                                    int64_t L, int64_t n_b, KindsArg kk, Gate g) {
  if (gate_closed(g)) return;
  using K = KSet<KS>;
  constexpr int NC = K::NC, NO = K::NO;
  const int n_o = K::n_o(kk);
  const int lane = threadIdx.x & 31;
  const int64_t n8 = (n_t + 7) >> 3;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t ub = (int64_t)blockIdx.x * blockDim.x + threadIdx.x - lane; ub < n8;
       ub += stride) {
    const int64_t u = ub + lane;
    int key = -1;
    float acc[NO];
#pragma unroll
    for (int o = 0; o < NO; ++o) acc[o] = 0.f;
    if (u < n8) {
      int p[8];
      float c[8], s[8];
      load8(pix, cc, ss, u, n_t, p, c, s);
      // the map row is gathered once per run of equal pixels in the thread's samples
      float m[8][NC];
      bool dup[8];
#pragma unroll
      for (int k = 0; k < 8; ++k) dup[k] = k > 0 && p[k] >= 0 && p[k] == p[k - 1];
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        if (p[k] >= 0 && !dup[k]) {
          load_map<NC, float>(map, p[k], m[k]);
        } else {
#pragma unroll
          for (int j = 0; j < NC; ++j) m[k][j] = 0.f;
        }
      }
#pragma unroll
      for (int k = 1; k < 8; ++k)
        if (dup[k]) {
#pragma unroll
          for (int j = 0; j < NC; ++j) m[k][j] = m[k - 1][j];
        }
      const int64_t t0 = u << 3;
      int64_t b = t0 / L;
      int64_t bend = (b + 1) * L;
      float zb[NO];
#pragma unroll
      for (int o = 0; o < NO; ++o) zb[o] = o < n_o ? __ldg(x + o * n_b + b) : 0.f;
      key = (int)b;
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        const int64_t t = t0 + k;
        if (t >= n_t) break;
        if (t >= bend) {
#pragma unroll
          for (int o = 0; o < NO; ++o) {
            if (o < n_o && acc[o] != 0.f) atomicAdd(out + o * n_b + b, to_f64(acc[o]));
            acc[o] = 0.f;
          }
          b += 1;
          bend += L;
          key = (int)b;
#pragma unroll
          for (int o = 0; o < NO; ++o) zb[o] = o < n_o ? __ldg(x + o * n_b + b) : 0.f;
        }
        if (p[k] < 0) continue;
#pragma unroll
        for (int o = 0; o < NO; ++o)
          if (o < n_o) acc[o] += zb[o] - row_dot<NC, float>(K::kind(o, kk), c[k], s[k], m[k]);
      }
    }
    warp_segment_flush<NO, float>(key, acc, n_o, out, n_b);
  }
}

// x rounded to float32 once per operator apply, so that the float32 passes read
// float32 baselines (no float64 conversion per sample group)
__global__ void __launch_bounds__(kBlock) k_to_f32(const double* __restrict__ x,
                                                   float* __restrict__ x32, int64_t n, Gate g) {
  if (gate_closed(g)) return;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride)
    x32[i] = (float)x[i];
}

// ---- per-pixel solve: m_p = M_p^-1 s_p on kept pixels, 0 elsewhere ---------------
// Reads the float64 sums, clears them for the next pass, writes the map in the
// working precision (and optionally component-major float64 for the caller).
template <int NC, typename T, typename BT>
__global__ void __launch_bounds__(kBlock) k_pixel_solve(BT* __restrict__ bins,
                                                        const double* __restrict__ minv,
                                                        const uint8_t* __restrict__ mask,
                                                        T* __restrict__ map,
                                                        double* __restrict__ out_map, int64_t npix,
                                                        unsigned* __restrict__ mmax, Gate g) {
  if (gate_closed(g)) return;
  constexpr int NM = NC * (NC + 1) / 2;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  float big = 0.f;  // largest |m| of this thread's pixels (mmax: the grid's, as float bits)
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < npix; p += stride) {
    double s[NC], m[NC];
    if constexpr (std::is_same<BT, float>::value && std::is_same<T, float>::value) {
      // The float32 operator's pass.  A pixel no run touched has zero sums, and a cut
      // pixel's map entry is zero from the plan's creation on (every pass leaves it
      // so): both cost two loads here and no float64 work, which is narrow on this
      // GPU.  The sums of a kept pixel widen on the integer pipes.
      const float4 v = reinterpret_cast<const float4*>(bins)[p];
      if (v.x != 0.f || v.y != 0.f || v.z != 0.f || v.w != 0.f)
        reinterpret_cast<float4*>(bins)[p] = make_float4(0.f, 0.f, 0.f, 0.f);
      if (!mask[p]) {
        if (out_map != nullptr)
#pragma unroll
          for (int j = 0; j < NC; ++j) out_map[(int64_t)j * npix + p] = 0.0;
        continue;
      }
      s[0] = f64_of_f32(v.x);
      if constexpr (NC > 1) s[1] = f64_of_f32(v.y);
      if constexpr (NC > 2) s[2] = f64_of_f32(v.z);
      double mi[NM];
#pragma unroll
      for (int j = 0; j < NM; ++j) mi[j] = minv[p * NM + j];
      sym_mul<NC>(mi, s, m);
      float4 o4 = make_float4(0.f, 0.f, 0.f, 0.f);
      o4.x = (float)m[0];
      if constexpr (NC > 1) o4.y = (float)m[1];
      if constexpr (NC > 2) o4.z = (float)m[2];
      reinterpret_cast<float4*>(map)[p] = o4;
      big = __uint_as_float(max(__float_as_uint(big),
                                max(__float_as_uint(fabsf(o4.x)),
                                    max(__float_as_uint(fabsf(o4.y)), __float_as_uint(fabsf(o4.z))))));
      if (out_map != nullptr)
#pragma unroll
        for (int j = 0; j < NC; ++j) out_map[(int64_t)j * npix + p] = m[j];
      continue;
    }
    if constexpr (std::is_same<BT, float>::value) {
      const float4 v = reinterpret_cast<const float4*>(bins)[p];
      s[0] = v.x;
      if constexpr (NC > 1) s[1] = v.y;
      if constexpr (NC > 2) s[2] = v.z;
      reinterpret_cast<float4*>(bins)[p] = make_float4(0.f, 0.f, 0.f, 0.f);
    } else {
      const double2 s01 = reinterpret_cast<const double2*>(bins)[2 * p];
      s[0] = s01.x;
      if constexpr (NC > 1) s[1] = s01.y;
      if constexpr (NC > 2) s[2] = bins[4 * p + 2];
      reinterpret_cast<double2*>(bins)[2 * p] = make_double2(0.0, 0.0);
      if constexpr (NC > 2) bins[4 * p + 2] = 0.0;
    }
    if (mask[p]) {
      double mi[NM];
#pragma unroll
      for (int j = 0; j < NM; ++j) mi[j] = minv[p * NM + j];
      sym_mul<NC>(mi, s, m);
    } else {
#pragma unroll
      for (int j = 0; j < NC; ++j) m[j] = 0.0;
    }
    if constexpr (std::is_same<T, float>::value) {
      float4 o4 = make_float4(0.f, 0.f, 0.f, 0.f);
      o4.x = (float)m[0];
      if constexpr (NC > 1) o4.y = (float)m[1];
      if constexpr (NC > 2) o4.z = (float)m[2];
      reinterpret_cast<float4*>(map)[p] = o4;
      // the largest |m| by the bits of non-negative floats, which order as the values
      // do and keep a NaN (above +inf; fmaxf would drop it)
      big = __uint_as_float(max(__float_as_uint(big),
                                max(__float_as_uint(fabsf(o4.x)),
                                    max(__float_as_uint(fabsf(o4.y)), __float_as_uint(fabsf(o4.z))))));
    } else {
      reinterpret_cast<double2*>(map)[2 * p] = make_double2(m[0], NC > 1 ? m[NC > 1 ? 1 : 0] : 0.0);
      if constexpr (NC > 2) map[4 * p + 2] = m[2];
    }
    if (out_map != nullptr) {
#pragma unroll
      for (int j = 0; j < NC; ++j) out_map[(int64_t)j * npix + p] = m[j];
    }
  }
  if (mmax != nullptr) {  // one atomic per block: a warp's each would queue on one address
    __shared__ unsigned s_big[kBlock / 32];
    const unsigned w = __reduce_max_sync(0xffffffffu, __float_as_uint(big));
    if ((threadIdx.x & 31) == 0) s_big[threadIdx.x >> 5] = w;
    __syncthreads();
    if (threadIdx.x == 0) {
      unsigned m = 0u;
      for (int q = 0; q < kBlock / 32; ++q) m = max(m, s_big[q]);
      atomicMax(mmax, m);
    }
  }
}

// ---- rescan + per-baseline sum: out[o][b] += sum_{t in b} v (z_o(t) - w_o(t) . m_p(t))
template <int KS, typename T, bool ZY, typename YT, bool DEDUP = false, typename XT = double>
__global__ void __launch_bounds__(kBlock) k_rescan(const int32_t* __restrict__ pix,
                                                   const float* __restrict__ cc,
                                                   const float* __restrict__ ss,
                                                   const XT* __restrict__ x,
                                                   const YT* __restrict__ y,
                                                   const T* __restrict__ map,
                                                   double* __restrict__ out, int64_t n_t,
                                                   int64_t L, int64_t n_b, KindsArg kk, Gate g) {
  if (gate_closed(g)) return;
  using K = KSet<KS>;
  constexpr int NC = K::NC, NO = K::NO;
  const int n_o = K::n_o(kk);
  const int lane = threadIdx.x & 31;
  const int64_t nvec = (n_t + 3) >> 2;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t vb = (int64_t)blockIdx.x * blockDim.x + threadIdx.x - lane; vb < nvec;
       vb += stride) {
    const int64_t v = vb + lane;
    int key = -1;
    T acc[NO];
#pragma unroll
    for (int o = 0; o < NO; ++o) acc[o] = T(0);
    if (v < nvec) {
      int p[4];
      float c[4], s[4];
      load4(pix, cc, ss, v, n_t, p, c, s);
      T m[4][NC];
      if constexpr (DEDUP) {
        // a sample on the same pixel as the one before it reuses that map value:
        // the other gathers are all issued first, the copies made after
        bool dup[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) dup[k] = k > 0 && p[k] >= 0 && p[k] == p[k - 1];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          if (p[k] >= 0 && !dup[k]) {
            load_map<NC, T>(map, p[k], m[k]);
          } else {
#pragma unroll
            for (int j = 0; j < NC; ++j) m[k][j] = T(0);
          }
        }
#pragma unroll
        for (int k = 1; k < 4; ++k)
          if (dup[k]) {
#pragma unroll
            for (int j = 0; j < NC; ++j) m[k][j] = m[k - 1][j];
          }
      } else {
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          if (p[k] >= 0) {
            load_map<NC, T>(map, p[k], m[k]);
          } else {
#pragma unroll
            for (int j = 0; j < NC; ++j) m[k][j] = T(0);
          }
        }
      }
      const int64_t t0 = v << 2;
      int64_t b = t0 / L;
      int64_t bend = (b + 1) * L;
      T zb[NO];
#pragma unroll
      for (int o = 0; o < NO; ++o)
        zb[o] = (o < n_o && x != nullptr) ? (T)__ldg(x + o * n_b + b) : T(0);
      key = (int)b;
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const int64_t t = t0 + k;
        if (t >= n_t) break;
        if (t >= bend) {
#pragma unroll
          for (int o = 0; o < NO; ++o) {
            if (o < n_o && acc[o] != T(0)) atomicAdd(out + o * n_b + b, to_f64(acc[o]));
            acc[o] = T(0);
          }
          b += 1;
          bend += L;
          key = (int)b;
#pragma unroll
          for (int o = 0; o < NO; ++o)
            zb[o] = (o < n_o && x != nullptr) ? (T)__ldg(x + o * n_b + b) : T(0);
        }
        if (p[k] < 0) continue;
#pragma unroll
        for (int o = 0; o < NO; ++o) {
          if (o < n_o) {
            T z = zb[o];
            if constexpr (ZY) z = (T)y[(int64_t)o * n_t + t] - z;
            acc[o] += z - row_dot<NC, T>(K::kind(o, kk), (T)c[k], (T)s[k], m[k]);
          }
        }
      }
    }
    warp_segment_flush<NO, T>(key, acc, n_o, out, n_b);
  }
}

}  // namespace

int stream_grid(const Plan& P, int64_t work_items, int block, int per_sm) {
  int64_t need = (work_items + block - 1) / block;
  int64_t cap = (int64_t)P.num_sms * per_sm;
  if (need < 1) need = 1;
  return (int)(need < cap ? need : cap);
}

static bool f32_bins(const Plan& P, bool fp64) { return !fp64 && P.bin_mode == 1; }

void launch_bin_x(const Plan& P, cudaStream_t st, bool fp64, const double* x, Gate g) {
  const int grid = stream_grid(P, (P.n_t + 3) / 4, kBlock, P.blocks_per_sm);
  with_kindset(P.kindset, [&](auto ksc) {
    constexpr int KS = decltype(ksc)::value;
    if (fp64)
      k_bin<KS, double, false, double, double><<<grid, kBlock, 0, st>>>(
          P.pix, P.c, P.s, x, nullptr, P.bins, P.n_t, P.L, P.n_b, P.kinds, g);
    else if (f32_bins(P, fp64) && P.x32 != nullptr && P.samples_per_thread == 8)
      k_bin8<KS><<<stream_grid(P, (P.n_t + 7) / 8, kBlock, P.blocks_per_sm), kBlock, 0, st>>>(
          P.pix, P.c, P.s, P.x32, P.bins32, P.n_t, P.L, P.n_b, P.kinds, g);
    else if (f32_bins(P, fp64) && P.x32 != nullptr)
      k_bin<KS, float, false, float, float, float><<<grid, kBlock, 0, st>>>(
          P.pix, P.c, P.s, P.x32, nullptr, P.bins32, P.n_t, P.L, P.n_b, P.kinds, g);
    else if (f32_bins(P, fp64))
      k_bin<KS, float, false, float, float><<<grid, kBlock, 0, st>>>(
          P.pix, P.c, P.s, x, nullptr, P.bins32, P.n_t, P.L, P.n_b, P.kinds, g);
    else
      k_bin<KS, float, false, float, double><<<grid, kBlock, 0, st>>>(
          P.pix, P.c, P.s, x, nullptr, P.bins, P.n_t, P.L, P.n_b, P.kinds, g);
  });
}

void launch_bin_y(const Plan& P, cudaStream_t st, const void* y, const double* a, Gate g) {
  const int grid = stream_grid(P, (P.n_t + 3) / 4, kBlock, P.blocks_per_sm);
  with_kindset(P.kindset, [&](auto ksc) {
    constexpr int KS = decltype(ksc)::value;
    if (P.desc.precision == DS_PREC_FP64)
      k_bin<KS, double, true, double, double><<<grid, kBlock, 0, st>>>(
          P.pix, P.c, P.s, a, static_cast<const double*>(y), P.bins, P.n_t, P.L, P.n_b, P.kinds, g);
    else
      k_bin<KS, double, true, float, double><<<grid, kBlock, 0, st>>>(
          P.pix, P.c, P.s, a, static_cast<const float*>(y), P.bins, P.n_t, P.L, P.n_b, P.kinds, g);
  });
}

void launch_pixel_solve(const Plan& P, cudaStream_t st, bool fp64, double* out_map, Gate g) {
  const int grid = stream_grid(P, P.npix, kBlock, 8);
  auto go = [&](auto ncc) {
    constexpr int NC = decltype(ncc)::value;
    if (fp64)
      k_pixel_solve<NC, double, double><<<grid, kBlock, 0, st>>>(P.bins, P.minv, P.mask, P.map64,
                                                                  out_map, P.npix, nullptr, g);
    else if (f32_bins(P, fp64))
      k_pixel_solve<NC, float, float><<<grid, kBlock, 0, st>>>(
          P.bins32, P.minv, P.mask, P.map32, out_map, P.npix, tl_ready(P) ? P.tl_mmax : nullptr,
          g);
    else
      k_pixel_solve<NC, float, double><<<grid, kBlock, 0, st>>>(P.bins, P.minv, P.mask, P.map32,
                                                                 out_map, P.npix, nullptr, g);
  };
  if (P.n_c == 1) go(std::integral_constant<int, 1>{});
  else if (P.n_c == 2) go(std::integral_constant<int, 2>{});
  else go(std::integral_constant<int, 3>{});
}

void launch_rescan_x(const Plan& P, cudaStream_t st, bool fp64, const double* x, double* out,
                     Gate g) {
  const int grid = stream_grid(P, (P.n_t + 3) / 4, kBlock, P.blocks_per_sm);
  with_kindset(P.kindset, [&](auto ksc) {
    constexpr int KS = decltype(ksc)::value;
    if (fp64)
      k_rescan<KS, double, false, double><<<grid, kBlock, 0, st>>>(
          P.pix, P.c, P.s, x, nullptr, P.map64, out, P.n_t, P.L, P.n_b, P.kinds, g);
    else if (P.x32 != nullptr && P.samples_per_thread == 8)
      k_rescan8<KS><<<stream_grid(P, (P.n_t + 7) / 8, kBlock, P.blocks_per_sm), kBlock, 0, st>>>(
          P.pix, P.c, P.s, P.x32, P.map32, out, P.n_t, P.L, P.n_b, P.kinds, g);
    else if (P.rescan_dedup && P.x32 != nullptr)
      k_rescan<KS, float, false, float, true, float><<<grid, kBlock, 0, st>>>(
          P.pix, P.c, P.s, P.x32, nullptr, P.map32, out, P.n_t, P.L, P.n_b, P.kinds, g);
    else if (P.rescan_dedup)
      k_rescan<KS, float, false, float, true><<<grid, kBlock, 0, st>>>(
          P.pix, P.c, P.s, x, nullptr, P.map32, out, P.n_t, P.L, P.n_b, P.kinds, g);
    else
      k_rescan<KS, float, false, float><<<grid, kBlock, 0, st>>>(
          P.pix, P.c, P.s, x, nullptr, P.map32, out, P.n_t, P.L, P.n_b, P.kinds, g);
  });
}

void launch_rescan_y(const Plan& P, cudaStream_t st, const void* y, double* out, Gate g) {
  const int grid = stream_grid(P, (P.n_t + 3) / 4, kBlock, P.blocks_per_sm);
  with_kindset(P.kindset, [&](auto ksc) {
    constexpr int KS = decltype(ksc)::value;
    if (P.desc.precision == DS_PREC_FP64)
      k_rescan<KS, double, true, double><<<grid, kBlock, 0, st>>>(
          P.pix, P.c, P.s, static_cast<const double*>(nullptr), static_cast<const double*>(y),
          P.map64, out, P.n_t, P.L, P.n_b,
          P.kinds, g);
    else
      k_rescan<KS, double, true, float><<<grid, kBlock, 0, st>>>(
          P.pix, P.c, P.s, static_cast<const double*>(nullptr), static_cast<const float*>(y),
          P.map64, out, P.n_t, P.L, P.n_b,
          P.kinds, g);
  });
}

// The pixel sums the next pixel solve reads: float32 [n_pix][4] for the float32
// operator with vector reductions, float64 [n_pix][4] otherwise.  A sharded plan
// sums them over the ranks here (the Export / Import step of Sect. 4).
static void exchange_sums(const Plan& P, cudaStream_t st, bool f32) {
  if (P.shard_allreduce == nullptr) return;
  if (f32) shard_exchange(P, st, P.bins32, P.npix * 4, DS_DT_F32);
  else shard_exchange(P, st, P.bins, P.npix * 4, DS_DT_F64);
}

static bool use_df(const Plan& P) {
  return P.desc.precision == DS_PREC_MIXED && P.accurate_df && P.maplo != nullptr;
}

// ev (optional): events recorded before binning, after binning, after the pixel
// solve and after the rescan.  fp64 selects the accurate operator: float64
// arithmetic, or double-float in mixed plans.
void enqueue_apply(const Plan& P, cudaStream_t st, bool fp64, const double* x, double* out,
                   Gate g, cudaEvent_t* ev) {
  if (fp64 && use_df(P)) {
    const bool runs = rl_df_ready(P);
    if (ev) cudaEventRecordWithFlags(ev[0], st, cudaEventRecordExternal);
    launch_split_df(P, st, x, g);
    if (runs) launch_bin_rl_df(P, st, g);
    else launch_bin_df(P, st, x, nullptr, g);
    exchange_sums(P, st, false);
    if (ev) cudaEventRecordWithFlags(ev[1], st, cudaEventRecordExternal);
    launch_pixel_solve_df(P, st, nullptr, g);
    if (ev) cudaEventRecordWithFlags(ev[2], st, cudaEventRecordExternal);
    if (runs && !P.rescan_samples) launch_rescan_rl_df(P, st, out, g);
    else launch_rescan_df(P, st, x, nullptr, out, g);
    if (ev) cudaEventRecordWithFlags(ev[3], st, cudaEventRecordExternal);
    return;
  }
  if (!fp64 && P.bin_mode == 1 && rl_ready(P)) {
    k_to_f32<<<stream_grid(P, P.n_u, kBlock, 8), kBlock, 0, st>>>(x, P.x32, P.n_u, g);
    if (ev) cudaEventRecordWithFlags(ev[0], st, cudaEventRecordExternal);
    launch_bin_rl(P, st, g);
    exchange_sums(P, st, true);
    if (ev) cudaEventRecordWithFlags(ev[1], st, cudaEventRecordExternal);
    launch_pixel_solve(P, st, false, nullptr, g);
    if (ev) cudaEventRecordWithFlags(ev[2], st, cudaEventRecordExternal);
    if (P.rescan_samples) launch_rescan_x(P, st, false, x, out, g);
    else launch_rescan_rl(P, st, out, g);
    if (ev) cudaEventRecordWithFlags(ev[3], st, cudaEventRecordExternal);
    return;
  }
  if (!fp64 && P.bin_mode == 1 && tl_ready(P)) {
    launch_pack_tl(P, st, x, g);
    if (ev) cudaEventRecordWithFlags(ev[0], st, cudaEventRecordExternal);
    launch_bin_tl(P, st, g);
    exchange_sums(P, st, true);
    if (ev) cudaEventRecordWithFlags(ev[1], st, cudaEventRecordExternal);
    launch_pixel_solve(P, st, false, nullptr, g);
    if (ev) cudaEventRecordWithFlags(ev[2], st, cudaEventRecordExternal);
    launch_rescan_tl(P, st, out, g);
    if (ev) cudaEventRecordWithFlags(ev[3], st, cudaEventRecordExternal);
    return;
  }
  if (!fp64 && P.bin_mode == 1 && ck_ready(P)) {
    if (ev) cudaEventRecordWithFlags(ev[0], st, cudaEventRecordExternal);
    launch_bin_ck(P, st, x, g);
    exchange_sums(P, st, true);
    if (ev) cudaEventRecordWithFlags(ev[1], st, cudaEventRecordExternal);
    launch_pixel_solve(P, st, false, nullptr, g);
    if (ev) cudaEventRecordWithFlags(ev[2], st, cudaEventRecordExternal);
    launch_rescan_ck(P, st, x, out, g);
    if (ev) cudaEventRecordWithFlags(ev[3], st, cudaEventRecordExternal);
    return;
  }
  // External records become event nodes when the stream is being captured.
  if (!fp64 && P.x32 != nullptr)
    k_to_f32<<<stream_grid(P, P.n_u, kBlock, 8), kBlock, 0, st>>>(x, P.x32, P.n_u, g);
  if (ev) cudaEventRecordWithFlags(ev[0], st, cudaEventRecordExternal);
  launch_bin_x(P, st, fp64, x, g);
  exchange_sums(P, st, f32_bins(P, fp64));
  if (ev) cudaEventRecordWithFlags(ev[1], st, cudaEventRecordExternal);
  launch_pixel_solve(P, st, fp64, nullptr, g);
  if (ev) cudaEventRecordWithFlags(ev[2], st, cudaEventRecordExternal);
  launch_rescan_x(P, st, fp64, x, out, g);
  if (ev) cudaEventRecordWithFlags(ev[3], st, cudaEventRecordExternal);
}

void enqueue_rhs(const Plan& P, cudaStream_t st, const void* y, double* out, Gate g) {
  if (use_df(P)) {
    launch_bin_df(P, st, nullptr, static_cast<const float*>(y), g);
    exchange_sums(P, st, false);
    launch_pixel_solve_df(P, st, nullptr, g);
    launch_rescan_df(P, st, nullptr, static_cast<const float*>(y), out, g);
    return;
  }
  launch_bin_y(P, st, y, nullptr, g);
  exchange_sums(P, st, false);
  launch_pixel_solve(P, st, true, nullptr, g);
  launch_rescan_y(P, st, y, out, g);
}

void enqueue_map(const Plan& P, cudaStream_t st, const void* y, const double* a, double* out_map) {
  Gate g{nullptr, nullptr};
  if (use_df(P)) {
    if (a != nullptr) launch_split_df(P, st, a, g);
    launch_bin_df(P, st, a, static_cast<const float*>(y), g);
    exchange_sums(P, st, false);
    launch_pixel_solve_df(P, st, out_map, g);
    return;
  }
  launch_bin_y(P, st, y, a, g);
  exchange_sums(P, st, false);
  launch_pixel_solve(P, st, true, out_map, g);
}

}  // namespace ds
