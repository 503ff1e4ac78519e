// Device helpers shared by the single-problem and batched streaming kernels:
// 4-sample vector loads of the pointing, run flushes into pixel sums, map
// gathers and the warp-segmented per-baseline sum.
#pragma once

#include <type_traits>

#include "df.cuh"
#include "internal.cuh"
#include "rows.cuh"

namespace ds {

// Load 4 samples starting at t0 = 4 v; samples past n_t get pixel -1.
__device__ __forceinline__ void load4(const int32_t* __restrict__ pix, const float* __restrict__ cc,
                                      const float* __restrict__ ss, int64_t v, int64_t n_t,
                                      int (&p)[4], float (&c)[4], float (&s)[4]) {
  const int64_t t0 = v << 2;
  if (t0 + 4 <= n_t) {
    const int4 pp = ld_stream(reinterpret_cast<const int4*>(pix) + v);
    const float4 c4 = ld_stream(reinterpret_cast<const float4*>(cc) + v);
    const float4 s4 = ld_stream(reinterpret_cast<const float4*>(ss) + v);
    p[0] = pp.x; p[1] = pp.y; p[2] = pp.z; p[3] = pp.w;
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
}

// Value for a float64 atomic: float32 sums are widened by bit re-encoding
// (f64_of_f32), which keeps the conversion off the narrow float64 pipe.
__device__ __forceinline__ double to_f64(float v) { return f64_of_f32(v); }
__device__ __forceinline__ double to_f64(double v) { return v; }

template <int NC, typename T>
__device__ __forceinline__ void flush_bins(double* __restrict__ bins, int p, const T (&acc)[NC]) {
  double* dst = bins + (int64_t)p * 4;
#pragma unroll
  for (int j = 0; j < NC; ++j) atomicAdd(dst + j, (double)acc[j]);
}

// One vector reduction (red.global.add.v4.f32) adds all components of a run to
// the float32 pixel sums; a single L2 atomic operation instead of NC.
template <int NC, typename T>
__device__ __forceinline__ void flush_bins(float* __restrict__ bins, int p, const T (&acc)[NC]) {
  float v[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
  for (int j = 0; j < NC; ++j) v[j] = (float)acc[j];
  float* dst = bins + (int64_t)p * 4;
  asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(dst), "f"(v[0]), "f"(v[1]),
               "f"(v[2]), "f"(v[3])
               : "memory");
}

template <int NC, typename T>
__device__ __forceinline__ void load_map(const T* __restrict__ map, int p, T (&m)[NC]) {
  if constexpr (std::is_same<T, float>::value) {
    const float4 v = __ldg(reinterpret_cast<const float4*>(map) + p);
    const float a[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
    for (int j = 0; j < NC; ++j) m[j] = a[j];
  } else {
    const double2 v0 = __ldg(reinterpret_cast<const double2*>(map) + 2 * (int64_t)p);
    m[0] = v0.x;
    if constexpr (NC > 1) m[1] = v0.y;
    if constexpr (NC > 2) m[2] = __ldg(map + 4 * (int64_t)p + 2);
  }
}

// Segmented sum across the warp of per-lane partials keyed by baseline index
// (keys non-decreasing with the lane; -1 = nothing).  The first lane of every
// run of equal keys adds the run total to out[o * n_b + key].
template <int NO, typename T>
__device__ __forceinline__ void warp_segment_flush(int key, T (&val)[NO], int n_o,
                                                   double* __restrict__ out, int64_t n_b) {
  const unsigned full = 0xffffffffu;
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const int k2 = __shfl_down_sync(full, key, d);
#pragma unroll
    for (int o = 0; o < NO; ++o) {
      const T v2 = __shfl_down_sync(full, val[o], d);
      if (lane + d < 32 && k2 == key) val[o] += v2;
    }
  }
  const int kp = __shfl_up_sync(full, key, 1);
  if (key >= 0 && (lane == 0 || kp != key)) {
#pragma unroll
    for (int o = 0; o < NO; ++o)
      if (o < n_o) atomicAdd(out + (int64_t)o * n_b + key, to_f64(val[o]));
  }
}

}  // namespace ds
