// Double-float helpers shared by the single-problem and batched accurate passes:
// rows applied to double-float values, 4-sample loads, flushes into float64
// pixel sums and the warp-segmented per-baseline sum.
#pragma once

#include "df.cuh"
#include "internal.cuh"
#include "rows.cuh"

namespace ds {

// acc += w_kind * z in double-float
template <int NC>
__device__ __forceinline__ void row_bin_df(int kind, float c, float s, df z, df (&acc)[NC]) {
  using F = Frame<NC>;
  if (kind == DS_KIND_I) {
    if constexpr (F::I >= 0) acc[F::I] = df_add(acc[F::I], z);
  } else if (kind == DS_KIND_Q) {
    if constexpr (F::Q >= 0) {
      acc[F::Q] = df_add(acc[F::Q], df_mul_f(z, c));
      acc[F::U] = df_add(acc[F::U], df_mul_f(z, s));
    }
  } else if (kind == DS_KIND_U) {
    if constexpr (F::Q >= 0) {
      acc[F::Q] = df_sub(acc[F::Q], df_mul_f(z, s));
      acc[F::U] = df_add(acc[F::U], df_mul_f(z, c));
    }
  } else {
    if constexpr (F::I >= 0 && F::Q >= 0) {
      acc[F::I] = df_add(acc[F::I], z);
      acc[F::Q] = df_add(acc[F::Q], df_mul_f(z, c));
      acc[F::U] = df_add(acc[F::U], df_mul_f(z, s));
    }
  }
}

// w_kind . m in double-float
template <int NC>
__device__ __forceinline__ df row_dot_df(int kind, float c, float s, const df (&m)[NC]) {
  using F = Frame<NC>;
  if (kind == DS_KIND_I) {
    if constexpr (F::I >= 0) return m[F::I];
  } else if (kind == DS_KIND_Q) {
    if constexpr (F::Q >= 0) return df_add(df_mul_f(m[F::Q], c), df_mul_f(m[F::U], s));
  } else if (kind == DS_KIND_U) {
    if constexpr (F::Q >= 0) return df_sub(df_mul_f(m[F::U], c), df_mul_f(m[F::Q], s));
  } else {
    if constexpr (F::I >= 0 && F::Q >= 0)
      return df_add(m[F::I], df_add(df_mul_f(m[F::Q], c), df_mul_f(m[F::U], s)));
  }
  return df{0.f, 0.f};
}

__device__ __forceinline__ void load4_df(const int32_t* __restrict__ pix,
                                         const float* __restrict__ cc,
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

template <int NC>
__device__ __forceinline__ void flush_bins_df(double* __restrict__ bins, int p, const df (&acc)[NC]) {
  double* dst = bins + (int64_t)p * 4;
#pragma unroll
  for (int j = 0; j < NC; ++j) atomicAdd(dst + j, df_to_double(acc[j]));
}

template <int NO>
__device__ __forceinline__ void warp_segment_flush_df(int key, df (&val)[NO], int n_o,
                                                      double* __restrict__ out, int64_t n_b) {
  const unsigned full = 0xffffffffu;
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const int k2 = __shfl_down_sync(full, key, d);
#pragma unroll
    for (int o = 0; o < NO; ++o) {
      const df v2 = df_shfl_down(val[o], d);
      if (lane + d < 32 && k2 == key) val[o] = df_add(val[o], v2);
    }
  }
  const int kp = __shfl_up_sync(full, key, 1);
  if (key >= 0 && (lane == 0 || kp != key)) {
#pragma unroll
    for (int o = 0; o < NO; ++o)
      if (o < n_o) atomicAdd(out + (int64_t)o * n_b + key, df_to_double(val[o]));
  }
}

}  // namespace ds
