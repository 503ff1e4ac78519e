// Helpers shared by the single-problem and batched accurate passes: rows applied
// to double-float values in compensated sums (df.cuh), 4-sample loads, flushes
// into float64 pixel sums and the warp-segmented per-baseline sum.
#pragma once

#include "df.cuh"
#include "internal.cuh"
#include "rows.cuh"

namespace ds {

// A split baseline (hi, lo) through the read-only path
__device__ __forceinline__ df df_ldg(const float2* __restrict__ xs, int64_t i) {
  const float2 v = __ldg(xs + i);
  return df{v.x, v.y};
}

// acc += w_kind * z for a pair z (compensated sums)
template <int NC>
__device__ __forceinline__ void row_bin_ds(int kind, float c, float s, df z, dsum (&acc)[NC]) {
  using F = Frame<NC>;
  if (kind == DS_KIND_I) {
    if constexpr (F::I >= 0) ds_add(acc[F::I], z);
  } else if (kind == DS_KIND_Q) {
    if constexpr (F::Q >= 0) {
      ds_add_prod(acc[F::Q], z, c);
      ds_add_prod(acc[F::U], z, s);
    }
  } else if (kind == DS_KIND_U) {
    if constexpr (F::Q >= 0) {
      ds_add_prod(acc[F::Q], z, -s);
      ds_add_prod(acc[F::U], z, c);
    }
  } else {
    if constexpr (F::I >= 0 && F::Q >= 0) {
      ds_add(acc[F::I], z);
      ds_add_prod(acc[F::Q], z, c);
      ds_add_prod(acc[F::U], z, s);
    }
  }
}

// acc += w_kind * y for a float32 y (exact products)
template <int NC>
__device__ __forceinline__ void row_bin_ds(int kind, float c, float s, float y, dsum (&acc)[NC]) {
  using F = Frame<NC>;
  if (kind == DS_KIND_I) {
    if constexpr (F::I >= 0) ds_add(acc[F::I], y);
  } else if (kind == DS_KIND_Q) {
    if constexpr (F::Q >= 0) {
      ds_add_prod(acc[F::Q], y, c);
      ds_add_prod(acc[F::U], y, s);
    }
  } else if (kind == DS_KIND_U) {
    if constexpr (F::Q >= 0) {
      ds_add_prod(acc[F::Q], y, -s);
      ds_add_prod(acc[F::U], y, c);
    }
  } else {
    if constexpr (F::I >= 0 && F::Q >= 0) {
      ds_add(acc[F::I], y);
      ds_add_prod(acc[F::Q], y, c);
      ds_add_prod(acc[F::U], y, s);
    }
  }
}

// acc -= w_kind . m for a double-float map m
template <int NC>
__device__ __forceinline__ void row_sub_dot_ds(int kind, float c, float s, const df (&m)[NC],
                                               dsum& acc) {
  using F = Frame<NC>;
  if (kind == DS_KIND_I) {
    if constexpr (F::I >= 0) ds_add(acc, df_neg(m[F::I]));
  } else if (kind == DS_KIND_Q) {
    if constexpr (F::Q >= 0) {
      ds_add_prod(acc, m[F::Q], -c);
      ds_add_prod(acc, m[F::U], -s);
    }
  } else if (kind == DS_KIND_U) {
    if constexpr (F::Q >= 0) {
      ds_add_prod(acc, m[F::Q], s);
      ds_add_prod(acc, m[F::U], -c);
    }
  } else {
    if constexpr (F::I >= 0 && F::Q >= 0) {
      ds_add(acc, df_neg(m[F::I]));
      ds_add_prod(acc, m[F::Q], -c);
      ds_add_prod(acc, m[F::U], -s);
    }
  }
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
__device__ __forceinline__ void flush_bins_ds(double* __restrict__ bins, int p, const dsum (&acc)[NC]) {
  double* dst = bins + (int64_t)p * 4;
#pragma unroll
  for (int j = 0; j < NC; ++j) atomicAdd(dst + j, ds_to_double(acc[j]));
}

// Segmented sum across the warp of per-lane compensated partials keyed by
// baseline (each key's lanes contiguous, -1 for none); the first lane of every
// segment adds it to out[o][key] in float64.
template <int NO>
__device__ __forceinline__ void warp_segment_flush_ds(int key, dsum (&val)[NO], int n_o,
                                                      double* __restrict__ out, int64_t n_b) {
  const unsigned full = 0xffffffffu;
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int o = 0; o < NO; ++o) ds_norm(val[o]);
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const int k2 = __shfl_down_sync(full, key, d);
#pragma unroll
    for (int o = 0; o < NO; ++o) {
      const df v2 = df{__shfl_down_sync(full, val[o].hi, d), __shfl_down_sync(full, val[o].lo, d)};
      if (lane + d < 32 && k2 == key) ds_add(val[o], v2);
    }
  }
  const int kp = __shfl_up_sync(full, key, 1);
  if (key >= 0 && (lane == 0 || kp != key)) {
#pragma unroll
    for (int o = 0; o < NO; ++o)
      if (o < n_o) atomicAdd(out + (int64_t)o * n_b + key, ds_to_double(val[o]));
  }
}


}  // namespace ds
