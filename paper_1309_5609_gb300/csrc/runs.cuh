// Device helpers of the run-length operator shared by the single-problem and
// batched passes: a run (pixel, count n, C = sum cos 2psi, S = sum sin 2psi)
// enters every row of Sect. 3 through (n, C, S).
#pragma once

#include "df.cuh"
#include "internal.cuh"
#include "rows.cuh"

namespace ds {

// acc += (row of one output summed over the run) * z
template <int NC>
__device__ __forceinline__ void run_bin(int kind, float n, float C, float S, float z,
                                        float (&acc)[NC]) {
  using F = Frame<NC>;
  if (kind == DS_KIND_I) {
    if constexpr (F::I >= 0) acc[F::I] = fmaf(n, z, acc[F::I]);
  } else if (kind == DS_KIND_Q) {
    if constexpr (F::Q >= 0) {
      acc[F::Q] = fmaf(C, z, acc[F::Q]);
      acc[F::U] = fmaf(S, z, acc[F::U]);
    }
  } else if (kind == DS_KIND_U) {
    if constexpr (F::Q >= 0) {
      acc[F::Q] = fmaf(-S, z, acc[F::Q]);
      acc[F::U] = fmaf(C, z, acc[F::U]);
    }
  } else {
    if constexpr (F::I >= 0 && F::Q >= 0) {
      acc[F::I] = fmaf(n, z, acc[F::I]);
      acc[F::Q] = fmaf(C, z, acc[F::Q]);
      acc[F::U] = fmaf(S, z, acc[F::U]);
    }
  }
}

// (row of one output summed over the run) . m
template <int NC>
__device__ __forceinline__ float run_dot(int kind, float n, float C, float S, const float (&m)[NC]) {
  using F = Frame<NC>;
  if (kind == DS_KIND_I) {
    if constexpr (F::I >= 0) return n * m[F::I];
  } else if (kind == DS_KIND_Q) {
    if constexpr (F::Q >= 0) return fmaf(C, m[F::Q], S * m[F::U]);
  } else if (kind == DS_KIND_U) {
    if constexpr (F::Q >= 0) return fmaf(C, m[F::U], -S * m[F::Q]);
  } else {
    if constexpr (F::I >= 0 && F::Q >= 0) return fmaf(n, m[F::I], fmaf(C, m[F::Q], S * m[F::U]));
  }
  return 0.f;
}

__device__ __forceinline__ RunRec load_run(const RunRec* __restrict__ rec, int64_t i) {
  const int4 v = __ldcs(reinterpret_cast<const int4*>(rec) + i);
  return RunRec{v.x, __int_as_float(v.y), __int_as_float(v.z), __int_as_float(v.w)};
}

// acc += w_kind-run sums * z: I n z, q (C z, S z), u (-S z, C z)
template <int NC>
__device__ __forceinline__ void run_bin_ds(int kind, float n, df C, df S, df z, dsum (&acc)[NC]) {
  using F = Frame<NC>;
  if (kind == DS_KIND_I) {
    if constexpr (F::I >= 0) ds_add_prod(acc[F::I], z, n);
  } else if (kind == DS_KIND_Q) {
    if constexpr (F::Q >= 0) {
      ds_add_prod(acc[F::Q], z, C);
      ds_add_prod(acc[F::U], z, S);
    }
  } else if (kind == DS_KIND_U) {
    if constexpr (F::Q >= 0) {
      ds_add_prod(acc[F::Q], z, df_neg(S));
      ds_add_prod(acc[F::U], z, C);
    }
  } else {
    if constexpr (F::I >= 0 && F::Q >= 0) {
      ds_add_prod(acc[F::I], z, n);
      ds_add_prod(acc[F::Q], z, C);
      ds_add_prod(acc[F::U], z, S);
    }
  }
}

}  // namespace ds
