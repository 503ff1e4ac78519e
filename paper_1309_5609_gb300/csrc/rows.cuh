// Rows w_o(t) of the pointing-and-rotation operator (Sect. 3, rotation matrices
// R_Q, R_U) in the map's component frame, with c = cos 2psi and s = sin 2psi:
//   I   : (1)          on I
//   q   : ( c, s)      on (Q, U)
//   u   : (-s, c)      on (Q, U)
//   iqu : (1, c, s)    on (I, Q, U)
// Component frame: NC = 1 -> (I); NC = 2 -> (Q, U); NC = 3 -> (I, Q, U).
#pragma once

#include <type_traits>

#include "internal.cuh"

namespace ds {

template <int NC>
struct Frame {
  static constexpr int I = (NC == 2) ? -1 : 0;
  static constexpr int Q = (NC == 1) ? -1 : NC - 2;
  static constexpr int U = (NC == 1) ? -1 : NC - 1;
};

// acc += w_kind * z  (the transpose of the row: what binning adds to the sums)
template <int NC, typename T>
__device__ __forceinline__ void row_bin(int kind, T c, T s, T z, T (&acc)[NC]) {
  using F = Frame<NC>;
  if (kind == DS_KIND_I) {
    if constexpr (F::I >= 0) acc[F::I] += z;
  } else if (kind == DS_KIND_Q) {
    if constexpr (F::Q >= 0) {
      acc[F::Q] = fma(c, z, acc[F::Q]);
      acc[F::U] = fma(s, z, acc[F::U]);
    }
  } else if (kind == DS_KIND_U) {
    if constexpr (F::Q >= 0) {
      acc[F::Q] = fma(-s, z, acc[F::Q]);
      acc[F::U] = fma(c, z, acc[F::U]);
    }
  } else {
    if constexpr (F::I >= 0 && F::Q >= 0) {
      acc[F::I] += z;
      acc[F::Q] = fma(c, z, acc[F::Q]);
      acc[F::U] = fma(s, z, acc[F::U]);
    }
  }
}

// The row of output `kind` averaged over some samples, from their moments
// (m1 = the samples' share, mc and ms = their cos 2psi and sin 2psi sums, all
// divided by the same count): every row is linear in (1, c, s), so these three
// numbers give the average row of each output kind.
template <int NC>
__device__ __forceinline__ void row_moments(int kind, float m1, float mc, float ms, float (&v)[NC]) {
  using F = Frame<NC>;
#pragma unroll
  for (int j = 0; j < NC; ++j) v[j] = 0.f;
  if (kind == DS_KIND_I) {
    if constexpr (F::I >= 0) v[F::I] = m1;
  } else if (kind == DS_KIND_Q) {
    if constexpr (F::Q >= 0) { v[F::Q] = mc; v[F::U] = ms; }
  } else if (kind == DS_KIND_U) {
    if constexpr (F::Q >= 0) { v[F::Q] = -ms; v[F::U] = mc; }
  } else {
    if constexpr (F::I >= 0 && F::Q >= 0) { v[F::I] = m1; v[F::Q] = mc; v[F::U] = ms; }
  }
}

// w_kind . m  (what rescanning the map gives for this output)
template <int NC, typename T>
__device__ __forceinline__ T row_dot(int kind, T c, T s, const T (&m)[NC]) {
  using F = Frame<NC>;
  if (kind == DS_KIND_I) {
    if constexpr (F::I >= 0) return m[F::I];
  } else if (kind == DS_KIND_Q) {
    if constexpr (F::Q >= 0) return fma(c, m[F::Q], s * m[F::U]);
  } else if (kind == DS_KIND_U) {
    if constexpr (F::Q >= 0) return fma(c, m[F::U], -s * m[F::Q]);
  } else {
    if constexpr (F::I >= 0 && F::Q >= 0) return m[F::I] + fma(c, m[F::Q], s * m[F::U]);
  }
  return T(0);
}

// Kind sets: number of outputs / components and the kind of output o.
template <int KS> struct KSet;
template <> struct KSet<KS_QU> {
  static constexpr int NC = 2, NO = 2;
  __device__ static constexpr int n_o(const KindsArg&) { return 2; }
  __device__ static constexpr int kind(int o, const KindsArg&) { return o == 0 ? DS_KIND_Q : DS_KIND_U; }
};
template <> struct KSet<KS_IQU3> {
  static constexpr int NC = 3, NO = 3;
  __device__ static constexpr int n_o(const KindsArg&) { return 3; }
  __device__ static constexpr int kind(int o, const KindsArg&) {
    return o == 0 ? DS_KIND_I : (o == 1 ? DS_KIND_Q : DS_KIND_U);
  }
};
template <> struct KSet<KS_IQU1> {
  static constexpr int NC = 3, NO = 1;
  __device__ static constexpr int n_o(const KindsArg&) { return 1; }
  __device__ static constexpr int kind(int, const KindsArg&) { return DS_KIND_IQU; }
};
template <> struct KSet<KS_I> {
  static constexpr int NC = 1, NO = 1;
  __device__ static constexpr int n_o(const KindsArg&) { return 1; }
  __device__ static constexpr int kind(int, const KindsArg&) { return DS_KIND_I; }
};
template <int NC_> struct KSetGen {
  static constexpr int NC = NC_, NO = DS_MAX_OUTPUTS;
  __device__ static int n_o(const KindsArg& k) { return k.n_o; }
  __device__ static int kind(int o, const KindsArg& k) { return k.kind[o]; }
};
template <> struct KSet<KS_QU12> {
  static constexpr int NC = 2, NO = 2;
  __device__ static int n_o(const KindsArg& k) { return k.n_o; }
  __device__ static int kind(int o, const KindsArg& k) { return k.kind[o]; }
};
template <> struct KSet<KS_GEN1> : KSetGen<1> {};
template <> struct KSet<KS_GEN2> : KSetGen<2> {};
template <> struct KSet<KS_GEN3> : KSetGen<3> {};

// Calls f(std::integral_constant<int, KS>{}) for the run-time kind set ks, so that
// kernels are instantiated per kind set and chosen on the host.
template <typename F>
void with_kindset(int ks, F&& f) {
  switch (ks) {
    case KS_QU: f(std::integral_constant<int, KS_QU>{}); break;
    case KS_IQU3: f(std::integral_constant<int, KS_IQU3>{}); break;
    case KS_IQU1: f(std::integral_constant<int, KS_IQU1>{}); break;
    case KS_I: f(std::integral_constant<int, KS_I>{}); break;
    case KS_QU12: f(std::integral_constant<int, KS_QU12>{}); break;
    case KS_GEN1: f(std::integral_constant<int, KS_GEN1>{}); break;
    case KS_GEN2: f(std::integral_constant<int, KS_GEN2>{}); break;
    default: f(std::integral_constant<int, KS_GEN3>{}); break;
  }
}

// Packed symmetric inverse times a vector: m = Minv s.
template <int NC>
__device__ __forceinline__ void sym_mul(const double* __restrict__ mi, const double (&s)[NC],
                                        double (&m)[NC]) {
  if constexpr (NC == 1) {
    m[0] = mi[0] * s[0];
  } else if constexpr (NC == 2) {
    m[0] = mi[0] * s[0] + mi[1] * s[1];
    m[1] = mi[1] * s[0] + mi[2] * s[1];
  } else {
    m[0] = mi[0] * s[0] + mi[1] * s[1] + mi[2] * s[2];
    m[1] = mi[1] * s[0] + mi[3] * s[1] + mi[4] * s[2];
    m[2] = mi[2] * s[0] + mi[4] * s[1] + mi[5] * s[2];
  }
}

// Streaming loads that skip L1 allocation (read-once pointing data).
__device__ __forceinline__ int4 ld_stream(const int4* p) { return __ldcs(p); }
__device__ __forceinline__ float4 ld_stream(const float4* p) { return __ldcs(p); }

}  // namespace ds
