// Chunk-local pixel index and the float32 operator passes that use it.
//
// The timeline is cut into chunks of C consecutive samples (C a power of two,
// 2048-16384).  At plan time every chunk gets
//   upix[c0 + u]  its distinct kept pixels, sorted (u < ucnt[chunk])
//   lid[t]        per sample, the rank u of its pixel in that list (uint16),
//                 or 0xFFFF when the sample has weight 0 (flagged, cut or past n_t).
// The per-iteration passes then read 2 bytes of pixel index per sample instead
// of 4, and keep the chunk's pixels in shared memory:
//   binning  adds each sample's w z into shared per-chunk sums (one shared
//            atomic per run of equal pixels), then adds the chunk's sums to the
//            float32 pixel sums with one vector reduction per distinct pixel,
//            in sorted pixel order (neighbouring addresses);
//   rescan   stages the chunk's map values from the float32 map into shared
//            memory in sorted order, so the per-sample map reads are shared
//            memory loads instead of scattered global gathers.
// This is the same operator (Sect. 3: P~^T R^T binning, R P~ rescan); only the
// order of the float32 additions changes.
#include <type_traits>

#include "internal.cuh"
#include "rows.cuh"
#include "stream_common.cuh"

namespace ds {

namespace {

constexpr uint16_t kNoPix = 0xFFFF;
constexpr int kBuildThreads = 1024;

// ---- plan time: sort each chunk's (pixel, position) keys, rank the distinct pixels
// One block per chunk.  Keys are (pixel << 32 | position in chunk); weight-0
// samples carry pixel 0xFFFFFFFF and sort last.  Bitonic sort in shared memory.
template <int C>
__global__ void __launch_bounds__(kBuildThreads) k_ck_build(const int32_t* __restrict__ pix,
                                                            int64_t n_t, int64_t n_chunks,
                                                            uint16_t* __restrict__ lid,
                                                            int32_t* __restrict__ upix,
                                                            int32_t* __restrict__ ucnt,
                                                            unsigned long long* __restrict__ umax) {
  extern __shared__ unsigned long long keys[];
  __shared__ int wsum[kBuildThreads / 32];
  constexpr int E = C / kBuildThreads;  // sorted positions per thread in the ranking
  constexpr unsigned kInv = 0xFFFFFFFFu;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  for (int64_t ch = blockIdx.x; ch < n_chunks; ch += gridDim.x) {
    const int64_t c0 = ch * C;
    for (int i = tid; i < C; i += kBuildThreads) {
      const int64_t t = c0 + i;
      const int p = t < n_t ? pix[t] : -1;
      const unsigned hi = p >= 0 ? (unsigned)p : kInv;
      keys[i] = ((unsigned long long)hi << 32) | (unsigned)i;
    }
    __syncthreads();
    for (int k = 2; k <= C; k <<= 1) {
      for (int j = k >> 1; j > 0; j >>= 1) {
        for (int q = tid; q < C / 2; q += kBuildThreads) {
          const int i = 2 * q - (q & (j - 1));
          const unsigned long long a = keys[i], b = keys[i + j];
          if ((a > b) == ((i & k) == 0)) {
            keys[i] = b;
            keys[i + j] = a;
          }
        }
        __syncthreads();
      }
    }
    // distinct pixels: a sorted position starts a new one when its pixel differs
    // from the previous position's
    int cnt = 0;
#pragma unroll
    for (int e = 0; e < E; ++e) {
      const int i = tid * E + e;
      const unsigned hi = (unsigned)(keys[i] >> 32);
      if (hi != kInv && (i == 0 || (unsigned)(keys[i - 1] >> 32) != hi)) ++cnt;
    }
    int v = cnt;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const int n = __shfl_up_sync(0xffffffffu, v, d);
      if (lane >= d) v += n;
    }
    if (lane == 31) wsum[warp] = v;
    __syncthreads();
    if (warp == 0) {
      int w = wsum[lane];
#pragma unroll
      for (int d = 1; d < 32; d <<= 1) {
        const int n = __shfl_up_sync(0xffffffffu, w, d);
        if (lane >= d) w += n;
      }
      wsum[lane] = w;
    }
    __syncthreads();
    int rank = (warp > 0 ? wsum[warp - 1] : 0) + v - cnt - 1;
    const int total = wsum[kBuildThreads / 32 - 1];
#pragma unroll
    for (int e = 0; e < E; ++e) {
      const int i = tid * E + e;
      const unsigned hi = (unsigned)(keys[i] >> 32);
      const int pos = (int)(keys[i] & 0xFFFFFFFFu);
      if (hi != kInv) {
        if (i == 0 || (unsigned)(keys[i - 1] >> 32) != hi) {
          ++rank;
          upix[c0 + rank] = (int32_t)hi;
        }
        lid[c0 + pos] = (uint16_t)rank;
      } else {
        lid[c0 + pos] = kNoPix;
      }
    }
    if (tid == 0) {
      ucnt[ch] = total;
      atomicMax(umax, (unsigned long long)total);
    }
    __syncthreads();
  }
}

// Eight consecutive samples from t0 (a multiple of 8): chunk-local indices,
// cos 2psi and sin 2psi; samples past n_t read as weight 0.
__device__ __forceinline__ void load8(const uint16_t* __restrict__ lid,
                                      const float* __restrict__ cc, const float* __restrict__ ss,
                                      int64_t t0, int64_t n_t, uint16_t (&u)[8], float (&c)[8],
                                      float (&s)[8]) {
  const uint4 l4 = __ldcs(reinterpret_cast<const uint4*>(lid + t0));
  const uint32_t lw[4] = {l4.x, l4.y, l4.z, l4.w};
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    u[2 * k] = (uint16_t)(lw[k] & 0xFFFFu);
    u[2 * k + 1] = (uint16_t)(lw[k] >> 16);
  }
  if (t0 + 8 <= n_t) {
    const float4 c0 = __ldcs(reinterpret_cast<const float4*>(cc + t0));
    const float4 c1 = __ldcs(reinterpret_cast<const float4*>(cc + t0) + 1);
    const float4 s0 = __ldcs(reinterpret_cast<const float4*>(ss + t0));
    const float4 s1 = __ldcs(reinterpret_cast<const float4*>(ss + t0) + 1);
    c[0] = c0.x; c[1] = c0.y; c[2] = c0.z; c[3] = c0.w;
    c[4] = c1.x; c[5] = c1.y; c[6] = c1.z; c[7] = c1.w;
    s[0] = s0.x; s[1] = s0.y; s[2] = s0.z; s[3] = s0.w;
    s[4] = s1.x; s[5] = s1.y; s[6] = s1.z; s[7] = s1.w;
  } else {
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      const bool in = t0 + k < n_t;
      c[k] = in ? cc[t0 + k] : 0.f;
      s[k] = in ? ss[t0 + k] : 0.f;
    }
  }
}

// Every thread owns two 8-sample groups of a chunk (blockDim = C / 16) and
// issues the loads of both before using either, so that a chunk's pointing is in
// flight at once; per-chunk gathers (pixel list, map) are batched the same way.
constexpr int kGroupsPerThread = 2;

// Binning of one 8-sample group into the shared sums (weight-0 samples skipped).
template <int KS>
__device__ __forceinline__ void bin_group(const uint16_t (&u)[8], const float (&c)[8],
                                          const float (&s)[8], int64_t t0, int64_t L,
                                          int64_t n_b, const double* __restrict__ x,
                                          float* __restrict__ sb, int ustride,
                                          const KindsArg& kk) {
  using K = KSet<KS>;
  constexpr int NC = K::NC, NO = K::NO;
  const int n_o = K::n_o(kk);
  int64_t b = t0 / L;
  int64_t bend = (b + 1) * L;
  float zb[NO];
#pragma unroll
  for (int o = 0; o < NO; ++o) zb[o] = o < n_o ? (float)__ldg(x + o * n_b + b) : 0.f;
  float acc[NC];
#pragma unroll
  for (int j = 0; j < NC; ++j) acc[j] = 0.f;
  int cur = kNoPix;
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    if (t0 + k >= bend) {
      b += 1;
      bend += L;
      if (b < n_b) {
#pragma unroll
        for (int o = 0; o < NO; ++o) zb[o] = o < n_o ? (float)__ldg(x + o * n_b + b) : 0.f;
      }
    }
    if (u[k] == kNoPix) continue;
    float w[NC];
#pragma unroll
    for (int j = 0; j < NC; ++j) w[j] = 0.f;
#pragma unroll
    for (int o = 0; o < NO; ++o)
      if (o < n_o) row_bin<NC, float>(K::kind(o, kk), c[k], s[k], zb[o], w);
    if (u[k] != cur) {
      if (cur != kNoPix) {
#pragma unroll
        for (int j = 0; j < NC; ++j) atomicAdd(sb + j * ustride + cur, acc[j]);
      }
      cur = u[k];
#pragma unroll
      for (int j = 0; j < NC; ++j) acc[j] = w[j];
    } else {
#pragma unroll
      for (int j = 0; j < NC; ++j) acc[j] += w[j];
    }
  }
  if (cur != kNoPix) {
#pragma unroll
    for (int j = 0; j < NC; ++j) atomicAdd(sb + j * ustride + cur, acc[j]);
  }
}

// ---- binning of F~ x into the float32 pixel sums ----------------------------------
// Shared sums are component-major [NC][ustride]; they are zero on entry to every
// chunk (cleared at start, then by the flush that reads them).
template <int KS>
__global__ void __launch_bounds__(1024) k_ck_bin(const uint16_t* __restrict__ lid,
                                                const int32_t* __restrict__ upix,
                                                const int32_t* __restrict__ ucnt,
                                                const float* __restrict__ cc,
                                                const float* __restrict__ ss,
                                                const double* __restrict__ x,
                                                float* __restrict__ bins, int64_t n_t, int64_t L,
                                                int64_t n_b, int C, int64_t n_chunks, int ustride,
                                                KindsArg kk, Gate g) {
  if (gate_closed(g)) return;
  extern __shared__ float sb[];
  constexpr int NC = KSet<KS>::NC;
  const int nthr = blockDim.x;
  for (int i = threadIdx.x; i < NC * ustride; i += nthr) sb[i] = 0.f;
  __syncthreads();
  for (int64_t ch = blockIdx.x; ch < n_chunks; ch += gridDim.x) {
    const int64_t c0 = ch * (int64_t)C;
    const int64_t ta = c0 + ((int64_t)threadIdx.x << 3);
    const int64_t tb = ta + ((int64_t)nthr << 3);
    uint16_t ua[8], ub[8];
    float ca[8], sa[8], cb[8], sbv[8];
    if (ta < n_t) load8(lid, cc, ss, ta, n_t, ua, ca, sa);
    if (tb < n_t) load8(lid, cc, ss, tb, n_t, ub, cb, sbv);
    const int U = ucnt[ch];
    if (ta < n_t) bin_group<KS>(ua, ca, sa, ta, L, n_b, x, sb, ustride, kk);
    if (tb < n_t) bin_group<KS>(ub, cb, sbv, tb, L, n_b, x, sb, ustride, kk);
    __syncthreads();
    // one vector reduction per distinct pixel, four pixels' indices fetched together
    for (int i0 = threadIdx.x; i0 < U; i0 += 4 * nthr) {
      int pp[4];
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const int i = i0 + k * nthr;
        pp[k] = i < U ? __ldg(upix + c0 + i) : -1;
      }
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const int i = i0 + k * nthr;
        if (pp[k] < 0) continue;
        float v[NC];
#pragma unroll
        for (int j = 0; j < NC; ++j) {
          v[j] = sb[j * ustride + i];
          sb[j * ustride + i] = 0.f;
        }
        flush_bins<NC, float>(bins, pp[k], v);
      }
    }
    __syncthreads();
  }
}

// Rescan of one group against the shared map, per-baseline sums of the residual.
template <int KS>
__device__ __forceinline__ void rescan_group(const uint16_t (&u)[8], const float (&c)[8],
                                             const float (&s)[8], int64_t t0, int64_t n_t,
                                             int64_t L, int64_t n_b,
                                             const double* __restrict__ x,
                                             const float* __restrict__ sm, int ustride,
                                             double* __restrict__ out, const KindsArg& kk) {
  using K = KSet<KS>;
  constexpr int NC = K::NC, NO = K::NO;
  const int n_o = K::n_o(kk);
  int key = -1;
  float acc[NO];
#pragma unroll
  for (int o = 0; o < NO; ++o) acc[o] = 0.f;
  if (t0 < n_t) {
    int64_t b = t0 / L;
    int64_t bend = (b + 1) * L;
    float zb[NO];
#pragma unroll
    for (int o = 0; o < NO; ++o) zb[o] = o < n_o ? (float)__ldg(x + o * n_b + b) : 0.f;
    key = (int)b;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      const int64_t t = t0 + k;
      if (t >= n_t) break;
      if (t >= bend) {
#pragma unroll
        for (int o = 0; o < NO; ++o) {
          if (o < n_o && acc[o] != 0.f) atomicAdd(out + o * n_b + b, (double)acc[o]);
          acc[o] = 0.f;
        }
        b += 1;
        bend += L;
        key = (int)b;
#pragma unroll
        for (int o = 0; o < NO; ++o) zb[o] = o < n_o ? (float)__ldg(x + o * n_b + b) : 0.f;
      }
      if (u[k] == kNoPix) continue;
      float m[NC];
#pragma unroll
      for (int j = 0; j < NC; ++j) m[j] = sm[j * ustride + u[k]];
#pragma unroll
      for (int o = 0; o < NO; ++o)
        if (o < n_o) acc[o] += zb[o] - row_dot<NC, float>(K::kind(o, kk), c[k], s[k], m);
    }
  }
  warp_segment_flush<NO, float>(key, acc, n_o, out, n_b);
}

// ---- rescan of the float32 map and per-baseline sums of the residual -------------
// out[o][b] += sum_{t in b} v (x[o][b] - w_o(t) . m_p(t)); shared map [NC][ustride].
template <int KS>
__global__ void __launch_bounds__(1024) k_ck_rescan(const uint16_t* __restrict__ lid,
                                                   const int32_t* __restrict__ upix,
                                                   const int32_t* __restrict__ ucnt,
                                                   const float* __restrict__ cc,
                                                   const float* __restrict__ ss,
                                                   const double* __restrict__ x,
                                                   const float* __restrict__ map,
                                                   double* __restrict__ out, int64_t n_t,
                                                   int64_t L, int64_t n_b, int C,
                                                   int64_t n_chunks, int ustride, KindsArg kk,
                                                   Gate g) {
  if (gate_closed(g)) return;
  extern __shared__ float sm[];
  constexpr int NC = KSet<KS>::NC;
  const int nthr = blockDim.x;
  for (int64_t ch = blockIdx.x; ch < n_chunks; ch += gridDim.x) {
    const int64_t c0 = ch * (int64_t)C;
    const int64_t ta = c0 + ((int64_t)threadIdx.x << 3);
    const int64_t tb = ta + ((int64_t)nthr << 3);
    uint16_t ua[8], ub[8];
    float ca[8], sa[8], cb[8], sbv[8];
    if (ta < n_t) load8(lid, cc, ss, ta, n_t, ua, ca, sa);
    if (tb < n_t) load8(lid, cc, ss, tb, n_t, ub, cb, sbv);
    const int U = ucnt[ch];
    for (int i0 = threadIdx.x; i0 < U; i0 += 4 * nthr) {
      int pp[4];
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const int i = i0 + k * nthr;
        pp[k] = i < U ? __ldg(upix + c0 + i) : -1;
      }
      float m[4][NC];
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        if (pp[k] >= 0) {
          load_map<NC, float>(map, pp[k], m[k]);
        } else {
#pragma unroll
          for (int j = 0; j < NC; ++j) m[k][j] = 0.f;
        }
      }
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const int i = i0 + k * nthr;
        if (i < U) {
#pragma unroll
          for (int j = 0; j < NC; ++j) sm[j * ustride + i] = m[k][j];
        }
      }
    }
    __syncthreads();
    rescan_group<KS>(ua, ca, sa, ta, n_t, L, n_b, x, sm, ustride, out, kk);
    rescan_group<KS>(ub, cb, sbv, tb, n_t, L, n_b, x, sm, ustride, out, kk);
    __syncthreads();
  }
}

template <int C>
cudaError_t build_with(Plan& P, unsigned long long* umax) {
  const size_t smem = sizeof(unsigned long long) * C;
  cudaError_t e = cudaFuncSetAttribute(k_ck_build<C>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  const int64_t grid = P.ck_nchunks < (int64_t)P.num_sms * 2 ? P.ck_nchunks : (int64_t)P.num_sms * 2;
  k_ck_build<C><<<(int)grid, kBuildThreads, smem, P.stream>>>(P.pix, P.n_t, P.ck_nchunks, P.lid,
                                                              P.upix, P.ucnt, umax);
  return cudaGetLastError();
}

// Threads per block and resident blocks of the two passes for this plan's
// shared-memory size.  The dynamic shared-memory limit is an attribute of the
// kernel, shared by every plan: it is raised to the device's opt-in maximum
// (a plan needing less must not lower it under another plan's launches).
cudaError_t ck_configure(Plan& P) {
  const size_t smem = sizeof(float) * (size_t)P.n_c * P.ck_ustride;
  int optin = 0;
  cudaError_t e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, P.device);
  if (e != cudaSuccess) return e;
  if (smem > (size_t)optin) return cudaErrorInvalidValue;
  int nb = 1, nr = 1;
  with_kindset(P.kindset, [&](auto ksc) {
    constexpr int KS = decltype(ksc)::value;
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(k_ck_bin<KS>, cudaFuncAttributeMaxDynamicSharedMemorySize, optin);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(k_ck_rescan<KS>, cudaFuncAttributeMaxDynamicSharedMemorySize, optin);
    if (e == cudaSuccess)
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_ck_bin<KS>, P.ck_threads, smem);
    if (e == cudaSuccess)
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nr, k_ck_rescan<KS>, P.ck_threads, smem);
  });
  if (e != cudaSuccess) return e;
  P.ck_bin_blocks = nb > 0 ? nb : 1;
  P.ck_rescan_blocks = nr > 0 ? nr : 1;
  return cudaSuccess;
}

int ck_grid(const Plan& P, int per_sm) {
  const int64_t cap = (int64_t)P.num_sms * per_sm;
  return (int)(P.ck_nchunks < cap ? P.ck_nchunks : cap);
}

}  // namespace

int ck_default_chunk(int64_t n_t, int num_sms) {
  int C = 8192;
  while (C > 2048 && (n_t + C - 1) / C < 8 * (int64_t)num_sms) C >>= 1;
  return C;
}

// Builds the index for chunk length C on the plan's stream; *umax (device) gets
// the largest number of distinct pixels in a chunk.  P.pix must be final.
cudaError_t ck_build(Plan& P, int C, unsigned long long* umax) {
  if (P.lid == nullptr) return cudaErrorInvalidValue;
  P.ck_C = C;
  P.ck_nchunks = (P.n_t + C - 1) / C;
  switch (C) {
    case 2048: return build_with<2048>(P, umax);
    case 4096: return build_with<4096>(P, umax);
    case 8192: return build_with<8192>(P, umax);
    case 16384: return build_with<16384>(P, umax);
    default: return cudaErrorInvalidValue;
  }
}

// After the build has completed: size the shared arrays from the largest chunk.
cudaError_t ck_finish(Plan& P, int64_t umax) {
  P.ck_umax = (int)umax;
  P.ck_ustride = (int)((umax + 32) & ~int64_t(31));  // >= umax + 1, a multiple of 32
  P.ck_threads = P.ck_C / (8 * kGroupsPerThread);
  return ck_configure(P);
}

bool ck_ready(const Plan& P) { return P.lid != nullptr && P.layout == 1 && P.ck_bin_blocks > 0; }

void launch_bin_ck(const Plan& P, cudaStream_t st, const double* x, Gate g) {
  const size_t smem = sizeof(float) * (size_t)P.n_c * P.ck_ustride;
  const int grid = ck_grid(P, P.ck_bin_blocks);
  with_kindset(P.kindset, [&](auto ksc) {
    constexpr int KS = decltype(ksc)::value;
    k_ck_bin<KS><<<grid, P.ck_threads, smem, st>>>(P.lid, P.upix, P.ucnt, P.c, P.s, x, P.bins32,
                                                   P.n_t, P.L, P.n_b, P.ck_C, P.ck_nchunks,
                                                   P.ck_ustride, P.kinds, g);
  });
}

void launch_rescan_ck(const Plan& P, cudaStream_t st, const double* x, double* out, Gate g) {
  const size_t smem = sizeof(float) * (size_t)P.n_c * P.ck_ustride;
  const int grid = ck_grid(P, P.ck_rescan_blocks);
  with_kindset(P.kindset, [&](auto ksc) {
    constexpr int KS = decltype(ksc)::value;
    k_ck_rescan<KS><<<grid, P.ck_threads, smem, st>>>(P.lid, P.upix, P.ucnt, P.c, P.s, x, P.map32,
                                                      out, P.n_t, P.L, P.n_b, P.ck_C,
                                                      P.ck_nchunks, P.ck_ustride, P.kinds, g);
  });
}

}  // namespace ds
