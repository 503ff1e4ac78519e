// Two-level preconditioner of the destriping CG: construction of the coarse
// space and of its coarse matrix (the per-iteration kernels are in cg.cu).
//
// The paper solves the destriping equation (Sect. 3) with an unpreconditioned
// Krylov method (GMRES in Sect. 4, CG named as the alternative).  With short
// baselines the slow modes of A = F~^T Z F~ are baseline patterns that look like
// large-scale sky: offsets a with F~ a close to A_p m for a map m that is smooth
// over one baseline's sweep, which the map absorbs almost entirely.  A coarse
// space spans them.  The sphere is cut into cells (coarse_cell below), and the
// coarse column (k, c) holds, per baseline, the average over the baseline's
// valid samples of row component c restricted to the samples in cell k:
//
//     R[(o,b), (k,c)] = (1 / n_b) sum_{t in b, cell(p(t)) = k} v(t) w_{o,c}(t),
//
// the best baseline fit of the map that is 1 on component c of cell k.  A
// baseline keeps at most kPcSlots cells (the ones holding most of its samples;
// any R gives a valid preconditioner, and the coarse matrix below is built from
// the R actually stored).  Every row w_o is linear in (1, cos 2psi, sin 2psi), so
// a slot stores three numbers shared by all outputs (the cell's share of the
// baseline's valid samples and their cos and sin sums over the valid count) and
// each output's entries follow from its kind.  The preconditioner is additive:
//
//     z = D^-1 r + R E^+ R^T r,   D = diag(n_b),   E = R^T A R,
//
// with E = R^T D R - (K R)^T M^-1 (K R), K = A_p^T V F~: the first term from one
// pass over the baselines, the second from one pass over the pixel-major run
// records (one warp per pixel sums (K R)_p in registers and adds
// (K R)_p^T M_p^-1 (K R)_p into E).  E^+ is a generalised inverse by the sweep
// operator, skipping pivots that hold less than a 1e-6 share of their direction's
// R^T D R (null modes of A, where E is rounding noise); the I null mode (a common
// offset of the I-carrying outputs, which R reproduces) gets a rank-one term so
// that it is swept like the rest.
#include <climits>
#include <cmath>
#include <cstring>
#include <vector>

#include "df.cuh"
#include "internal.cuh"
#include "rows.cuh"

namespace ds {

namespace {

constexpr int kBlock = 256;
constexpr int kCand = 4;      // cells a baseline can hold while its samples are read
constexpr int kWarpCells = 8; // cells of one pixel's baselines merged per warp
constexpr int64_t kPcWarpRows = 256;  // baselines from this length get a warp each
constexpr double kPcKeptMin = 0.8;  // share of valid samples the kept slots must hold
constexpr double kPcPivotMin = 1e-6;  // share of diag(R^T D R) below which a pivot is skipped

// Floor of the square root of x >= 0 (exact for x < 2^52).
__device__ __forceinline__ int64_t isqrt64(int64_t x) {
  int64_t r = (int64_t)sqrtf((float)x);
  while (r * r > x) --r;
  while ((r + 1) * (r + 1) <= x) ++r;
  return r;
}

}  // namespace

// Coarse cell of a HEALPix RING pixel p at resolution nside.  Fine ring i goes
// to the nearest of the 4 nc - 1 coarse rings (the coarse ring k lies at the
// colatitude of fine ring k nside / nc), and within it to one of the coarse
// ring's sectors of equal longitude width (4k, 4nc or 4(4nc - k) of them, as in
// a HEALPix grid of resolution nc).  Cells are numbered ring by ring: 12 nc^2 in
// all, compact regions of about (60 / nc) degrees.
__host__ __device__ int coarse_cell(int64_t p, int64_t nside, int64_t nc) {
  const int64_t N = nside, npix = 12 * N * N, ncap = 2 * N * (N - 1);
  int64_t i, j, nring, twice_shift;
  if (p < ncap) {  // north cap: ring i has 4 i pixels, centres at (j + 1/2) 2 pi / 4i
#ifdef __CUDA_ARCH__
    i = (1 + isqrt64(1 + 2 * p)) >> 1;
#else
    i = (1 + (int64_t)std::sqrt((double)(1 + 2 * p))) >> 1;
    while (2 * i * (i - 1) > p) --i;
    while (2 * (i + 1) * i <= p) ++i;
#endif
    j = p - 2 * i * (i - 1);
    nring = 4 * i;
    twice_shift = 1;
  } else if (p < npix - ncap) {  // equatorial belt: 4N pixels, shift alternates
    const int64_t q = p - ncap;
    i = q / (4 * N) + N;
    j = q - (i - N) * 4 * N;
    nring = 4 * N;
    twice_shift = (i - N + 1) & 1;
  } else {  // south cap, mirrored
    const int64_t q = npix - 1 - p;
#ifdef __CUDA_ARCH__
    const int64_t ii = (1 + isqrt64(1 + 2 * q)) >> 1;
#else
    int64_t ii = (1 + (int64_t)std::sqrt((double)(1 + 2 * q))) >> 1;
    while (2 * ii * (ii - 1) > q) --ii;
    while (2 * (ii + 1) * ii <= q) ++ii;
#endif
    i = 4 * N - ii;
    j = 4 * ii - 1 - (q - 2 * ii * (ii - 1));
    nring = 4 * ii;
    twice_shift = 1;
  }
  int64_t k = (2 * i * nc + N) / (2 * N);
  if (k < 1) k = 1;
  if (k > 4 * nc - 1) k = 4 * nc - 1;
  int64_t nk, off;
  if (k < nc) {
    nk = 4 * k;
    off = 2 * k * (k - 1);
  } else if (k <= 3 * nc) {
    nk = 4 * nc;
    off = 2 * nc * (nc - 1) + (k - nc) * 4 * nc;
  } else {
    const int64_t kk = 4 * nc - k;
    nk = 4 * kk;
    off = 12 * nc * nc - 2 * kk * (kk + 1);
  }
  int64_t sec = ((2 * j + twice_shift) * nk) / (2 * nring);
  if (sec >= nk) sec = nk - 1;
  return (int)(off + sec);
}

namespace {

__global__ void __launch_bounds__(kBlock) k_pc_cell_table(int32_t* __restrict__ cell_of,
                                                          int64_t npix, int64_t nside, int64_t nc) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < npix; p += stride)
    cell_of[p] = coarse_cell(p, nside, nc);
}

// One thread per baseline: the cells its valid samples fall in (up to kCand, in
// order of appearance) with each output's row sums per cell; the kPcSlots cells
// with most samples are kept, their sums divided by the baseline's valid count.
__global__ void __launch_bounds__(kBlock) k_pc_rows(const int32_t* __restrict__ pix,
                                                    const float* __restrict__ cc,
                                                    const float* __restrict__ ss,
                                                    const int32_t* __restrict__ cell_of,
                                                    const int32_t* __restrict__ nvalid,
                                                    int64_t n_t, int64_t L, int64_t n_b,
                                                    float4* __restrict__ slot,
                                                    int32_t* __restrict__ used,
                                                    unsigned long long* __restrict__ kept_total) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  unsigned long long kept_all = 0, valid_all = 0;
  for (int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; b < n_b; b += stride) {
    int id[kCand];
    int cnt[kCand];
    float sc[kCand], sn[kCand];  // sums of cos 2psi and sin 2psi per candidate cell
#pragma unroll
    for (int j = 0; j < kCand; ++j) {
      id[j] = -1;
      cnt[j] = 0;
      sc[j] = sn[j] = 0.f;
    }
    const int64_t t1 = (b + 1) * L < n_t ? (b + 1) * L : n_t;
    for (int64_t t = b * L; t < t1; t += 4) {
      // four samples' loads and cell lookups in flight, then summed in order
      int p[4], k[4];
      float c[4], s[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) p[u] = t + u < t1 ? pix[t + u] : -1;
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        k[u] = p[u] >= 0 ? __ldg(cell_of + p[u]) : -1;
        c[u] = p[u] >= 0 ? cc[t + u] : 0.f;
        s[u] = p[u] >= 0 ? ss[t + u] : 0.f;
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        if (p[u] < 0) continue;
        bool placed = false;
#pragma unroll
        for (int j = 0; j < kCand; ++j) {
          if (!placed && (id[j] == k[u] || id[j] < 0)) {
            id[j] = k[u];
            cnt[j] += 1;
            sc[j] += c[u];
            sn[j] += s[u];
            placed = true;
          }
        }
      }
    }
    const int nv = nvalid[b];
    const float inv = nv > 0 ? 1.f / (float)nv : 0.f;
    // the kPcSlots cells with most samples, in decreasing order
#pragma unroll
    for (int s = 0; s < kPcSlots; ++s) {
      int best = -1, bc = 0;
#pragma unroll
      for (int j = 0; j < kCand; ++j)
        if (id[j] >= 0 && cnt[j] > bc) {
          best = j;
          bc = cnt[j];
        }
      kept_all += (unsigned long long)bc;
      int cell = -1;
      float4 v = make_float4(__int_as_float(-1), 0.f, 0.f, 0.f);
#pragma unroll
      for (int j = 0; j < kCand; ++j)
        if (j == best) {
          cell = id[j];
          v = make_float4(__int_as_float(id[j]), (float)cnt[j] * inv, sc[j] * inv, sn[j] * inv);
          cnt[j] = 0;
        }
      slot[b * kPcSlots + s] = v;
      if (cell >= 0) used[cell] = 1;
    }
    valid_all += (unsigned long long)(nv > 0 ? nv : 0);
  }
  for (int d = 16; d > 0; d >>= 1) {
    kept_all += __shfl_down_sync(0xffffffffu, kept_all, d);
    valid_all += __shfl_down_sync(0xffffffffu, valid_all, d);
  }
  if ((threadIdx.x & 31) == 0) {
    atomicAdd(kept_total, kept_all);
    atomicAdd(kept_total + 1, valid_all);
  }
}

// The same for long baselines, one warp per baseline (every step-th baseline; step > 1
// is a probe that only counts the kept samples): each lane takes every 32nd
// sample into its own kCand candidate cells, then the warp merges the lanes'
// candidates (smallest cell first, at most kWarpCells cells; sums in a fixed
// shuffle order, so the result does not depend on timing) and keeps the two
// cells with most samples.  A thread per baseline would walk L samples one
// dependent load after another.
__global__ void __launch_bounds__(kBlock) k_pc_rows_warp(const int32_t* __restrict__ pix,
                                                         const float* __restrict__ cc,
                                                         const float* __restrict__ ss,
                                                         const int32_t* __restrict__ cell_of,
                                                         const int32_t* __restrict__ nvalid,
                                                         int64_t n_t, int64_t L, int64_t n_b,
                                                         int64_t step, float4* __restrict__ slot,
                                                         int32_t* __restrict__ used,
                                                         unsigned long long* __restrict__ kept_total) {
  const unsigned full = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  unsigned long long kept_all = 0, valid_all = 0;
  for (int64_t j = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); j * step < n_b;
       j += warps) {
    const int64_t b = j * step;
    int id[kCand];
    int cnt[kCand];
    float sc[kCand], sn[kCand];
#pragma unroll
    for (int j = 0; j < kCand; ++j) {
      id[j] = -1;
      cnt[j] = 0;
      sc[j] = sn[j] = 0.f;
    }
    const int64_t t1 = (b + 1) * L < n_t ? (b + 1) * L : n_t;
    for (int64_t t = b * L + lane; t < t1; t += 32) {
      const int p = pix[t];
      if (p < 0) continue;
      const int k = __ldg(cell_of + p);
      const float c = cc[t], s = ss[t];
      bool placed = false;
#pragma unroll
      for (int j = 0; j < kCand; ++j) {
        if (!placed && (id[j] == k || id[j] < 0)) {
          id[j] = k;
          cnt[j] += 1;
          sc[j] += c;
          sn[j] += s;
          placed = true;
        }
      }
    }
    // merge: repeatedly the smallest candidate cell left in any lane
    int best_id[kPcSlots], best_cnt[kPcSlots];
    float best_c[kPcSlots], best_s[kPcSlots];
#pragma unroll
    for (int s = 0; s < kPcSlots; ++s) {
      best_id[s] = -1;
      best_cnt[s] = 0;
      best_c[s] = best_s[s] = 0.f;
    }
    for (int round = 0; round < kWarpCells; ++round) {
      int mine = INT_MAX;
#pragma unroll
      for (int j = 0; j < kCand; ++j)
        if (id[j] >= 0 && id[j] < mine) mine = id[j];
      const int cell = __reduce_min_sync(full, mine);
      if (cell == INT_MAX) break;  // warp-uniform
      int n = 0;
      float c = 0.f, s = 0.f;
#pragma unroll
      for (int j = 0; j < kCand; ++j)
        if (id[j] == cell) {
          n = cnt[j];
          c = sc[j];
          s = sn[j];
          id[j] = -1;
        }
      n = __reduce_add_sync(full, n);
      for (int d = 16; d > 0; d >>= 1) {
        c += __shfl_xor_sync(full, c, d);
        s += __shfl_xor_sync(full, s, d);
      }
      // insert into the two best (more samples first; the smaller cell on a tie)
      if (n > best_cnt[0]) {
        best_id[1] = best_id[0]; best_cnt[1] = best_cnt[0]; best_c[1] = best_c[0]; best_s[1] = best_s[0];
        best_id[0] = cell; best_cnt[0] = n; best_c[0] = c; best_s[0] = s;
      } else if (n > best_cnt[1]) {
        best_id[1] = cell; best_cnt[1] = n; best_c[1] = c; best_s[1] = s;
      }
    }
    if (lane == 0) {
      const int nv = nvalid[b];
      const float inv = nv > 0 ? 1.f / (float)nv : 0.f;
#pragma unroll
      for (int s = 0; s < kPcSlots; ++s) {
        kept_all += (unsigned long long)best_cnt[s];
        if (step > 1) continue;  // a probe of every step-th baseline counts only
        slot[b * kPcSlots + s] =
            best_id[s] >= 0 ? make_float4(__int_as_float(best_id[s]), (float)best_cnt[s] * inv,
                                          best_c[s] * inv, best_s[s] * inv)
                            : make_float4(__int_as_float(-1), 0.f, 0.f, 0.f);
        if (best_id[s] >= 0) used[best_id[s]] = 1;
      }
      valid_all += (unsigned long long)(nv > 0 ? nv : 0);
    }
  }
  for (int d = 16; d > 0; d >>= 1) {
    kept_all += __shfl_down_sync(full, kept_all, d);
    valid_all += __shfl_down_sync(full, valid_all, d);
  }
  if (lane == 0) {
    atomicAdd(kept_total, kept_all);
    atomicAdd(kept_total + 1, valid_all);
  }
}

// Cell numbers to kept-cell numbers (-1 stays -1).
__global__ void __launch_bounds__(kBlock) k_pc_remap(float4* __restrict__ slot, int64_t n,
                                                     const int32_t* __restrict__ cmap) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    const int c = __float_as_int(slot[i].x);
    slot[i].x = __int_as_float(c >= 0 ? cmap[c] : -1);
  }
}

// E += R^T D R: per unknown (o, b), n_b times the outer product of its R row.
template <int KS>
__global__ void __launch_bounds__(kBlock) k_pc_E_diag(const float4* __restrict__ slot,
                                                      const int32_t* __restrict__ nvalid,
                                                      int64_t n_b, KindsArg kk, int n,
                                                      double* __restrict__ E) {
  using K = KSet<KS>;
  constexpr int NC = K::NC;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int64_t n_u = (int64_t)K::n_o(kk) * n_b;
  for (int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; u < n_u; u += stride) {
    const int64_t b = u % n_b;
    const int kind = K::kind((int)(u / n_b), kk);
    const int nv = nvalid[b];
    if (nv <= 0) continue;
    int col[kPcSlots * NC];
    double val[kPcSlots * NC];
#pragma unroll
    for (int s = 0; s < kPcSlots; ++s) {
      const float4 m = slot[b * kPcSlots + s];
      const int cell = __float_as_int(m.x);
      float v[NC];
      row_moments<NC>(kind, m.y, m.z, m.w, v);
#pragma unroll
      for (int c = 0; c < NC; ++c) {
        col[s * NC + c] = cell >= 0 ? cell * NC + c : -1;
        val[s * NC + c] = cell >= 0 ? (double)v[c] : 0.0;
      }
    }
#pragma unroll
    for (int a = 0; a < kPcSlots * NC; ++a) {
      if (col[a] < 0 || val[a] == 0.0) continue;
#pragma unroll
      for (int e = 0; e < kPcSlots * NC; ++e) {
        if (col[e] < 0 || val[e] == 0.0) continue;
        atomicAdd(E + (int64_t)col[a] * n + col[e], (double)nv * val[a] * val[e]);
      }
    }
  }
}

// E -= (K R)^T M^-1 (K R), one warp per pixel over its runs.  A run (count n,
// sum cos, sum sin, baseline b) is one entry of K: the row sums k_o of each output
// on the pixel's components.  (K R)_p[c'][(cell, c)] = sum over runs and outputs of
// k_o[c'] R[(o,b), (cell, c)].  Each lane sums its runs for up to kCand cells in
// registers; the warp merges the lanes' cells in shared memory and adds the
// pixel's term into E.  The runs come from the pixel-major copy (k_pc_E_pix) or
// from the long tiles of the tiled operator, where a pixel's runs of each tile are
// contiguous (k_pc_E_tiles).
// A warp's sum of pixel terms over the cells its recent pixels touched (shared
// memory): neighbouring pixels mostly touch the same few cells, so their terms are
// added here and reach E (float64 atomics, contended by every pixel of a cell) once
// per change of cells instead of once per pixel.
template <int NC>
struct EBuf {
  int id[kWarpCells];  // the buffer's cells
  int n;               // cells in use
  int full;            // the current pixel's cells do not fit: flush first
  int map[kWarpCells]; // the current pixel's cells in the buffer
  double v[kWarpCells * NC][kWarpCells * NC];

  __device__ __forceinline__ void clear() {
    const int lane = threadIdx.x & 31;
    for (int q = lane; q < kWarpCells * NC * kWarpCells * NC; q += 32)
      v[q / (kWarpCells * NC)][q % (kWarpCells * NC)] = 0.0;
    if (lane == 0) n = 0;
    __syncwarp();
  }

  __device__ __forceinline__ void flush(double* __restrict__ E, int nE) {
    const int lane = threadIdx.x & 31;
    const int m = n * NC;
    for (int q = lane; q < m * m; q += 32) {
      const int e1 = q / m, e2 = q - (q / m) * m;
      const double x = v[e1][e2];
      if (x != 0.0)
        atomicAdd(E + (int64_t)(id[e1 / NC] * NC + e1 % NC) * nE + id[e2 / NC] * NC + e2 % NC, x);
    }
    __syncwarp();
    clear();
  }
};

template <int KS>
struct PixTerm {
  static constexpr int NC = KSet<KS>::NC, NO = KSet<KS>::NO;
  int id[kCand];
  double kr[kCand][NC][NC];

  __device__ __forceinline__ void clear() {
#pragma unroll
    for (int j = 0; j < kCand; ++j) {
      id[j] = -1;
#pragma unroll
      for (int a = 0; a < NC; ++a)
#pragma unroll
        for (int c = 0; c < NC; ++c) kr[j][a][c] = 0.0;
    }
  }

  // float32 operands widened by bit re-encoding (f64_of_f32: integer pipes), so
  // that GB300's narrow float64 pipe does only the multiply-adds
  template <int J>
  __device__ __forceinline__ void update(const double (&kv)[NC], const float (&rv)[NC]) {
    double r[NC];
#pragma unroll
    for (int c = 0; c < NC; ++c) r[c] = f64_of_f32(rv[c]);
#pragma unroll
    for (int a = 0; a < NC; ++a)
#pragma unroll
      for (int c = 0; c < NC; ++c) kr[J][a][c] = fma(kv[a], r[c], kr[J][a][c]);
  }

  // one run: n samples, sums C and S, the slots of its baseline
  __device__ __forceinline__ void add_run(float n, float C, float S,
                                          const float4 (&ms)[kPcSlots], const KindsArg& kk) {
    using K = KSet<KS>;
    const int n_o = K::n_o(kk);
#pragma unroll
    for (int o = 0; o < NO; ++o) {
      if (o >= n_o) continue;
      float kv[NC];
#pragma unroll
      for (int c = 0; c < NC; ++c) kv[c] = 0.f;
      {  // the output's row summed over the run (z = 1)
        using F = Frame<NC>;
        const int kind = K::kind(o, kk);
        if (kind == DS_KIND_I) {
          if constexpr (F::I >= 0) kv[F::I] = n;
        } else if (kind == DS_KIND_Q) {
          if constexpr (F::Q >= 0) { kv[F::Q] = C; kv[F::U] = S; }
        } else if (kind == DS_KIND_U) {
          if constexpr (F::Q >= 0) { kv[F::Q] = -S; kv[F::U] = C; }
        } else {
          if constexpr (F::I >= 0 && F::Q >= 0) { kv[F::I] = n; kv[F::Q] = C; kv[F::U] = S; }
        }
      }
      double dkv[NC];
#pragma unroll
      for (int c = 0; c < NC; ++c) dkv[c] = f64_of_f32(kv[c]);
#pragma unroll
      for (int s = 0; s < kPcSlots; ++s) {
        const float4 m = ms[s];
        const int cell = __float_as_int(m.x);
        if (cell < 0) continue;
        float rv[NC];
        row_moments<NC>(K::kind(o, kk), m.y, m.z, m.w, rv);
        // the candidate first, then one block of updates under a branch that is
        // nearly always warp-uniform (a pixel's runs mostly fall in its first
        // cell): GB300's float64 pipe is narrow, and predicated updates of every
        // candidate cost it kCand times over
        int jsel = -1;
#pragma unroll
        for (int j = 0; j < kCand; ++j)
          if (jsel < 0 && (id[j] == cell || id[j] < 0)) jsel = j;
#pragma unroll
        for (int j = 0; j < kCand; ++j)
          if (j == jsel) id[j] = cell;
        static_assert(kCand == 4, "one case per candidate");
        switch (jsel) {
          case 0: update<0>(dkv, rv); break;
          case 1: update<1>(dkv, rv); break;
          case 2: update<2>(dkv, rv); break;
          case 3: update<3>(dkv, rv); break;
          default: break;
        }
      }
    }
  }

  // the warp's merged cells and E -= (K R)_p^T M_p^-1 (K R)_p
  __device__ __forceinline__ void finish(int64_t p, const double* __restrict__ minv, int n,
                                         double* __restrict__ E, int (&s_id)[kWarpCells],
                                         double (&s_kr)[kWarpCells][NC][NC], EBuf<NC>& buf) {
    constexpr int NM = NC * (NC + 1) / 2;
    const unsigned full = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    if (lane < kWarpCells) s_id[lane] = -1;
    __syncwarp();
    int slot_of[kCand];
#pragma unroll
    for (int j = 0; j < kCand; ++j) {
      slot_of[j] = -1;
      if (id[j] < 0) continue;
      for (int t = 0; t < kWarpCells; ++t) {
        const int old = atomicCAS(&s_id[t], -1, id[j]);
        if (old == -1 || old == id[j]) {
          slot_of[j] = t;
          break;
        }
      }
    }
    __syncwarp();
    int ncell = 0;
    while (ncell < kWarpCells && s_id[ncell] >= 0) ++ncell;
    for (int t = 0; t < ncell; ++t) {  // warp sums of every (cell, a, c) entry
#pragma unroll
      for (int a = 0; a < NC; ++a)
#pragma unroll
        for (int c = 0; c < NC; ++c) {
          double v = 0.0;
#pragma unroll
          for (int j = 0; j < kCand; ++j)
            if (slot_of[j] == t) v += kr[j][a][c];
          for (int d = 16; d > 0; d >>= 1) v += __shfl_xor_sync(full, v, d);
          if (lane == 0) s_kr[t][a][c] = v;
        }
    }
    __syncwarp();
    double mi[NC][NC];  // the pixel's M^-1 (packed symmetric)
    {
      const double* mp = minv + p * NM;
      if constexpr (NC == 1) {
        mi[0][0] = mp[0];
      } else if constexpr (NC == 2) {
        mi[0][0] = mp[0]; mi[0][1] = mi[1][0] = mp[1]; mi[1][1] = mp[2];
      } else {
        mi[0][0] = mp[0]; mi[0][1] = mi[1][0] = mp[1]; mi[0][2] = mi[2][0] = mp[2];
        mi[1][1] = mp[3]; mi[1][2] = mi[2][1] = mp[4]; mi[2][2] = mp[5];
      }
    }
    // the pixel's cells in the warp's buffer: new ones appended while there is
    // room, else the buffer goes to E and starts over with this pixel's cells
    if (lane == 0) {
      const int n0 = buf.n;
      int nb = n0;
      bool fits = true;
      for (int t = 0; t < ncell; ++t) {
        int idx = -1;
        for (int u = 0; u < n0; ++u)  // the buffer's cells (the pixel's are distinct)
          if (buf.id[u] == s_id[t]) idx = u;
        if (idx < 0) {
          if (nb < kWarpCells) idx = nb++;
          else fits = false;
        }
        buf.map[t] = idx;
      }
      if (fits) {
        for (int t = 0; t < ncell; ++t) buf.id[buf.map[t]] = s_id[t];
        buf.n = nb;
      }
      buf.full = fits ? 0 : 1;
    }
    __syncwarp();
    if (buf.full) {
      buf.flush(E, n);
      if (lane == 0) {
        for (int t = 0; t < ncell; ++t) {
          buf.id[t] = s_id[t];
          buf.map[t] = t;
        }
        buf.n = ncell;
      }
      __syncwarp();
    }
    const int m = ncell * NC;
    for (int q = lane; q < m * m; q += 32) {
      const int e1 = q / m, e2 = q - (q / m) * m;
      const int t1 = e1 / NC, c1 = e1 - t1 * NC, t2 = e2 / NC, c2 = e2 - t2 * NC;
      double v = 0.0;
#pragma unroll
      for (int a = 0; a < NC; ++a)
#pragma unroll
        for (int a2 = 0; a2 < NC; ++a2)
          v += s_kr[t1][a][c1] * mi[a][a2] * s_kr[t2][a2][c2];
      buf.v[buf.map[t1] * NC + c1][buf.map[t2] * NC + c2] -= v;
    }
    __syncwarp();
  }
};

template <int KS>
__global__ void __launch_bounds__(kBlock) k_pc_E_pix(const uint32_t* __restrict__ off,
                                                     const float4* __restrict__ rec,
                                                     const float4* __restrict__ slot,
                                                     const double* __restrict__ minv,
                                                     const uint8_t* __restrict__ mask,
                                                     int64_t npix, KindsArg kk, int n,
                                                     double* __restrict__ E) {
  constexpr int NC = KSet<KS>::NC;
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  __shared__ int s_id[kBlock / 32][kWarpCells];
  __shared__ double s_kr[kBlock / 32][kWarpCells][NC][NC];
  __shared__ EBuf<NC> s_buf[kBlock / 32];
  s_buf[wib].clear();
  // each warp a contiguous range of pixels (neighbours share cells)
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  const int64_t per = (npix + warps - 1) / warps;
  const int64_t w = (int64_t)blockIdx.x * (blockDim.x >> 5) + wib;
  const int64_t p1 = (w + 1) * per < npix ? (w + 1) * per : npix;
  for (int64_t p = w * per; p < p1; ++p) {
    if (!mask[p]) continue;  // warp-uniform
    const uint32_t beg = __ldg(off + p), end = __ldg(off + p + 1);
    if (beg == end) continue;
    PixTerm<KS> pt;
    pt.clear();
    for (uint32_t i = beg + lane; i < end; i += 64) {
      // two runs per lane: their records, then their slots, in flight together
      const bool two = i + 32 < end;
      const float4 r0 = __ldg(rec + i);
      const float4 r1 = two ? __ldg(rec + i + 32) : make_float4(0.f, 0.f, 0.f, 0.f);
      float4 m0[kPcSlots], m1[kPcSlots];
#pragma unroll
      for (int s = 0; s < kPcSlots; ++s) {
        m0[s] = __ldg(slot + (int64_t)__float_as_int(r0.w) * kPcSlots + s);
        m1[s] = two ? __ldg(slot + (int64_t)__float_as_int(r1.w) * kPcSlots + s)
                    : make_float4(__int_as_float(-1), 0.f, 0.f, 0.f);
      }
      pt.add_run(r0.x, r0.y, r0.z, m0, kk);
      if (two) pt.add_run(r1.x, r1.y, r1.z, m1, kk);
    }
    pt.finish(p, minv, n, E, s_id[wib], s_kr[wib], s_buf[wib]);
  }
  s_buf[wib].flush(E, n);
}

// The same over the long tiles: pixel rank r's runs of tile t are records
// [end[t nkeys + r - 1], end[t nkeys + r]) (16-byte tiled records: pixel,
// n << 24 | baseline in the tile, sum cos, sum sin).
template <int KS>
__global__ void __launch_bounds__(kBlock) k_pc_E_tiles(const int4* __restrict__ rec,
                                                       const uint32_t* __restrict__ end,
                                                       int64_t n_tiles, int64_t nkeys, int64_t Tb,
                                                       const float4* __restrict__ slot,
                                                       const double* __restrict__ minv,
                                                       KindsArg kk, int n, double* __restrict__ E) {
  constexpr int NC = KSet<KS>::NC;
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  __shared__ int s_id[kBlock / 32][kWarpCells];
  __shared__ double s_kr[kBlock / 32][kWarpCells][NC][NC];
  __shared__ EBuf<NC> s_buf[kBlock / 32];
  s_buf[wib].clear();
  // each warp a contiguous range of ranks (neighbours along the scan share cells)
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  const int64_t per = (nkeys + warps - 1) / warps;
  const int64_t w = (int64_t)blockIdx.x * (blockDim.x >> 5) + wib;
  const int64_t r1 = (w + 1) * per < nkeys ? (w + 1) * per : nkeys;
  const unsigned full = 0xffffffffu;
  for (int64_t r = w * per; r < r1; ++r) {
    PixTerm<KS> pt;
    pt.clear();
    int p = -1;
    // the rank's runs of 32 tiles at a time, numbered through so that every lane
    // has one (a pixel holds a dozen or two runs per tile)
    for (int64_t tg = 0; tg < n_tiles; tg += 32) {
      const int64_t t = tg + lane;
      uint32_t b0 = 0, len = 0;
      if (t < n_tiles) {
        const int64_t k = t * nkeys + r;
        b0 = k > 0 ? __ldg(end + k - 1) : 0u;
        len = __ldg(end + k) - b0;
      }
      uint32_t pre = len;  // inclusive prefix over the lanes' tiles
#pragma unroll
      for (int d = 1; d < 32; d <<= 1) {
        const uint32_t u = __shfl_up_sync(full, pre, d);
        if (lane >= d) pre += u;
      }
      const uint32_t total = __shfl_sync(full, pre, 31);
      pre -= len;  // exclusive
      if (p < 0 && total > 0) {  // the pixel, from the first record of the group
        const unsigned nz = __ballot_sync(full, len > 0);
        const uint32_t bf = __shfl_sync(full, b0, __ffs(nz) - 1);
        p = __ldg(rec + bf).x;
      }
      for (uint32_t base = 0; base < total; base += 32) {
        const uint32_t f = base + lane;
        // the lane whose tile holds run f: the last with pre <= f
        int lo = 0;
#pragma unroll
        for (int step = 16; step > 0; step >>= 1) {
          const uint32_t pc = __shfl_sync(full, pre, lo + step);
          if (lo + step < 32 && pc <= f) lo += step;
        }
        const uint32_t b0l = __shfl_sync(full, b0, lo), prel = __shfl_sync(full, pre, lo);
        if (f >= total) continue;
        const int4 v = __ldcs(rec + b0l + (f - prel));
        const int64_t bb = (tg + lo) * Tb + (int64_t)((unsigned)v.y & 0xFFFFFFu);
        float4 m[kPcSlots];
#pragma unroll
        for (int s = 0; s < kPcSlots; ++s) m[s] = __ldg(slot + bb * kPcSlots + s);
        pt.add_run((float)((unsigned)v.y >> 24), __int_as_float(v.z), __int_as_float(v.w), m, kk);
      }
    }
    if (p >= 0) pt.finish(p, minv, n, E, s_id[wib], s_kr[wib], s_buf[wib]);
  }
  s_buf[wib].flush(E, n);
}

// Rank-one term mu/m on every pair of the m I-component columns.
__global__ void k_pc_null_term(double* __restrict__ E, int n, int nc, int ci, int cells, double mu) {
  const int64_t total = (int64_t)cells * cells;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < total; q += stride) {
    const int64_t a = q / cells, b = q - (q / cells) * cells;
    E[(a * nc + ci) * n + b * nc + ci] += mu / (double)cells;
  }
}

// One step of the sweep operator on pivot k (out = sweep_k(in)); a pivot whose
// value has fallen to tol_rel of its original diagonal is skipped (in copied to
// out) and flagged.
__global__ void __launch_bounds__(kBlock) k_pc_sweep(const double* __restrict__ in,
                                                     double* __restrict__ out, int n, int k,
                                                     const double* __restrict__ diag0,
                                                     double tol_rel, int32_t* __restrict__ skipped) {
  __shared__ double s_inv;
  __shared__ int s_skip;
  if (threadIdx.x == 0) {
    const double d = in[(int64_t)k * n + k];
    s_skip = !(d > tol_rel * diag0[k]);
    s_inv = s_skip ? 0.0 : 1.0 / d;
    if (s_skip && blockIdx.x == 0) skipped[k] = 1;
  }
  __syncthreads();
  const double inv = s_inv;
  const bool skip = s_skip != 0;
  const int64_t total = (int64_t)n * n;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < total; q += stride) {
    const int64_t i = q / n, j = q - (q / n) * n;
    double v = in[q];
    if (!skip) {
      if (i == k && j == k) v = -inv;
      else if (i == k || j == k) v = v * inv;
      else v = v - in[i * n + k] * in[(int64_t)k * n + j] * inv;
    }
    out[q] = v;
  }
}

// E^+ = -(swept matrix) with the rows and columns of skipped pivots set to 0.
__global__ void __launch_bounds__(kBlock) k_pc_finish(const double* __restrict__ in,
                                                      double* __restrict__ out, int n,
                                                      const int32_t* __restrict__ skipped) {
  const int64_t total = (int64_t)n * n;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < total; q += stride) {
    const int64_t i = q / n, j = q - (q / n) * n;
    out[q] = (skipped[i] || skipped[j]) ? 0.0 : -in[q];
  }
}

__global__ void k_pc_diag(const double* __restrict__ E, double* __restrict__ d, int n) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    d[i] = E[(int64_t)i * n + i];
}

}  // namespace

void pc_free(Plan& P, cudaStream_t st) {
  void** held[] = {reinterpret_cast<void**>(&P.pc_slot), reinterpret_cast<void**>(&P.pc_einv), reinterpret_cast<void**>(&P.pc_u),
                   reinterpret_cast<void**>(&P.pc_c)};
  for (void** h : held)
    if (*h != nullptr) {
      cudaFreeAsync(*h, st);
      *h = nullptr;
    }
  P.pc_n = 0;
  P.pc_cells = 0;
  P.pc_built = 0;
  P.pc_fallback = 0;
  P.pc_probed = 0;
}

bool pc_ready(const Plan& P) {
  return P.precond == 2 && P.pc_built && P.pc_n > 0 && !P.pc_fallback;
}

// The preconditioner the iteration applies: 0 none, 1 D^-1, 2 two-level.  A
// two-level plan whose coarse space was not built (it would not span the slow
// modes, or has no room) iterates plain CG: D^-1 alone is nearly a scalar where
// baselines hold equal counts, and costs a kernel per iteration; after a breakdown
// with the coarse correction it keeps D^-1.
int pc_mode(const Plan& P) {
  if (P.precond != 2) return P.precond;
  if (pc_ready(P)) return 2;
  return P.pc_built && !P.pc_fallback ? 0 : 1;
}

// Long baselines often sweep too many cells for their two slots to hold most of
// their samples.  A probe of about 4096 of them (counting only) decides first:
// where the slots would keep too few samples the plan gets no coarse space and
// iterates plain CG.  The host waits for the count, so a solve probes before it
// queues its right-hand side.
ds_status pc_probe(Plan& P) {
  if (P.precond != 2 || P.pc_built || P.pc_probed) return DS_OK;
  const int64_t step = P.n_b / 4096 > 1 ? P.n_b / 4096 : 1;
  if (P.L < kPcWarpRows || step <= 1) {
    P.pc_probed = 1;
    return DS_OK;
  }
  cudaStream_t st = P.stream;
  const int64_t nc = P.pc_nside < P.desc.nside ? P.pc_nside : P.desc.nside;
  int32_t* cell_of = nullptr;
  unsigned long long* kept = nullptr;  // samples in kept slots, valid samples
  unsigned long long h_probe[2] = {0, 0};
  cudaError_t e = plan_alloc(P, reinterpret_cast<void**>(&cell_of), sizeof(int32_t) * P.npix, false);
  if (e == cudaSuccess) e = plan_alloc(P, reinterpret_cast<void**>(&kept), sizeof(h_probe), false);
  if (e == cudaSuccess) e = cudaMemsetAsync(kept, 0, sizeof(h_probe), st);
  if (e == cudaSuccess) {
    k_pc_cell_table<<<stream_grid(P, P.npix, kBlock, 8), kBlock, 0, st>>>(cell_of, P.npix,
                                                                        P.desc.nside, nc);
    // with step > 1 the kernel writes neither slots nor the used-cell flags
    k_pc_rows_warp<<<stream_grid(P, (P.n_b / step + 1) * 32, kBlock, 8), kBlock, 0, st>>>(
        P.pix, P.c, P.s, cell_of, P.nvalid, P.n_t, P.L, P.n_b, step, nullptr, nullptr, kept);
    P.launches += 2;
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(h_probe, kept, sizeof(h_probe), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (cell_of) cudaFreeAsync(cell_of, st);
  if (kept) cudaFreeAsync(kept, st);
  if (e == cudaErrorMemoryAllocation) {  // the coarse-space build reports it
    (void)cudaGetLastError();
    return DS_OK;
  }
  if (e != cudaSuccess) return DS_ECUDA;
  P.pc_probed = 1;
  if (h_probe[1] > 0 && (double)h_probe[0] < (kPcKeptMin - 0.1) * (double)h_probe[1]) {
    pc_free(P, st);
    P.pc_built = 1;
  }
  return DS_OK;
}

// Builds the coarse space and E^+ on the plan's stream (synchronises it).  The
// second term of E reads the pixel-major copy of the run records; a plan whose
// operator does not keep one gets it for the purpose (made_runs / made_pm) and
// gives it back afterwards.
ds_status pc_build(Plan& P, bool* made_runs, bool* made_pm) {
  *made_runs = *made_pm = false;
  if (P.pc_built) return DS_OK;
  const ds_status sp = pc_probe(P);
  if (sp != DS_OK || P.pc_built) return sp;
  cudaStream_t st = P.stream;
  const int64_t nc = P.pc_nside < P.desc.nside ? P.pc_nside : P.desc.nside;
  const int64_t ncell = 12 * nc * nc;
  int32_t *cell_of = nullptr, *used = nullptr, *cmap = nullptr, *skipped = nullptr;
  unsigned long long* kept = nullptr;  // samples in kept slots, valid samples
  double *E = nullptr, *E2 = nullptr, *diag0 = nullptr;
  auto fail = [&](cudaError_t e) {
    void* tmp[] = {cell_of, used, cmap, skipped, E, E2, diag0, kept};
    for (void* t : tmp)
      if (t) cudaFreeAsync(t, st);
    pc_free(P, st);
    return e == cudaErrorMemoryAllocation ? DS_ENOMEM : DS_ECUDA;
  };
  cudaError_t e = plan_alloc(P, reinterpret_cast<void**>(&cell_of), sizeof(int32_t) * P.npix, false);
  if (e == cudaSuccess) e = plan_alloc(P, reinterpret_cast<void**>(&used), sizeof(int32_t) * ncell, false);
  if (e == cudaSuccess) e = plan_alloc(P, reinterpret_cast<void**>(&cmap), sizeof(int32_t) * ncell, false);
  if (e == cudaSuccess)
    e = plan_alloc(P, reinterpret_cast<void**>(&P.pc_slot), sizeof(float4) * P.n_b * kPcSlots, true);
  if (e == cudaSuccess) e = plan_alloc(P, reinterpret_cast<void**>(&kept), sizeof(unsigned long long) * 2, false);
  if (e == cudaSuccess) e = cudaMemsetAsync(used, 0, sizeof(int32_t) * ncell, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(kept, 0, sizeof(unsigned long long) * 2, st);
  if (e != cudaSuccess) return fail(e);
  const int g_pix = stream_grid(P, P.npix, kBlock, 8);
  k_pc_cell_table<<<g_pix, kBlock, 0, st>>>(cell_of, P.npix, P.desc.nside, nc);
  const int g_b = stream_grid(P, P.n_b, kBlock, 8);
  if (P.L >= kPcWarpRows) {
    k_pc_rows_warp<<<stream_grid(P, P.n_b * 32, kBlock, 8), kBlock, 0, st>>>(
        P.pix, P.c, P.s, cell_of, P.nvalid, P.n_t, P.L, P.n_b, 1, P.pc_slot, used, kept);
  } else
    k_pc_rows<<<g_b, kBlock, 0, st>>>(P.pix, P.c, P.s, cell_of, P.nvalid, P.n_t, P.L, P.n_b,
                                      P.pc_slot, used, kept);
  P.launches += 2;
  e = cudaGetLastError();
  // kept cells: numbered in cell order on the host
  std::vector<int32_t> h_used(ncell), h_map(ncell, -1);
  unsigned long long h_kept[2] = {0, 0};
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(h_used.data(), used, sizeof(int32_t) * ncell, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(h_kept, kept, sizeof(h_kept), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return fail(e);
  int n_kept = 0;
  for (int64_t c = 0; c < ncell; ++c)
    if (h_used[c]) h_map[c] = n_kept++;
  const int n = n_kept * P.n_c;
  // Baselines that sweep many cells (long baselines) keep only part of their
  // samples in kPcSlots cells; such a coarse space spans the slow modes badly
  // and costs more than it saves, so the plan keeps D^-1 alone.
  const bool spans = h_kept[1] > 0 && (double)h_kept[0] >= kPcKeptMin * (double)h_kept[1];
  // the restriction sums a block's share of R^T r in shared memory
  if (n == 0 || !spans || !pc_restrict_fits(P, n)) {
    void* tmp[] = {cell_of, used, cmap, kept};
    for (void* t : tmp) cudaFreeAsync(t, st);
    pc_free(P, st);
    P.pc_built = 1;
    return DS_OK;
  }
  // the runs of each pixel for the second term of E: the tiled operator's long
  // tiles, else the pixel-major copy (made for the purpose when the plan has none)
  const bool tiles = P.layout == 3 && P.tl2_end != nullptr && P.tl2_rec != nullptr;
  if (!tiles && P.pm_rec == nullptr) {
    ds_status sr = DS_OK;
    if (P.rl_rec == nullptr) {
      sr = rl_build(P);
      *made_runs = true;
    }
    if (sr == DS_OK) {
      sr = pm_build(P, st);
      *made_pm = true;
    }
    if (sr != DS_OK || P.pm_rec == nullptr) {  // no room or too many runs: D^-1 alone
      void* tmp[] = {cell_of, used, cmap, kept};
      for (void* t : tmp) cudaFreeAsync(t, st);
      pc_free(P, st);
      P.pc_built = 1;
      return sr == DS_ENOMEM ? DS_OK : sr;
    }
  }
  e = cudaMemcpyAsync(cmap, h_map.data(), sizeof(int32_t) * ncell, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess)
    e = plan_alloc(P, reinterpret_cast<void**>(&P.pc_einv), sizeof(double) * n * n, true);
  if (e == cudaSuccess) e = plan_alloc(P, reinterpret_cast<void**>(&E), sizeof(double) * n * n, false);
  if (e == cudaSuccess) e = plan_alloc(P, reinterpret_cast<void**>(&E2), sizeof(double) * n * n, false);
  if (e == cudaSuccess) e = plan_alloc(P, reinterpret_cast<void**>(&diag0), sizeof(double) * n, false);
  if (e == cudaSuccess) e = plan_alloc(P, reinterpret_cast<void**>(&skipped), sizeof(int32_t) * n, false);
  if (e == cudaSuccess) e = plan_alloc(P, reinterpret_cast<void**>(&P.pc_u), sizeof(double) * n, true);
  if (e == cudaSuccess) e = plan_alloc(P, reinterpret_cast<void**>(&P.pc_c), sizeof(float) * n, true);
  if (e == cudaSuccess) e = cudaMemsetAsync(E, 0, sizeof(double) * n * n, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(P.pc_u, 0, sizeof(double) * n, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(P.pc_c, 0, sizeof(float) * n, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(skipped, 0, sizeof(int32_t) * n, st);
  if (e != cudaSuccess) return fail(e);
  k_pc_remap<<<g_b, kBlock, 0, st>>>(P.pc_slot, P.n_b * kPcSlots, cmap);
  const int g_u = stream_grid(P, P.n_u, kBlock, 8);
  with_kindset(P.kindset, [&](auto ksc) {
    constexpr int KS = decltype(ksc)::value;
    k_pc_E_diag<KS><<<g_u, kBlock, 0, st>>>(P.pc_slot, P.nvalid, P.n_b, P.kinds, n, E);
  });
  // the scale of each coarse direction: diag(R^T D R), before the pixel term
  k_pc_diag<<<(n + 255) / 256, 256, 0, st>>>(E, diag0, n);
  with_kindset(P.kindset, [&](auto ksc) {
    constexpr int KS = decltype(ksc)::value;
    if (tiles)
      k_pc_E_tiles<KS><<<stream_grid(P, P.tl2_nkeys * 32, kBlock, 8), kBlock, 0, st>>>(
          P.tl2_rec, P.tl2_end, P.tl2_tiles, P.tl2_nkeys, P.tl2_tb, P.pc_slot, P.minv, P.kinds,
          n, E);
    else
      k_pc_E_pix<KS><<<stream_grid(P, P.npix * 32, kBlock, 8), kBlock, 0, st>>>(
          P.pm_off, P.pm_rec, P.pc_slot, P.minv, P.mask, P.npix, P.kinds, n, E);
  });
  P.launches += 3;
  e = cudaGetLastError();
  if (e != cudaSuccess) return fail(e);
  // the I null mode: rank-one term at the mean diagonal of R^T D R, on the
  // I-component columns
  if (P.has_I_outputs) {
    std::vector<double> hd(n);
    e = cudaMemcpyAsync(hd.data(), diag0, sizeof(double) * n, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return fail(e);
    double mu = 0.0;
    for (double v : hd) mu += v;
    mu /= (double)n;
    const int ci = 0;  // I is the first component whenever outputs carry I
    k_pc_null_term<<<stream_grid(P, (int64_t)n_kept * n_kept, kBlock, 8), kBlock, 0, st>>>(
        E, n, P.n_c, ci, n_kept, mu);
    P.launches += 2;
  }
  // sweep every pivot, ping-ponging between E and E2; a pivot is skipped when it
  // holds less than kPcPivotMin of its direction's R^T D R: the direction is
  // (numerically) a null mode of A, and E is known there only to the float32
  // rounding of R and of the run sums
  const int g_s = stream_grid(P, (int64_t)n * n, kBlock, 8);
  double* a = E;
  double* bbuf = E2;
  for (int k = 0; k < n; ++k) {
    k_pc_sweep<<<g_s, kBlock, 0, st>>>(a, bbuf, n, k, diag0, kPcPivotMin, skipped);
    double* t = a;
    a = bbuf;
    bbuf = t;
  }
  k_pc_finish<<<g_s, kBlock, 0, st>>>(a, P.pc_einv, n, skipped);
  P.launches += n + 2;
  e = cudaGetLastError();
  if (e != cudaSuccess) return fail(e);
  void* tmp[] = {cell_of, used, cmap, skipped, E, E2, diag0, kept};
  for (void* t : tmp) cudaFreeAsync(t, st);
  P.pc_n = n;
  P.pc_cells = n_kept;
  P.pc_built = 1;
  return DS_OK;
}

ds_status pc_prepare(Plan& P) {
  if (P.pc_built) return DS_OK;
  cudaStream_t st = P.stream;
  const bool runs_kept = P.layout == 2 && P.desc.precision == DS_PREC_MIXED;
  bool made_runs = false, made_pm = false;
  ds_status s = pc_build(P, &made_runs, &made_pm);
  // records the operator does not read are given back once E is built
  if (made_pm && !(runs_kept && P.bin_order == 1)) pm_release(P, st);
  if (made_runs && !runs_kept) rl_release(P, st);
  if (s == DS_ENOMEM) {  // no room for the coarse space: D^-1 alone
    cudaGetLastError();
    pc_free(P, st);
    P.pc_built = 1;
    s = DS_OK;
  }
  if (s != DS_OK) return s;
  return cudaStreamSynchronize(st) == cudaSuccess ? DS_OK : DS_ECUDA;
}

}  // namespace ds
