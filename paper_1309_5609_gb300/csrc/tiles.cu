// Time-tiled, pixel-sorted run records: the float32 operator of plans whose runs
// are short (about one pixel per sample, e.g. nside 512 at 50 Hz), where neither
// the time-ordered samples nor the pixel-major copy pays.
//
// The runs of consecutive samples on one pixel within a baseline (runs_build.cu)
// are cut into tiles of Tb consecutive baselines, and within each tile sorted by
// pixel (one counting sort per tile at plan time).  A record is 16 bytes:
//     (pixel, n << 24 | baseline - first baseline of the tile, sum cos 2psi, sum sin 2psi)
// with n <= 255 samples (plans with longer runs keep the other forms).
//
// Both passes of an iteration give each tile to one block, which streams the
// tile's records once (Sect. 3 operator, exact reformulation: only the float32
// rounding order changes):
//  * binning (P~^T R^T F~ x): the tile's baselines are staged in shared memory;
//    a warp walks a contiguous share of the tile's records in rounds of 32, sums
//    the contributions of equal pixels across the lanes (a segmented sum over the
//    sorted keys) and carries the last pixel's sums into its next round, so that
//    one vector reduction (red.global.add.v4.f32) is issued per pixel and warp
//    share instead of one per run;
//  * rescan and per-baseline sums (F~^T (z - R P~ m)): the tile's baseline sums
//    live in shared memory (float32 atomics; the runs of one pixel lie in
//    different baselines, so lanes rarely collide); the map row of a pixel is
//    gathered by every lane of its run group at one address; the block stores
//    its baselines' sums once (each baseline belongs to one tile: no atomics in
//    global memory).
#include <vector>

#include "internal.cuh"
#include "rows.cuh"
#include "runs.cuh"
#include "stream_common.cuh"

namespace ds {

namespace {

constexpr int kBlock = 256;
constexpr int kTileThreads = 512;
constexpr int kTileFloats = 12288;  // shared floats per block: baselines x outputs of a tile

// ---- construction ------------------------------------------------------------------

// tile_off[t] = first run of tile t (runs are in baseline order), t = 0 .. n_tiles.
__global__ void k_tl_bounds(const int32_t* __restrict__ rb, int64_t n_runs, int64_t n_tiles,
                            int64_t Tb, int64_t* __restrict__ tile_off) {
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t <= n_tiles;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t b = t * Tb;
    int64_t lo = 0, hi = n_runs;  // first run with baseline >= b
    while (lo < hi) {
      const int64_t mid = (lo + hi) >> 1;
      if ((int64_t)rb[mid] < b) lo = mid + 1;
      else hi = mid;
    }
    tile_off[t] = lo;
  }
}

// *longest = the largest sample count of any run
__global__ void __launch_bounds__(kBlock) k_tl_longest(const RunRec* __restrict__ rec,
                                                       int64_t n_runs, int* __restrict__ longest) {
  int m = 0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n_runs;
       i += (int64_t)gridDim.x * blockDim.x)
    m = max(m, (int)rec[i].n);
  for (int d = 16; d > 0; d >>= 1) m = max(m, __shfl_down_sync(0xffffffffu, m, d));
  if ((threadIdx.x & 31) == 0) atomicMax(longest, m);
}

// Runs per pixel within tile t (cnt zeroed before).
__global__ void __launch_bounds__(kBlock) k_tl_hist(const RunRec* __restrict__ rec,
                                                    const int64_t* __restrict__ tile_off, int64_t t,
                                                    uint32_t* __restrict__ cnt) {
  const int64_t r0 = tile_off[t], r1 = tile_off[t + 1];
  for (int64_t i = r0 + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < r1;
       i += (int64_t)gridDim.x * blockDim.x)
    atomicAdd(cnt + rec[i].pix, 1u);
}

// Exclusive scan of cnt[0 .. n) into run positions, in three steps: block sums
// (each block S consecutive pixels), their scan from the tile's first run, and
// the positions within each block.  cnt becomes the scatter cursor.
__global__ void __launch_bounds__(kBlock) k_tl_scan_up(const uint32_t* __restrict__ cnt, int64_t n,
                                                       int64_t S, int64_t* __restrict__ blk) {
  __shared__ int64_t sh[kBlock / 32];
  const int64_t lo = (int64_t)blockIdx.x * S, hi = lo + S < n ? lo + S : n;
  int64_t v = 0;
  for (int64_t i = lo + threadIdx.x; i < hi; i += blockDim.x) v += cnt[i];
  for (int d = 16; d > 0; d >>= 1) v += __shfl_down_sync(0xffffffffu, v, d);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    int64_t t = 0;
    for (int q = 0; q < kBlock / 32; ++q) t += sh[q];
    blk[blockIdx.x] = t;
  }
}

// blk[j] = tile start + sum of blk[0 .. j) (one thread; G is at most a few thousand)
__global__ void k_tl_scan_top(int64_t* __restrict__ blk, int64_t G,
                              const int64_t* __restrict__ tile_off, int64_t t) {
  int64_t run = tile_off[t];
  for (int64_t j = 0; j < G; ++j) {
    const int64_t x = blk[j];
    blk[j] = run;
    run += x;
  }
}

__global__ void __launch_bounds__(kBlock) k_tl_scan_down(uint32_t* __restrict__ cnt, int64_t n,
                                                         int64_t S, const int64_t* __restrict__ blk,
                                                         int64_t* __restrict__ pos) {
  __shared__ int64_t wsum[kBlock / 32];
  const unsigned full = 0xffffffffu;
  const int lane = threadIdx.x & 31, wq = threadIdx.x >> 5;
  const int64_t lo = (int64_t)blockIdx.x * S, hi = lo + S < n ? lo + S : n;
  int64_t carry = blk[blockIdx.x];
  for (int64_t base = lo; base < hi; base += blockDim.x) {
    const int64_t i = base + threadIdx.x;
    const int64_t v = i < hi ? cnt[i] : 0;
    int64_t inc = v;
    for (int d = 1; d < 32; d <<= 1) {
      const int64_t u = __shfl_up_sync(full, inc, d);
      if (lane >= d) inc += u;
    }
    if (lane == 31) wsum[wq] = inc;
    __syncthreads();
    int64_t before = 0, tile = 0;
    for (int q = 0; q < (int)(blockDim.x >> 5); ++q) {
      if (q < wq) before += wsum[q];
      tile += wsum[q];
    }
    if (i < hi) pos[i] = carry + before + inc - v;
    carry += tile;
    __syncthreads();
  }
}

// Each run of tile t to its pixel's next slot, as a 16-byte record.
__global__ void __launch_bounds__(kBlock) k_tl_scatter(const RunRec* __restrict__ rec,
                                                       const int32_t* __restrict__ rb,
                                                       const int64_t* __restrict__ tile_off,
                                                       int64_t t, int64_t Tb,
                                                       unsigned long long* __restrict__ cursor,
                                                       int4* __restrict__ out) {
  const int64_t r0 = tile_off[t], r1 = tile_off[t + 1];
  const int64_t b0 = t * Tb;
  for (int64_t i = r0 + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < r1;
       i += (int64_t)gridDim.x * blockDim.x) {
    const RunRec r = rec[i];
    const unsigned bl = (unsigned)((int64_t)rb[i] - b0);
    const unsigned long long slot = atomicAdd(cursor + r.pix, 1ull);
    out[slot] = make_int4(r.pix, (int)(((unsigned)r.n << 24) | bl), __float_as_int(r.c),
                          __float_as_int(r.s));
  }
}

// ---- the operator's passes --------------------------------------------------------

constexpr int kUnroll = 4;  // records per lane loaded before any is used (bytes in flight)
constexpr int64_t kChunk = 32 * kUnroll * 16;  // records per warp chunk of the long-tile binning

// One round of 32 records of a warp's share: lane sums of equal pixels (the
// records are sorted by pixel within the tile), the carried pixel of the previous
// round joined to lane 0, one reduction per other segment, the last segment
// carried on.
template <int NC>
__device__ __forceinline__ void tl_bin_round(int key, float (&acc)[NC], int& ckey,
                                             float (&carry)[NC], float* __restrict__ bins) {
  const unsigned full = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  if (lane == 0 && ckey >= 0) {
    if (key == ckey) {
#pragma unroll
      for (int j = 0; j < NC; ++j) acc[j] += carry[j];
    } else {
      flush_bins<NC, float>(bins, ckey, carry);
    }
  }
  const int nxt = __shfl_down_sync(full, key, 1);
  bool stop = lane == 31 || nxt != key;
#pragma unroll
  for (int w = 1; w < 32; w <<= 1) {
    float v2[NC];
#pragma unroll
    for (int j = 0; j < NC; ++j) v2[j] = __shfl_down_sync(full, acc[j], w);
    const bool s2 = __shfl_down_sync(full, stop, w);
    if (!stop) {
#pragma unroll
      for (int j = 0; j < NC; ++j) acc[j] += v2[j];
      stop = s2;
    }
  }
  const int prv = __shfl_up_sync(full, key, 1);
  const bool head = key >= 0 && (lane == 0 || prv != key);
  const unsigned heads = __ballot_sync(full, head);
  const int last = heads ? 31 - __clz(heads) : -1;
  const int lkey = __shfl_sync(full, key, 31);
  const bool carry_last = last >= 0 && __shfl_sync(full, key, last) == lkey && lkey >= 0;
  if (head && !(carry_last && lane == last)) flush_bins<NC, float>(bins, key, acc);
  ckey = carry_last ? lkey : -1;
#pragma unroll
  for (int j = 0; j < NC; ++j) carry[j] = __shfl_sync(full, acc[j], last >= 0 ? last : 0);
}

// bins[p] += sum over the tile's runs on p of the rows summed over the run times
// the run's baselines (float32).  A warp takes kUnroll rounds of 32 records at a
// time: all their loads are issued before the first round is summed.
template <int KS>
__global__ void __launch_bounds__(kTileThreads) k_tl_bin(const int4* __restrict__ rec,
                                                         const int64_t* __restrict__ tile_off,
                                                         int64_t n_tiles, int64_t Tb,
                                                         const float* __restrict__ x,
                                                         float* __restrict__ bins, int64_t n_b,
                                                         KindsArg kk, Gate g) {
  if (gate_closed(g)) return;
  using K = KSet<KS>;
  constexpr int NC = K::NC, NO = K::NO;
  const int n_o = K::n_o(kk);
  extern __shared__ float xs[];  // [n_o][Tb]
  const int lane = threadIdx.x & 31, wq = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int64_t t = blockIdx.x; t < n_tiles; t += gridDim.x) {
    const int64_t b0 = t * Tb;
    const int64_t nb = b0 + Tb < n_b ? Tb : n_b - b0;
    for (int o = 0; o < n_o; ++o)
      for (int64_t j = threadIdx.x; j < nb; j += blockDim.x) xs[o * Tb + j] = __ldg(x + o * n_b + b0 + j);
    __syncthreads();
    const int64_t r0 = tile_off[t], r1 = tile_off[t + 1];
    // warp wq takes a contiguous share of the tile's runs, whole rounds of 32
    const int64_t per = ((r1 - r0 + nw - 1) / nw + 31) & ~int64_t(31);
    const int64_t lo = r0 + wq * per;
    const int64_t hi = lo + per < r1 ? lo + per : r1;
    int ckey = -1;  // the pixel whose sums are carried from the previous round
    float carry[NC];
#pragma unroll
    for (int j = 0; j < NC; ++j) carry[j] = 0.f;
    for (int64_t base = lo; base < hi; base += 32 * kUnroll) {
      int4 v[kUnroll];
#pragma unroll
      for (int u = 0; u < kUnroll; ++u) {
        const int64_t i = base + 32 * u + lane;
        v[u] = i < hi ? __ldcs(rec + i) : make_int4(-1, 0, 0, 0);
      }
#pragma unroll
      for (int u = 0; u < kUnroll; ++u) {
        if (base + 32 * u >= hi) break;  // warp-uniform
        float acc[NC];
#pragma unroll
        for (int j = 0; j < NC; ++j) acc[j] = 0.f;
        const int key = v[u].x;
        if (key >= 0) {
          const float n = (float)((unsigned)v[u].y >> 24);
          const int bl = (int)((unsigned)v[u].y & 0xFFFFFFu);
          const float c = __int_as_float(v[u].z), sn = __int_as_float(v[u].w);
#pragma unroll
          for (int o = 0; o < NO; ++o)
            if (o < n_o) run_bin<NC>(K::kind(o, kk), n, c, sn, xs[o * Tb + bl], acc);
        }
        tl_bin_round<NC>(key, acc, ckey, carry, bins);
      }
    }
    if (lane == 0 && ckey >= 0) flush_bins<NC, float>(bins, ckey, carry);
    __syncthreads();
  }
}

// out[o][b] = sum over the tile's runs in baseline b of n x[o][b] - (row sums) . m_p
// (float32 sums in shared memory, one float64 store per baseline).  Each thread
// issues the loads of kUnroll records, then their map rows and baselines, before
// any sum.
template <int KS>
__global__ void __launch_bounds__(kTileThreads) k_tl_rescan(const int4* __restrict__ rec,
                                                            const int64_t* __restrict__ tile_off,
                                                            int64_t n_tiles, int64_t Tb,
                                                            const float* __restrict__ x,
                                                            const float* __restrict__ map,
                                                            double* __restrict__ out, int64_t n_b,
                                                            KindsArg kk, Gate g) {
  if (gate_closed(g)) return;
  using K = KSet<KS>;
  constexpr int NC = K::NC, NO = K::NO;
  const int n_o = K::n_o(kk);
  extern __shared__ float sums[];  // [n_o][Tb]
  for (int64_t t = blockIdx.x; t < n_tiles; t += gridDim.x) {
    const int64_t b0 = t * Tb;
    const int64_t nb = b0 + Tb < n_b ? Tb : n_b - b0;
    for (int64_t j = threadIdx.x; j < (int64_t)n_o * Tb; j += blockDim.x) sums[j] = 0.f;
    __syncthreads();
    const int64_t r0 = tile_off[t], r1 = tile_off[t + 1];
    for (int64_t base = r0 + threadIdx.x; base < r1; base += (int64_t)kUnroll * blockDim.x) {
      int4 v[kUnroll];
#pragma unroll
      for (int u = 0; u < kUnroll; ++u) {
        const int64_t i = base + (int64_t)u * blockDim.x;
        v[u] = i < r1 ? __ldcs(rec + i) : make_int4(-1, 0, 0, 0);
      }
      float m[kUnroll][NC];
      float z[kUnroll][NO];
#pragma unroll
      for (int u = 0; u < kUnroll; ++u) {
        const int bl = (int)((unsigned)v[u].y & 0xFFFFFFu);
        if (v[u].x >= 0) {
          load_map<NC, float>(map, v[u].x, m[u]);
#pragma unroll
          for (int o = 0; o < NO; ++o) z[u][o] = o < n_o ? __ldg(x + o * n_b + b0 + bl) : 0.f;
        }
      }
#pragma unroll
      for (int u = 0; u < kUnroll; ++u) {
        if (v[u].x < 0) continue;
        const float n = (float)((unsigned)v[u].y >> 24);
        const int bl = (int)((unsigned)v[u].y & 0xFFFFFFu);
        const float c = __int_as_float(v[u].z), sn = __int_as_float(v[u].w);
#pragma unroll
        for (int o = 0; o < NO; ++o)
          if (o < n_o)
            atomicAdd(sums + o * Tb + bl,
                      fmaf(n, z[u][o], -run_dot<NC>(K::kind(o, kk), n, c, sn, m[u])));
      }
    }
    __syncthreads();
    for (int o = 0; o < n_o; ++o)
      for (int64_t j = threadIdx.x; j < nb; j += blockDim.x)
        out[o * n_b + b0 + j] = to_f64(sums[o * Tb + j]);
    __syncthreads();
  }
}

// The binning over long tiles (many days: each pixel's runs of a tile are summed
// in registers, so that reductions are few): warps take chunks of kChunk records
// of one tile, gather the baselines from L2 (the tile's baselines span a few MB),
// and carry their last pixel across rounds as k_tl_bin does.
template <int KS>
__global__ void __launch_bounds__(kBlock) k_tl_bin_long(const int4* __restrict__ rec,
                                                        const int64_t* __restrict__ tile_off,
                                                        const int64_t* __restrict__ chunk_first,
                                                        int64_t n_tiles, int64_t n_chunks,
                                                        int64_t Tb, const float* __restrict__ x,
                                                        float* __restrict__ bins, int64_t n_b,
                                                        KindsArg kk, Gate g) {
  if (gate_closed(g)) return;
  using K = KSet<KS>;
  constexpr int NC = K::NC, NO = K::NO;
  const int n_o = K::n_o(kk);
  const int lane = threadIdx.x & 31;
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t ch = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); ch < n_chunks;
       ch += warps) {
    int64_t t = 0;  // the chunk's tile: few tiles, a linear walk
    while (t + 1 < n_tiles && chunk_first[t + 1] <= ch) ++t;
    const int64_t lo = tile_off[t] + (ch - chunk_first[t]) * kChunk;
    const int64_t hi = lo + kChunk < tile_off[t + 1] ? lo + kChunk : tile_off[t + 1];
    const float* xb = x + t * Tb;
    int ckey = -1;
    float carry[NC];
#pragma unroll
    for (int j = 0; j < NC; ++j) carry[j] = 0.f;
    for (int64_t base = lo; base < hi; base += 32 * kUnroll) {
      int4 v[kUnroll];
#pragma unroll
      for (int u = 0; u < kUnroll; ++u) {
        const int64_t i = base + 32 * u + lane;
        v[u] = i < hi ? __ldcs(rec + i) : make_int4(-1, 0, 0, 0);
      }
      float z[kUnroll][NO];
#pragma unroll
      for (int u = 0; u < kUnroll; ++u) {
        const int bl = (int)((unsigned)v[u].y & 0xFFFFFFu);
#pragma unroll
        for (int o = 0; o < NO; ++o)
          z[u][o] = (o < n_o && v[u].x >= 0) ? __ldg(xb + o * n_b + bl) : 0.f;
      }
#pragma unroll
      for (int u = 0; u < kUnroll; ++u) {
        if (base + 32 * u >= hi) break;  // warp-uniform
        float acc[NC];
#pragma unroll
        for (int j = 0; j < NC; ++j) acc[j] = 0.f;
        const int key = v[u].x;
        if (key >= 0) {
          const float n = (float)((unsigned)v[u].y >> 24);
          const float c = __int_as_float(v[u].z), sn = __int_as_float(v[u].w);
#pragma unroll
          for (int o = 0; o < NO; ++o)
            if (o < n_o) run_bin<NC>(K::kind(o, kk), n, c, sn, z[u][o], acc);
        }
        tl_bin_round<NC>(key, acc, ckey, carry, bins);
      }
    }
    if (lane == 0 && ckey >= 0) flush_bins<NC, float>(bins, ckey, carry);
  }
}

}  // namespace

bool tl_ready(const Plan& P) { return P.layout == 3 && P.tl_rec != nullptr && P.x32 != nullptr; }

static int tl_grid(const Plan& P, int per_sm) {
  const int64_t g = (int64_t)P.num_sms * (per_sm > 0 ? per_sm : 1);
  return (int)(P.tl_tiles < g ? P.tl_tiles : g);
}

void launch_bin_tl(const Plan& P, cudaStream_t st, Gate g) {
  if (P.tl2_rec != nullptr) {
    with_kindset(P.kindset, [&](auto ksc) {
      constexpr int KS = decltype(ksc)::value;
      k_tl_bin_long<KS><<<stream_grid(P, P.tl2_chunks * 32, kBlock, 8), kBlock, 0, st>>>(
          P.tl2_rec, P.tl2_off, P.tl2_chunk, P.tl2_tiles, P.tl2_chunks, P.tl2_tb, P.x32, P.bins32,
          P.n_b, P.kinds, g);
    });
    return;
  }
  const size_t smem = sizeof(float) * (size_t)P.n_o * P.tl_tb;
  with_kindset(P.kindset, [&](auto ksc) {
    constexpr int KS = decltype(ksc)::value;
    k_tl_bin<KS><<<tl_grid(P, P.tl_bin_blocks), kTileThreads, smem, st>>>(
        P.tl_rec, P.tl_off, P.tl_tiles, P.tl_tb, P.x32, P.bins32, P.n_b, P.kinds, g);
  });
}

void launch_rescan_tl(const Plan& P, cudaStream_t st, double* out, Gate g) {
  const size_t smem = sizeof(float) * (size_t)P.n_o * P.tl_tb;
  with_kindset(P.kindset, [&](auto ksc) {
    constexpr int KS = decltype(ksc)::value;
    k_tl_rescan<KS><<<tl_grid(P, P.tl_rescan_blocks), kTileThreads, smem, st>>>(
        P.tl_rec, P.tl_off, P.tl_tiles, P.tl_tb, P.x32, P.map32, out, P.n_b, P.kinds, g);
  });
}

// Sorts the time-ordered runs by pixel within tiles of Tb baselines into *out_rec
// (16-byte records), with the tiles' first records in *out_off (stream-ordered on
// the plan's stream; one counting sort per tile over the pixels).
static cudaError_t tl_sort(Plan& P, int64_t Tb, int4** out_rec, int64_t** out_off) {
  cudaStream_t st = P.stream;
  const int64_t n_tiles = (P.n_b + Tb - 1) / Tb;
  const int64_t npix = P.npix;
  const int64_t g = stream_grid(P, npix, kBlock, 8);
  const int64_t S = (npix + g - 1) / g, G = (npix + S - 1) / S;
  uint32_t* cnt = nullptr;
  int64_t *blk = nullptr, *pos = nullptr;
  cudaError_t e = plan_alloc(P, reinterpret_cast<void**>(out_rec), sizeof(int4) * P.rl_n, true);
  if (e == cudaSuccess)
    e = plan_alloc(P, reinterpret_cast<void**>(out_off), sizeof(int64_t) * (n_tiles + 1), true);
  if (e == cudaSuccess) e = plan_alloc(P, reinterpret_cast<void**>(&cnt), sizeof(uint32_t) * npix, false);
  if (e == cudaSuccess) e = plan_alloc(P, reinterpret_cast<void**>(&blk), sizeof(int64_t) * G, false);
  if (e == cudaSuccess) e = plan_alloc(P, reinterpret_cast<void**>(&pos), sizeof(int64_t) * npix, false);
  if (e == cudaSuccess) {
    k_tl_bounds<<<(unsigned)((n_tiles + 1 + 127) / 128), 128, 0, st>>>(P.rl_b, P.rl_n, n_tiles,
                                                                       Tb, *out_off);
    const int rg = stream_grid(P, (P.rl_n + n_tiles - 1) / n_tiles, kBlock, 8);
    for (int64_t t = 0; t < n_tiles && e == cudaSuccess; ++t) {
      e = cudaMemsetAsync(cnt, 0, sizeof(uint32_t) * npix, st);
      if (e != cudaSuccess) break;
      k_tl_hist<<<rg, kBlock, 0, st>>>(P.rl_rec, *out_off, t, cnt);
      k_tl_scan_up<<<(unsigned)G, kBlock, 0, st>>>(cnt, npix, S, blk);
      k_tl_scan_top<<<1, 1, 0, st>>>(blk, G, *out_off, t);
      k_tl_scan_down<<<(unsigned)G, kBlock, 0, st>>>(cnt, npix, S, blk, pos);
      k_tl_scatter<<<rg, kBlock, 0, st>>>(P.rl_rec, P.rl_b, *out_off, t, Tb,
                                          reinterpret_cast<unsigned long long*>(pos), *out_rec);
      P.launches += 5;
      e = cudaGetLastError();
    }
  }
  for (void* t : {(void*)cnt, (void*)blk, (void*)pos})
    if (t) cudaFreeAsync(t, st);
  return e;
}

static void tl_free(Plan& P) {
  void* mine[] = {P.tl_rec, P.tl_off, P.tl2_rec, P.tl2_off, P.tl2_chunk};
  for (void* t : mine)
    if (t) cudaFreeAsync(t, P.stream);
  P.tl_rec = nullptr;
  P.tl_off = nullptr;
  P.tl2_rec = nullptr;
  P.tl2_off = nullptr;
  P.tl2_chunk = nullptr;
}

// Builds the tiled records from the time-ordered run records: tiles of a few
// hours for the rescan (their baseline sums fit in shared memory), and tiles of
// about 2^26 samples for the binning (each pixel's runs of many days summed in
// registers).  One host synchronisation for the longest run, one for the chunk
// table.  Returns DS_ESTATE, leaving nothing behind, when a run is longer than
// 255 samples.
ds_status tl_build(Plan& P) {
  if (P.rl_rec == nullptr || P.rl_n <= 0) return DS_ESTATE;
  cudaStream_t st = P.stream;
  int64_t Tb = kTileFloats / P.n_o;
  if (Tb > P.n_b) Tb = P.n_b;
  int64_t Tb2 = (int64_t(1) << 26) / P.L;
  if (Tb2 > (int64_t(1) << 24) - 1) Tb2 = (int64_t(1) << 24) - 1;
  if (Tb2 < Tb) Tb2 = Tb;
  if (Tb2 > P.n_b) Tb2 = P.n_b;
  const int64_t n_tiles = (P.n_b + Tb - 1) / Tb, n_tiles2 = (P.n_b + Tb2 - 1) / Tb2;
  int* longest = nullptr;
  const int64_t held_before = P.device_bytes;
  auto release = [&](cudaError_t e) {
    if (longest) cudaFreeAsync(longest, st);
    tl_free(P);
    P.device_bytes = held_before;
    return e == cudaErrorMemoryAllocation ? DS_ENOMEM : DS_ECUDA;
  };
  cudaError_t e = plan_alloc(P, reinterpret_cast<void**>(&longest), sizeof(int), false);
  if (e == cudaSuccess) e = cudaMemsetAsync(longest, 0, sizeof(int), st);
  if (e != cudaSuccess) return release(e);
  k_tl_longest<<<stream_grid(P, P.rl_n, kBlock, 8), kBlock, 0, st>>>(P.rl_rec, P.rl_n, longest);
  int h_longest = 0;
  e = cudaMemcpyAsync(&h_longest, longest, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return release(e);
  cudaFreeAsync(longest, st);
  longest = nullptr;
  if (h_longest > 255) {
    release(cudaSuccess);
    return DS_ESTATE;
  }
  e = tl_sort(P, Tb, &P.tl_rec, &P.tl_off);
  if (e != cudaSuccess) return release(e);
  // the long tiles and their chunk table (tile t's chunks start at chunk_first[t])
  if (n_tiles2 < n_tiles) {
    e = tl_sort(P, Tb2, &P.tl2_rec, &P.tl2_off);
    std::vector<int64_t> off(n_tiles2 + 1), first(n_tiles2 + 1);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(off.data(), P.tl2_off, sizeof(int64_t) * (n_tiles2 + 1),
                          cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return release(e);
    first[0] = 0;
    for (int64_t t = 0; t < n_tiles2; ++t)
      first[t + 1] = first[t] + (off[t + 1] - off[t] + kChunk - 1) / kChunk;
    e = plan_alloc(P, reinterpret_cast<void**>(&P.tl2_chunk), sizeof(int64_t) * (n_tiles2 + 1), true);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(P.tl2_chunk, first.data(), sizeof(int64_t) * (n_tiles2 + 1),
                          cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);  // first[] leaves scope
    if (e != cudaSuccess) return release(e);
    P.tl2_tiles = n_tiles2;
    P.tl2_tb = Tb2;
    P.tl2_chunks = first[n_tiles2];
  }
  P.tl_tiles = n_tiles;
  P.tl_tb = Tb;
  // shared arrays above 48 KB need the kernels' opt-in; resident blocks per SM
  const size_t smem = sizeof(float) * (size_t)P.n_o * Tb;
  with_kindset(P.kindset, [&](auto ksc) {
    constexpr int KS = decltype(ksc)::value;
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(k_tl_bin<KS>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(k_tl_rescan<KS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)smem);
    if (e == cudaSuccess)
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&P.tl_bin_blocks, k_tl_bin<KS>,
                                                        kTileThreads, smem);
    if (e == cudaSuccess)
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&P.tl_rescan_blocks, k_tl_rescan<KS>,
                                                        kTileThreads, smem);
  });
  if (e != cudaSuccess || P.tl_bin_blocks < 1 || P.tl_rescan_blocks < 1) {
    tl_free(P);
    P.device_bytes = held_before;
    return e == cudaSuccess ? DS_ESTATE : DS_ECUDA;
  }
  return DS_OK;
}

}  // namespace ds
