// Time-tiled, pixel-sorted run records: the float32 operator of plans whose runs
// are short (about one pixel per sample, e.g. nside 512 at 50 Hz), where neither
// the time-ordered samples nor the pixel-major copy pays.
//
// The runs of consecutive samples on one pixel within a baseline (runs_build.cu)
// are cut into tiles of consecutive baselines, and within each tile sorted by a
// key per pixel (counting sorts over batches of tiles at plan time).  A record is
// 16 bytes:
//     (pixel, n << 24 | baseline - first baseline of the tile, sum cos 2psi, sum sin 2psi)
// with n <= 255 samples (plans with longer runs keep the other forms).  Two
// copies are kept, sorted within tiles of two lengths (Sect. 3 operator, exact
// reformulation: only the float32 rounding order changes):
//  * binning (P~^T R^T F~ x) reads long tiles (about two weeks of data), pixels in
//    the order of their first visit: a pixel is revisited every sidereal day, so
//    its runs of a tile are many and contiguous, and its neighbours along the scan
//    follow it, their runs sharing baselines.  Each lane sums consecutive records
//    of one pixel in registers, gathering each run's baselines (one float32, or a
//    16-byte vector of all outputs), and about one vector reduction per pixel and
//    tile reaches L2, instead of one per run as in time order;
//  * rescan and per-baseline sums (F~^T (z - R P~ m)) read short tiles (a few
//    hours), pixels in pixel order: each block keeps its tile's map-term sums per
//    baseline in shared memory (fixed-point integer atomics; the runs of one pixel
//    lie in different baselines, so lanes rarely collide), gathers the map row of each
//    run, and stores each baseline's valid samples times its baseline minus that
//    sum once (each baseline belongs to one tile: no atomics in global memory).
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

// Order of the pixels within a tile: by first visit.  first[p] = the first run on
// p (first zeroed to all ones before); rank[p] = how many pixels were visited
// before p first was.  A pixel's neighbours along the scan then sit next to it in
// the sorted records, and their runs share baselines (the baseline gathers of the
// passes hit in L1).
__global__ void __launch_bounds__(kBlock) k_tl_first(const RunRec* __restrict__ rec,
                                                     int64_t n_runs, uint32_t* __restrict__ first) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n_runs;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int p = rec[i].pix;
    if (i == 0 || rec[i - 1].pix != p) atomicMin(first + p, (uint32_t)i);
  }
}

// Pixels first visited in runs [g S, (g + 1) S) -> cnt[g]
__global__ void __launch_bounds__(kBlock) k_tl_rank_count(const RunRec* __restrict__ rec,
                                                          int64_t n_runs,
                                                          const uint32_t* __restrict__ first,
                                                          int64_t S, int64_t* __restrict__ cnt) {
  __shared__ int64_t sh[kBlock / 32];
  const int64_t lo = (int64_t)blockIdx.x * S, hi = lo + S < n_runs ? lo + S : n_runs;
  int64_t c = 0;
  for (int64_t i = lo + threadIdx.x; i < hi; i += blockDim.x)
    c += first[rec[i].pix] == (uint32_t)i ? 1 : 0;
  for (int d = 16; d > 0; d >>= 1) c += __shfl_down_sync(0xffffffffu, c, d);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = c;
  __syncthreads();
  if (threadIdx.x == 0) {
    int64_t s = 0;
    for (int q = 0; q < kBlock / 32; ++q) s += sh[q];
    cnt[blockIdx.x] = s;
  }
}

// rank[p] for the pixels first visited in runs [g S, (g + 1) S), in run order from
// the block's offset off[g]
__global__ void __launch_bounds__(kBlock) k_tl_rank_write(const RunRec* __restrict__ rec,
                                                          int64_t n_runs,
                                                          const uint32_t* __restrict__ first,
                                                          int64_t S, const int64_t* __restrict__ off,
                                                          int32_t* __restrict__ rank) {
  __shared__ int wsum[kBlock / 32];
  const int lane = threadIdx.x & 31, wq = threadIdx.x >> 5;
  const int64_t lo = (int64_t)blockIdx.x * S, hi = lo + S < n_runs ? lo + S : n_runs;
  int64_t base = off[blockIdx.x];
  for (int64_t b0 = lo; b0 < hi; b0 += blockDim.x) {
    const int64_t i = b0 + threadIdx.x;
    const int p = i < hi ? rec[i].pix : -1;
    const bool mark = i < hi && first[p] == (uint32_t)i;
    const unsigned bal = __ballot_sync(0xffffffffu, mark);
    if (lane == 0) wsum[wq] = __popc(bal);
    __syncthreads();
    int before = 0, total = 0;
    for (int q = 0; q < (int)(blockDim.x >> 5); ++q) {
      if (q < wq) before += wsum[q];
      total += wsum[q];
    }
    if (mark) rank[p] = (int32_t)(base + before + __popc(bal & ((1u << lane) - 1u)));
    base += total;
    __syncthreads();
  }
}

// seen[p] = 1 for the pixels some run visits (scanned into their numbering)
__global__ void __launch_bounds__(kBlock) k_tl_seen(const uint32_t* __restrict__ first,
                                                    int64_t npix, uint32_t* __restrict__ seen) {
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < npix;
       p += (int64_t)gridDim.x * blockDim.x)
    seen[p] = first[p] != 0xFFFFFFFFu ? 1u : 0u;
}

// Sort key of run i within a batch of tiles [t0, ..): (tile - t0) x nkeys + the
// pixel's rank (rank == nullptr: the pixel)
__device__ __forceinline__ int64_t tl_key(const RunRec& r, int32_t b, const int32_t* rank,
                                          int64_t Tb, int64_t t0, int64_t nkeys) {
  const int64_t k = rank != nullptr ? rank[r.pix] : r.pix;
  return ((int64_t)b / Tb - t0) * nkeys + k;
}

// Runs per key over the runs of tiles [t0, t1) (cnt zeroed before).
__global__ void __launch_bounds__(kBlock) k_tl_hist(const RunRec* __restrict__ rec,
                                                    const int32_t* __restrict__ rb,
                                                    const int32_t* __restrict__ rank,
                                                    const int64_t* __restrict__ tile_off,
                                                    int64_t t0, int64_t t1, int64_t Tb,
                                                    int64_t nkeys, uint32_t* __restrict__ cnt) {
  const int64_t r0 = tile_off[t0], r1 = tile_off[t1];
  for (int64_t i = r0 + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < r1;
       i += (int64_t)gridDim.x * blockDim.x)
    atomicAdd(cnt + tl_key(rec[i], rb[i], rank, Tb, t0, nkeys), 1u);
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

// blk[j] = start + sum of blk[0 .. j), start = tile_off[t] (or 0 without tile_off):
// one block of kScanTop threads, each over a contiguous share of the G entries.
constexpr int kScanTop = 1024;
__global__ void __launch_bounds__(kScanTop) k_tl_scan_top(int64_t* __restrict__ blk, int64_t G,
                                                          const int64_t* __restrict__ tile_off,
                                                          int64_t t) {
  __shared__ int64_t sh[kScanTop / 32];
  const int lane = threadIdx.x & 31, wq = threadIdx.x >> 5;
  const int64_t per = (G + kScanTop - 1) / kScanTop;
  const int64_t lo = (int64_t)threadIdx.x * per, hi = lo + per < G ? lo + per : G;
  int64_t s = 0;
  for (int64_t j = lo; j < hi; ++j) s += blk[j];
  int64_t inc = s;
  for (int d = 1; d < 32; d <<= 1) {
    const int64_t u = __shfl_up_sync(0xffffffffu, inc, d);
    if (lane >= d) inc += u;
  }
  if (lane == 31) sh[wq] = inc;
  __syncthreads();
  int64_t before = tile_off != nullptr ? tile_off[t] : 0;
  for (int q = 0; q < wq; ++q) before += sh[q];
  int64_t run = before + inc - s;
  for (int64_t j = lo; j < hi; ++j) {
    const int64_t x = blk[j];
    blk[j] = run;
    run += x;
  }
}

__global__ void __launch_bounds__(kBlock) k_tl_scan_down(uint32_t* __restrict__ cnt, int64_t n,
                                                         int64_t S, const int64_t* __restrict__ blk) {
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
    if (i < hi) cnt[i] = (uint32_t)(carry + before + inc - v);
    carry += tile;
    __syncthreads();
  }
}

// Each run of tiles [t0, t1) to its key's next slot (absolute cursors), as a
// 16-byte record with the baseline relative to its tile.
__global__ void __launch_bounds__(kBlock) k_tl_scatter(const RunRec* __restrict__ rec,
                                                       const int32_t* __restrict__ rb,
                                                       const int32_t* __restrict__ rank,
                                                       const int64_t* __restrict__ tile_off,
                                                       int64_t t0, int64_t t1, int64_t Tb,
                                                       int64_t nkeys, uint32_t* __restrict__ cursor,
                                                       int4* __restrict__ out) {
  const int64_t r0 = tile_off[t0], r1 = tile_off[t1];
  for (int64_t i = r0 + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < r1;
       i += (int64_t)gridDim.x * blockDim.x) {
    const RunRec r = rec[i];
    const int32_t b = rb[i];
    const unsigned bl = (unsigned)((int64_t)b % Tb);
    const int64_t slot = atomicAdd(cursor + tl_key(r, b, rank, Tb, t0, nkeys), 1u);
    out[slot] = make_int4(r.pix, (int)(((unsigned)r.n << 24) | bl), __float_as_int(r.c),
                          __float_as_int(r.s));
  }
}

// ---- the operator's passes --------------------------------------------------------

constexpr int kUnroll = 4;     // records per thread loaded before any is used (rescan)
constexpr int kLaneRecs = 8;   // consecutive records a lane sums per round (binning)
constexpr int kRound = 32 * kLaneRecs;  // records per warp round
constexpr int kBinWarps = 8;   // warps per block of the binning
constexpr int64_t kChunk = kRound * 8;  // records per warp chunk of the binning

// x32[o][b] = x[o][b] rounded to float32, and (several outputs) x4[b] = every
// output's baseline b (one 16-byte gather per run record in the tiled binning).
// Two baselines per thread and iteration, so that two loads per output are in
// flight.  The first kernel of an operator application: it also clears the map
// maximum that the pixel solve raises for the rescan.
template <int NO>
__global__ void __launch_bounds__(kBlock) k_tl_pack(const double* __restrict__ x,
                                                    float* __restrict__ x32,
                                                    float4* __restrict__ x4, int64_t n_b, int n_o,
                                                    unsigned* __restrict__ mmax, Gate g) {
  if (gate_closed(g)) return;
  if (blockIdx.x == 0 && threadIdx.x == 0) *mmax = 0u;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int64_t half = (n_b + 1) >> 1;
  for (int64_t h = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; h < half; h += stride) {
    const int64_t b0 = h, b1 = h + half;  // two coalesced streams
    float v0[4] = {0.f, 0.f, 0.f, 0.f}, v1[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
    for (int o = 0; o < NO; ++o)
      if (o < n_o) {
        v0[o] = (float)x[o * n_b + b0];
        if (b1 < n_b) v1[o] = (float)x[o * n_b + b1];
      }
#pragma unroll
    for (int o = 0; o < NO; ++o)
      if (o < n_o) {
        x32[o * n_b + b0] = v0[o];
        if (b1 < n_b) x32[o * n_b + b1] = v1[o];
      }
    if constexpr (NO > 1) {
      x4[b0] = make_float4(v0[0], v0[1], v0[2], v0[3]);
      if (b1 < n_b) x4[b1] = make_float4(v1[0], v1[1], v1[2], v1[3]);
    }
  }
}

// The baselines of every output at baseline b.
template <int NO>
__device__ __forceinline__ void tl_gather(const float* __restrict__ x32,
                                          const float4* __restrict__ x4, int64_t b,
                                          float (&z)[NO]) {
  if constexpr (NO == 1) {
    z[0] = __ldg(x32 + b);
  } else {
    const float4 q = __ldg(x4 + b);
    const float a[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
    for (int o = 0; o < NO; ++o) z[o] = a[o];
  }
}

// Shared-memory slot of record j of a warp's round: an XOR swizzle over the eight
// 16-byte bank groups, so that both the coalesced stores (lane = j mod 32) and the
// lane-sequential loads (lane = j / kLaneRecs) are free of bank conflicts.
__device__ __forceinline__ int tl_swz(int j) { return j ^ ((j >> 3) & 7); }

// bins[p] += sum over the runs on p of the rows summed over the run times the
// run's baselines (float32), over long tiles whose records are sorted by pixel
// (pixels in first-visit order).  A warp takes chunks of kChunk records of one
// tile in rounds of kRound: the round is loaded with coalesced 16-byte loads,
// staged in shared memory, and each lane then sums kLaneRecs consecutive records
// in registers (one 16-byte baseline gather per record, issued for all its
// records first).  A pixel's records are contiguous, so a lane issues a
// reduction only for a pixel that starts and ends within its records; pixels
// that cross lanes are joined by one segmented scan over the lanes per round, and
// the round's last pixel is carried into the next round.  About one vector
// reduction per pixel and tile remains.
template <int KS>
__global__ void __launch_bounds__(32 * kBinWarps, 3) k_tl_bin_lanes(
    const int4* __restrict__ rec, const int64_t* __restrict__ tile_off,
    const int64_t* __restrict__ chunk_first, int64_t n_tiles, int64_t n_chunks, int64_t Tb,
    const float* __restrict__ x32, const float4* __restrict__ x4, float* __restrict__ bins,
    KindsArg kk, Gate g) {
  if (gate_closed(g)) return;
  using K = KSet<KS>;
  constexpr int NC = K::NC, NO = K::NO;
  const int n_o = K::n_o(kk);
  const unsigned full = 0xffffffffu;
  __shared__ int4 stage[kBinWarps][kRound];
  const int lane = threadIdx.x & 31, wq = threadIdx.x >> 5;
  int4* st = stage[wq];
  const int64_t warps = (int64_t)gridDim.x * kBinWarps;
  for (int64_t ch = (int64_t)blockIdx.x * kBinWarps + wq; ch < n_chunks; ch += warps) {
    int64_t t = 0, tb = n_tiles - 1;  // the chunk's tile: last t with chunk_first[t] <= ch
    while (t < tb) {
      const int64_t mid = (t + tb + 1) >> 1;
      if (__ldg(chunk_first + mid) <= ch) t = mid;
      else tb = mid - 1;
    }
    const int64_t lo = __ldg(tile_off + t) + (ch - __ldg(chunk_first + t)) * kChunk;
    const int64_t end = __ldg(tile_off + t + 1);
    const int64_t hi = lo + kChunk < end ? lo + kChunk : end;
    const int64_t b0 = t * Tb;
    int ckey = -1;  // the pixel carried from the previous round, and its sums
    float carry[NC];
#pragma unroll
    for (int j = 0; j < NC; ++j) carry[j] = 0.f;
    for (int64_t base = lo; base < hi; base += kRound) {
      int4 v[kLaneRecs];
#pragma unroll
      for (int u = 0; u < kLaneRecs; ++u) {
        const int64_t i = base + 32 * u + lane;
        v[u] = i < hi ? __ldcs(rec + i) : make_int4(-1, 0, 0, 0);
      }
      __syncwarp();  // the previous round's shared reads are done
#pragma unroll
      for (int u = 0; u < kLaneRecs; ++u) st[tl_swz(32 * u + lane)] = v[u];
      __syncwarp();
#pragma unroll
      for (int k = 0; k < kLaneRecs; ++k) v[k] = st[tl_swz(kLaneRecs * lane + k)];
      float z[kLaneRecs][NO];
#pragma unroll
      for (int k = 0; k < kLaneRecs; ++k) {
        if (v[k].x >= 0) {
          tl_gather<NO>(x32, x4, b0 + (int64_t)((unsigned)v[k].y & 0xFFFFFFu), z[k]);
        } else {
#pragma unroll
          for (int o = 0; o < NO; ++o) z[k][o] = 0.f;
        }
      }
      // the lane's records: its first pixel (head, when another follows), complete
      // pixels in between (reduced at once), and its last pixel (tail)
      int cur = -1, hkey = -1;
      bool has_head = false;
      float acc[NC], hacc[NC];
#pragma unroll
      for (int j = 0; j < NC; ++j) acc[j] = hacc[j] = 0.f;
#pragma unroll
      for (int k = 0; k < kLaneRecs; ++k) {
        const int key = v[k].x;
        if (key < 0) continue;  // past the chunk's end
        float w[NC];
#pragma unroll
        for (int j = 0; j < NC; ++j) w[j] = 0.f;
        const float n = (float)((unsigned)v[k].y >> 24);
        const float c = __int_as_float(v[k].z), sn = __int_as_float(v[k].w);
#pragma unroll
        for (int o = 0; o < NO; ++o)
          if (o < n_o) run_bin<NC>(K::kind(o, kk), n, c, sn, z[k][o], w);
        if (key != cur) {
          if (cur >= 0) {
            if (!has_head) {
              has_head = true;
              hkey = cur;
#pragma unroll
              for (int j = 0; j < NC; ++j) hacc[j] = acc[j];
            } else {
              flush_bins<NC, float>(bins, cur, acc);
            }
          }
          cur = key;
#pragma unroll
          for (int j = 0; j < NC; ++j) acc[j] = w[j];
        } else {
#pragma unroll
          for (int j = 0; j < NC; ++j) acc[j] += w[j];
        }
      }
      const int first = has_head ? hkey : cur;
      // the carried pixel joins lane 0's first pixel, or is complete
      if (lane == 0 && ckey >= 0) {
        if (first == ckey) {
#pragma unroll
          for (int j = 0; j < NC; ++j) {
            if (has_head) hacc[j] += carry[j];
            else acc[j] += carry[j];
          }
        } else {
          flush_bins<NC, float>(bins, ckey, carry);
        }
      }
      // segmented inclusive scan of the tails over the lanes: a segment starts at
      // a lane whose tail began inside it (it has a head) or whose tail pixel
      // differs from the previous lane's
      const int prev = __shfl_up_sync(full, cur, 1);
      bool f = lane == 0 || has_head || prev != cur;
#pragma unroll
      for (int d = 1; d < 32; d <<= 1) {
        const bool fu = __shfl_up_sync(full, f, d);
#pragma unroll
        for (int j = 0; j < NC; ++j) {
          const float su = __shfl_up_sync(full, acc[j], d);
          if (lane >= d && !f) acc[j] += su;
        }
        if (lane >= d && !f) f = fu;
      }
      // a head completes the pixel of the previous lanes' tails
      float before[NC];
#pragma unroll
      for (int j = 0; j < NC; ++j) before[j] = __shfl_up_sync(full, acc[j], 1);
      if (has_head) {
        if (lane > 0 && prev == hkey) {
#pragma unroll
          for (int j = 0; j < NC; ++j) hacc[j] += before[j];
        }
        flush_bins<NC, float>(bins, hkey, hacc);
      }
      // a tail is complete unless the next lane starts with the same pixel; the
      // last lane's tail is carried
      const int next_first = __shfl_down_sync(full, first, 1);
      if (lane < 31 && cur >= 0 && next_first != cur) flush_bins<NC, float>(bins, cur, acc);
      ckey = __shfl_sync(full, cur, 31);
#pragma unroll
      for (int j = 0; j < NC; ++j) carry[j] = __shfl_sync(full, acc[j], 31);
    }
    if (lane == 0 && ckey >= 0) flush_bins<NC, float>(bins, ckey, carry);
  }
}

// out[o][b] = nvalid[b] x[o][b] - sum over the tile's runs in baseline b of
// (row sums) . m_p: the baseline term of every run of b adds up to the valid
// samples of b times x, so only the map term is summed per run, in shared memory,
// and each baseline is stored once.  The shared sums are fixed-point integers
// (integer atomics on random addresses run about 4.5x faster than float ones):
// a run's term times 2^e, e set so that L x 3 x max|m| x 2^e <= 2^30 (a run's
// term is at most n x 3 max|m|, a baseline holds at most L samples), split into
// its rounded integer (hi) and the rest times 2^f (lo, f = 16 while L < 2^14,
// fewer beyond), so that no partial sum overflows and the result is exact to far
// below float32 rounding.  A map with a non-finite value gives NaN baselines.
// Each thread issues the loads of kUnroll records, then their map rows, before
// any sum.
template <int KS>
__global__ void __launch_bounds__(kTileThreads) k_tl_rescan(const int4* __restrict__ rec,
                                                            const int64_t* __restrict__ tile_off,
                                                            int64_t n_tiles, int64_t Tb,
                                                            const float* __restrict__ x32,
                                                            const int32_t* __restrict__ nvalid,
                                                            const float* __restrict__ map,
                                                            const unsigned* __restrict__ mmax,
                                                            int64_t L, double* __restrict__ out,
                                                            int64_t n_b, KindsArg kk, Gate g) {
  if (gate_closed(g)) return;
  using K = KSet<KS>;
  constexpr int NC = K::NC, NO = K::NO;
  const int n_o = K::n_o(kk);
  extern __shared__ int hi[];  // [n_o][Tb] integer parts, then [n_o][Tb] fractions x 2^f
  int* lo = hi + (int64_t)n_o * Tb;
  const float big = __uint_as_float(*mmax);
  const bool finite = big <= 3.0e38f;  // false for +inf and NaN
  int e = 0;
  if (finite && big > 0.f) {
    int ex = 0;
    frexp((double)L * 3.0 * (double)big, &ex);  // the bound is below 2^ex
    e = 30 - ex;
    e = e < -126 ? -126 : (e > 126 ? 126 : e);
  }
  // lo: at most L terms of at most 2^(f - 1) each stay below 2^29
  int f = 30 - (64 - __clzll((unsigned long long)L));
  f = f < 0 ? 0 : (f > 16 ? 16 : f);
  const float scale = ldexpf(1.f, e), inv = ldexpf(1.f, -e), frac = ldexpf(1.f, f),
              inv_lo = ldexpf(1.f, -e - f);
  for (int64_t t = blockIdx.x; t < n_tiles; t += gridDim.x) {
    const int64_t b0 = t * Tb;
    const int64_t nb = b0 + Tb < n_b ? Tb : n_b - b0;
    for (int64_t j = threadIdx.x; j < 2 * (int64_t)n_o * Tb; j += blockDim.x) hi[j] = 0;
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
#pragma unroll
      for (int u = 0; u < kUnroll; ++u)
        if (v[u].x >= 0) load_map<NC, float>(map, v[u].x, m[u]);
#pragma unroll
      for (int u = 0; u < kUnroll; ++u) {
        if (v[u].x < 0) continue;
        const float n = (float)((unsigned)v[u].y >> 24);
        const int bl = (int)((unsigned)v[u].y & 0xFFFFFFu);
        const float c = __int_as_float(v[u].z), sn = __int_as_float(v[u].w);
#pragma unroll
        for (int o = 0; o < NO; ++o)
          if (o < n_o) {
            // |q| <= 2^30 n / L; q - h is exact (q is a whole number from 2^23 up)
            const float q = -run_dot<NC>(K::kind(o, kk), n, c, sn, m[u]) * scale;
            const float h = rintf(q);
            atomicAdd(hi + o * Tb + bl, (int)h);
            atomicAdd(lo + o * Tb + bl, __float2int_rn((q - h) * frac));
          }
      }
    }
    __syncthreads();
    for (int o = 0; o < n_o; ++o)
      for (int64_t j = threadIdx.x; j < nb; j += blockDim.x) {
        const int64_t i = o * n_b + b0 + j;
        const float s =
            __int2float_rn(hi[o * Tb + j]) * inv + __int2float_rn(lo[o * Tb + j]) * inv_lo;
        out[i] = finite ? to_f64(fmaf((float)nvalid[b0 + j], x32[i], s))
                        : __longlong_as_double(0x7ff8000000000000LL);
      }
    __syncthreads();
  }
}

}  // namespace

// whether the plan's kind set gathers packed baselines (more than one output slot);
// with one, the passes gather x32 directly
static bool tl_packs(const Plan& P) {
  int no = 0;
  with_kindset(P.kindset, [&](auto ksc) { no = KSet<decltype(ksc)::value>::NO; });
  return no > 1;
}

bool tl_ready(const Plan& P) {
  return P.layout == 3 && P.tl_rec != nullptr && P.tl2_rec != nullptr && P.x32 != nullptr &&
         P.tl_mmax != nullptr &&
         (P.tl_x4 != nullptr || !tl_packs(P));
}

void launch_pack_tl(const Plan& P, cudaStream_t st, const double* x, Gate g) {
  const int grid = stream_grid(P, (P.n_b + 1) / 2, kBlock, 8);
  with_kindset(P.kindset, [&](auto ksc) {
    constexpr int NO = KSet<decltype(ksc)::value>::NO;
    k_tl_pack<NO><<<grid, kBlock, 0, st>>>(x, P.x32, P.tl_x4, P.n_b, P.n_o, P.tl_mmax, g);
  });
}

void launch_bin_tl(const Plan& P, cudaStream_t st, Gate g) {
  const int64_t warps = (int64_t)P.num_sms * P.tl_bin_blocks * kBinWarps;
  const int64_t need = (P.tl2_chunks + kBinWarps - 1) / kBinWarps;
  int grid = (int)(need < warps / kBinWarps ? need : warps / kBinWarps);
  if (grid < 1) grid = 1;
  with_kindset(P.kindset, [&](auto ksc) {
    constexpr int KS = decltype(ksc)::value;
    k_tl_bin_lanes<KS><<<grid, 32 * kBinWarps, 0, st>>>(P.tl2_rec, P.tl2_off, P.tl2_chunk,
                                                        P.tl2_tiles, P.tl2_chunks, P.tl2_tb, P.x32,
                                                        P.tl_x4, P.bins32, P.kinds, g);
  });
}

void launch_rescan_tl(const Plan& P, cudaStream_t st, double* out, Gate g) {
  const int64_t per_sm = P.tl_rescan_blocks > 0 ? P.tl_rescan_blocks : 1;
  const int64_t cap = (int64_t)P.num_sms * per_sm;
  const int grid = (int)(P.tl_tiles < cap ? P.tl_tiles : cap);
  const size_t smem = 2 * sizeof(int) * (size_t)P.n_o * P.tl_tb;
  with_kindset(P.kindset, [&](auto ksc) {
    constexpr int KS = decltype(ksc)::value;
    k_tl_rescan<KS><<<grid, kTileThreads, smem, st>>>(P.tl_rec, P.tl_off, P.tl_tiles, P.tl_tb,
                                                      P.x32, P.nvalid, P.map32, P.tl_mmax, P.L,
                                                      out, P.n_b, P.kinds, g);
  });
}

// Sorts the time-ordered runs by a key per pixel (rank[p], nkeys keys; or, with
// rank == nullptr, the pixel over nkeys = n_pix) within tiles of Tb baselines into
// *out_rec (16-byte records), with the tiles' first records in *out_off.  One
// counting sort per batch of tiles over the keys (tile, key).  One host
// synchronisation for the tile offsets; the rest is stream-ordered on the plan's
// stream.  keep_ends: every key's end (absolute) per tile, [n_tiles][nkeys].
static cudaError_t tl_sort(Plan& P, int64_t Tb, const int32_t* rank, int64_t nkeys,
                           int4** out_rec, int64_t** out_off, uint32_t** keep_ends = nullptr) {
  // counters per batch: kept within L2, where the histogram's and the scatter's
  // atomic updates stay (a batch of a few tiles; at least one)
  constexpr int64_t kSortCounts = int64_t(1) << 24;
  cudaStream_t st = P.stream;
  const int64_t n_tiles = (P.n_b + Tb - 1) / Tb;
  uint32_t* cnt = nullptr;
  int64_t* blk = nullptr;
  const int64_t per = kSortCounts / nkeys > 0 ? kSortCounts / nkeys : 1;  // tiles per batch
  const int64_t cap = (per < n_tiles ? per : n_tiles) * nkeys;
  const int64_t gmax = stream_grid(P, cap, kBlock, 8);
  // kept ends: the counters of every batch side by side (after the scatter each
  // cursor holds its key's end), 4 bytes per key and tile
  const bool keep = keep_ends != nullptr;
  const int64_t n_cnt = keep ? n_tiles * nkeys : cap;
  cudaError_t e = plan_alloc(P, reinterpret_cast<void**>(out_rec), sizeof(int4) * P.rl_n, true);
  if (e == cudaSuccess)
    e = plan_alloc(P, reinterpret_cast<void**>(out_off), sizeof(int64_t) * (n_tiles + 1), true);
  if (e == cudaSuccess) e = plan_alloc(P, reinterpret_cast<void**>(&cnt), sizeof(uint32_t) * n_cnt, keep);
  if (e == cudaSuccess) e = plan_alloc(P, reinterpret_cast<void**>(&blk), sizeof(int64_t) * gmax, false);
  std::vector<int64_t> off(n_tiles + 1);
  if (e == cudaSuccess) {
    k_tl_bounds<<<(unsigned)((n_tiles + 1 + 127) / 128), 128, 0, st>>>(P.rl_b, P.rl_n, n_tiles,
                                                                       Tb, *out_off);
    e = cudaMemcpyAsync(off.data(), *out_off, sizeof(int64_t) * (n_tiles + 1),
                        cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  }
  for (int64_t t0 = 0; t0 < n_tiles && e == cudaSuccess;) {
    const int64_t t1 = t0 + per < n_tiles ? t0 + per : n_tiles;
    const int64_t n = (t1 - t0) * nkeys;
    const int64_t g = stream_grid(P, n, kBlock, 8);
    const int64_t S = (n + g - 1) / g, G = (n + S - 1) / S;
    const int rg = stream_grid(P, off[t1] - off[t0] > 0 ? off[t1] - off[t0] : 1, kBlock, 8);
    uint32_t* c = keep ? cnt + t0 * nkeys : cnt;
    e = cudaMemsetAsync(c, 0, sizeof(uint32_t) * n, st);
    if (e != cudaSuccess) break;
    // positions are absolute (runs are fewer than 2^32)
    k_tl_hist<<<rg, kBlock, 0, st>>>(P.rl_rec, P.rl_b, rank, *out_off, t0, t1, Tb, nkeys, c);
    k_tl_scan_up<<<(unsigned)G, kBlock, 0, st>>>(c, n, S, blk);
    k_tl_scan_top<<<1, kScanTop, 0, st>>>(blk, G, *out_off, t0);
    k_tl_scan_down<<<(unsigned)G, kBlock, 0, st>>>(c, n, S, blk);
    k_tl_scatter<<<rg, kBlock, 0, st>>>(P.rl_rec, P.rl_b, rank, *out_off, t0, t1, Tb, nkeys, c,
                                        *out_rec);
    P.launches += 5;
    e = cudaGetLastError();
    t0 = t1;
  }
  if (keep && e == cudaSuccess) {
    *keep_ends = cnt;
    cnt = nullptr;
  }
  for (void* t : {(void*)cnt, (void*)blk})
    if (t) cudaFreeAsync(t, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);  // off[] leaves scope
  return e;
}

// rank[p] = first-visit order of the observed pixels (*nkeys of them); stream-
// ordered, one host synchronisation for the count.
// and cidx[p] = the number of observed pixels below p (the observed pixels
// numbered in pixel order: keys of the rescan's tiles over observed pixels only)
static cudaError_t tl_rank(Plan& P, int32_t** rank, int32_t** cidx, int64_t* nkeys) {
  cudaStream_t st = P.stream;
  const int64_t g = stream_grid(P, P.rl_n, kBlock, 8);
  const int64_t S = (P.rl_n + g - 1) / g, G = (P.rl_n + S - 1) / S;
  const int64_t gp = stream_grid(P, P.npix, kBlock, 8);
  const int64_t Sp = (P.npix + gp - 1) / gp, Gp = (P.npix + Sp - 1) / Sp;
  uint32_t* first = nullptr;
  int64_t* blk = nullptr;
  int64_t* blkp = nullptr;
  cudaError_t e = plan_alloc(P, reinterpret_cast<void**>(&first), sizeof(uint32_t) * P.npix, false);
  if (e == cudaSuccess) e = plan_alloc(P, reinterpret_cast<void**>(rank), sizeof(int32_t) * P.npix, false);
  if (e == cudaSuccess) e = plan_alloc(P, reinterpret_cast<void**>(cidx), sizeof(int32_t) * P.npix, false);
  if (e == cudaSuccess) e = plan_alloc(P, reinterpret_cast<void**>(&blk), sizeof(int64_t) * (G + 1), false);
  if (e == cudaSuccess) e = plan_alloc(P, reinterpret_cast<void**>(&blkp), sizeof(int64_t) * Gp, false);
  if (e == cudaSuccess) e = cudaMemsetAsync(first, 0xFF, sizeof(uint32_t) * P.npix, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(blk + G, 0, sizeof(int64_t), st);
  int64_t h_total = 0;
  if (e == cudaSuccess) {
    k_tl_first<<<stream_grid(P, P.rl_n, kBlock, 8), kBlock, 0, st>>>(P.rl_rec, P.rl_n, first);
    k_tl_rank_count<<<(unsigned)G, kBlock, 0, st>>>(P.rl_rec, P.rl_n, first, S, blk);
    k_tl_scan_top<<<1, kScanTop, 0, st>>>(blk, G + 1, nullptr, 0);  // blk[G] = the total
    k_tl_rank_write<<<(unsigned)G, kBlock, 0, st>>>(P.rl_rec, P.rl_n, first, S, blk, *rank);
    uint32_t* seen = reinterpret_cast<uint32_t*>(*cidx);
    k_tl_seen<<<(unsigned)gp, kBlock, 0, st>>>(first, P.npix, seen);
    k_tl_scan_up<<<(unsigned)Gp, kBlock, 0, st>>>(seen, P.npix, Sp, blkp);
    k_tl_scan_top<<<1, kScanTop, 0, st>>>(blkp, Gp, nullptr, 0);
    k_tl_scan_down<<<(unsigned)Gp, kBlock, 0, st>>>(seen, P.npix, Sp, blkp);
    P.launches += 8;
    e = cudaGetLastError();
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(&h_total, blk + G, sizeof(int64_t), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  }
  for (void* t : {(void*)first, (void*)blk, (void*)blkp})
    if (t) cudaFreeAsync(t, st);
  *nkeys = h_total;
  return e;
}

static void tl_free(Plan& P) {
  void* mine[] = {P.tl_rec, P.tl_off, P.tl2_rec, P.tl2_off, P.tl2_chunk, P.tl_x4, P.tl2_end,
                  P.tl_mmax};
  for (void* t : mine)
    if (t) cudaFreeAsync(t, P.stream);
  P.tl_mmax = nullptr;
  P.tl2_end = nullptr;
  P.tl_rec = nullptr;
  P.tl_off = nullptr;
  P.tl2_rec = nullptr;
  P.tl2_off = nullptr;
  P.tl2_chunk = nullptr;
  P.tl_x4 = nullptr;
}

// Builds the tiled records from the time-ordered run records: tiles of a few
// hours for the rescan (their baseline sums fit in shared memory), and tiles of
// P.tl_bin_samples samples (2^26 by default, about two weeks at 50 Hz) for the
// binning, so that each pixel's runs of many days are summed in registers.  One
// host synchronisation for the longest run, one for the chunk table.  Returns
// DS_ESTATE, leaving nothing behind, when a run is longer than 255 samples (or
// there are 2^32 - 1 runs or more).
ds_status tl_build(Plan& P) {
  // run indices are ranked as 32-bit numbers
  if (P.rl_rec == nullptr || P.rl_n <= 0 || P.rl_n >= (int64_t)0xFFFFFFFF) return DS_ESTATE;
  cudaStream_t st = P.stream;
  int64_t Tb = kTileFloats / P.n_o;
  if (Tb > P.n_b) Tb = P.n_b;
  int64_t Tb2 = P.tl_bin_samples / P.L;
  if (Tb2 < 1) Tb2 = 1;
  if (Tb2 > (int64_t(1) << 24) - 1) Tb2 = (int64_t(1) << 24) - 1;
  if (Tb2 > P.n_b) Tb2 = P.n_b;
  const int64_t n_tiles = (P.n_b + Tb - 1) / Tb, n_tiles2 = (P.n_b + Tb2 - 1) / Tb2;
  int* longest = nullptr;
  int32_t *rank = nullptr, *cidx = nullptr;
  const int64_t held_before = P.device_bytes;
  auto release = [&](cudaError_t e) {
    if (longest) cudaFreeAsync(longest, st);
    if (rank) cudaFreeAsync(rank, st);
    if (cidx) cudaFreeAsync(cidx, st);
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
  if (tl_packs(P)) e = plan_alloc(P, reinterpret_cast<void**>(&P.tl_x4), sizeof(float4) * P.n_b, true);
  if (e == cudaSuccess) e = plan_alloc(P, reinterpret_cast<void**>(&P.tl_mmax), sizeof(unsigned), true);
  if (e == cudaSuccess) e = cudaMemsetAsync(P.tl_mmax, 0, sizeof(unsigned), st);
  int64_t nkeys = 0;
  if (e == cudaSuccess) e = tl_rank(P, &rank, &cidx, &nkeys);
  if (e == cudaSuccess && nkeys <= 0) e = cudaErrorInvalidValue;
  // the rescan's tiles in pixel order (keys: the observed pixels numbered in pixel
  // order): the runs of neighbouring pixels along the scan share baselines, and
  // would collide on the tile's shared baseline sums
  if (e == cudaSuccess) e = tl_sort(P, Tb, cidx, nkeys, &P.tl_rec, &P.tl_off);
  if (e == cudaSuccess) {
    cudaFreeAsync(cidx, st);
    cidx = nullptr;
  }
  if (e != cudaSuccess) return release(e);
  // the long tiles and their chunk table (tile t's chunks start at chunk_first[t])
  e = tl_sort(P, Tb2, rank, nkeys, &P.tl2_rec, &P.tl2_off, &P.tl2_end);
  P.tl2_nkeys = nkeys;
  if (e == cudaSuccess) {
    cudaFreeAsync(rank, st);
    rank = nullptr;
  }
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
  P.tl_runs = P.rl_n;
  P.tl2_chunks = first[n_tiles2];
  P.tl_tiles = n_tiles;
  P.tl_tb = Tb;
  // the rescan's shared arrays above 48 KB need the kernel's opt-in; resident
  // blocks per SM of both passes
  const size_t smem = 2 * sizeof(int) * (size_t)P.n_o * Tb;
  with_kindset(P.kindset, [&](auto ksc) {
    constexpr int KS = decltype(ksc)::value;
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(k_tl_rescan<KS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)smem);
    if (e == cudaSuccess)
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&P.tl_bin_blocks, k_tl_bin_lanes<KS>,
                                                        32 * kBinWarps, 0);
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

// Builds the records a plan chose at its creation (synchronises); where they cannot be
// built (a run above 255 samples, too many runs, no room) the plan keeps the
// time-ordered operator.
ds_status tl_ensure(Plan& P) {
  if (!P.tl_pending) return DS_OK;
  P.tl_pending = 0;
  const bool made = P.rl_rec == nullptr;
  ds_status s = made ? rl_build(P, false) : DS_OK;
  if (s == DS_OK) s = tl_build(P);
  if (s == DS_OK && cudaStreamSynchronize(P.stream) != cudaSuccess) s = DS_ECUDA;
  if (s == DS_ESTATE || s == DS_ENOMEM) {
    cudaGetLastError();
    rl_release(P, P.stream);
    P.layout = 0;
    return DS_OK;
  }
  // the tiled records hold everything the passes read: the runs they came from go
  // (a later switch to the run-length layout builds them again)
  if (s == DS_OK && made) rl_release(P, P.stream);
  return s;
}

}  // namespace ds
