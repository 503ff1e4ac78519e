// Plan-time construction of the run-length records used by runs.cu: the runs of
// consecutive samples on one pixel within a baseline (samples of weight 0 end a
// run), each summarised by its pixel, sample count and the sums of cos 2psi and
// sin 2psi (float32 for the float32 operator, double-float pairs for the
// accurate passes), in sample order.
#include "df.cuh"
#include "internal.cuh"

namespace ds {

namespace {

constexpr int kBlock = 256;
constexpr int kSub = 512;  // samples per warp in the construction: 16 rounds of 32
constexpr int kScanThreads = 1024;

// Baseline cursor of a warp walking the timeline in rounds of 32 samples: the
// baseline b0 and offset r0 (< L) of the round's first sample t0, advanced without
// a 64-bit division per sample.
struct Cursor {
  int64_t b0, r0;
  __device__ __forceinline__ Cursor(int64_t t0, int64_t L) : b0(t0 / L), r0(t0 - (t0 / L) * L) {}
  // baselines crossed between t0 and t0 + k (k < 64), and the offset of t0 + k
  __device__ __forceinline__ void at(int k, int64_t L, int64_t& b, int64_t& off) const {
    const int64_t q = r0 + k;
    if (L >= 32) {
      const bool wrap = q >= L;  // q < L + 32 <= 2 L
      b = b0 + (wrap ? 1 : 0);
      off = wrap ? q - L : q;
    } else {
      const unsigned w = (unsigned)q / (unsigned)L;  // q < 64
      b = b0 + w;
      off = q - (int64_t)w * L;
    }
  }
  __device__ __forceinline__ void advance(int64_t L) {
    int64_t b, off;
    at(32, L, b, off);
    b0 = b;
    r0 = off;
  }
};

// A run starts at a valid sample whose predecessor is another pixel or in
// another baseline (off: the sample's offset in its baseline; prev: the pixel
// before it).
__device__ __forceinline__ bool run_start(int p, int prev, int64_t off) {
  return p >= 0 && (off == 0 || prev != p);
}

// Round loads: the pixel (-1 past the end) and the angles of sample t0 + lane.
// Issued one round ahead of their use, so that a warp's next round is in flight
// while it works on the current one.
__device__ __forceinline__ void fetch_round(const int32_t* __restrict__ pix,
                                            const float* __restrict__ cc,
                                            const float* __restrict__ ss, int64_t t0, int64_t n_t,
                                            int lane, int& p, float& c, float& s) {
  const int64_t t = t0 + lane;
  const bool in = t < n_t;
  p = in ? pix[t] : -1;
  c = in && cc != nullptr ? cc[t] : 0.f;
  s = in && ss != nullptr ? ss[t] : 0.f;
}

// Runs starting in each stretch of kSub samples.  Block j takes the S consecutive
// stretches [j S, (j + 1) S), each warp a contiguous share of them, walked in
// coalesced rounds of 32 samples (ballots of the run starts).  sub_off[w] gets the
// runs before stretch w within its block, blk[j] the block's total (made into
// block offsets by k_rl_scan).
__global__ void __launch_bounds__(kBlock) k_rl_count(const int32_t* __restrict__ pix, int64_t n_t,
                                                     int64_t L, int64_t n_sub, int64_t S,
                                                     int64_t* __restrict__ sub_off,
                                                     int64_t* __restrict__ blk) {
  __shared__ int64_t wsum[kBlock / 32];
  const unsigned full = 0xffffffffu;
  const int lane = threadIdx.x & 31, wq = threadIdx.x >> 5;
  constexpr int kWarps = kBlock / 32;
  const int64_t b0 = (int64_t)blockIdx.x * S;
  const int64_t b1 = b0 + S < n_sub ? b0 + S : n_sub;
  const int64_t per = (S + kWarps - 1) / kWarps;
  const int64_t lo = b0 + wq * per < b1 ? b0 + wq * per : b1;
  const int64_t hi = lo + per < b1 ? lo + per : b1;
  int64_t run = 0;
  if (lo < hi) {
    int64_t t0 = lo * kSub;
    Cursor cur(t0, L);
    int prev0 = t0 > 0 ? pix[t0 - 1] : -1;  // pixel before the round's lane 0
    int pn;
    float unused_c, unused_s;
    fetch_round(pix, nullptr, nullptr, t0, n_t, lane, pn, unused_c, unused_s);
    for (int64_t w = lo; w < hi; ++w) {
      int cnt = 0;
      for (int k = 0; k < kSub / 32; ++k, t0 += 32) {
        const int p = pn;
        fetch_round(pix, nullptr, nullptr, t0 + 32, n_t, lane, pn, unused_c, unused_s);
        int prev = __shfl_up_sync(full, p, 1);
        if (lane == 0) prev = prev0;
        prev0 = __shfl_sync(full, p, 31);
        int64_t b, off;
        cur.at(lane, L, b, off);
        cnt += __popc(__ballot_sync(full, run_start(p, prev, off)));
        cur.advance(L);
      }
      if (lane == 0) sub_off[w] = run;
      run += cnt;
    }
  }
  if (lane == 0) wsum[wq] = run;
  __syncthreads();
  if (threadIdx.x == 0) {
    int64_t acc = 0;
    for (int q = 0; q < kWarps; ++q) {
      const int64_t x = wsum[q];
      wsum[q] = acc;
      acc += x;
    }
    blk[blockIdx.x] = acc;
  }
  __syncthreads();
  if (lane == 0) {
    const int64_t wo = wsum[wq];
    for (int64_t w = lo; w < hi; ++w) sub_off[w] += wo;
  }
}

// Exclusive prefix sum in place, total in *total (one block; used on the block totals).
__global__ void __launch_bounds__(kScanThreads) k_rl_scan(int64_t* __restrict__ v, int64_t n,
                                                          int64_t* __restrict__ total) {
  __shared__ int64_t part[kScanThreads];
  const int64_t per = (n + kScanThreads - 1) / kScanThreads;
  const int64_t lo = (int64_t)threadIdx.x * per;
  const int64_t hi = lo + per < n ? lo + per : n;
  int64_t s = 0;
  for (int64_t i = lo; i < hi; ++i) s += v[i];
  part[threadIdx.x] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    int64_t run = 0;
    for (int i = 0; i < kScanThreads; ++i) {
      const int64_t x = part[i];
      part[i] = run;
      run += x;
    }
    *total = run;
  }
  __syncthreads();
  int64_t run = part[threadIdx.x];
  for (int64_t i = lo; i < hi; ++i) {
    const int64_t x = v[i];
    v[i] = run;
    run += x;
  }
}

// One record per run.  Each warp fills the runs that start in its stretch, in
// rounds of 32 consecutive samples (one per lane): a ballot of the run starts
// gives every run its place in sample order, a segmented shuffle scan sums
// (count, cos 2psi, sin 2psi) over the lanes of each run, and the lane where a run
// ends writes it.  A run still open at the end of a round carries its partial
// sums into the next round (runs end at baseline ends, so a warp may carry past
// its stretch and finish the run in the samples after it).
__global__ void __launch_bounds__(kBlock) k_rl_fill(const int32_t* __restrict__ pix,
                                                    const float* __restrict__ cc,
                                                    const float* __restrict__ ss, int64_t n_t,
                                                    int64_t L, int64_t n_sub, int64_t S,
                                                    const int64_t* __restrict__ sub_off,
                                                    const int64_t* __restrict__ blk,
                                                    RunRec* __restrict__ rec,
                                                    int32_t* __restrict__ rb,
                                                    float4* __restrict__ rdf) {
  const unsigned full = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  const unsigned upto = lane == 31 ? full : (2u << lane) - 1u;
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t w = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); w < n_sub;
       w += warps) {
    int64_t base = sub_off[w] + blk[w / S];
    // partial sums of a run opened in an earlier round (cr < 0: none)
    float cn = 0.f;
    df cC{0.f, 0.f}, cS{0.f, 0.f};
    int64_t cr = -1;
    Cursor cur(w * kSub, L);
    int prev0 = w > 0 ? pix[w * kSub - 1] : -1;  // pixel before the round's lane 0
    int pn;
    float cv_n, sv_n;
    fetch_round(pix, cc, ss, w * kSub, n_t, lane, pn, cv_n, sv_n);
    for (int64_t t0 = w * kSub; ; t0 += 32, cur.advance(L)) {
      const bool own = t0 < (w + 1) * kSub;  // rounds past the stretch only finish a carried run
      if (!own && cr < 0) break;
      const int p = pn;
      const float cv = cv_n, sv = sv_n;
      fetch_round(pix, cc, ss, t0 + 32, n_t, lane, pn, cv_n, sv_n);
      int prev = __shfl_up_sync(full, p, 1);
      if (lane == 0) prev = prev0;
      prev0 = __shfl_sync(full, p, 31);
      const int64_t t = t0 + lane;
      int64_t bl, off;
      cur.at(lane, L, bl, off);
      const bool valid = p >= 0;
      const bool rstart = run_start(p, prev, off);
      const unsigned rmask = __ballot_sync(full, rstart);
      const unsigned smask = own ? rmask : 0u;  // runs this warp fills
      const bool start = own && rstart;
      const unsigned hm = rmask & upto;
      const int head = hm ? 31 - __clz(hm) : -1;  // lane of the last run start at or before this one
      // a run started in this round is ours only inside the stretch; with no start
      // at or before this lane the sample continues the carried run, if any
      const bool member = valid && (head >= 0 ? own : cr >= 0);
      float n = member ? 1.f : 0.f;
      df C = member ? df_make(cv) : df{0.f, 0.f};
      df S = member ? df_make(sv) : df{0.f, 0.f};
      const int seg0 = head >= 0 ? head : 0;
      // the scan needs only the steps that reach the longest run's first lane
      const unsigned reach = __reduce_max_sync(full, member ? (unsigned)(lane - seg0) : 0u);
#pragma unroll
      for (int d = 1; d < 32; d <<= 1) {
        if ((unsigned)d > reach) break;
        const float n2 = __shfl_up_sync(full, n, d);
        const df C2 = df{__shfl_up_sync(full, C.hi, d), __shfl_up_sync(full, C.lo, d)};
        const df S2 = df{__shfl_up_sync(full, S.hi, d), __shfl_up_sync(full, S.lo, d)};
        if (lane - d >= seg0) {
          n += n2;
          C = df_add(C, C2);
          S = df_add(S, S2);
        }
      }
      if (head < 0 && cr >= 0) {
        n += cn;
        C = df_add(C, cC);
        S = df_add(S, cS);
      }
      // does the next sample continue this lane's run?
      const bool nstart = __shfl_down_sync(full, start, 1);
      const bool nmember = __shfl_down_sync(full, member, 1);
      const int pnext = __shfl_sync(full, pn, 0);  // the sample after lane 31 (-1 past the end)
      bool cont;
      if (lane < 31) {
        cont = nmember && !nstart;
      } else {
        cont = member && t + 1 < n_t && off + 1 != L && pnext == p;
      }
      const int64_t r = head >= 0 ? base + __popc(smask & ((1u << head) - 1u)) : cr;
      if (member && !cont) {
        rec[r] = RunRec{p, n, C.hi, S.hi};
        rb[r] = (int32_t)bl;
        if (rdf != nullptr) rdf[r] = make_float4(C.hi, C.lo, S.hi, S.lo);
      }
      // carry lane 31's open run into the next round
      const bool carry = __shfl_sync(full, member && cont, 31);
      cn = __shfl_sync(full, n, 31);
      cC = df{__shfl_sync(full, C.hi, 31), __shfl_sync(full, C.lo, 31)};
      cS = df{__shfl_sync(full, S.hi, 31), __shfl_sync(full, S.lo, 31)};
      const int64_t r31 = __shfl_sync(full, r, 31);
      cr = carry ? r31 : -1;
      base += __popc(smask);
    }
  }
}

// ---- pixel-major copy of the records (runs_pm.cu bins from it) ------------------

// Runs per pixel (cnt zeroed by the caller).
__global__ void __launch_bounds__(kBlock) k_pm_hist(const RunRec* __restrict__ rec, int64_t n_runs,
                                                    uint32_t* __restrict__ cnt) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n_runs; i += stride)
    atomicAdd(cnt + __ldcs(reinterpret_cast<const int*>(rec + i)), 1u);
}

__device__ __forceinline__ int64_t block_sum(int64_t v, int64_t* sh) {
  const int lane = threadIdx.x & 31, wq = threadIdx.x >> 5;
  for (int d = 16; d > 0; d >>= 1) v += __shfl_down_sync(0xffffffffu, v, d);
  if (lane == 0) sh[wq] = v;
  __syncthreads();
  int64_t t = 0;
  for (int q = 0; q < (int)(blockDim.x >> 5); ++q) t += sh[q];
  __syncthreads();
  return t;
}

// blk[j] = sum of cnt over block j's S consecutive pixels.
__global__ void __launch_bounds__(kBlock) k_pm_scan_up(const uint32_t* __restrict__ cnt, int64_t n,
                                                       int64_t S, int64_t* __restrict__ blk) {
  __shared__ int64_t sh[kBlock / 32];
  const int64_t lo = (int64_t)blockIdx.x * S, hi = lo + S < n ? lo + S : n;
  int64_t v = 0;
  for (int64_t i = lo + threadIdx.x; i < hi; i += blockDim.x) v += cnt[i];
  const int64_t t = block_sum(v, sh);
  if (threadIdx.x == 0) blk[blockIdx.x] = t;
}

// off[p] = first run of pixel p: block j's offset (blk, made exclusive by k_rl_scan)
// plus the prefix within the block, in tiles of blockDim pixels; cnt becomes the
// scatter cursor (= off).  off[n] = the total.
__global__ void __launch_bounds__(kBlock) k_pm_scan_down(uint32_t* __restrict__ cnt, int64_t n,
                                                         int64_t S, const int64_t* __restrict__ blk,
                                                         const int64_t* __restrict__ total,
                                                         uint32_t* __restrict__ off) {
  __shared__ int64_t wsum[kBlock / 32];
  const unsigned full = 0xffffffffu;
  const int lane = threadIdx.x & 31, wq = threadIdx.x >> 5;
  const int64_t lo = (int64_t)blockIdx.x * S, hi = lo + S < n ? lo + S : n;
  int64_t carry = blk[blockIdx.x];
  for (int64_t base = lo; base < hi; base += blockDim.x) {
    const int64_t i = base + threadIdx.x;
    const int64_t v = i < hi ? cnt[i] : 0;
    int64_t inc = v;  // inclusive scan within the warp
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
    if (i < hi) {
      const uint32_t o = (uint32_t)(carry + before + inc - v);
      off[i] = o;
      cnt[i] = o;
    }
    carry += tile;
    __syncthreads();
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) off[n] = (uint32_t)*total;
}

// Each run to its pixel's next slot: (count, sum cos, sum sin, baseline bits) and
// the low parts of the double-float sums (the record's sums are their high
// parts).  The order of the runs within a pixel is arbitrary.
__global__ void __launch_bounds__(kBlock) k_pm_scatter(const RunRec* __restrict__ rec,
                                                       const int32_t* __restrict__ rb,
                                                       const float4* __restrict__ rdf,
                                                       int64_t n_runs, uint32_t* __restrict__ cursor,
                                                       float4* __restrict__ pm_rec,
                                                       float2* __restrict__ pm_lo) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n_runs; i += stride) {
    const int4 r = __ldcs(reinterpret_cast<const int4*>(rec) + i);
    const int b = __ldcs(rb + i);
    const float4 cs = __ldcs(rdf + i);
    const uint32_t slot = atomicAdd(cursor + r.x, 1u);
    pm_rec[slot] = make_float4(__int_as_float(r.y), __int_as_float(r.z), __int_as_float(r.w),
                               __int_as_float(b));
    pm_lo[slot] = make_float2(cs.y, cs.w);
  }
}

}  // namespace

// Run records are built in two steps around the plan's synchronisation: the
// count (and its prefix over tiles) is enqueued first; once the host knows the
// total it allocates the records and enqueues the fill.
// Stretches per counting block (S) and counting blocks (G) for n_sub stretches:
// G x S >= n_sub with S a whole number of warp shares.
static void count_split(const Plan& P, int64_t n_sub, int64_t& S, int64_t& G) {
  const int64_t g = stream_grid(P, n_sub * 32, kBlock, 8);
  S = (n_sub + g - 1) / g;
  G = (n_sub + S - 1) / S;
}

ds_status rl_count(Plan& P, int64_t* d_total) {
  const int64_t n_sub = (P.n_t + kSub - 1) / kSub;
  int64_t S, G;
  count_split(P, n_sub, S, G);
  // per-stretch offsets within their block, then the block offsets
  DS_CUDA_TRY(plan_alloc(P, reinterpret_cast<void**>(&P.rl_tiles), sizeof(int64_t) * (n_sub + G),
                         false));
  k_rl_count<<<(unsigned)G, kBlock, 0, P.stream>>>(P.pix, P.n_t, P.L, n_sub, S, P.rl_tiles,
                                                   P.rl_tiles + n_sub);
  k_rl_scan<<<1, kScanThreads, 0, P.stream>>>(P.rl_tiles + n_sub, G, d_total);
  P.launches += 2;
  DS_CUDA_TRY(cudaGetLastError());
  return DS_OK;
}

ds_status rl_fill(Plan& P, int64_t n_runs, bool with_df) {
  const int64_t n_sub = (P.n_t + kSub - 1) / kSub;
  P.rl_n = n_runs;
  DS_CUDA_TRY(plan_alloc(P, reinterpret_cast<void**>(&P.rl_rec),
                         sizeof(RunRec) * (n_runs > 0 ? n_runs : 1), true));
  DS_CUDA_TRY(plan_alloc(P, reinterpret_cast<void**>(&P.rl_b),
                         sizeof(int32_t) * (n_runs > 0 ? n_runs : 1), true));
  const int grid = stream_grid(P, n_sub * 32, kBlock, 8);
  if (with_df)
    DS_CUDA_TRY(plan_alloc(P, reinterpret_cast<void**>(&P.rl_df),
                           sizeof(float4) * (n_runs > 0 ? n_runs : 1), true));
  int64_t S, G;
  count_split(P, n_sub, S, G);
  k_rl_fill<<<grid, kBlock, 0, P.stream>>>(P.pix, P.c, P.s, P.n_t, P.L, n_sub, S, P.rl_tiles,
                                           P.rl_tiles + n_sub, P.rl_rec, P.rl_b, P.rl_df);
  P.launches += 1;
  DS_CUDA_TRY(cudaGetLastError());
  cudaFreeAsync(P.rl_tiles, P.stream);
  P.rl_tiles = nullptr;
  return DS_OK;
}

// On request after the plan exists (synchronises once).
// The pixel-major copy of the records: runs per pixel, their prefix, a scatter
// with one atomic cursor per pixel.  Stream-ordered; no host synchronisation.
// Built on first use by a single-problem solve or operator application (batched
// problems bin with their own kernels and never need it).
ds_status pm_build(Plan& P, cudaStream_t st) {
  // run offsets are 32-bit, with room for the binning loop's stride past the end
  // (and the runs' double-float sums, whose low parts it keeps)
  if (P.rl_rec == nullptr || P.rl_df == nullptr || P.rl_n <= 0 ||
      P.rl_n > (int64_t)UINT32_MAX - 256)
    return DS_OK;
  const int64_t npix = P.npix;
  const int64_t g = stream_grid(P, npix, kBlock, 8);
  const int64_t S = (npix + g - 1) / g, G = (npix + S - 1) / S;
  uint32_t* cnt = nullptr;  // runs per pixel, then the scatter cursor (scratch)
  int64_t* blk = nullptr;   // block totals and the total (scratch)
  const int64_t held_before = P.device_bytes;
  cudaError_t e = plan_alloc_on(P, st, reinterpret_cast<void**>(&P.pm_off), sizeof(uint32_t) * (npix + 1), true);
  if (e == cudaSuccess) e = plan_alloc_on(P, st, reinterpret_cast<void**>(&P.pm_rec), sizeof(float4) * P.rl_n, true);
  if (e == cudaSuccess) e = plan_alloc_on(P, st, reinterpret_cast<void**>(&P.pm_lo), sizeof(float2) * P.rl_n, true);
  if (e == cudaSuccess) e = plan_alloc_on(P, st, reinterpret_cast<void**>(&P.x4), sizeof(float4) * P.n_b, true);
  if (e == cudaSuccess) e = plan_alloc_on(P, st, reinterpret_cast<void**>(&P.xd4), sizeof(float4) * 2 * P.n_b, true);
  if (e == cudaSuccess) e = plan_alloc_on(P, st, reinterpret_cast<void**>(&cnt), sizeof(uint32_t) * npix, false);
  if (e == cudaSuccess) e = plan_alloc_on(P, st, reinterpret_cast<void**>(&blk), sizeof(int64_t) * (G + 1), false);
  // On any failure give back what was taken and leave no half-built copy behind:
  // without the copy the binning reads the runs in time order.
  auto release = [&](cudaError_t err) {
    void** held[] = {reinterpret_cast<void**>(&P.pm_off), reinterpret_cast<void**>(&P.pm_rec),
                     reinterpret_cast<void**>(&P.pm_lo), reinterpret_cast<void**>(&P.x4),
                     reinterpret_cast<void**>(&P.xd4), reinterpret_cast<void**>(&cnt),
                     reinterpret_cast<void**>(&blk)};
    for (void** h : held)
      if (*h != nullptr) {
        cudaFreeAsync(*h, st);
        *h = nullptr;
      }
    P.device_bytes = held_before;
    return err == cudaErrorMemoryAllocation ? DS_ENOMEM : DS_ECUDA;
  };
  if (e != cudaSuccess) return release(e);
  e = cudaMemsetAsync(cnt, 0, sizeof(uint32_t) * npix, st);
  if (e != cudaSuccess) return release(e);
  const int rgrid = stream_grid(P, P.rl_n, kBlock, 8);
  k_pm_hist<<<rgrid, kBlock, 0, st>>>(P.rl_rec, P.rl_n, cnt);
  k_pm_scan_up<<<(unsigned)G, kBlock, 0, st>>>(cnt, npix, S, blk);
  k_rl_scan<<<1, kScanThreads, 0, st>>>(blk, G, blk + G);
  k_pm_scan_down<<<(unsigned)G, kBlock, 0, st>>>(cnt, npix, S, blk, blk + G, P.pm_off);
  k_pm_scatter<<<rgrid, kBlock, 0, st>>>(P.rl_rec, P.rl_b, P.rl_df, P.rl_n, cnt, P.pm_rec, P.pm_lo);
  P.launches += 5;
  e = cudaGetLastError();
  if (e != cudaSuccess) return release(e);
  cudaFreeAsync(cnt, st);
  cudaFreeAsync(blk, st);
  return DS_OK;
}

// Frees a pixel-major copy (built or not) ordered after the work on st.
void pm_release(Plan& P, cudaStream_t st) {
  void** held[] = {reinterpret_cast<void**>(&P.pm_off), reinterpret_cast<void**>(&P.pm_rec),
                   reinterpret_cast<void**>(&P.pm_lo), reinterpret_cast<void**>(&P.x4),
                   reinterpret_cast<void**>(&P.xd4)};
  for (void** h : held)
    if (*h != nullptr) {
      cudaFreeAsync(*h, st);
      *h = nullptr;
    }
  P.pm_pending = 0;
}

static bool pm_needed(const Plan& P) {
  return P.layout == 2 && P.bin_order == 1 && P.pm_rec == nullptr && P.rl_rec != nullptr;
}

// Without room for the copy the binning reads the runs in time order instead.
static ds_status pm_outcome(Plan& P, ds_status s) {
  if (s == DS_ENOMEM) {
    cudaGetLastError();
    P.bin_order = 0;
    return DS_OK;
  }
  return s;
}

ds_status pm_ensure(Plan& P) {
  if (!pm_needed(P)) return DS_OK;
  return pm_outcome(P, pm_build(P, P.stream));
}

ds_status pm_begin(Plan& P, bool* started) {
  *started = false;
  if (!pm_needed(P)) return DS_OK;
  if (P.side_stream == nullptr) {
    DS_CUDA_TRY(cudaStreamCreateWithFlags(&P.side_stream, cudaStreamNonBlocking));
    for (cudaEvent_t& e : P.side_ev) DS_CUDA_TRY(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
  }
  // the run records come from the plan's stream
  DS_CUDA_TRY(cudaEventRecord(P.side_ev[0], P.stream));
  DS_CUDA_TRY(cudaStreamWaitEvent(P.side_stream, P.side_ev[0], 0));
  const ds_status s = pm_build(P, P.side_stream);
  if (s != DS_OK) return pm_outcome(P, s);
  // until pm_join orders the plan's stream after the build, nothing may bin from
  // the copy (a warm start's first operator application comes before the join)
  P.pm_pending = 1;
  if (cudaEventRecord(P.side_ev[1], P.side_stream) != cudaSuccess) {
    cudaStreamSynchronize(P.side_stream);
    pm_release(P, P.side_stream);
    return DS_ECUDA;
  }
  *started = true;
  return DS_OK;
}

ds_status pm_join(Plan& P, bool started) {
  if (!started) return DS_OK;
  if (cudaStreamWaitEvent(P.stream, P.side_ev[1], 0) != cudaSuccess) {
    // the plan's stream cannot be ordered after the build: wait for it here
    if (cudaStreamSynchronize(P.side_stream) != cudaSuccess) {
      pm_release(P, P.side_stream);
      return DS_ECUDA;
    }
  }
  P.pm_pending = 0;
  return DS_OK;
}

void rl_release(Plan& P, cudaStream_t st) {
  void** held[] = {reinterpret_cast<void**>(&P.rl_rec), reinterpret_cast<void**>(&P.rl_b),
                   reinterpret_cast<void**>(&P.rl_df), reinterpret_cast<void**>(&P.rl_tiles)};
  for (void** h : held)
    if (*h != nullptr) {
      cudaFreeAsync(*h, st);
      *h = nullptr;
    }
  P.rl_n = 0;
}

ds_status rl_build(Plan& P, bool with_df) {
  int64_t* total = nullptr;
  DS_CUDA_TRY(plan_alloc(P, reinterpret_cast<void**>(&total), sizeof(int64_t), false));
  ds_status s = rl_count(P, total);
  int64_t n_runs = 0;
  if (s == DS_OK &&
      cudaMemcpyAsync(&n_runs, total, sizeof(int64_t), cudaMemcpyDeviceToHost, P.stream) != cudaSuccess)
    s = DS_ECUDA;
  if (s == DS_OK && cudaStreamSynchronize(P.stream) != cudaSuccess) s = DS_ECUDA;
  cudaFreeAsync(total, P.stream);
  if (s == DS_OK) s = rl_fill(P, n_runs, with_df);
  if (s == DS_OK && cudaStreamSynchronize(P.stream) != cudaSuccess) s = DS_ECUDA;
  return s;
}

}  // namespace ds
