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

__device__ __forceinline__ bool run_start(const int32_t* __restrict__ pix, int64_t t, int64_t L) {
  const int p = pix[t];
  return p >= 0 && (t % L == 0 || pix[t - 1] != p);
}

// Runs starting in each stretch of kSub samples, one warp per stretch (ballots
// over coalesced rounds of 32 samples; no block-wide synchronisation).
__global__ void __launch_bounds__(kBlock) k_rl_count(const int32_t* __restrict__ pix, int64_t n_t,
                                                     int64_t L, int64_t n_sub,
                                                     int64_t* __restrict__ sub_runs) {
  const int lane = threadIdx.x & 31;
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t w = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); w < n_sub;
       w += warps) {
    int cnt = 0;
    for (int k = 0; k < kSub / 32; ++k) {
      const int64_t t = w * kSub + k * 32 + lane;
      cnt += __popc(__ballot_sync(0xffffffffu, t < n_t && run_start(pix, t, L)));
    }
    if (lane == 0) sub_runs[w] = cnt;
  }
}

// Exclusive prefix sum of the per-stretch counts in place, total in *total (one block).
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
                                                    int64_t L, int64_t n_sub,
                                                    const int64_t* __restrict__ sub_off,
                                                    RunRec* __restrict__ rec,
                                                    int32_t* __restrict__ rb,
                                                    float4* __restrict__ rdf) {
  const unsigned full = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  const unsigned below = (1u << lane) - 1u;
  const unsigned upto = lane == 31 ? full : (2u << lane) - 1u;
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t w = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); w < n_sub;
       w += warps) {
    int64_t base = sub_off[w];
    // partial sums of a run opened in an earlier round (cr < 0: none)
    float cn = 0.f;
    df cC{0.f, 0.f}, cS{0.f, 0.f};
    int64_t cr = -1;
    for (int64_t t0 = w * kSub; ; t0 += 32) {
      const bool own = t0 < (w + 1) * kSub;  // rounds past the stretch only finish a carried run
      if (!own && cr < 0) break;
      const int64_t t = t0 + lane;
      const int p = t < n_t ? pix[t] : -1;
      const bool valid = p >= 0;
      const bool rstart = valid && run_start(pix, t, L);
      const unsigned rmask = __ballot_sync(full, rstart);
      const unsigned smask = own ? rmask : 0u;  // runs this warp fills
      const bool start = own && rstart;
      const unsigned hm = rmask & upto;
      const int head = hm ? 31 - __clz(hm) : -1;  // lane of the last run start at or before this one
      // a run started in this round is ours only inside the stretch; with no start
      // at or before this lane the sample continues the carried run, if any
      const bool member = valid && (head >= 0 ? own : cr >= 0);
      float n = member ? 1.f : 0.f;
      df C = member ? df_make(cc[t]) : df{0.f, 0.f};
      df S = member ? df_make(ss[t]) : df{0.f, 0.f};
      const int seg0 = head >= 0 ? head : 0;
#pragma unroll
      for (int d = 1; d < 32; d <<= 1) {
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
      bool cont;
      if (lane < 31) {
        cont = nmember && !nstart;
      } else {
        const int64_t u = t + 1;
        cont = member && u < n_t && u % L != 0 && pix[u] == p;
      }
      const int64_t r = head >= 0 ? base + __popc(smask & ((1u << head) - 1u)) : cr;
      if (member && !cont) {
        rec[r] = RunRec{p, n, C.hi, S.hi};
        rb[r] = (int32_t)(t / L);
        rdf[r] = make_float4(C.hi, C.lo, S.hi, S.lo);
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

}  // namespace

// Run records are built in two steps around the plan's synchronisation: the
// count (and its prefix over tiles) is enqueued first; once the host knows the
// total it allocates the records and enqueues the fill.
ds_status rl_count(Plan& P, int64_t* d_total) {
  const int64_t n_sub = (P.n_t + kSub - 1) / kSub;
  DS_CUDA_TRY(plan_alloc(P, reinterpret_cast<void**>(&P.rl_tiles), sizeof(int64_t) * n_sub, false));
  const int grid = stream_grid(P, n_sub * 32, kBlock, 8);
  k_rl_count<<<grid, kBlock, 0, P.stream>>>(P.pix, P.n_t, P.L, n_sub, P.rl_tiles);
  k_rl_scan<<<1, kScanThreads, 0, P.stream>>>(P.rl_tiles, n_sub, d_total);
  P.launches += 2;
  DS_CUDA_TRY(cudaGetLastError());
  return DS_OK;
}

ds_status rl_fill(Plan& P, int64_t n_runs) {
  const int64_t n_sub = (P.n_t + kSub - 1) / kSub;
  P.rl_n = n_runs;
  DS_CUDA_TRY(plan_alloc(P, reinterpret_cast<void**>(&P.rl_rec),
                         sizeof(RunRec) * (n_runs > 0 ? n_runs : 1), true));
  DS_CUDA_TRY(plan_alloc(P, reinterpret_cast<void**>(&P.rl_b),
                         sizeof(int32_t) * (n_runs > 0 ? n_runs : 1), true));
  const int grid = stream_grid(P, n_sub * 32, kBlock, 8);
  DS_CUDA_TRY(plan_alloc(P, reinterpret_cast<void**>(&P.rl_df),
                         sizeof(float4) * (n_runs > 0 ? n_runs : 1), true));
  k_rl_fill<<<grid, kBlock, 0, P.stream>>>(P.pix, P.c, P.s, P.n_t, P.L, n_sub, P.rl_tiles,
                                           P.rl_rec, P.rl_b, P.rl_df);
  P.launches += 1;
  DS_CUDA_TRY(cudaGetLastError());
  cudaFreeAsync(P.rl_tiles, P.stream);
  P.rl_tiles = nullptr;
  return DS_OK;
}

// On request after the plan exists (synchronises once).
ds_status rl_build(Plan& P) {
  int64_t* total = nullptr;
  DS_CUDA_TRY(plan_alloc(P, reinterpret_cast<void**>(&total), sizeof(int64_t), false));
  ds_status s = rl_count(P, total);
  int64_t n_runs = 0;
  if (s == DS_OK &&
      cudaMemcpyAsync(&n_runs, total, sizeof(int64_t), cudaMemcpyDeviceToHost, P.stream) != cudaSuccess)
    s = DS_ECUDA;
  if (s == DS_OK && cudaStreamSynchronize(P.stream) != cudaSuccess) s = DS_ECUDA;
  cudaFreeAsync(total, P.stream);
  if (s == DS_OK) s = rl_fill(P, n_runs);
  if (s == DS_OK && cudaStreamSynchronize(P.stream) != cudaSuccess) s = DS_ECUDA;
  return s;
}

}  // namespace ds
