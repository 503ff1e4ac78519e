// Streaming kernels of the mixed-precision CG operator with the pointing staged
// through shared memory by TMA bulk copies (cp.async.bulk, mbarrier completion).
//
// Each block is persistent (two per SM) and runs a kStages-deep pipeline: one
// producer warp issues the bulk copies of the pixel, cos 2psi and sin 2psi
// streams of a 2048-sample tile into a free stage; eight consumer warps wait for
// the stage to fill, process it, and hand it back.  The copies keep about 192 KB
// in flight per SM, independent of the consumers' registers, which is what an
// HBM-bound stream needs; the consumers only touch shared memory and L2.
//
// Work per consumer round: each lane takes 4 consecutive samples of a 128-sample
// slice (one 16-byte shared load per stream), exactly the split of apply.cu, so
// the binning run aggregation and the warp-segmented baseline sums carry over.
//
// Every wait on an mbarrier is bounded by a clock budget; on expiry the kernel
// sets ERR_TIMEOUT in the plan's error word, stops issuing, waits (again
// bounded) for its own copies in flight and returns.
#include <type_traits>

#include "internal.cuh"
#include "rows.cuh"

namespace ds {

namespace {

constexpr int kConsumerWarps = 8;
constexpr int kThreads = (kConsumerWarps + 1) * 32;
constexpr long long kWaitBudget = 4000000000LL;  // clock cycles (~2 s at 2 GHz)

// Pipeline shapes: samples per stage, stages, resident blocks per SM.
//   deep : 2048 x 4 stages, 2 blocks/SM (192 KB of copies in flight per SM)
//   wide : 1024 x 3 stages, 3 blocks/SM (more consumer warps per SM)
template <int TILE_, int STAGES_, int BPS_>
struct PipeCfg {
  static constexpr int TILE = TILE_, STAGES = STAGES_, BPS = BPS_;
  static constexpr int ROUNDS = TILE / (kConsumerWarps * 128);  // 128-sample slices per warp
};
using CfgDeep = PipeCfg<2048, 4, 2>;
using CfgWide = PipeCfg<1024, 3, 3>;

template <int TILE>
struct __align__(128) StageBuf {
  int32_t pix[TILE];
  float c[TILE];
  float s[TILE];
};

template <class Cfg>
struct PipeSmem {
  StageBuf<Cfg::TILE> st[Cfg::STAGES];
  unsigned long long full[Cfg::STAGES];
  unsigned long long empty[Cfg::STAGES];
};

__device__ __forceinline__ unsigned smem_u32(const void* p) {
  return static_cast<unsigned>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(unsigned long long* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive(unsigned long long* bar) {
  asm volatile(
      "{\n\t.reg .b64 st;\n\tmbarrier.arrive.shared::cta.b64 st, [%0];\n\t}" ::"r"(smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(unsigned long long* bar, unsigned bytes) {
  asm volatile(
      "{\n\t.reg .b64 st;\n\tmbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n\t}" ::"r"(
          smem_u32(bar)),
      "r"(bytes)
      : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(unsigned long long* bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Bounded wait for the phase with the given parity to complete.
__device__ __forceinline__ bool mbar_wait(unsigned long long* bar, unsigned parity) {
  if (mbar_try_wait(bar, parity)) return true;
  const long long t0 = clock64();
  while (!mbar_try_wait(bar, parity)) {
    if (clock64() - t0 > kWaitBudget) return false;
  }
  return true;
}

__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, unsigned bytes,
                                         unsigned long long* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

// Producer: lane 0 of the last warp.  Fills stage k % STAGES with tile k of this block.
template <class Cfg>
__device__ void produce(PipeSmem<Cfg>& sm, const int32_t* __restrict__ pix,
                        const float* __restrict__ cc, const float* __restrict__ ss, int64_t n_t,
                        int64_t n_tiles, int32_t* __restrict__ err, volatile int* abort_flag) {
  constexpr int kTile = Cfg::TILE, kStages = Cfg::STAGES;
  int k = 0;
  for (int64_t tile = blockIdx.x; tile < n_tiles; tile += gridDim.x, ++k) {
    const int stage = k % kStages;
    if (k >= kStages) {
      if (!mbar_wait(&sm.empty[stage], ((k / kStages) - 1) & 1)) {
        atomicOr(err, ERR_TIMEOUT);
        *abort_flag = 1;
        break;
      }
    }
    if (*abort_flag) break;
    const int64_t t0 = tile * kTile;
    const int64_t n = (n_t - t0 < kTile) ? (n_t - t0) : kTile;
    const unsigned nb = (unsigned)((n >> 2) << 4);  // whole 16-byte groups only
    if (nb == 0) {
      mbar_arrive(&sm.full[stage]);
    } else {
      mbar_arrive_expect_tx(&sm.full[stage], 3u * nb);
      bulk_g2s(sm.st[stage].pix, pix + t0, nb, &sm.full[stage]);
      bulk_g2s(sm.st[stage].c, cc + t0, nb, &sm.full[stage]);
      bulk_g2s(sm.st[stage].s, ss + t0, nb, &sm.full[stage]);
    }
  }
  // Copies still in flight write into this block's shared memory: before the
  // block may retire, wait (bounded) until every issued stage has landed.
  const int issued = k;
  for (int j = (issued > kStages ? issued - kStages : 0); j < issued; ++j)
    mbar_wait(&sm.full[j % kStages], (j / kStages) & 1);
}

// Samples 4 lane .. 4 lane + 3 of a 128-sample slice: shared memory for the
// bulk-copied part, global memory for the last (n mod 4) samples of the stream.
template <int TILE>
__device__ __forceinline__ void read4(const StageBuf<TILE>& b, const int32_t* __restrict__ pix,
                                      const float* __restrict__ cc, const float* __restrict__ ss,
                                      int64_t t_tile, int off, int n, int (&p)[4], float (&c)[4],
                                      float (&s)[4]) {
  const int ncopy = n & ~3;
  if (off + 4 <= ncopy) {
    const int4 pp = *reinterpret_cast<const int4*>(&b.pix[off]);
    const float4 c4 = *reinterpret_cast<const float4*>(&b.c[off]);
    const float4 s4 = *reinterpret_cast<const float4*>(&b.s[off]);
    p[0] = pp.x; p[1] = pp.y; p[2] = pp.z; p[3] = pp.w;
    c[0] = c4.x; c[1] = c4.y; c[2] = c4.z; c[3] = c4.w;
    s[0] = s4.x; s[1] = s4.y; s[2] = s4.z; s[3] = s4.w;
  } else {
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const int i = off + k;
      const bool in = i < n;
      p[k] = in ? (i < ncopy ? b.pix[i] : pix[t_tile + i]) : -1;
      c[k] = in ? (i < ncopy ? b.c[i] : cc[t_tile + i]) : 0.f;
      s[k] = in ? (i < ncopy ? b.s[i] : ss[t_tile + i]) : 0.f;
    }
  }
}

// ---- binning consumer: float32 products, runs of equal pixels, one vector atomic ----
template <int KS>
struct BinBody {
  using K = KSet<KS>;
  static constexpr int NC = K::NC, NO = K::NO;
  const double* __restrict__ x;
  float* __restrict__ bins;
  int64_t L, n_b;
  KindsArg kk;

  __device__ __forceinline__ void flush(int p, const float (&acc)[NC]) const {
    float v[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
    for (int j = 0; j < NC; ++j) v[j] = acc[j];
    float* dst = bins + (int64_t)p * 4;
    asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(dst), "f"(v[0]),
                 "f"(v[1]), "f"(v[2]), "f"(v[3])
                 : "memory");
  }

  __device__ __forceinline__ void slice(int64_t t0, int nvalid, const int (&p)[4],
                                        const float (&c)[4], const float (&s)[4]) const {
    const int n_o = K::n_o(kk);
    if (nvalid <= 0) return;
    int64_t b = t0 / L;
    int64_t bend = (b + 1) * L;
    float zb[NO];
#pragma unroll
    for (int o = 0; o < NO; ++o) zb[o] = (o < n_o) ? (float)__ldg(x + o * n_b + b) : 0.f;
    float acc[NC];
#pragma unroll
    for (int j = 0; j < NC; ++j) acc[j] = 0.f;
    int cur = -1;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      if (k >= nvalid) break;
      if (t0 + k >= bend) {
        b += 1;
        bend += L;
#pragma unroll
        for (int o = 0; o < NO; ++o) zb[o] = (o < n_o) ? (float)__ldg(x + o * n_b + b) : 0.f;
      }
      if (p[k] < 0) continue;
      float w[NC];
#pragma unroll
      for (int j = 0; j < NC; ++j) w[j] = 0.f;
#pragma unroll
      for (int o = 0; o < NO; ++o)
        if (o < n_o) row_bin<NC, float>(K::kind(o, kk), c[k], s[k], zb[o], w);
      if (p[k] != cur) {
        if (cur >= 0) flush(cur, acc);
        cur = p[k];
#pragma unroll
        for (int j = 0; j < NC; ++j) acc[j] = w[j];
      } else {
#pragma unroll
        for (int j = 0; j < NC; ++j) acc[j] += w[j];
      }
    }
    if (cur >= 0) flush(cur, acc);
  }
};

// ---- rescan consumer: r = z - w . m, warp-segmented per-baseline sums ----------
template <int KS>
struct RescanBody {
  using K = KSet<KS>;
  static constexpr int NC = K::NC, NO = K::NO;
  const double* __restrict__ x;
  const float* __restrict__ map;
  double* __restrict__ out;
  int64_t L, n_b;
  KindsArg kk;

  // all lanes of the warp call this together (warp-uniform)
  __device__ __forceinline__ void slice(int64_t t0, int nvalid, const int (&p)[4],
                                        const float (&c)[4], const float (&s)[4]) const {
    const int n_o = K::n_o(kk);
    const unsigned full = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    int key = -1;
    float acc[NO];
#pragma unroll
    for (int o = 0; o < NO; ++o) acc[o] = 0.f;
    if (nvalid > 0) {
      float m[4][NC];
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        if (p[k] >= 0) {
          const float4 v = __ldg(reinterpret_cast<const float4*>(map) + p[k]);
          const float a[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
          for (int j = 0; j < NC; ++j) m[k][j] = a[j];
        } else {
#pragma unroll
          for (int j = 0; j < NC; ++j) m[k][j] = 0.f;
        }
      }
      int64_t b = t0 / L;
      int64_t bend = (b + 1) * L;
      float zb[NO];
#pragma unroll
      for (int o = 0; o < NO; ++o) zb[o] = (o < n_o) ? (float)__ldg(x + o * n_b + b) : 0.f;
      key = (int)b;
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        if (k >= nvalid) break;
        if (t0 + k >= bend) {
#pragma unroll
          for (int o = 0; o < NO; ++o) {
            if (o < n_o && acc[o] != 0.f) atomicAdd(out + o * n_b + b, (double)acc[o]);
            acc[o] = 0.f;
          }
          b += 1;
          bend += L;
          key = (int)b;
#pragma unroll
          for (int o = 0; o < NO; ++o) zb[o] = (o < n_o) ? (float)__ldg(x + o * n_b + b) : 0.f;
        }
        if (p[k] < 0) continue;
#pragma unroll
        for (int o = 0; o < NO; ++o)
          if (o < n_o) acc[o] += zb[o] - row_dot<NC, float>(K::kind(o, kk), c[k], s[k], m[k]);
      }
    }
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const int k2 = __shfl_down_sync(full, key, d);
#pragma unroll
      for (int o = 0; o < NO; ++o) {
        const float v2 = __shfl_down_sync(full, acc[o], d);
        if (lane + d < 32 && k2 == key) acc[o] += v2;
      }
    }
    const int kp = __shfl_up_sync(full, key, 1);
    if (key >= 0 && (lane == 0 || kp != key)) {
#pragma unroll
      for (int o = 0; o < NO; ++o)
        if (o < n_o) atomicAdd(out + (int64_t)o * n_b + key, (double)acc[o]);
    }
  }
};

template <class Cfg, class Body>
__global__ void __launch_bounds__(kThreads, Cfg::BPS) k_stream_tma(const int32_t* __restrict__ pix,
                                                                   const float* __restrict__ cc,
                                                                   const float* __restrict__ ss,
                                                                   int64_t n_t, Body body,
                                                                   int32_t* __restrict__ err,
                                                                   Gate g) {
  constexpr int kTile = Cfg::TILE, kStages = Cfg::STAGES, kRounds = Cfg::ROUNDS;
  if (gate_closed(g)) return;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  PipeSmem<Cfg>& sm = *reinterpret_cast<PipeSmem<Cfg>*>(smem_raw);
  __shared__ int abort_flag;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int i = 0; i < kStages; ++i) {
      mbar_init(&sm.full[i], 1);
      mbar_init(&sm.empty[i], kConsumerWarps);
    }
    abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  const int64_t n_tiles = (n_t + kTile - 1) / kTile;
  if (warp == kConsumerWarps) {
    if (lane == 0) produce<Cfg>(sm, pix, cc, ss, n_t, n_tiles, err, &abort_flag);
    return;
  }
  int k = 0;
  for (int64_t tile = blockIdx.x; tile < n_tiles; tile += gridDim.x, ++k) {
    const int stage = k % kStages;
    bool ok = mbar_wait(&sm.full[stage], (k / kStages) & 1);
    // warp-uniform decision: the lanes of a warp wait on the same barrier
    ok = __all_sync(0xffffffffu, ok) != 0;
    if (!ok || *(volatile int*)&abort_flag) {
      if (lane == 0) {
        atomicOr(err, ERR_TIMEOUT);
        *(volatile int*)&abort_flag = 1;
      }
      break;
    }
    const int64_t t_tile = tile * kTile;
    const int n = (int)((n_t - t_tile < kTile) ? (n_t - t_tile) : kTile);
    const StageBuf<kTile>& buf = sm.st[stage];
#pragma unroll
    for (int r = 0; r < kRounds; ++r) {
      const int off = (warp * kRounds + r) * 128 + 4 * lane;
      int p[4];
      float c[4], s[4];
      read4(buf, pix, cc, ss, t_tile, off, n, p, c, s);
      const int nvalid = n - off;  // samples of this lane inside the tile (may be <= 0)
      body.slice(t_tile + off, nvalid, p, c, s);
    }
    __syncwarp();
    if (lane == 0) mbar_arrive(&sm.empty[stage]);
  }
}

template <class Cfg, class Body>
void launch_stream_cfg(const Plan& P, cudaStream_t st, const Body& body, Gate g) {
  constexpr size_t kSmemBytes = sizeof(PipeSmem<Cfg>);
  // the limit is per kernel and per device: set it on every launch (a host call)
  cudaFuncSetAttribute(k_stream_tma<Cfg, Body>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)kSmemBytes);
  const int64_t n_tiles = (P.n_t + Cfg::TILE - 1) / Cfg::TILE;
  int64_t grid = (int64_t)P.num_sms * Cfg::BPS;
  if (grid > n_tiles) grid = n_tiles;
  if (grid < 1) grid = 1;
  k_stream_tma<Cfg, Body><<<(int)grid, kThreads, kSmemBytes, st>>>(P.pix, P.c, P.s, P.n_t, body,
                                                                     P.err, g);
}

template <class Body>
void launch_stream(const Plan& P, cudaStream_t st, const Body& body, Gate g) {
  if (P.stream_mode == 2) launch_stream_cfg<CfgWide>(P, st, body, g);
  else launch_stream_cfg<CfgDeep>(P, st, body, g);
}

}  // namespace

bool tma_supported(const Plan& P) {
  // 16-byte aligned streams (checked at plan time) and a float32 operator
  return P.desc.precision == DS_PREC_MIXED && P.bins32 != nullptr;
}

void launch_bin_tma(const Plan& P, cudaStream_t st, const double* x, Gate g) {
  with_kindset(P.kindset, [&](auto ksc) {
    constexpr int KS = decltype(ksc)::value;
    BinBody<KS> body{x, P.bins32, P.L, P.n_b, P.kinds};
    launch_stream(P, st, body, g);
  });
}

void launch_rescan_tma(const Plan& P, cudaStream_t st, const double* x, double* out, Gate g) {
  with_kindset(P.kindset, [&](auto ksc) {
    constexpr int KS = decltype(ksc)::value;
    RescanBody<KS> body{x, P.map32, out, P.L, P.n_b, P.kinds};
    launch_stream(P, st, body, g);
  });
}

}  // namespace ds
