// destripe_bin_noalloc: binned map straight from the pointing and the data,
// with no device allocation at all.
//
// Some callers cannot allocate device memory when they need a map: a process
// whose device memory is already owned by another allocator (a framework's
// caching pool that has reserved the GPU, so a cudaMalloc would fail or steal
// its budget), or an acquisition / control loop that forbids allocation after
// start-up because allocation may block the device or fail at an arbitrary
// moment.  This entry point serves them: the caller passes inputs and outputs,
// and all intermediate per-pixel sums live in one fixed array in device global
// memory that the library declares at file scope.  Every GPU that loads the
// library holds that array (4.2 MB) until the process exits.  The hits, the
// pixel matrices, the rcond cut and the inverses come from the very kernels a plan
// of the same descriptor uses (plan.cu, pixmat.cuh), written into that array, so
// that every pixel is kept or cut exactly as destripe_plan keeps or cuts it.
//
// Limits and sharing rules:
//  - maps of at most DS_NOALLOC_MAX_PIX pixels (nside <= 64);
//  - every call reuses the same array and clears the part it needs before
//    using it; calls that overlap on the GPU (for example on two streams, or
//    from two host threads without ordering) race on the array and must be
//    serialised by the caller;
//  - the first call on each device looks up the array's device address
//    (cudaGetSymbolAddress with that device current); make that first call
//    before any stream capture on the device.
#include <cstdint>
#include <mutex>

#include "internal.cuh"
#include "rows.cuh"

namespace ds {
namespace {

constexpr int kBlock = 256;
constexpr int64_t kMaxPix = DS_NOALLOC_MAX_PIX;
// Layout (in doubles): sums [kMaxPix][4] | normal matrices, then their inverses,
// packed [kMaxPix][NM <= 6] | hits int32 [kMaxPix] | mask uint8 [kMaxPix] |
// error word and kept-pixel count.
constexpr int64_t kSumOff = 0;
constexpr int64_t kMatOff = kSumOff + 4 * kMaxPix;
constexpr int64_t kHitOff = kMatOff + 6 * kMaxPix;
constexpr int64_t kMaskOff = kHitOff + kMaxPix / 2;
constexpr int64_t kErrOff = kMaskOff + kMaxPix / 8;
constexpr int64_t kScratchDoubles = kErrOff + 32;

static __device__ __align__(256) double g_noalloc_scratch[kScratchDoubles];

constexpr int kMaxDevices = 64;
std::mutex g_setup_lock;
double* g_scratch_addr[kMaxDevices] = {};

// Device address of the scratch array on the current device (set up once per device).
cudaError_t scratch_address(int device, double** out) {
  std::lock_guard<std::mutex> guard(g_setup_lock);
  if (g_scratch_addr[device] == nullptr) {
    void* ptr = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_addr[device] = static_cast<double*>(ptr);
  }
  *out = g_scratch_addr[device];
  return cudaSuccess;
}

__global__ void __launch_bounds__(kBlock) k_na_clear(double* __restrict__ scratch, int64_t npix) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < 10 * npix; i += stride) {
    if (i < 4 * npix) scratch[kSumOff + i] = 0.0;
    else scratch[kMatOff + (i - 4 * npix)] = 0.0;
  }
  int32_t* hits = reinterpret_cast<int32_t*>(scratch + kHitOff);
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < npix; i += stride)
    hits[i] = 0;
  if (blockIdx.x == 0 && threadIdx.x < 32) scratch[kErrOff + threadIdx.x] = 0.0;
}

// One pass over the samples: sums of w_o(t) y_o(t) on the kept pixels.
template <int KS, typename YT>
__global__ void __launch_bounds__(kBlock) k_na_sums(const int32_t* __restrict__ pix,
                                                    const float* __restrict__ cc,
                                                    const float* __restrict__ ss,
                                                    const uint8_t* __restrict__ valid,
                                                    const YT* __restrict__ y,
                                                    double* __restrict__ scratch, int64_t n_t,
                                                    int64_t npix, KindsArg kk) {
  using K = KSet<KS>;
  constexpr int NC = K::NC, NO = K::NO;
  const int n_o = K::n_o(kk);
  const uint8_t* mask = reinterpret_cast<const uint8_t*>(scratch + kMaskOff);
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n_t; t += stride) {
    if (valid != nullptr && valid[t] == 0) continue;
    const int p = pix[t];
    if (p < 0 || p >= npix || !mask[p]) continue;  // out of range: flagged by the matrix pass
    const double c = cc[t], s = ss[t];
    double sum[NC];
#pragma unroll
    for (int j = 0; j < NC; ++j) sum[j] = 0.0;
#pragma unroll
    for (int o = 0; o < NO; ++o)
      if (o < n_o) row_bin<NC, double>(K::kind(o, kk), c, s, (double)y[(int64_t)o * n_t + t], sum);
#pragma unroll
    for (int j = 0; j < NC; ++j) atomicAdd(scratch + kSumOff + 4 * (int64_t)p + j, sum[j]);
  }
}

// Per pixel: m_p = M_p^-1 s_p on kept pixels (0 elsewhere), hits and mask out.
template <int NC>
__global__ void __launch_bounds__(kBlock) k_na_map(const double* __restrict__ scratch,
                                                   int64_t npix, double* __restrict__ map,
                                                   int32_t* __restrict__ hits_out,
                                                   uint8_t* __restrict__ mask_out) {
  constexpr int NM = NC * (NC + 1) / 2;
  const int32_t* hits = reinterpret_cast<const int32_t*>(scratch + kHitOff);
  const uint8_t* mask = reinterpret_cast<const uint8_t*>(scratch + kMaskOff);
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < npix; p += stride) {
    double mi[NM], s[NC], m[NC];
#pragma unroll
    for (int j = 0; j < NM; ++j) mi[j] = scratch[kMatOff + NM * p + j];
#pragma unroll
    for (int j = 0; j < NC; ++j) s[j] = scratch[kSumOff + 4 * p + j];
    const bool keep = mask[p] != 0;
    if (keep) {
      sym_mul<NC>(mi, s, m);
    } else {
#pragma unroll
      for (int j = 0; j < NC; ++j) m[j] = 0.0;
    }
#pragma unroll
    for (int j = 0; j < NC; ++j) map[(int64_t)j * npix + p] = m[j];
    if (hits_out) hits_out[p] = hits[p];
    if (mask_out) mask_out[p] = keep ? 1 : 0;
  }
}

template <typename YT>
void na_launch_sums(int ks, int grid, cudaStream_t st, const int32_t* pix, const float* c,
                    const float* s, const uint8_t* valid, const YT* y, double* scratch,
                    int64_t n_t, int64_t npix, KindsArg kk) {
  with_kindset(ks, [&](auto ksc) {
    constexpr int KS = decltype(ksc)::value;
    k_na_sums<KS, YT><<<grid, kBlock, 0, st>>>(pix, c, s, valid, y, scratch, n_t, npix, kk);
  });
}

}  // namespace
}  // namespace ds

using namespace ds;

extern "C" ds_status destripe_bin_noalloc(const ds_desc* desc, const int32_t* d_pix,
                                          const float* d_cos2psi, const float* d_sin2psi,
                                          const uint8_t* d_valid, const void* d_y,
                                          double* d_map, int32_t* d_hits, uint8_t* d_mask) {
  if (desc == nullptr || d_pix == nullptr || d_cos2psi == nullptr || d_sin2psi == nullptr ||
      d_y == nullptr || d_map == nullptr)
    return DS_EINVAL;
  if (desc->n_samples < 1 || desc->n_samples >= (int64_t(1) << 31)) return DS_EINVAL;
  if (desc->nside < 1 || (desc->nside & (desc->nside - 1)) != 0) return DS_EINVAL;
  if (desc->n_outputs < 1 || desc->n_outputs > DS_MAX_OUTPUTS) return DS_EINVAL;
  if (desc->precision != DS_PREC_FP64 && desc->precision != DS_PREC_MIXED) return DS_EINVAL;
  if (desc->reserved != 0) return DS_EINVAL;
  const int64_t npix = int64_t(12) * desc->nside * desc->nside;
  if (npix > kMaxPix) return DS_EINVAL;  // map larger than the fixed scratch array
  // the matrix pass is the plan's own (vector loads of cos / sin)
  if ((reinterpret_cast<uintptr_t>(d_cos2psi) & 15) || (reinterpret_cast<uintptr_t>(d_sin2psi) & 15))
    return DS_EINVAL;
  bool has_i = false, has_p = false;
  KindsArg kk{};
  kk.n_o = desc->n_outputs;
  for (int o = 0; o < desc->n_outputs; ++o) {
    const int k = desc->kinds[o];
    if (k < DS_KIND_I || k > DS_KIND_IQU) return DS_EINVAL;
    kk.kind[o] = k;
    has_i |= (k == DS_KIND_I || k == DS_KIND_IQU);
    has_p |= (k != DS_KIND_I);
  }
  const int n_c = (has_i && has_p) ? 3 : (has_p ? 2 : 1);
  const double rcond_min = desc->rcond_min > 0.0 ? desc->rcond_min : 1e-3;
  int device = 0, sms = 0;
  if (cudaGetDevice(&device) != cudaSuccess || device < 0 || device >= kMaxDevices) return DS_ECUDA;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess)
    return DS_ECUDA;
  double* scratch = nullptr;
  if (scratch_address(device, &scratch) != cudaSuccess) return DS_ECUDA;
  (void)cudaGetLastError();
  cudaStream_t st = static_cast<cudaStream_t>(desc->stream);
  const int64_t n_t = desc->n_samples;
  auto grid_for = [&](int64_t n) {
    int64_t g = (n + kBlock - 1) / kBlock, cap = (int64_t)sms * 8;
    return (int)(g < 1 ? 1 : (g < cap ? g : cap));
  };
  k_na_clear<<<grid_for(10 * npix), kBlock, 0, st>>>(scratch, npix);
  const int ks = kindset_of(desc->kinds, desc->n_outputs, n_c);
  int32_t* hits = reinterpret_cast<int32_t*>(scratch + kHitOff);
  uint8_t* mask = reinterpret_cast<uint8_t*>(scratch + kMaskOff);
  int32_t* err = reinterpret_cast<int32_t*>(scratch + kErrOff);
  // hits, M_p, the cut and M_p^-1 exactly as a plan of this descriptor builds them
  launch_plan_matrices(ks, desc->precision == DS_PREC_MIXED, grid_for((n_t + 3) / 4), st, d_pix,
                       d_cos2psi, d_sin2psi, d_valid, hits, scratch + kMatOff, n_t, npix, kk, err);
  launch_pixel_invert(n_c, grid_for(npix), st, scratch + kMatOff, hits, mask, npix, rcond_min,
                      reinterpret_cast<unsigned long long*>(scratch + kErrOff + 1));
  if (desc->precision == DS_PREC_FP64)
    na_launch_sums<double>(ks, grid_for(n_t), st, d_pix, d_cos2psi, d_sin2psi, d_valid,
                           static_cast<const double*>(d_y), scratch, n_t, npix, kk);
  else
    na_launch_sums<float>(ks, grid_for(n_t), st, d_pix, d_cos2psi, d_sin2psi, d_valid,
                          static_cast<const float*>(d_y), scratch, n_t, npix, kk);
  const int pg = grid_for(npix);
  if (n_c == 1) k_na_map<1><<<pg, kBlock, 0, st>>>(scratch, npix, d_map, d_hits, d_mask);
  else if (n_c == 2) k_na_map<2><<<pg, kBlock, 0, st>>>(scratch, npix, d_map, d_hits, d_mask);
  else k_na_map<3><<<pg, kBlock, 0, st>>>(scratch, npix, d_map, d_hits, d_mask);
  if (cudaGetLastError() != cudaSuccess) return DS_ECUDA;
  int32_t err_h = 0;
  if (cudaMemcpyAsync(&err_h, scratch + kErrOff, sizeof(int32_t), cudaMemcpyDeviceToHost, st) !=
          cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return DS_ECUDA;
  return (err_h & ERR_PIX) ? DS_EPIX : DS_OK;
}
