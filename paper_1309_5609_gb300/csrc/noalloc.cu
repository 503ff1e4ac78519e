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
// library holds that array (4.2 MB) until the process exits.
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
// Layout (in doubles): sums [kMaxPix][4] | normal matrices [kMaxPix][6] |
// hits int32 [kMaxPix] | error word.
constexpr int64_t kSumOff = 0;
constexpr int64_t kMatOff = kSumOff + 4 * kMaxPix;
constexpr int64_t kHitOff = kMatOff + 6 * kMaxPix;
constexpr int64_t kErrOff = kHitOff + kMaxPix / 2;
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
  if (blockIdx.x == 0 && threadIdx.x == 0) reinterpret_cast<int32_t*>(scratch + kErrOff)[0] = 0;
}

template <int NC>
__device__ __forceinline__ constexpr int na_sym(int i, int j) {
  if (i > j) { int t = i; i = j; j = t; }
  return i * NC - i * (i - 1) / 2 + (j - i);
}

// One pass over the samples: hits, normal matrices and sums of w_o(t) y_o(t).
template <int KS, typename YT>
__global__ void __launch_bounds__(kBlock) k_na_accum(const int32_t* __restrict__ pix,
                                                     const float* __restrict__ cc,
                                                     const float* __restrict__ ss,
                                                     const uint8_t* __restrict__ valid,
                                                     const YT* __restrict__ y,
                                                     double* __restrict__ scratch, int64_t n_t,
                                                     int64_t npix, KindsArg kk) {
  using K = KSet<KS>;
  constexpr int NC = K::NC, NO = K::NO, NM = NC * (NC + 1) / 2;
  const int n_o = K::n_o(kk);
  int32_t* hits = reinterpret_cast<int32_t*>(scratch + kHitOff);
  int32_t* err = reinterpret_cast<int32_t*>(scratch + kErrOff);
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n_t; t += stride) {
    if (valid != nullptr && valid[t] == 0) continue;
    const int p = pix[t];
    if (p < 0 || p >= npix) {
      atomicOr(err, 1);
      continue;
    }
    const double c = cc[t], s = ss[t];
    double sum[NC], mat[NM];
#pragma unroll
    for (int j = 0; j < NC; ++j) sum[j] = 0.0;
#pragma unroll
    for (int j = 0; j < NM; ++j) mat[j] = 0.0;
#pragma unroll
    for (int o = 0; o < NO; ++o) {
      if (o < n_o) {
        double row[NC];
#pragma unroll
        for (int j = 0; j < NC; ++j) row[j] = 0.0;
        row_bin<NC, double>(K::kind(o, kk), c, s, 1.0, row);
        const double yo = (double)y[(int64_t)o * n_t + t];
#pragma unroll
        for (int i = 0; i < NC; ++i) {
          sum[i] += row[i] * yo;
#pragma unroll
          for (int j = i; j < NC; ++j) mat[na_sym<NC>(i, j)] += row[i] * row[j];
        }
      }
    }
    atomicAdd(hits + p, 1);
#pragma unroll
    for (int j = 0; j < NC; ++j) atomicAdd(scratch + kSumOff + 4 * (int64_t)p + j, sum[j]);
#pragma unroll
    for (int j = 0; j < NM; ++j) atomicAdd(scratch + kMatOff + 6 * (int64_t)p + j, mat[j]);
  }
}

// Per pixel: rcond = lambda_min / lambda_max of M_p in closed form, the cut, and
// m_p = M_p^-1 s_p on kept pixels (0 elsewhere).
template <int NC>
__global__ void __launch_bounds__(kBlock) k_na_finish(const double* __restrict__ scratch,
                                                      int64_t npix, double rcond_min,
                                                      double* __restrict__ map,
                                                      int32_t* __restrict__ hits_out,
                                                      uint8_t* __restrict__ mask_out) {
  constexpr int NM = NC * (NC + 1) / 2;
  const int32_t* hits = reinterpret_cast<const int32_t*>(scratch + kHitOff);
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < npix; p += stride) {
    double a[NM], s[NC], m[NC];
#pragma unroll
    for (int j = 0; j < NM; ++j) a[j] = scratch[kMatOff + 6 * p + j];
#pragma unroll
    for (int j = 0; j < NC; ++j) s[j] = scratch[kSumOff + 4 * p + j];
    const int h = hits[p];
    double rc = 0.0;
    if (h > 0) {
      if constexpr (NC == 1) {
        rc = a[0] > 0.0 ? 1.0 : 0.0;
      } else if constexpr (NC == 2) {
        const double mid = 0.5 * (a[0] + a[2]), half = 0.5 * (a[0] - a[2]);
        const double lmax = mid + sqrt(half * half + a[1] * a[1]);
        rc = lmax > 0.0 ? ((a[0] * a[2] - a[1] * a[1]) / lmax) / lmax : 0.0;
      } else {
        const double p1 = a[1] * a[1] + a[2] * a[2] + a[4] * a[4];
        double e1, e3;
        if (p1 == 0.0) {
          e1 = fmax(a[0], fmax(a[3], a[5]));
          e3 = fmin(a[0], fmin(a[3], a[5]));
        } else {
          const double q = (a[0] + a[3] + a[5]) / 3.0;
          const double d0 = a[0] - q, d1 = a[3] - q, d2 = a[5] - q;
          const double pp = sqrt((d0 * d0 + d1 * d1 + d2 * d2 + 2.0 * p1) / 6.0);
          const double ip = 1.0 / pp;
          const double b00 = d0 * ip, b11 = d1 * ip, b22 = d2 * ip;
          const double b01 = a[1] * ip, b02 = a[2] * ip, b12 = a[4] * ip;
          double r = 0.5 * (b00 * (b11 * b22 - b12 * b12) - b01 * (b01 * b22 - b12 * b02) +
                            b02 * (b01 * b12 - b11 * b02));
          r = fmin(1.0, fmax(-1.0, r));
          const double phi = acos(r) / 3.0;
          e1 = q + 2.0 * pp * cos(phi);
          e3 = q + 2.0 * pp * cos(phi + 2.0943951023931954923);
        }
        rc = e1 > 0.0 ? e3 / e1 : 0.0;
      }
    }
    const bool keep = h > 0 && rc >= rcond_min;
    if (keep) {
      if constexpr (NC == 1) {
        m[0] = s[0] / a[0];
      } else if constexpr (NC == 2) {
        const double det = a[0] * a[2] - a[1] * a[1];
        m[0] = (a[2] * s[0] - a[1] * s[1]) / det;
        m[1] = (a[0] * s[1] - a[1] * s[0]) / det;
      } else {
        const double c00 = a[3] * a[5] - a[4] * a[4], c01 = a[2] * a[4] - a[1] * a[5];
        const double c02 = a[1] * a[4] - a[2] * a[3], c11 = a[0] * a[5] - a[2] * a[2];
        const double c12 = a[1] * a[2] - a[0] * a[4], c22 = a[0] * a[3] - a[1] * a[1];
        const double id = 1.0 / (a[0] * c00 + a[1] * c01 + a[2] * c02);
        m[0] = (c00 * s[0] + c01 * s[1] + c02 * s[2]) * id;
        m[1] = (c01 * s[0] + c11 * s[1] + c12 * s[2]) * id;
        m[2] = (c02 * s[0] + c12 * s[1] + c22 * s[2]) * id;
      }
    } else {
#pragma unroll
      for (int j = 0; j < NC; ++j) m[j] = 0.0;
    }
#pragma unroll
    for (int j = 0; j < NC; ++j) map[(int64_t)j * npix + p] = m[j];
    if (hits_out) hits_out[p] = h;
    if (mask_out) mask_out[p] = keep ? 1 : 0;
  }
}

int na_kindset(const int* k, int n_o, int n_c) {
  if (n_o == 2 && k[0] == DS_KIND_Q && k[1] == DS_KIND_U) return KS_QU;
  if (n_o == 3 && k[0] == DS_KIND_I && k[1] == DS_KIND_Q && k[2] == DS_KIND_U) return KS_IQU3;
  if (n_o == 1 && k[0] == DS_KIND_IQU) return KS_IQU1;
  if (n_o == 1 && k[0] == DS_KIND_I) return KS_I;
  return n_c == 1 ? KS_GEN1 : (n_c == 2 ? KS_GEN2 : KS_GEN3);
}

template <typename YT>
void na_launch_accum(int ks, int grid, cudaStream_t st, const int32_t* pix, const float* c,
                     const float* s, const uint8_t* valid, const YT* y, double* scratch,
                     int64_t n_t, int64_t npix, KindsArg kk) {
  switch (ks) {
    case KS_QU: k_na_accum<KS_QU, YT><<<grid, kBlock, 0, st>>>(pix, c, s, valid, y, scratch, n_t, npix, kk); break;
    case KS_IQU3: k_na_accum<KS_IQU3, YT><<<grid, kBlock, 0, st>>>(pix, c, s, valid, y, scratch, n_t, npix, kk); break;
    case KS_IQU1: k_na_accum<KS_IQU1, YT><<<grid, kBlock, 0, st>>>(pix, c, s, valid, y, scratch, n_t, npix, kk); break;
    case KS_I: k_na_accum<KS_I, YT><<<grid, kBlock, 0, st>>>(pix, c, s, valid, y, scratch, n_t, npix, kk); break;
    case KS_GEN1: k_na_accum<KS_GEN1, YT><<<grid, kBlock, 0, st>>>(pix, c, s, valid, y, scratch, n_t, npix, kk); break;
    case KS_GEN2: k_na_accum<KS_GEN2, YT><<<grid, kBlock, 0, st>>>(pix, c, s, valid, y, scratch, n_t, npix, kk); break;
    default: k_na_accum<KS_GEN3, YT><<<grid, kBlock, 0, st>>>(pix, c, s, valid, y, scratch, n_t, npix, kk); break;
  }
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
  const int ks = na_kindset(desc->kinds, desc->n_outputs, n_c);
  if (desc->precision == DS_PREC_FP64)
    na_launch_accum<double>(ks, grid_for(n_t), st, d_pix, d_cos2psi, d_sin2psi, d_valid,
                            static_cast<const double*>(d_y), scratch, n_t, npix, kk);
  else
    na_launch_accum<float>(ks, grid_for(n_t), st, d_pix, d_cos2psi, d_sin2psi, d_valid,
                           static_cast<const float*>(d_y), scratch, n_t, npix, kk);
  const int pg = grid_for(npix);
  if (n_c == 1) k_na_finish<1><<<pg, kBlock, 0, st>>>(scratch, npix, rcond_min, d_map, d_hits, d_mask);
  else if (n_c == 2) k_na_finish<2><<<pg, kBlock, 0, st>>>(scratch, npix, rcond_min, d_map, d_hits, d_mask);
  else k_na_finish<3><<<pg, kBlock, 0, st>>>(scratch, npix, rcond_min, d_map, d_hits, d_mask);
  if (cudaGetLastError() != cudaSuccess) return DS_ECUDA;
  int32_t err = 0;
  if (cudaMemcpyAsync(&err, scratch + kErrOff, sizeof(int32_t), cudaMemcpyDeviceToHost, st) !=
          cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return DS_ECUDA;
  return err ? DS_EPIX : DS_OK;
}
