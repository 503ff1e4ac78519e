// Time-domain steps around the destriper (C ABI in destripe.h):
//
//  * destripe_gapfill -- white-noise gap filling (Sect. 2): every flagged sample
//    of every output becomes Gaussian white noise with the mean and standard
//    deviation (population) of that output's good samples in the same day of data
//    (a block of block_len samples; a block without good samples is filled with
//    0).  The draws come from the counter-based generator Philox4x32-10 (Salmon,
//    Moraes, Dror & Shaw 2011) with counter (t mod 2^32, t div 2^32, o, 0) and key
//    (seed mod 2^32, seed div 2^32): its first two words give the uniforms
//    (u + 1/2) 2^-32 and one normal draw by Box-Muller, sqrt(-2 ln u0) cos(2 pi u1).
//    Two streaming passes give each day's sums (mean, then squared deviations);
//    a third writes the flagged samples.
//  * destripe_spectrum -- amplitude spectra of the timelines y and y - F~ a
//    (Sect. 6, frequency domain): non-overlapping segments of seg_len samples
//    transformed by cuFFT, the one-sided power spectral density 2 |X_k|^2 /
//    (f_samp seg_len) averaged over segments (k = 0 and the Nyquist term not
//    doubled), its square root averaged over n_bins bins of linearly growing length
//    (edges floor(K j (j + 1) / (n (n + 1))), K = seg_len / 2, DC left out).
#include <cmath>
#include <cufft.h>

#include "internal.cuh"

namespace ds {

namespace {

constexpr int kBlock = 256;
constexpr int kPerThread = 8;  // consecutive samples a thread sums before the warp flush

// ---- Philox4x32-10 and one normal draw --------------------------------------------
__device__ __forceinline__ double philox_normal(uint64_t t, uint32_t o, uint64_t seed) {
  uint32_t c0 = (uint32_t)t, c1 = (uint32_t)(t >> 32), c2 = o, c3 = 0u;
  uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint32_t hi0 = __umulhi(0xD2511F53u, c0), lo0 = 0xD2511F53u * c0;
    const uint32_t hi1 = __umulhi(0xCD9E8D57u, c2), lo1 = 0xCD9E8D57u * c2;
    const uint32_t n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
    c0 = n0;
    c1 = lo1;
    c2 = n2;
    c3 = lo0;
    if (r < 9) {
      k0 += 0x9E3779B9u;
      k1 += 0xBB67AE85u;
    }
  }
  const double u0 = ((double)c0 + 0.5) * 0x1p-32;
  const double u1 = ((double)c1 + 0.5) * 0x1p-32;
  return sqrt(-2.0 * log(u0)) * cospi(2.0 * u1);
}

template <typename YT>
__device__ __forceinline__ double ld_y(const YT* y, int64_t i) { return (double)y[i]; }

// Per (output, day): pass 0 sums the good samples and counts them; pass 1 sums
// the squared deviations from the day's mean.  acc = [n_o][n_days][3] (count,
// sum, squared deviations).  Threads sum kPerThread consecutive samples; a warp
// flushes each day's total once (segmented over the lanes, whose keys do not
// decrease); a day that ends inside a thread's samples is flushed there.
__device__ __forceinline__ void gf_flush(double* __restrict__ acc, int64_t row, int pass,
                                         double n, double s) {
  if (n <= 0.0) return;
  double* a = acc + row * 3;
  if (pass == 0) {
    atomicAdd(a + 0, n);
    atomicAdd(a + 1, s);
  } else {
    atomicAdd(a + 2, s);
  }
}

__device__ __forceinline__ double gf_mean(const double* __restrict__ acc, int64_t row) {
  const double n = acc[row * 3];
  return n > 0.0 ? acc[row * 3 + 1] / n : 0.0;
}

template <typename YT>
__global__ void __launch_bounds__(kBlock) k_gf_stats(const YT* __restrict__ y,
                                                     const uint8_t* __restrict__ valid,
                                                     int64_t n_t, int n_o, int64_t day,
                                                     int64_t n_days, int pass,
                                                     double* __restrict__ acc) {
  const unsigned full = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  const int64_t groups = (n_t + kPerThread - 1) / kPerThread;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int o = 0; o < n_o; ++o) {
    for (int64_t gb = (int64_t)blockIdx.x * blockDim.x + threadIdx.x - lane; gb < groups;
         gb += stride) {
      const int64_t g = gb + lane;
      int key = -1;
      double s = 0.0, n = 0.0;
      if (g < groups) {
        const int64_t t0 = g * kPerThread;
        const int64_t t1 = t0 + kPerThread < n_t ? t0 + kPerThread : n_t;
        int64_t d = t0 / day, dend = (d + 1) * day;
        key = (int)d;
        double mu = pass == 1 ? gf_mean(acc, (int64_t)o * n_days + d) : 0.0;
        for (int64_t t = t0; t < t1; ++t) {
          if (t >= dend) {  // a day ends inside the thread's samples
            gf_flush(acc, (int64_t)o * n_days + d, pass, n, s);
            d += 1;
            dend += day;
            key = (int)d;
            s = n = 0.0;
            if (pass == 1) mu = gf_mean(acc, (int64_t)o * n_days + d);
          }
          if (valid[t] == 0) continue;
          const double v = ld_y(y, (int64_t)o * n_t + t);
          s += pass == 0 ? v : (v - mu) * (v - mu);
          n += 1.0;
        }
      }
      for (int w = 1; w < 32; w <<= 1) {
        const int k2 = __shfl_down_sync(full, key, w);
        const double s2 = __shfl_down_sync(full, s, w);
        const double n2 = __shfl_down_sync(full, n, w);
        if (lane + w < 32 && k2 == key) {
          s += s2;
          n += n2;
        }
      }
      const int kp = __shfl_up_sync(full, key, 1);
      if (key >= 0 && (lane == 0 || kp != key)) gf_flush(acc, (int64_t)o * n_days + key, pass, n, s);
    }
  }
}

template <typename YT>
__global__ void __launch_bounds__(kBlock) k_gf_fill(YT* __restrict__ y,
                                                    const uint8_t* __restrict__ valid,
                                                    int64_t n_t, int n_o, int64_t day,
                                                    int64_t n_days, uint64_t seed,
                                                    const double* __restrict__ acc) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n_t; t += stride) {
    if (valid[t] != 0) continue;
    const int64_t d = t / day;
    for (int o = 0; o < n_o; ++o) {
      const double* a = acc + ((int64_t)o * n_days + d) * 3;
      double v = 0.0;
      if (a[0] > 0.0) {
        const double mu = a[1] / a[0];
        const double sd = sqrt(a[2] / a[0]);
        v = mu + sd * philox_normal((uint64_t)t, (uint32_t)o, seed);
      }
      y[(int64_t)o * n_t + t] = (YT)v;
    }
  }
}

// z[s][i] = y[o][s0 + s N + i] - a[o][(s0 + s N + i) / L] for the segments of a chunk
template <typename YT>
__global__ void __launch_bounds__(kBlock) k_sp_timeline(const YT* __restrict__ y,
                                                        const double* __restrict__ a,
                                                        int64_t t0, int64_t len, int64_t L,
                                                        double* __restrict__ z) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < len; i += stride) {
    const int64_t t = t0 + i;
    double v = (double)y[t];
    if (a != nullptr) v -= a[t / L];
    z[i] = v;
  }
}

// pw[k] += sum over the chunk's segments of |X_k|^2 (one thread per k)
__global__ void __launch_bounds__(kBlock) k_sp_power(const cufftDoubleComplex* __restrict__ X,
                                                     int64_t nseg, int64_t nk,
                                                     double* __restrict__ pw) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < nk; k += stride) {
    double s = 0.0;
    for (int64_t g = 0; g < nseg; ++g) {
      const cufftDoubleComplex v = X[g * nk + k];
      s += v.x * v.x + v.y * v.y;
    }
    pw[k] += s;
  }
}

// Bin j: mean frequency and mean amplitude over k = e_{j-1} + 1 .. e_j.
__global__ void k_sp_bins(const double* __restrict__ pw, int64_t seg_len, int64_t nseg,
                          int n_bins, double f_samp, double* __restrict__ freq,
                          double* __restrict__ amp) {
  const int64_t K = seg_len / 2;
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n_bins; j += gridDim.x * blockDim.x) {
    const int64_t e0 = (K * (int64_t)j * (j + 1)) / ((int64_t)n_bins * (n_bins + 1));
    const int64_t e1 = (K * (int64_t)(j + 1) * (j + 2)) / ((int64_t)n_bins * (n_bins + 1));
    double fs = 0.0, as = 0.0;
    for (int64_t k = e0 + 1; k <= e1; ++k) {
      double p = pw[k] * 2.0 / (f_samp * (double)seg_len * (double)nseg);
      if (k == K && (seg_len % 2) == 0) p *= 0.5;
      fs += (double)k * f_samp / (double)seg_len;
      as += sqrt(p);
    }
    const double cnt = (double)(e1 - e0);
    if (freq != nullptr) freq[j] = fs / cnt;
    amp[j] = as / cnt;
  }
}

}  // namespace

}  // namespace ds

using namespace ds;

extern "C" {

ds_status destripe_gapfill(const ds_desc* desc, const uint8_t* d_valid, int64_t block_len,
                           uint64_t seed, void* d_y) {
  if (desc == nullptr || d_valid == nullptr || d_y == nullptr || block_len < 1) return DS_EINVAL;
  if (desc->n_samples < 1 || desc->n_samples >= (int64_t(1) << 31)) return DS_EINVAL;
  if (desc->n_outputs < 1 || desc->n_outputs > DS_MAX_OUTPUTS) return DS_EINVAL;
  if (desc->precision != DS_PREC_FP64 && desc->precision != DS_PREC_MIXED) return DS_EINVAL;
  cudaStream_t st = static_cast<cudaStream_t>(desc->stream);
  const int64_t n_t = desc->n_samples;
  const int n_o = desc->n_outputs;
  const int64_t n_days = (n_t + block_len - 1) / block_len;
  (void)cudaGetLastError();
  int device = 0, sms = 0;
  DS_CUDA_TRY(cudaGetDevice(&device));
  DS_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device));
  double* acc = nullptr;
  DS_CUDA_TRY(cudaMallocAsync(reinterpret_cast<void**>(&acc), sizeof(double) * 3 * n_o * n_days, st));
  cudaError_t e = cudaMemsetAsync(acc, 0, sizeof(double) * 3 * n_o * n_days, st);
  const int64_t groups = (n_t + kPerThread - 1) / kPerThread;
  const int g1 = (int)std::min<int64_t>((groups + kBlock - 1) / kBlock, (int64_t)sms * 8);
  const int g2 = (int)std::min<int64_t>((n_t + kBlock - 1) / kBlock, (int64_t)sms * 8);
  if (e == cudaSuccess) {
    if (desc->precision == DS_PREC_FP64) {
      const double* y = static_cast<const double*>(d_y);
      k_gf_stats<double><<<g1, kBlock, 0, st>>>(y, d_valid, n_t, n_o, block_len, n_days, 0, acc);
      k_gf_stats<double><<<g1, kBlock, 0, st>>>(y, d_valid, n_t, n_o, block_len, n_days, 1, acc);
      k_gf_fill<double><<<g2, kBlock, 0, st>>>(static_cast<double*>(d_y), d_valid, n_t, n_o,
                                               block_len, n_days, seed, acc);
    } else {
      const float* y = static_cast<const float*>(d_y);
      k_gf_stats<float><<<g1, kBlock, 0, st>>>(y, d_valid, n_t, n_o, block_len, n_days, 0, acc);
      k_gf_stats<float><<<g1, kBlock, 0, st>>>(y, d_valid, n_t, n_o, block_len, n_days, 1, acc);
      k_gf_fill<float><<<g2, kBlock, 0, st>>>(static_cast<float*>(d_y), d_valid, n_t, n_o,
                                              block_len, n_days, seed, acc);
    }
    e = cudaGetLastError();
  }
  cudaFreeAsync(acc, st);
  if (e != cudaSuccess) return e == cudaErrorMemoryAllocation ? DS_ENOMEM : DS_ECUDA;
  return DS_OK;
}

ds_status destripe_spectrum(ds_plan_t plan, const void* d_y, const double* d_a, int64_t seg_len,
                            int32_t n_bins, double f_samp, double* d_freq, double* d_amp) {
  if (plan == nullptr || d_y == nullptr || d_amp == nullptr) return DS_EINVAL;
  Plan& P = *reinterpret_cast<Plan*>(plan);
  if (seg_len < 2 || seg_len > P.n_t || n_bins < 1 || !(f_samp > 0.0)) return DS_EINVAL;
  const int64_t K = seg_len / 2;
  if ((int64_t)n_bins * (n_bins + 1) / 2 > K) return DS_EINVAL;  // every bin holds a k
  cudaStream_t st = P.stream;
  (void)cudaGetLastError();
  const int64_t nk = K + 1;
  const int64_t nseg_all = P.n_t / seg_len;
  // chunks of whole segments, about 2^25 samples each
  int64_t per_chunk = (int64_t(1) << 25) / seg_len;
  if (per_chunk < 1) per_chunk = 1;
  if (per_chunk > nseg_all) per_chunk = nseg_all;
  double* z = nullptr;
  cufftDoubleComplex* X = nullptr;
  double* pw = nullptr;
  cufftHandle fft = 0;
  bool have_fft = false;
  ds_status s = DS_OK;
  cudaError_t e = plan_alloc(P, reinterpret_cast<void**>(&z), sizeof(double) * per_chunk * seg_len, false);
  if (e == cudaSuccess)
    e = plan_alloc(P, reinterpret_cast<void**>(&X), sizeof(cufftDoubleComplex) * per_chunk * nk, false);
  if (e == cudaSuccess) e = plan_alloc(P, reinterpret_cast<void**>(&pw), sizeof(double) * nk, false);
  if (e != cudaSuccess) s = e == cudaErrorMemoryAllocation ? DS_ENOMEM : DS_ECUDA;
  int n = (int)seg_len;
  if (s == DS_OK) {
    if (cufftPlanMany(&fft, 1, &n, nullptr, 1, n, nullptr, 1, (int)nk, CUFFT_D2Z,
                      (int)per_chunk) != CUFFT_SUCCESS ||
        cufftSetStream(fft, st) != CUFFT_SUCCESS)
      s = DS_ECUDA;
    else
      have_fft = true;
  }
  const bool f64 = P.desc.precision == DS_PREC_FP64;
  for (int o = 0; o < P.n_o && s == DS_OK; ++o) {
    if (cudaMemsetAsync(pw, 0, sizeof(double) * nk, st) != cudaSuccess) {
      s = DS_ECUDA;
      break;
    }
    for (int64_t g0 = 0; g0 < nseg_all && s == DS_OK; g0 += per_chunk) {
      const int64_t ns = (g0 + per_chunk <= nseg_all) ? per_chunk : nseg_all - g0;
      if (ns < per_chunk)  // the last chunk: clear the unused segments' input
        if (cudaMemsetAsync(z, 0, sizeof(double) * per_chunk * seg_len, st) != cudaSuccess) {
          s = DS_ECUDA;
          break;
        }
      const int64_t len = ns * seg_len;
      const int grid = stream_grid(P, len, kBlock, 8);
      const double* a = d_a != nullptr ? d_a + (int64_t)o * P.n_b : nullptr;
      if (f64)
        k_sp_timeline<double><<<grid, kBlock, 0, st>>>(
            static_cast<const double*>(d_y) + (int64_t)o * P.n_t, a, g0 * seg_len, len, P.L, z);
      else
        k_sp_timeline<float><<<grid, kBlock, 0, st>>>(
            static_cast<const float*>(d_y) + (int64_t)o * P.n_t, a, g0 * seg_len, len, P.L, z);
      if (cufftExecD2Z(fft, z, X) != CUFFT_SUCCESS) {
        s = DS_ECUDA;
        break;
      }
      k_sp_power<<<stream_grid(P, nk, kBlock, 8), kBlock, 0, st>>>(X, ns, nk, pw);
      P.launches += 3;
    }
    if (s != DS_OK) break;
    k_sp_bins<<<(n_bins + 127) / 128, 128, 0, st>>>(pw, seg_len, nseg_all, n_bins, f_samp,
                                                   o == 0 ? d_freq : nullptr,
                                                   d_amp + (int64_t)o * n_bins);
    P.launches += 1;
    if (cudaGetLastError() != cudaSuccess) s = DS_ECUDA;
  }
  if (have_fft) cufftDestroy(fft);
  if (s == DS_OK && cudaStreamSynchronize(st) != cudaSuccess) s = DS_ECUDA;
  for (void* b : {(void*)z, (void*)X, (void*)pw})
    if (b) cudaFreeAsync(b, st);
  return s;
}

}  // extern "C"
