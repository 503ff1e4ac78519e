// Pointing of an analytic ground scan computed on the device (destripe_scan_pointing):
// the spin scan of Sect. 5 (fixed elevation, constant azimuth rate, the sky turning
// with the Earth) converted to equatorial coordinates, the parallactic angle psi
// (Sect. 3, the polarimeter's orientation), an optional polarisation modulator, and
// the HEALPix RING pixel of each sample (Gorski et al. 2005, as cited in Sect. 3).
//
//     t        = k (1 / f_samp)
//     az       = az0 + (2 pi / T_spin) t,    lst = lst0 + (2 pi / T_sidereal) t
//     sin dec  = sin el sin lat + cos el cos lat cos az
//     H        = atan2(-sin az cos el, sin el cos lat - cos el sin lat cos az)
//     RA       = (lst - H) mod 2 pi
//     psi      = atan2(sin H, tan lat cos dec - sin dec cos H) + (2 pi / T_mod) t
//
// Every step is one IEEE float64 operation in a fixed order (the products and sums
// are written with round-to-nearest intrinsics, so none is contracted into a fused
// multiply-add), so the result is a deterministic function of the scan parameters,
// identical wherever the same operations run in the same order.  cos 2psi and sin 2psi are rounded once to
// float32, as the plan reads them.
//
// The arithmetic is float64 throughout; on GB300, whose float64 pipe is narrow,
// this makes the pass slower than copying 12 bytes per sample of precomputed
// pointing from the host (see the design notes), so it is a plan-time generator,
// not a replacement for the pointing streams of the CG iteration.
#include <cmath>

#include "internal.cuh"

namespace ds {

namespace {

constexpr int kBlock = 256;

struct ScanConst {
  double inv_fs;                // 1 / f_samp
  double w_spin, w_sid, w_mod;  // 2 pi / period (w_mod = 0: no modulator)
  double az0, lst0;
  double a_sd, b_sd;            // sin el sin lat, cos el cos lat
  double cos_el;
  double c_h, d_h;              // sin el cos lat, cos el sin lat
  double tan_lat;
  double two_pi, half_pi, two_over_pi;
};

// x mod y with the sign of y (y > 0): fmod, moved into [0, y)
__device__ __forceinline__ double mod_pos(double x, double y) {
  double m = fmod(x, y);
  if (m != 0.0 && ((y < 0.0) != (m < 0.0))) m = __dadd_rn(m, y);
  return m;
}

// HEALPix RING pixel of (theta, phi): the belt from the two families of edge lines,
// the caps from the ring number counted from the nearest pole.
__device__ __forceinline__ int64_t ring_pixel(int64_t nside, double theta, double phi,
                                              const ScanConst& k) {
  phi = mod_pos(phi, k.two_pi);
  const double z = cos(theta);
  const double za = fabs(z);
  double tt = __dmul_rn(phi, k.two_over_pi);
  if (tt >= 4.0) tt = __dadd_rn(tt, -4.0);
  const double ns = (double)nside;
  const int64_t npix = 12 * nside * nside, ncap = 2 * nside * (nside - 1);
  if (za <= 2.0 / 3.0) {
    const double t1 = __dmul_rn(ns, __dadd_rn(0.5, tt));
    const double t2 = __dmul_rn(__dmul_rn(ns, z), 0.75);
    const int64_t jp = (int64_t)floor(__dadd_rn(t1, -t2));
    const int64_t jm = (int64_t)floor(__dadd_rn(t1, t2));
    const int64_t ir = nside + 1 + jp - jm;
    const int64_t kshift = 1 - (ir & 1);
    int64_t ip = jp + jm - nside + kshift + 1;
    ip = ip >= 0 ? ip / 2 : -((-ip + 1) / 2);  // floor division by 2
    const int64_t nr = 4 * nside;
    ip %= nr;
    if (ip < 0) ip += nr;
    return ncap + (ir - 1) * nr + ip;
  }
  const double tp = __dadd_rn(tt, -floor(tt));
  double q = __dmul_rn(3.0, __dadd_rn(1.0, -za));
  if (q < 0.0) q = 0.0;
  const double tmp = __dmul_rn(ns, sqrt(q));
  const int64_t jp = (int64_t)floor(__dmul_rn(tp, tmp));
  const int64_t jm = (int64_t)floor(__dmul_rn(__dadd_rn(1.0, -tp), tmp));
  const int64_t ir = jp + jm + 1;
  int64_t ip = (int64_t)floor(__dmul_rn(tt, (double)ir));
  ip %= 4 * ir;
  if (ip < 0) ip += 4 * ir;
  return z > 0.0 ? 2 * ir * (ir - 1) + ip : npix - 2 * ir * (ir + 1) + ip;
}

__global__ void __launch_bounds__(kBlock) k_scan_pointing(ScanConst k, int64_t first, int64_t n,
                                                          int64_t nside, int32_t* __restrict__ pix,
                                                          float* __restrict__ c2,
                                                          float* __restrict__ s2) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    const double t = __dmul_rn((double)(first + i), k.inv_fs);
    const double az = __dadd_rn(k.az0, __dmul_rn(k.w_spin, t));
    const double lst = __dadd_rn(k.lst0, __dmul_rn(k.w_sid, t));
    const double cos_az = cos(az), sin_az = sin(az);
    double sin_dec = __dadd_rn(k.a_sd, __dmul_rn(k.b_sd, cos_az));
    sin_dec = fmin(fmax(sin_dec, -1.0), 1.0);
    const double dec = asin(sin_dec);
    const double ha = atan2(__dmul_rn(-sin_az, k.cos_el), __dadd_rn(k.c_h, -__dmul_rn(k.d_h, cos_az)));
    const double ra = mod_pos(__dadd_rn(lst, -ha), k.two_pi);
    double psi = atan2(sin(ha), __dadd_rn(__dmul_rn(k.tan_lat, cos(dec)), -__dmul_rn(sin_dec, cos(ha))));
    if (k.w_mod != 0.0) psi = __dadd_rn(psi, __dmul_rn(k.w_mod, t));
    const double theta = __dadd_rn(k.half_pi, -dec);
    pix[i] = (int32_t)ring_pixel(nside, theta, ra, k);
    const double two_psi = __dmul_rn(2.0, psi);
    c2[i] = __double2float_rn(cos(two_psi));
    s2[i] = __double2float_rn(sin(two_psi));
  }
}

}  // namespace

}  // namespace ds

using namespace ds;

extern "C" ds_status destripe_scan_pointing(const ds_scan* scan, int64_t first_sample,
                                            int64_t n_samples, int32_t nside, int32_t* d_pix,
                                            float* d_cos2psi, float* d_sin2psi, void* stream) {
  if (scan == nullptr || d_pix == nullptr || d_cos2psi == nullptr || d_sin2psi == nullptr)
    return DS_EINVAL;
  if (n_samples < 0 || first_sample < 0) return DS_EINVAL;
  if (nside < 1 || nside > 8192 || (nside & (nside - 1)) != 0) return DS_EINVAL;
  if (!(scan->f_samp > 0.0) || !(scan->spin_period > 0.0) || !(scan->sidereal_day > 0.0) ||
      scan->pol_rotation_period < 0.0)
    return DS_EINVAL;
  if (n_samples == 0) return DS_OK;
  const double pi = 3.141592653589793;
  ScanConst k{};
  k.inv_fs = 1.0 / scan->f_samp;
  k.w_spin = 2.0 * pi / scan->spin_period;
  k.w_sid = 2.0 * pi / scan->sidereal_day;
  k.w_mod = scan->pol_rotation_period > 0.0 ? 2.0 * pi / scan->pol_rotation_period : 0.0;
  k.az0 = scan->az0;
  k.lst0 = scan->lst0;
  const double el = scan->elevation_deg * (pi / 180.0), lat = scan->latitude_deg * (pi / 180.0);
  const double sin_el = std::sin(el), cos_el = std::cos(el);
  const double sin_lat = std::sin(lat), cos_lat = std::cos(lat);
  k.a_sd = sin_el * sin_lat;
  k.b_sd = cos_el * cos_lat;
  k.cos_el = cos_el;
  k.c_h = sin_el * cos_lat;
  k.d_h = cos_el * sin_lat;
  k.tan_lat = std::tan(lat);
  k.two_pi = 2.0 * pi;
  k.half_pi = 0.5 * pi;
  k.two_over_pi = 2.0 / pi;
  int device = 0, sms = 0;
  DS_CUDA_TRY(cudaGetDevice(&device));
  DS_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device));
  const int64_t need = (n_samples + kBlock - 1) / kBlock;
  const int grid = (int)(need < (int64_t)sms * 8 ? need : (int64_t)sms * 8);
  (void)cudaGetLastError();
  k_scan_pointing<<<grid, kBlock, 0, static_cast<cudaStream_t>(stream)>>>(
      k, first_sample, n_samples, nside, d_pix, d_cos2psi, d_sin2psi);
  return cudaGetLastError() == cudaSuccess ? DS_OK : DS_ECUDA;
}
