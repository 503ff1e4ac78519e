// Per-pixel normal matrices M_p (packed upper triangle, NC = 1, 2 or 3): the
// rcond of the pixel cut from closed-form eigenvalues, and the inverse.  Shared by
// the plan build (plan.cu) and the allocation-free binned map (noalloc.cu), so that
// both cut and invert every pixel alike.
#pragma once

namespace ds {

// Closed-form eigenvalues of a packed symmetric matrix; rcond = lambda_min / lambda_max.
// 2x2: mid +- radius.  3x3: the trigonometric solution of the characteristic cubic.
template <int NC>
__device__ double rcond_of(const double (&a)[NC * (NC + 1) / 2]) {
  if constexpr (NC == 1) {
    return a[0] > 0.0 ? 1.0 : 0.0;
  } else if constexpr (NC == 2) {
    const double mid = 0.5 * (a[0] + a[2]);
    const double half = 0.5 * (a[0] - a[2]);
    const double rad = sqrt(half * half + a[1] * a[1]);
    const double lmax = mid + rad;
    if (!(lmax > 0.0)) return 0.0;
    const double det = a[0] * a[2] - a[1] * a[1];
    return (det / lmax) / lmax;  // lambda_min = det / lambda_max
  } else {
    const double a00 = a[0], a01 = a[1], a02 = a[2], a11 = a[3], a12 = a[4], a22 = a[5];
    const double p1 = a01 * a01 + a02 * a02 + a12 * a12;
    double e1, e3;
    if (p1 == 0.0) {
      e1 = fmax(a00, fmax(a11, a22));
      e3 = fmin(a00, fmin(a11, a22));
    } else {
      const double q = (a00 + a11 + a22) / 3.0;
      const double d0 = a00 - q, d1 = a11 - q, d2 = a22 - q;
      const double p2 = d0 * d0 + d1 * d1 + d2 * d2 + 2.0 * p1;
      const double pp = sqrt(p2 / 6.0);
      const double ip = 1.0 / pp;
      const double b00 = d0 * ip, b11 = d1 * ip, b22 = d2 * ip;
      const double b01 = a01 * ip, b02 = a02 * ip, b12 = a12 * ip;
      const double detb = b00 * (b11 * b22 - b12 * b12) - b01 * (b01 * b22 - b12 * b02) +
                          b02 * (b01 * b12 - b11 * b02);
      double r = 0.5 * detb;
      r = fmin(1.0, fmax(-1.0, r));
      const double phi = acos(r) / 3.0;
      e1 = q + 2.0 * pp * cos(phi);
      e3 = q + 2.0 * pp * cos(phi + 2.0943951023931954923);  // + 2 pi / 3
    }
    if (!(e1 > 0.0)) return 0.0;
    return e3 / e1;
  }
}

template <int NC>
__device__ void sym_inverse(const double (&a)[NC * (NC + 1) / 2], double (&inv)[NC * (NC + 1) / 2]) {
  if constexpr (NC == 1) {
    inv[0] = 1.0 / a[0];
  } else if constexpr (NC == 2) {
    const double det = a[0] * a[2] - a[1] * a[1];
    inv[0] = a[2] / det;
    inv[1] = -a[1] / det;
    inv[2] = a[0] / det;
  } else {
    const double a00 = a[0], a01 = a[1], a02 = a[2], a11 = a[3], a12 = a[4], a22 = a[5];
    const double c00 = a11 * a22 - a12 * a12;
    const double c01 = a02 * a12 - a01 * a22;
    const double c02 = a01 * a12 - a02 * a11;
    const double c11 = a00 * a22 - a02 * a02;
    const double c12 = a01 * a02 - a00 * a12;
    const double c22 = a00 * a11 - a01 * a01;
    const double det = a00 * c00 + a01 * c01 + a02 * c02;
    const double id = 1.0 / det;
    inv[0] = c00 * id; inv[1] = c01 * id; inv[2] = c02 * id;
    inv[3] = c11 * id; inv[4] = c12 * id; inv[5] = c22 * id;
  }
}

}  // namespace ds
