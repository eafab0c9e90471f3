// One-electron integrals over normalised primitive s Gaussians, g_a(r) = (2a/pi)^{3/4}
// exp(-a |r - A|^2), with point nuclei: the input matrices S, T, V and W0 = sum_k p_k V p_k of
// the modified Dirac equation (Sec. II, Eqs. 4-7).  Host and device code (the host build is
// checked against an independent host implementation in the tests).
//
// For a pair (a, A), (b, B): p = a + b, mu = a b / p, P = (a A + b B) / p,
// K = N_a N_b exp(-mu |A - B|^2) and, per nucleus C of charge Z_C, T_C = p |P - C|^2:
//   S  = K (pi / p)^{3/2}
//   T  = mu (3 - 2 mu |A - B|^2) S
//   V  = -(2 pi K / p) sum_C Z_C F0(T_C)
//   W0 = -(8 pi a b K / p) sum_C Z_C [ (3 F0 - e^{-T_C}) / (2 p) + (C - P).(2P - A - B) F1
//                                      + (P - A).(P - B) F0 ]
// (the gradient of an s Gaussian is -2a (r - A) g_a; expanding (r - A).(r - B) about P gives
// the three terms, with <|r - P|^2 ...> reduced by the Boys recurrence).
#pragma once

#include <math.h>

namespace x2c {

// Boys functions F_m(T) = int_0^1 t^{2m} e^{-T t^2} dt for m = 0, 1, 2, T >= 0.  Small and
// moderate T: F_2 from its convergent series e^{-T} sum_k (2T)^k / prod_{i=0..k} (5 + 2i),
// then F_1 and F_0 by the downward recurrence F_m = (2T F_{m+1} + e^{-T}) / (2m + 1), which
// only adds positive terms.  Large T: F_0 from the error function and the upward recurrence
// F_{m+1} = ((2m + 1) F_m - e^{-T}) / (2T), which no longer cancels there.
__host__ __device__ inline void boys_f012(double T, double &f0, double &f1, double &f2) {
  const double e = exp(-T);
  if (T < 25.0) {
    const double t2 = T + T;
    double term = 0.2, sum = 0.2;
    for (int k = 1; k < 400 && term > 1e-18 * sum; ++k) {
      term = term * t2 / (5.0 + 2.0 * k);
      sum += term;
    }
    f2 = e * sum;
    f1 = (t2 * f2 + e) * (1.0 / 3.0);
    f0 = t2 * f1 + e;
  } else {
    const double rt = sqrt(T);
    f0 = 0.5 * sqrt(3.14159265358979323846 / T) * (T < 40.0 ? erf(rt) : 1.0);
    f1 = (f0 - e) / (T + T);
    f2 = (3.0 * f1 - e) / (T + T);
  }
}

// S, T, V, W0 of one primitive pair; nuclei as (x, y, z) triples and charges.
__host__ __device__ inline void s_pair_integrals(const double *A, double a, const double *B, double b, int n_nuc,
                                                 const double *nuc_xyz, const double *nuc_z, double &s, double &t,
                                                 double &v, double &w0) {
  const double pi = 3.14159265358979323846;
  const double p = a + b, mu = a * b / p;
  const double dx = A[0] - B[0], dy = A[1] - B[1], dz = A[2] - B[2];
  const double x = mu * (dx * dx + dy * dy + dz * dz);
  if (x > 745.0) {  // the Gaussian product underflows: every integral is 0
    s = t = v = w0 = 0.0;
    return;
  }
  const double K = pow(4.0 * a * b / (pi * pi), 0.75) * exp(-x);
  s = K * pow(pi / p, 1.5);
  t = mu * (3.0 - 2.0 * x) * s;
  const double Px = (a * A[0] + b * B[0]) / p, Py = (a * A[1] + b * B[1]) / p, Pz = (a * A[2] + b * B[2]) / p;
  // 2P - A - B = (b - a)(B - A)/p and (P - A).(P - B) = -mu |A - B|^2 / p
  const double gx = (b - a) * (-dx) / p, gy = (b - a) * (-dy) / p, gz = (b - a) * (-dz) / p;
  const double papb = -x / p;
  double sv = 0.0, sw = 0.0;
  for (int c = 0; c < n_nuc; ++c) {
    const double cx = nuc_xyz[3 * c] - Px, cy = nuc_xyz[3 * c + 1] - Py, cz = nuc_xyz[3 * c + 2] - Pz;
    const double T = p * (cx * cx + cy * cy + cz * cz);
    double f0, f1, f2;
    boys_f012(T, f0, f1, f2);
    const double z = nuc_z[c];
    sv += z * f0;
    sw += z * ((3.0 * f0 - exp(-T)) / (2.0 * p) + (cx * gx + cy * gy + cz * gz) * f1 + papb * f0);
  }
  const double pref = 2.0 * pi * K / p;
  v = -pref * sv;
  w0 = -4.0 * a * b * pref * sw;
}

}  // namespace x2c
