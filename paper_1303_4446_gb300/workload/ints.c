/*
 * Closed-form one-electron integrals over normalised primitive s-type Gaussians
 *   g_a(r) = (2 a / pi)^{3/4} exp(-a |r - A|^2)
 * with point nuclei (charges Z_C at positions C).
 *
 * These are the input matrices of the relativistic transformation: the overlap S,
 * the kinetic energy T, the nuclear attraction V and the scalar part W0 = sum_k p_k V p_k
 * of the spin-dependent potential matrix W (Sec. II, Eqs. (5)-(7) of the paper: the
 * modified Dirac equation needs only S, T, V and W).  This file is a workload
 * generator: it holds none of the decoupling arithmetic.
 *
 * Textbook Gaussian formulas.  With p = a + b, mu = a b / p, P = (a A + b B)/p,
 * K = N_a N_b exp(-mu |A-B|^2):
 *   S  = K (pi/p)^{3/2}
 *   T  = mu (3 - 2 mu |A-B|^2) S
 *   V  = - sum_C Z_C K (2 pi / p) F0(p |P-C|^2)
 *   W0 = <grad g_a | V | grad g_b> = 4 a b <g_a| (r-A).(r-B) V |g_b>, and with
 *        (r-A).(r-B) = |r-P|^2 + (r-P).(2P-A-B) + (P-A).(P-B):
 *   W0 = - sum_C Z_C 4 a b K (2 pi/p) [ (3 F0 - e^{-T}) / (2p)
 *                                     + (C-P).(2P-A-B) F1 + (P-A).(P-B) F0 ]
 * where F_m is the Boys function at T = p |P-C|^2.
 *
 * Portable C99 + OpenMP; no architecture-specific code.
 */
#include <math.h>
#include <stddef.h>
#include <stdint.h>

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

/* Boys functions F0, F1, F2 at T >= 0.
 * T < 25: F2 from the series with positive terms
 *   F_m(T) = e^{-T} sum_k (2T)^k / ((2m+1)(2m+3)...(2m+2k+1)),
 * then the (stable) downward recurrence F_m = (2T F_{m+1} + e^{-T}) / (2m+1).
 * T >= 25: F0 = (1/2) sqrt(pi/T) erf(sqrt T) and the upward recurrence
 *   F_{m+1} = ((2m+1) F_m - e^{-T}) / (2T), which does not cancel there. */
void x2c_boys012(double T, double F[3]) {
  if (T < 25.0) {
    const double twoT = 2.0 * T;
    double term = 1.0 / 5.0, sum = term;
    for (int k = 1; k < 400; ++k) {
      term *= twoT / (5.0 + 2.0 * k);
      sum += term;
      if (term < 1e-18 * sum) break;
    }
    const double e = exp(-T);
    F[2] = e * sum;
    F[1] = (twoT * F[2] + e) / 3.0;
    F[0] = twoT * F[1] + e;
  } else {
    const double e = exp(-T);
    const double erfv = (T < 40.0) ? erf(sqrt(T)) : 1.0; /* erfc(sqrt 40) < 1e-18 */
    F[0] = 0.5 * sqrt(M_PI / T) * erfv;
    F[1] = (F[0] - e) / (2.0 * T);
    F[2] = (3.0 * F[1] - e) / (2.0 * T);
  }
}

/* One matrix element of each requested integral (any output pointer may be NULL). */
static void one_pair(int nnuc, const double *nuc_xyz, const double *nuc_Z,
                     const double *A, double a, const double *B, double b,
                     double *s, double *t, double *v, double *w0) {
  const double p = a + b, mu = a * b / p;
  const double AB[3] = {A[0] - B[0], A[1] - B[1], A[2] - B[2]};
  const double R2 = AB[0] * AB[0] + AB[1] * AB[1] + AB[2] * AB[2];
  const double x = mu * R2;
  if (x > 745.0) { /* exp underflows to exactly zero: every integral is zero */
    if (s) *s = 0.0;
    if (t) *t = 0.0;
    if (v) *v = 0.0;
    if (w0) *w0 = 0.0;
    return;
  }
  const double Na = pow(2.0 * a / M_PI, 0.75), Nb = pow(2.0 * b / M_PI, 0.75);
  const double K = Na * Nb * exp(-x);
  const double S = K * pow(M_PI / p, 1.5);
  if (s) *s = S;
  if (t) *t = mu * (3.0 - 2.0 * x) * S;
  if (!v && !w0) return;
  const double P[3] = {(a * A[0] + b * B[0]) / p, (a * A[1] + b * B[1]) / p,
                       (a * A[2] + b * B[2]) / p};
  /* (P-A).(P-B) = -mu |A-B|^2 / p ;  2P-A-B = (b-a)(B-A)/p */
  const double PAPB = -x / p;
  const double Q[3] = {(b - a) * (-AB[0]) / p, (b - a) * (-AB[1]) / p,
                       (b - a) * (-AB[2]) / p};
  const double pref = K * 2.0 * M_PI / p;
  double vs = 0.0, ws = 0.0;
  for (int c = 0; c < nnuc; ++c) {
    const double *C = nuc_xyz + 3 * c;
    const double PC[3] = {P[0] - C[0], P[1] - C[1], P[2] - C[2]};
    const double T = p * (PC[0] * PC[0] + PC[1] * PC[1] + PC[2] * PC[2]);
    double F[3];
    x2c_boys012(T, F);
    vs += nuc_Z[c] * F[0];
    if (w0) {
      const double CPQ = -(PC[0] * Q[0] + PC[1] * Q[1] + PC[2] * Q[2]);
      ws += nuc_Z[c] * ((3.0 * F[0] - exp(-T)) / (2.0 * p) + CPQ * F[1] + PAPB * F[0]);
    }
  }
  if (v) *v = -pref * vs;
  if (w0) *w0 = -4.0 * a * b * pref * ws;
}

/* Rectangular block of the integral matrices: rows i in [i0, i1), columns j in [j0, j1),
 * written row-major with leading dimension ld at out[(i - i0) * ld + (j - j0)].
 * nuc_xyz: 3*nnuc; bf_xyz: 3*nbf (centre of each primitive); bf_alpha: nbf exponents.
 * Any of S, T, V, W0 may be NULL. */
void x2c_ints_block(int nnuc, const double *nuc_xyz, const double *nuc_Z, int nbf,
                    const double *bf_xyz, const double *bf_alpha, int i0, int i1, int j0,
                    int j1, double *S, double *T, double *V, double *W0, int64_t ld) {
  (void)nbf;
#pragma omp parallel for schedule(dynamic, 4)
  for (int i = i0; i < i1; ++i) {
    for (int j = j0; j < j1; ++j) {
      const int64_t o = (int64_t)(i - i0) * ld + (j - j0);
      one_pair(nnuc, nuc_xyz, nuc_Z, bf_xyz + 3 * i, bf_alpha[i], bf_xyz + 3 * j,
               bf_alpha[j], S ? S + o : NULL, T ? T + o : NULL, V ? V + o : NULL,
               W0 ? W0 + o : NULL);
    }
  }
}

/* Full symmetric N x N matrices (row-major, leading dimension N): the upper triangle is
 * evaluated and mirrored, so the result is exactly symmetric. */
void x2c_ints_full(int nnuc, const double *nuc_xyz, const double *nuc_Z, int nbf,
                   const double *bf_xyz, const double *bf_alpha, double *S, double *T,
                   double *V, double *W0) {
  const int64_t n = nbf;
#pragma omp parallel for schedule(dynamic, 1)
  for (int i = 0; i < nbf; ++i) {
    for (int j = i; j < nbf; ++j) {
      double s, t, v, w;
      one_pair(nnuc, nuc_xyz, nuc_Z, bf_xyz + 3 * i, bf_alpha[i], bf_xyz + 3 * j,
               bf_alpha[j], &s, &t, V ? &v : NULL, W0 ? &w : NULL);
      if (S) { S[i * n + j] = s; S[j * n + i] = s; }
      if (T) { T[i * n + j] = t; T[j * n + i] = t; }
      if (V) { V[i * n + j] = v; V[j * n + i] = v; }
      if (W0) { W0[i * n + j] = w; W0[j * n + i] = w; }
    }
  }
}
