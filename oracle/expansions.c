/*
 * Oracle: basis functions, rotations and axial transforms of the
 * rotation-based FMM operators.  TEST INFRASTRUCTURE ONLY (see fmm_oracle.h).
 *
 * Basis recursions follow App. A; rotations and diagonal transforms follow
 * App. B.  Readings taken where the paper is ambiguous or garbled:
 *  - App. A.3: the leading minus sign of grad R^n_n is a typo; differentiating
 *    the App. A.1 diagonal recursion gives a plus sign, used here.
 *  - App. B.2: d^{|m|}_{n,k}(b) is the Wigner small-d matrix element
 *    d^n_{|m|,k}(b) = <n |m| | exp(-i b J_y) | n k>; the W cases "|k|=0,
 *    |m|>=0" and "|k|=0, |m|<0" are read as k=0 with m>=0 and with m<0.
 *  - "C(phi + dphi)" and "C(theta + dtheta)" are the coefficients in a frame
 *    turned by +dphi about z (by +dtheta about y); a translation vector
 *    t = c_old - c_new with spherical angles (theta_t, phi_t) is brought onto
 *    +z by an azimuthal turn of phi_t followed by a polar turn of theta_t, and
 *    the App. B.3 diagonal transforms use r = |t|.
 *  - The Wigner matrix elements come from the Jacobi-polynomial form of
 *    d^n_{m,k} with the three-term recurrence of Abramowitz & Stegun 22.7.1;
 *    the paper cites Jacobi recursions (Sec. II.D) whose text is not given.
 */
#include "fmm_oracle.h"
#include <math.h>
#include <stdlib.h>
#include <string.h>

static inline int ix(int n, int m) { return n * n + n + m; }
static inline int iabs(int a) { return a < 0 ? -a : a; }

static double fact(int n) {
  double f = 1.0;
  for (int i = 2; i <= n; i++) f *= (double)i;
  return f;
}

static double binom(int n, int k) {
  if (k < 0 || k > n) return 0.0;
  double b = 1.0;
  for (int i = 1; i <= k; i++) b = b * (double)(n - k + i) / (double)i;
  return b;
}

/* App. A.1: real regular basis R^m_n(x, y, z). */
void orc_rhat(int p, double x, double y, double z, double* R) {
  double r2 = x * x + y * y + z * z;
  R[ix(0, 0)] = 1.0;
  if (p >= 1) {
    R[ix(1, 1)] = x / 2.0;
    R[ix(1, -1)] = -y / 2.0;
  }
  for (int n = 2; n <= p; n++) {
    R[ix(n, n)] = (x * R[ix(n - 1, n - 1)] + y * R[ix(n - 1, 1 - n)]) / (2.0 * n);
    R[ix(n, -n)] = (x * R[ix(n - 1, 1 - n)] - y * R[ix(n - 1, n - 1)]) / (2.0 * n);
  }
  for (int n = 0; n <= p - 1; n++) {
    R[ix(n + 1, n)] = z * R[ix(n, n)];
    R[ix(n + 1, -n)] = z * R[ix(n, -n)];
  }
  for (int n = 2; n <= p; n++)
    for (int m = 2 - n; m <= n - 2; m++)
      R[ix(n, m)] = ((2.0 * n - 1.0) * z * R[ix(n - 1, m)] - r2 * R[ix(n - 2, m)]) /
                    ((double)(n - iabs(m)) * (double)(n + iabs(m)));
}

/* App. A.2: real singular basis S^m_n(x, y, z). */
void orc_shat(int p, double x, double y, double z, double* S) {
  double r2 = x * x + y * y + z * z;
  double r = sqrt(r2);
  S[ix(0, 0)] = 1.0 / r;
  if (p >= 1) {
    S[ix(1, 1)] = x / (r2 * r);
    S[ix(1, -1)] = y / (r2 * r);
  }
  for (int n = 2; n <= p; n++) {
    S[ix(n, n)] = (2.0 * n - 1.0) * (x * S[ix(n - 1, n - 1)] - y * S[ix(n - 1, 1 - n)]) / r2;
    S[ix(n, -n)] = (2.0 * n - 1.0) * (x * S[ix(n - 1, 1 - n)] + y * S[ix(n - 1, n - 1)]) / r2;
  }
  for (int n = 0; n <= p - 1; n++) {
    S[ix(n + 1, n)] = (2.0 * n + 1.0) * z * S[ix(n, n)] / r2;
    S[ix(n + 1, -n)] = (2.0 * n + 1.0) * z * S[ix(n, -n)] / r2;
  }
  for (int n = 2; n <= p; n++)
    for (int m = 2 - n; m <= n - 2; m++)
      S[ix(n, m)] = ((2.0 * n - 1.0) * z * S[ix(n - 1, m)] -
                     (double)(n - 1 - m) * (double)(n - 1 + m) * S[ix(n - 2, m)]) / r2;
}

/* App. A.3: gradient of the regular basis; G[3*idx + c], c = x, y, z.
 * Diagonal term uses the sign obtained by differentiating App. A.1. */
void orc_grad_rhat(int p, double x, double y, double z, double* R, double* G) {
  orc_rhat(p, x, y, z, R);
  double r2 = x * x + y * y + z * z;
  double rv[3] = {x, y, z};
  int P = (p + 1) * (p + 1);
  memset(G, 0, sizeof(double) * 3 * P);
  if (p >= 1) {
    G[3 * ix(1, 1) + 0] = 0.5;
    G[3 * ix(1, -1) + 1] = -0.5;
  }
  for (int n = 2; n <= p; n++) {
    const double* ga = &G[3 * ix(n - 1, n - 1)];
    const double* gb = &G[3 * ix(n - 1, 1 - n)];
    double a = R[ix(n - 1, n - 1)], b = R[ix(n - 1, 1 - n)];
    double* gp = &G[3 * ix(n, n)];
    double* gm = &G[3 * ix(n, -n)];
    for (int c = 0; c < 3; c++) {
      double ex = (c == 0) ? 1.0 : 0.0, ey = (c == 1) ? 1.0 : 0.0;
      gp[c] = (x * ga[c] + y * gb[c] + a * ex + b * ey) / (2.0 * n);
      gm[c] = (x * gb[c] - y * ga[c] + b * ex - a * ey) / (2.0 * n);
    }
  }
  for (int n = 0; n <= p - 1; n++) {
    for (int sgn = 0; sgn < 2; sgn++) {
      int m = sgn ? -n : n;
      const double* g0 = &G[3 * ix(n, m)];
      double* g1 = &G[3 * ix(n + 1, m)];
      for (int c = 0; c < 3; c++) g1[c] = z * g0[c] + ((c == 2) ? R[ix(n, m)] : 0.0);
    }
  }
  for (int n = 2; n <= p; n++)
    for (int m = 2 - n; m <= n - 2; m++) {
      const double* g1 = &G[3 * ix(n - 1, m)];
      const double* g2 = &G[3 * ix(n - 2, m)];
      double* g = &G[3 * ix(n, m)];
      for (int c = 0; c < 3; c++)
        g[c] = ((2.0 * n - 1.0) * (z * g1[c] + ((c == 2) ? R[ix(n - 1, m)] : 0.0)) -
                r2 * g2[c] - 2.0 * R[ix(n - 2, m)] * rv[c]) /
               ((double)n * n - (double)m * m);
    }
}

/* Jacobi polynomial P_k^{(a,b)}(x) by the three-term recurrence in the degree
 * (Abramowitz & Stegun 22.7.1). */
static double jacobi_p(int k, int a, int b, double x) {
  if (k == 0) return 1.0;
  double p0 = 1.0;
  double p1 = (a + 1.0) + (a + b + 2.0) * (x - 1.0) / 2.0;
  for (int n = 1; n < k; n++) {
    double c = 2.0 * n + a + b;
    double p2 = ((c + 1.0) * (c * (c + 2.0) * x + (double)a * a - (double)b * b) * p1 -
                 2.0 * (n + a) * (n + b) * (c + 2.0) * p0) /
                (2.0 * (n + 1) * (n + a + b + 1.0) * c);
    p0 = p1;
    p1 = p2;
  }
  return p1;
}

/* Wigner small-d element d^j_{m,k}(beta) = <j m| exp(-i beta J_y) |j k> via
 * its Jacobi-polynomial form. */
static double wigner_elem(int j, int m, int k, double beta) {
  int kk = j + k, a, lam;
  if (j - k < kk) kk = j - k;
  if (j + m < kk) kk = j + m;
  if (j - m < kk) kk = j - m;
  if (kk == j + k) { a = m - k; lam = m - k; }
  else if (kk == j - k) { a = k - m; lam = 0; }
  else if (kk == j + m) { a = k - m; lam = 0; }
  else { a = m - k; lam = m - k; }
  int b = 2 * j - 2 * kk - a;
  double sgn = (lam % 2 == 0) ? 1.0 : -1.0;
  double norm = sqrt(binom(2 * j - kk, kk + a) / binom(kk + b, b));
  return sgn * norm * pow(sin(beta / 2.0), a) * pow(cos(beta / 2.0), b) *
         jacobi_p(kk, a, b, cos(beta));
}

void orc_wigner_d(int p, double beta, double* d) {
  int w = 2 * p + 1;
  memset(d, 0, sizeof(double) * (size_t)(p + 1) * w * w);
  for (int n = 0; n <= p; n++)
    for (int m = -n; m <= n; m++)
      for (int k = -n; k <= n; k++)
        d[((size_t)n * w + (m + p)) * w + (k + p)] = wigner_elem(n, m, k, beta);
}

/* App. B.1: rotation by dphi about z.  local = 0: multipole, 1: local. */
void orc_rotate_azimuthal(int p, int local, double dphi, const double* in, double* out) {
  for (int n = 0; n <= p; n++) {
    out[ix(n, 0)] = in[ix(n, 0)];
    for (int m = 1; m <= n; m++) {
      double c = cos(m * dphi), s = sin(m * dphi);
      double a = in[ix(n, m)], b = in[ix(n, -m)];
      if (!local) {
        out[ix(n, m)] = a * c - b * s;   /* C^m cos(m dphi) - C^{-m} sin(m dphi)   */
        out[ix(n, -m)] = b * c + a * s;  /* same rule at -m: C^{-m} cos + C^m sin   */
      } else {
        out[ix(n, m)] = a * c + b * s;   /* D^m cos(m dphi) + D^{-m} sin(m dphi)   */
        out[ix(n, -m)] = b * c - a * s;  /* same rule at -m */
      }
    }
  }
}

/* App. B.2: rotation by dtheta about y,
 *   C'^m_n = sum_{k=0}^{n} C^{sgn(m) k}_n N^m_{n,k} W^m_{n,k},
 *   D'^m_n = sum_{k=0}^{n} D^{sgn(m) k}_n W^m_{n,k} / N^m_{n,k}. */
void orc_rotate_polar(int p, int local, double dtheta, const double* in, double* out) {
  int w = 2 * p + 1;
  double* d = (double*)malloc(sizeof(double) * (size_t)(p + 1) * w * w);
  orc_wigner_d(p, dtheta, d);
#define DW(n, m, k) d[((size_t)(n) * w + ((m) + p)) * w + ((k) + p)]
  for (int n = 0; n <= p; n++)
    for (int m = -n; m <= n; m++) {
      int am = iabs(m);
      double sgm = (m >= 0) ? 1.0 : -1.0;
      double acc = 0.0;
      for (int k = 0; k <= n; k++) {
        double W;
        if (k > 0) {
          double pm = (k % 2 == 0) ? 1.0 : -1.0;
          W = DW(n, am, k) + sgm * pm * DW(n, am, -k);
        } else {
          W = (m >= 0) ? DW(n, am, 0) : 0.0;
        }
        double N = sqrt(fact(n - k) * fact(n + k) / (fact(n - m) * fact(n + m)));
        int src = (m >= 0) ? k : -k;
        acc += in[ix(n, src)] * (local ? W / N : N * W);
      }
      out[ix(n, m)] = acc;
    }
#undef DW
  free(d);
}

/* App. B.3 diagonal transforms along b = (0, 0, r). */
void orc_axial_m2m(int p, double r, const double* in, double* out) {
  for (int n = 0; n <= p; n++)
    for (int m = -n; m <= n; m++) {
      double acc = 0.0;
      for (int k = iabs(m); k <= n; k++)
        acc += pow(r, n - k) / fact(n - k) * in[ix(k, m)];
      out[ix(n, m)] = acc;
    }
}

void orc_axial_m2l(int p, double r, const double* in, double* out) {
  for (int n = 0; n <= p; n++)
    for (int m = -n; m <= n; m++) {
      double sgm = (m >= 0) ? 1.0 : -1.0;
      double acc = 0.0;
      for (int k = iabs(m); k <= p; k++) {
        double pm = ((k + iabs(m)) % 2 == 0) ? 1.0 : -1.0; /* (-1)^(k+m) */
        acc += sgm * pm * fact(n + k) / pow(r, n + k + 1) * in[ix(k, m)];
      }
      out[ix(n, m)] = acc;
    }
}

void orc_axial_l2l(int p, double r, const double* in, double* out) {
  for (int n = 0; n <= p; n++)
    for (int m = -n; m <= n; m++) {
      double acc = 0.0;
      for (int k = n; k <= p; k++)
        acc += pow(-r, k - n) / fact(k - n) * in[ix(k, m)];
      out[ix(n, m)] = acc;
    }
}

/* Spherical angles of t: polar angle theta in [0, pi], azimuth phi. */
static void sph_angles(const double t[3], double* r, double* th, double* ph) {
  double rho = sqrt(t[0] * t[0] + t[1] * t[1]);
  *r = sqrt(t[0] * t[0] + t[1] * t[1] + t[2] * t[2]);
  *th = atan2(rho, t[2]);
  *ph = atan2(t[1], t[0]);
}

enum { OP_M2M = 0, OP_M2L = 1, OP_L2L = 2 };

/* Rotate so that t = c_old - c_new lies on +z, apply the diagonal transform,
 * rotate back (Sec. II.D), and add the result into out. */
static void rotated_translate(int op, int p, const double* in, const double c_old[3],
                              const double c_new[3], double* out) {
  int P = (p + 1) * (p + 1);
  double t[3] = {c_old[0] - c_new[0], c_old[1] - c_new[1], c_old[2] - c_new[2]};
  double r, th, ph;
  sph_angles(t, &r, &th, &ph);
  double* a = (double*)malloc(sizeof(double) * P);
  double* b = (double*)malloc(sizeof(double) * P);
  int in_local = (op == OP_L2L);
  int out_local = (op != OP_M2M);
  orc_rotate_azimuthal(p, in_local, ph, in, a);
  orc_rotate_polar(p, in_local, th, a, b);
  if (op == OP_M2M) orc_axial_m2m(p, r, b, a);
  else if (op == OP_M2L) orc_axial_m2l(p, r, b, a);
  else orc_axial_l2l(p, r, b, a);
  orc_rotate_polar(p, out_local, -th, a, b);
  orc_rotate_azimuthal(p, out_local, -ph, b, a);
  for (int i = 0; i < P; i++) out[i] += a[i];
  free(a);
  free(b);
}

void orc_m2m(int p, const double* C, const double c_old[3], const double c_new[3], double* out) {
  rotated_translate(OP_M2M, p, C, c_old, c_new, out);
}
void orc_m2l(int p, const double* C, const double c_src[3], const double c_trg[3], double* out) {
  rotated_translate(OP_M2L, p, C, c_src, c_trg, out);
}
void orc_l2l(int p, const double* D, const double c_old[3], const double c_new[3], double* out) {
  rotated_translate(OP_L2L, p, D, c_old, c_new, out);
}

/* Sec. II.C: C^m_n = sum_i q_i R^m_n(r_i - c). */
void orc_p2m(int p, const double* pts, const double* q, int64_t n, const double c[3], double* out) {
  int P = (p + 1) * (p + 1);
  double* R = (double*)malloc(sizeof(double) * P);
  for (int64_t i = 0; i < n; i++) {
    orc_rhat(p, pts[3 * i] - c[0], pts[3 * i + 1] - c[1], pts[3 * i + 2] - c[2], R);
    for (int k = 0; k < P; k++) out[k] += q[i] * R[k];
  }
  free(R);
}

/* Local coefficients of point charges: D^m_n = sum_i q_i S^m_n(r_i - c)
 * (Eq. 11 in the real basis; used by the tests as an exact reference). */
void orc_p2l(int p, const double* pts, const double* q, int64_t n, const double c[3], double* out) {
  int P = (p + 1) * (p + 1);
  double* S = (double*)malloc(sizeof(double) * P);
  for (int64_t i = 0; i < n; i++) {
    orc_shat(p, pts[3 * i] - c[0], pts[3 * i + 1] - c[1], pts[3 * i + 2] - c[2], S);
    for (int k = 0; k < P; k++) out[k] += q[i] * S[k];
  }
  free(S);
}

/* Sec. II.C evaluation rule  sum_n sum_m (2 - delta_0m) sgn(m) D^m_n R^m_n(x - c),
 * returned without the -1/(4 pi) factor; grad is its gradient in x. */
double orc_l2p(int p, const double* D, const double c[3], const double x[3], double* grad) {
  int P = (p + 1) * (p + 1);
  double* R = (double*)malloc(sizeof(double) * P);
  double* G = (double*)malloc(sizeof(double) * 3 * P);
  orc_grad_rhat(p, x[0] - c[0], x[1] - c[1], x[2] - c[2], R, G);
  double u = 0.0, g0 = 0.0, g1 = 0.0, g2 = 0.0;
  for (int n = 0; n <= p; n++)
    for (int m = -n; m <= n; m++) {
      double wgt = (m == 0) ? 1.0 : ((m > 0) ? 2.0 : -2.0);
      int k = ix(n, m);
      u += wgt * D[k] * R[k];
      g0 += wgt * D[k] * G[3 * k];
      g1 += wgt * D[k] * G[3 * k + 1];
      g2 += wgt * D[k] * G[3 * k + 2];
    }
  if (grad) { grad[0] = g0; grad[1] = g1; grad[2] = g2; }
  free(R);
  free(G);
  return u;
}

/* Multipole evaluation with the same contraction against the singular basis
 * (Eq. 8 in the real basis), without the -1/(4 pi) factor. */
double orc_m2p(int p, const double* C, const double c[3], const double x[3]) {
  int P = (p + 1) * (p + 1);
  double* S = (double*)malloc(sizeof(double) * P);
  orc_shat(p, x[0] - c[0], x[1] - c[1], x[2] - c[2], S);
  double u = 0.0;
  for (int n = 0; n <= p; n++)
    for (int m = -n; m <= n; m++) {
      double wgt = (m == 0) ? 1.0 : ((m > 0) ? 2.0 : -2.0);
      u += wgt * C[ix(n, m)] * S[ix(n, m)];
    }
  free(S);
  return u;
}
