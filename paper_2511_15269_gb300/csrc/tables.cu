// Host-side FP64 constant tables of the evaluation kernels.
//
// The kernels keep expansions in a normalised, radius-scaled real basis:
//   multipole  M^m_n = C^m_n K_n^m / rho^n,
//   local      L^m_n = +-D^m_n rho^n / K_n^m   (minus sign for m < 0),
// with C, D the real coefficients of Sec. II.C, K_n^m = sqrt((n-|m|)!(n+|m|)!)
// and rho the box's scaling radius.  In this basis the azimuthal rotation of
// App. B.1 has the same form for multipoles and locals, and the polar
// rotation of App. B.2 is W^m_{n,k}(beta) for both (the N^m_{n,k} factors
// cancel).  A polar rotation is evaluated as Y(beta) = B^-1 Z(beta) B with the
// fixed per-degree matrices
//   B = Y(-pi/2) Z(-pi/2),   B^-1 = Z(pi/2) Y(pi/2),
// which follow from turning about y = (quarter turn taking y to z) o (turn
// about z) o (its inverse).  Y(+-pi/2) uses Wigner elements at a right angle,
//   d^n_{m,k}(pi/2) = 2^-n sqrt((n+m)!(n-m)!/((n+k)!(n-k)!))
//                     * sum_t (-1)^(m-k+t) C(n+k, t) C(n-k, n-m-t),
// whose sum is an exact integer.  About a quarter of B's entries vanish by
// parity, which the kernels skip at compile time.
//
// Diagonal (axial) transforms of App. B.3 in the scaled basis, for a shift of
// length r along +z, with u_S = rho_S/r, u_T = rho_T/r, a = r/rho_P,
// b = rho_C/rho_P:
//   M2L  L^m_n = sum_k (-1)^(k+m) (n+k)!/(K_n^m K_k^m) u_T^n u_S^k / r  M^m_k
//   M2M  M'^m_n = sum_{k<=n} sqrt(C(n-|m|,k-|m|) C(n+|m|,k+|m|)) a^(n-k) b^k M^m_k
//   L2L  L'^m_n = sum_{k>=n} (-1)^(k-n) sqrt(C(k-|m|,n-|m|) C(k+|m|,n+|m|)) a^(k-n) b^n L^m_k
// Normalised regular basis Rt^m_n = K_n^m R^m_n (App. A.1 times K):
//   Rt^0_0 = 1, Rt^1_1 = x/sqrt2, Rt^-1_1 = -y/sqrt2,
//   Rt^+-n_n = sqrt((2n-1)/(2n)) (x Rt.. +- y Rt..)          (diagonal)
//   Rt^+-n_{n+1} = sqrt(2n+1) z Rt^+-n_n                      (sub-diagonal)
//   Rt^m_n = (2n-1)/sqrt((n-m)(n+m)) z Rt^m_{n-1}
//            - sqrt((n-m-1)(n+m-1)/((n-m)(n+m))) r^2 Rt^m_{n-2}
#include <cmath>
#include <cstring>
#include <mutex>

#include "common.cuh"

namespace fmm {
namespace {

double fact(int n) {
  double f = 1.0;
  for (int i = 2; i <= n; i++) f *= i;
  return f;
}

double binom(int n, int k) {
  if (k < 0 || k > n) return 0.0;
  double b = 1.0;
  for (int i = 1; i <= k; i++) b = b * (n - k + i) / i;
  return b;
}

long long ibinom(int n, int k) {
  if (k < 0 || k > n) return 0;
  long long b = 1;
  for (int i = 1; i <= k; i++) b = b * (n - k + i) / i;
  return b;
}

// Wigner element at a right angle, d^n_{m,k}(pi/2).
double d_right(int n, int m, int k) {
  long long s = 0;
  for (int t = 0; t <= 2 * n; t++) {
    if (n + k - t < 0 || n - m - t < 0 || m - k + t < 0) continue;
    long long term = ibinom(n + k, t) * ibinom(n - k, n - m - t);
    s += ((m - k + t) % 2 == 0) ? term : -term;
  }
  double norm = std::sqrt(fact(n + m) * fact(n - m) / (fact(n + k) * fact(n - k)));
  return std::ldexp(norm * (double)s, -n);
}

// Internal-basis polar rotation by sign * pi/2 for degree n; Y[row][col],
// row = m + n, col = source index + n.
void polar_right(int n, int sign, double* Y) {
  int w = 2 * n + 1;
  std::memset(Y, 0, sizeof(double) * w * w);
  for (int m = -n; m <= n; m++) {
    int am = m < 0 ? -m : m;
    for (int k = 0; k <= n; k++) {
      auto d = [&](int a, int b) { return sign > 0 ? d_right(n, a, b) : d_right(n, b, a); };
      double W;
      if (k > 0) W = d(am, k) + (m >= 0 ? 1.0 : -1.0) * ((k % 2) ? -1.0 : 1.0) * d(am, -k);
      else W = (m >= 0) ? d(am, 0) : 0.0;
      int src = (m >= 0) ? k : -k;
      Y[(m + n) * w + (src + n)] = W;
    }
  }
}

// Azimuthal rotation by a quarter turn (sign * pi/2): entries are 0 or +-1.
void azimuth_right(int n, int sign, double* Z) {
  int w = 2 * n + 1;
  std::memset(Z, 0, sizeof(double) * w * w);
  Z[n * w + n] = 1.0;
  for (int m = 1; m <= n; m++) {
    // cos(m a), sin(m a) for a = sign * pi/2, exactly
    int q = ((m * sign) % 4 + 4) % 4;
    double c = (q == 0) ? 1 : (q == 2) ? -1 : 0;
    double s = (q == 1) ? 1 : (q == 3) ? -1 : 0;
    Z[(m + n) * w + (m + n)] = c;
    Z[(m + n) * w + (-m + n)] = -s;
    Z[(-m + n) * w + (-m + n)] = c;
    Z[(-m + n) * w + (m + n)] = s;
  }
}

void matmul(int w, const double* A, const double* B, double* C) {
  for (int i = 0; i < w; i++)
    for (int j = 0; j < w; j++) {
      double s = 0;
      for (int k = 0; k < w; k++) s += A[i * w + k] * B[k * w + j];
      C[i * w + j] = s;
    }
}

HostTables* g_tab = nullptr;
std::once_flag g_once;

void build_tables() {
  HostTables* T = new HostTables();
  std::memset(T, 0, sizeof(HostTables));
  const int P = kMaxP;
  static double Y[21 * 21], Z[21 * 21];
  for (int n = 0; n <= P; n++) {
    int w = 2 * n + 1;
    polar_right(n, -1, Y);
    azimuth_right(n, -1, Z);
    matmul(w, Y, Z, T->B + b_off(n));
    azimuth_right(n, +1, Z);
    polar_right(n, +1, Y);
    matmul(w, Z, Y, T->Binv + b_off(n));
  }
  auto K = [](int j, int m) { return std::sqrt(fact(j - m) * fact(j + m)); };
  for (int n = 0; n <= P; n++)
    for (int k = 0; k <= P; k++)
      for (int m = 0; m <= P; m++) {
        int id = (n * (P + 1) + k) * (P + 1) + m;
        if (m <= n && m <= k) {
          double sg = ((k + m) % 2) ? -1.0 : 1.0;
          T->ax_m2l[id] = sg * fact(n + k) / (K(n, m) * K(k, m));
        }
        if (m <= k && k <= n) T->ax_m2m[id] = std::sqrt(binom(n - m, k - m) * binom(n + m, k + m));
        if (m <= n && n <= k) {
          double sg = ((k - n) % 2) ? -1.0 : 1.0;
          T->ax_l2l[id] = sg * std::sqrt(binom(k - m, n - m) * binom(k + m, n + m));
        }
      }
  for (int n = 0; n <= P; n++) {
    T->r_diag[n] = (n >= 1) ? std::sqrt((2.0 * n - 1.0) / (2.0 * n)) : 0.0;
    T->r_sub[n] = std::sqrt(2.0 * n + 1.0);
    for (int m = 0; m <= P; m++) {
      int id = n * (P + 1) + m;
      if (m + 2 <= n) {
        double nm = (double)(n - m) * (n + m);
        T->r_a[id] = (2.0 * n - 1.0) / std::sqrt(nm);
        T->r_b[id] = std::sqrt((double)(n - m - 1) * (n + m - 1) / nm);
      }
    }
  }
  g_tab = T;
}

}  // namespace

const HostTables& host_tables() {
  std::call_once(g_once, build_tables);
  return *g_tab;
}

}  // namespace fmm
