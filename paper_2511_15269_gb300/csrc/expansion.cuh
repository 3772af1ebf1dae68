// Device-side expansion algebra, compiled once per precision: the including
// translation unit defines `real` (float or double) before including this
// header.  The rotations and the axial M2L are templates on the value type,
// so that the FP64-accurate path can also run them on double-float values.  Table entries come from tables_gen.h (written by gen_tables.py).
//
// Coefficient (n, m) of an order-P expansion is v[n*n + n + m].  All loops
// run over compile-time indices, so the coefficient vector stays in registers
// and every table entry is an instruction immediate (no constant-bank
// traffic).
#pragma once
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

#include <type_traits>

#include "common.cuh"
#include "tables_gen.h"

namespace fmm {
namespace {

// Parity pattern of the quarter-turn polar rotation in the internal basis:
// entry (row order m, source order l) of Y(+-pi/2) can be nonzero only if
// m, l >= 0 with n+m+l even, or m, l < 0 with n+|m|+|l| odd.
__host__ __device__ constexpr bool ymask(int n, int m, int l) {
  return (m >= 0 && l >= 0 && ((n + m + l) % 2 == 0)) ||
         (m < 0 && l < 0 && ((n - m - l) % 2 == 1));
}
// A quarter-turn azimuthal rotation maps order m to m (|m| even) or -m (odd).
__host__ __device__ constexpr int qmap(int m) { return ((m < 0 ? -m : m) % 2 == 0) ? m : -m; }
// Nonzero pattern of B = Y(-pi/2) Z(-pi/2) and B^-1 = Z(pi/2) Y(pi/2);
// i, j are row/column indices m + n, m' + n of degree n.
__host__ __device__ constexpr bool b_nz(int n, int i, int j) { return ymask(n, i - n, qmap(j - n)); }
__host__ __device__ constexpr bool bi_nz(int n, int i, int j) { return ymask(n, qmap(i - n), j - n); }

// Every structurally skipped entry of B and B^-1 must be zero.
void upload_tables() {
  for (int n = 0; n <= kMaxP; n++)
    for (int i = 0; i <= 2 * n; i++)
      for (int j = 0; j <= 2 * n; j++) {
        const int id = b_off(n) + i * (2 * n + 1) + j;
        if ((!b_nz(n, i, j) && gen::kB[id] != 0.0) || (!bi_nz(n, i, j) && gen::kBi[id] != 0.0)) {
          set_error("rotation table sparsity check failed at degree %d (%d, %d)", n, i, j);
          throw Fail{FMM_ERR_CUDA};
        }
      }
}

template <int B, int E, class F>
__device__ __forceinline__ void sfor(F&& f) {
  if constexpr (B < E) {
    f(std::integral_constant<int, B>{});
    sfor<B + 1, E>(f);
  }
}

__host__ __device__ constexpr int ix(int n, int m) { return n * n + n + m; }
__host__ __device__ constexpr int ax_id(int n, int k, int m) {
  return (n * (kMaxP + 1) + k) * (kMaxP + 1) + m;
}
__host__ __device__ constexpr int iabs_c(int a) { return a < 0 ? -a : a; }

__device__ __forceinline__ real fmar(real a, real b, real c) { return fma(a, b, c); }

// Azimuthal rotation (App. B.1 form, identical for multipoles and locals in
// the internal basis).  INV applies the opposite angle.
template <int P, bool INV, class T>
__device__ __forceinline__ void rot_z(T (&v)[ncoef(P)], const T (&c)[P], const T (&s)[P]) {
#pragma unroll
  for (int n = 1; n <= P; n++)
#pragma unroll
    for (int m = 1; m <= n; m++) {
      T a = v[ix(n, m)], b = v[ix(n, -m)];
      if (!INV) {
        v[ix(n, m)] = fmar(a, c[m - 1], -b * s[m - 1]);
        v[ix(n, -m)] = fmar(b, c[m - 1], a * s[m - 1]);
      } else {
        v[ix(n, m)] = fmar(a, c[m - 1], b * s[m - 1]);
        v[ix(n, -m)] = fmar(b, c[m - 1], -a * s[m - 1]);
      }
    }
}

// v <- B v (INV = false) or B^-1 v (INV = true), degree by degree, skipping
// the structural zeros.
template <int P, bool INV, class T>
__device__ __forceinline__ void apply_b(T (&v)[ncoef(P)]) {
  sfor<1, P + 1>([&](auto nn) {
    constexpr int n = decltype(nn)::value;
    constexpr int w = 2 * n + 1;
    T out[w];
    sfor<0, w>([&](auto ii) {
      constexpr int i = decltype(ii)::value;
      T acc = T(0.0);
      sfor<0, w>([&](auto jj) {
        constexpr int j = decltype(jj)::value;
        constexpr bool nz = INV ? bi_nz(n, i, j) : b_nz(n, i, j);
        if constexpr (nz) {
          constexpr double c = INV ? gen::kBi[b_off(n) + i * w + j] : gen::kB[b_off(n) + i * w + j];
          if constexpr (c != 0.0) {
            constexpr T cc = T(c);
            acc = fmar(cc, v[n * n + j], acc);
          }
        }
      });
      out[i] = acc;
    });
#pragma unroll
    for (int i = 0; i < w; i++) v[n * n + i] = out[i];
  });
}

// cos(m a), sin(m a) for m = 1..P from cos a, sin a by angle addition, in
// the arithmetic of T (FP32: the error grows by about one rounding per step,
// and the degree-m coefficients it touches carry the factor (rho/r)^m of the
// expansion, so the potential sees a few roundings at most).
template <int P, class T>
__device__ __forceinline__ void trig_multiples(T c1, T s1, T (&c)[P], T (&s)[P]) {
  c[0] = c1;
  s[0] = s1;
#pragma unroll
  for (int m = 1; m < P; m++) {
    c[m] = fmar(c[m - 1], c1, -(s[m - 1] * s1));
    s[m] = fmar(s[m - 1], c1, c[m - 1] * s1);
  }
}

// Rotate so that the translation vector lies on +z, apply the axial
// transform `axial`, rotate back.  Both polar rotations run through one copy
// of the quarter-turn products (a two-pass loop, the second pass with the
// opposite angle), which halves the instruction footprint of the kernels.
template <int P, class T, class Axial>
__device__ __forceinline__ void translate_rotated(T (&v)[ncoef(P)], const T (&cp)[P], const T (&sp)[P],
                                                  const T (&ct)[P], const T (&st)[P], Axial&& axial) {
  T s[P];
#pragma unroll
  for (int m = 0; m < P; m++) s[m] = st[m];
  rot_z<P, false>(v, cp, sp);
#pragma unroll 1
  for (int pass = 0; pass < 2; pass++) {
    if (pass == 1) axial(v);
    apply_b<P, false>(v);
    rot_z<P, false>(v, ct, s);
    apply_b<P, true>(v);
#pragma unroll
    for (int m = 0; m < P; m++) s[m] = -s[m];
  }
  rot_z<P, true>(v, cp, sp);
}

// Axial M2L in the scaled basis (App. B.3), in place: multipole -> local.
template <int P, class T>
__device__ __forceinline__ void axial_m2l(T (&v)[ncoef(P)], T uS, T uT, T rinv) {
  T pS[P + 1], pT[P + 1];
  pS[0] = T(1.0);
  pT[0] = rinv;
#pragma unroll
  for (int k = 1; k <= P; k++) {
    pS[k] = pS[k - 1] * uS;
    pT[k] = pT[k - 1] * uT;
  }
  sfor<0, 2 * P + 1>([&](auto mm) {
    constexpr int m = decltype(mm)::value - P;
    constexpr int am = m < 0 ? -m : m;
    T in[P + 1];
#pragma unroll
    for (int k = am; k <= P; k++) in[k] = v[ix(k, m)] * pS[k];
    sfor<am, P + 1>([&](auto nn) {
      constexpr int n = decltype(nn)::value;
      T acc = T(0.0);
      sfor<am, P + 1>([&](auto kk) {
        constexpr int k = decltype(kk)::value;
        constexpr double c = gen::kAxM2L[ax_id(n, k, am)];
        constexpr T cc = T(c);
        acc = fmar(cc, in[k], acc);
      });
      v[ix(n, m)] = acc * pT[n];
    });
  });
}

// Axial M2M (App. B.3), a = r/rho_parent, b = rho_child/rho_parent.
template <int P>
__device__ __forceinline__ void axial_m2m(real (&v)[ncoef(P)], real a, real b) {
  real pB[P + 1];
  pB[0] = real(1);
#pragma unroll
  for (int k = 1; k <= P; k++) pB[k] = pB[k - 1] * b;
  sfor<0, 2 * P + 1>([&](auto mm) {
    constexpr int m = decltype(mm)::value - P;
    constexpr int am = m < 0 ? -m : m;
    real in[P + 1];
#pragma unroll
    for (int k = am; k <= P; k++) in[k] = v[ix(k, m)] * pB[k];
    sfor<am, P + 1>([&](auto nn) {
      constexpr int n = decltype(nn)::value;
      // sum_k c_nk a^(n-k) in_k in Horner form, lowest k first
      real acc = real(0);
      sfor<am, n + 1>([&](auto kk) {
        constexpr int k = decltype(kk)::value;
        constexpr double c = gen::kAxM2M[ax_id(n, k, am)];
        acc = fmar(acc, a, real(c) * in[k]);
      });
      v[ix(n, m)] = acc;
    });
  });
}

// Axial L2L (App. B.3), a = r/rho_parent, b = rho_child/rho_parent.
template <int P>
__device__ __forceinline__ void axial_l2l(real (&v)[ncoef(P)], real a, real b) {
  real pB[P + 1];
  pB[0] = real(1);
#pragma unroll
  for (int k = 1; k <= P; k++) pB[k] = pB[k - 1] * b;
  sfor<0, 2 * P + 1>([&](auto mm) {
    constexpr int m = decltype(mm)::value - P;
    constexpr int am = m < 0 ? -m : m;
    real in[P + 1];
#pragma unroll
    for (int k = am; k <= P; k++) in[k] = v[ix(k, m)];
    sfor<am, P + 1>([&](auto nn) {
      constexpr int n = decltype(nn)::value;
      // sum_k c_nk a^(k-n) in_k in Horner form, highest k first
      real acc = real(0);
      sfor<0, P + 1 - n>([&](auto jj) {
        constexpr int k = P - decltype(jj)::value;
        constexpr double c = gen::kAxL2L[ax_id(n, k, am)];
        acc = fmar(acc, a, real(c) * in[k]);
      });
      v[ix(n, m)] = acc * pB[n];
    });
  });
}

// Normalised regular basis Rt(y) up to degree P (the recursions in the
// header comment above),
// evaluated degree by degree; f(n, R) is called after degree n is complete so
// that callers can consume it before older degrees die.
template <int P, class F>
__device__ __forceinline__ void regular_basis(real x, real y, real z, real (&R)[ncoef(P)], F&& consume) {
  const real r2 = fmar(x, x, fmar(y, y, z * z));
  R[0] = real(1);
  consume(std::integral_constant<int, 0>{});
  if constexpr (P >= 1) {
    const real h = real(0.70710678118654752440);
    R[ix(1, 1)] = x * h;
    R[ix(1, -1)] = -y * h;
    R[ix(1, 0)] = z;
    consume(std::integral_constant<int, 1>{});
  }
  sfor<2, P + 1>([&](auto nn) {
    constexpr int n = decltype(nn)::value;
    constexpr double cdd = gen::kRDiag[n];
    const real cd = real(cdd);
    R[ix(n, n)] = cd * fmar(x, R[ix(n - 1, n - 1)], y * R[ix(n - 1, 1 - n)]);
    R[ix(n, -n)] = cd * fmar(x, R[ix(n - 1, 1 - n)], -y * R[ix(n - 1, n - 1)]);
    constexpr double csub = gen::kRSub[n - 1];
    const real zs = real(csub) * z;
    R[ix(n, n - 1)] = zs * R[ix(n - 1, n - 1)];
    R[ix(n, 1 - n)] = zs * R[ix(n - 1, 1 - n)];
    sfor<0, 2 * n - 3>([&](auto mm) {
      constexpr int m = decltype(mm)::value + 2 - n;
      constexpr int am = m < 0 ? -m : m;
      constexpr double ca = gen::kRA[n * (kMaxP + 1) + am];
      constexpr double cb = gen::kRB[n * (kMaxP + 1) + am];
      R[ix(n, m)] = fmar(real(ca) * z, R[ix(n - 1, m)], -(real(cb) * r2) * R[ix(n - 2, m)]);
    });
    consume(nn);
  });
}

}  // namespace
}  // namespace fmm
