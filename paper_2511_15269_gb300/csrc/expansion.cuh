// Device-side expansion algebra, compiled once per precision: the including
// translation unit defines `real` (float or double) before including this
// header, and uploads the constant tables with upload_tables().
//
// Expansions live in the normalised, radius-scaled real basis described in
// tables.cu.  Coefficient (n, m) of an order-P expansion is v[n*n + n + m].
// All loops run over compile-time bounds and are fully unrolled, so the
// coefficient vector stays in registers and every table entry is a constant
// bank operand.
#pragma once

#include <type_traits>

#include "common.cuh"

namespace fmm {
namespace {

__constant__ real c_B[1771];
__constant__ real c_Bi[1771];
__constant__ real c_ax_m2l[(kMaxP + 1) * (kMaxP + 1) * (kMaxP + 1)];
__constant__ real c_ax_m2m[(kMaxP + 1) * (kMaxP + 1) * (kMaxP + 1)];
__constant__ real c_ax_l2l[(kMaxP + 1) * (kMaxP + 1) * (kMaxP + 1)];
__constant__ real c_rdiag[kMaxP + 1];
__constant__ real c_rsub[kMaxP + 1];
__constant__ real c_ra[(kMaxP + 1) * (kMaxP + 1)];
__constant__ real c_rb[(kMaxP + 1) * (kMaxP + 1)];

template <class Dst>
void upload(const Dst& sym, const double* src, size_t count) {
  real tmp[1771];
  for (size_t i = 0; i < count; i++) tmp[i] = (real)src[i];
  FMM_CUDA_TRY(cudaMemcpyToSymbol(sym, tmp, sizeof(real) * count));
}

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

void upload_tables() {
  const HostTables& T = host_tables();
  // every entry the kernels skip must be zero
  for (int n = 0; n <= kMaxP; n++)
    for (int i = 0; i <= 2 * n; i++)
      for (int j = 0; j <= 2 * n; j++) {
        int id = b_off(n) + i * (2 * n + 1) + j;
        if ((!b_nz(n, i, j) && T.B[id] != 0.0 && std::fabs(T.B[id]) > 1e-13) ||
            (!bi_nz(n, i, j) && T.Binv[id] != 0.0 && std::fabs(T.Binv[id]) > 1e-13)) {
          set_error("rotation table sparsity check failed at degree %d (%d, %d)", n, i, j);
          throw Fail{FMM_ERR_CUDA};
        }
      }
  upload(c_B, T.B, 1771);
  upload(c_Bi, T.Binv, 1771);
  upload(c_ax_m2l, T.ax_m2l, 1331);
  upload(c_ax_m2m, T.ax_m2m, 1331);
  upload(c_ax_l2l, T.ax_l2l, 1331);
  upload(c_rdiag, T.r_diag, kMaxP + 1);
  upload(c_rsub, T.r_sub, kMaxP + 1);
  upload(c_ra, T.r_a, 121);
  upload(c_rb, T.r_b, 121);
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
template <int P, bool INV>
__device__ __forceinline__ void rot_z(real (&v)[ncoef(P)], const real (&c)[P], const real (&s)[P]) {
#pragma unroll
  for (int n = 1; n <= P; n++)
#pragma unroll
    for (int m = 1; m <= n; m++) {
      real a = v[ix(n, m)], b = v[ix(n, -m)];
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
template <int P, bool INV>
__device__ __forceinline__ void apply_b(real (&v)[ncoef(P)]) {
  sfor<1, P + 1>([&](auto nn) {
    constexpr int n = decltype(nn)::value;
    constexpr int w = 2 * n + 1;
    real out[w];
    sfor<0, w>([&](auto ii) {
      constexpr int i = decltype(ii)::value;
      real acc = real(0);
      sfor<0, w>([&](auto jj) {
        constexpr int j = decltype(jj)::value;
        constexpr bool nz = INV ? bi_nz(n, i, j) : b_nz(n, i, j);
        if constexpr (nz) acc = fmar(INV ? c_Bi[b_off(n) + i * w + j] : c_B[b_off(n) + i * w + j],
                                     v[n * n + j], acc);
      });
      out[i] = acc;
    });
#pragma unroll
    for (int i = 0; i < w; i++) v[n * n + i] = out[i];
  });
}

// Polar rotation by the angle whose multiples' cosines/sines are (ct, st):
// Y = B^-1 Z B.
template <int P, bool INV>
__device__ __forceinline__ void rot_y(real (&v)[ncoef(P)], const real (&ct)[P], const real (&st)[P]) {
  apply_b<P, false>(v);
  rot_z<P, INV>(v, ct, st);
  apply_b<P, true>(v);
}

// Rotation bringing the translation vector onto +z (forward) and back.
template <int P>
__device__ __forceinline__ void rotate_to_z(real (&v)[ncoef(P)], const real (&cp)[P], const real (&sp)[P],
                                            const real (&ct)[P], const real (&st)[P]) {
  rot_z<P, false>(v, cp, sp);
  rot_y<P, false>(v, ct, st);
}
template <int P>
__device__ __forceinline__ void rotate_from_z(real (&v)[ncoef(P)], const real (&cp)[P], const real (&sp)[P],
                                              const real (&ct)[P], const real (&st)[P]) {
  rot_y<P, true>(v, ct, st);
  rot_z<P, true>(v, cp, sp);
}

// Axial M2L in the scaled basis (App. B.3), in place: multipole -> local.
template <int P>
__device__ __forceinline__ void axial_m2l(real (&v)[ncoef(P)], real uS, real uT, real rinv) {
  real pS[P + 1], pT[P + 1];
  pS[0] = real(1);
  pT[0] = rinv;
#pragma unroll
  for (int k = 1; k <= P; k++) {
    pS[k] = pS[k - 1] * uS;
    pT[k] = pT[k - 1] * uT;
  }
#pragma unroll
  for (int m = -P; m <= P; m++) {
    const int am = m < 0 ? -m : m;
    real in[P + 1];
#pragma unroll
    for (int k = am; k <= P; k++) in[k] = v[ix(k, m)] * pS[k];
#pragma unroll
    for (int n = am; n <= P; n++) {
      real acc = real(0);
#pragma unroll
      for (int k = am; k <= P; k++) acc = fmar(c_ax_m2l[ax_id(n, k, am)], in[k], acc);
      v[ix(n, m)] = acc * pT[n];
    }
  }
}

// Axial M2M (App. B.3), a = r/rho_parent, b = rho_child/rho_parent.
template <int P>
__device__ __forceinline__ void axial_m2m(real (&v)[ncoef(P)], real a, real b) {
  real pA[P + 1], pB[P + 1];
  pA[0] = real(1);
  pB[0] = real(1);
#pragma unroll
  for (int k = 1; k <= P; k++) {
    pA[k] = pA[k - 1] * a;
    pB[k] = pB[k - 1] * b;
  }
#pragma unroll
  for (int m = -P; m <= P; m++) {
    const int am = m < 0 ? -m : m;
    real in[P + 1];
#pragma unroll
    for (int k = am; k <= P; k++) in[k] = v[ix(k, m)] * pB[k];
#pragma unroll
    for (int n = P; n >= am; n--) {
      real acc = real(0);
#pragma unroll
      for (int k = am; k <= n; k++) acc = fmar(c_ax_m2m[ax_id(n, k, am)] * pA[n - k], in[k], acc);
      v[ix(n, m)] = acc;
    }
  }
}

// Axial L2L (App. B.3), a = r/rho_parent, b = rho_child/rho_parent.
template <int P>
__device__ __forceinline__ void axial_l2l(real (&v)[ncoef(P)], real a, real b) {
  real pA[P + 1], pB[P + 1];
  pA[0] = real(1);
  pB[0] = real(1);
#pragma unroll
  for (int k = 1; k <= P; k++) {
    pA[k] = pA[k - 1] * a;
    pB[k] = pB[k - 1] * b;
  }
#pragma unroll
  for (int m = -P; m <= P; m++) {
    const int am = m < 0 ? -m : m;
    real in[P + 1];
#pragma unroll
    for (int k = am; k <= P; k++) in[k] = v[ix(k, m)];
#pragma unroll
    for (int n = am; n <= P; n++) {
      real acc = real(0);
#pragma unroll
      for (int k = n; k <= P; k++) acc = fmar(c_ax_l2l[ax_id(n, k, am)] * pA[k - n], in[k], acc);
      v[ix(n, m)] = acc * pB[n];
    }
  }
}

// Normalised regular basis Rt(y) up to degree P (recursions in tables.cu),
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
    const real cd = c_rdiag[n];
    R[ix(n, n)] = cd * fmar(x, R[ix(n - 1, n - 1)], y * R[ix(n - 1, 1 - n)]);
    R[ix(n, -n)] = cd * fmar(x, R[ix(n - 1, 1 - n)], -y * R[ix(n - 1, n - 1)]);
    const real zs = c_rsub[n - 1] * z;
    R[ix(n, n - 1)] = zs * R[ix(n - 1, n - 1)];
    R[ix(n, 1 - n)] = zs * R[ix(n - 1, 1 - n)];
#pragma unroll
    for (int m = 2 - n; m <= n - 2; m++) {
      const int am = m < 0 ? -m : m;
      R[ix(n, m)] = fmar(c_ra[n * (kMaxP + 1) + am] * z, R[ix(n - 1, m)],
                         -(c_rb[n * (kMaxP + 1) + am] * r2) * R[ix(n - 2, m)]);
    }
    consume(nn);
  });
}

}  // namespace
}  // namespace fmm
