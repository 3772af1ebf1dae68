// Evaluation kernels of the FMM (stages of Sec. III.A: sort, P2M, M2M, M2L,
// L2L, L2P, P2P, inverse sort), compiled once per precision.  The including
// translation unit defines `real`, FMM_EVAL_FN and FMM_INIT_FN.
#pragma once

#include <cuda_runtime.h>

#include "common.cuh"
#include "expansion.cuh"
#include "dfloat.cuh"

namespace fmm {
namespace {

constexpr bool kF32 = std::is_same<real, float>::value;
using vec4 = typename std::conditional<kF32, float4, dvec4>::type;
constexpr double kInv4Pi = 0.079577471545947667884441881686257181;

// ---- small helpers ----------------------------------------------------------
__device__ __forceinline__ int lane_id() { return threadIdx.x & 31; }

// Knuth's two-sum: s + e == a + b exactly.
template <class T>
__device__ __forceinline__ void two_sum(T& s, T& e, T b) {
  T a = s;
  T t = a + b;
  T bb = t - a;
  T err = (a - (t - bb)) + (b - bb);
  s = t;
  e += err;
}

__device__ __forceinline__ const real* m2l_row(const real* base, int64_t stride, int f) {
  return base + (int64_t)f * stride;
}

template <int P>
__device__ __forceinline__ void load_trig(const real* geo, int64_t stride, int64_t e, int f0,
                                          real (&cp)[P], real (&sp)[P], real (&ct)[P], real (&st)[P]) {
#pragma unroll
  for (int m = 0; m < P; m++) {
    cp[m] = geo[(int64_t)(f0 + m) * stride + e];
    sp[m] = geo[(int64_t)(f0 + P + m) * stride + e];
    ct[m] = geo[(int64_t)(f0 + 2 * P + m) * stride + e];
    st[m] = geo[(int64_t)(f0 + 3 * P + m) * stride + e];
  }
}

// One expansion row (16-byte aligned, padded to ncoef_pad) in vector loads.
template <int P>
__device__ __forceinline__ void load_coef(const real* src, real (&v)[ncoef(P)]) {
  constexpr int NC = ncoef(P);
  if constexpr (kF32) {
    const float4* s4 = reinterpret_cast<const float4*>(src);
#pragma unroll
    for (int c = 0; c < (NC + 3) / 4; c++) {
      const float4 x = __ldg(s4 + c);
      v[4 * c] = x.x;
      if (4 * c + 1 < NC) v[4 * c + 1] = x.y;
      if (4 * c + 2 < NC) v[4 * c + 2] = x.z;
      if (4 * c + 3 < NC) v[4 * c + 3] = x.w;
    }
  } else {
    const double2* s2 = reinterpret_cast<const double2*>(src);
#pragma unroll
    for (int c = 0; c < (NC + 1) / 2; c++) {
      const double2 x = __ldg(s2 + c);
      v[2 * c] = x.x;
      if (2 * c + 1 < NC) v[2 * c + 1] = x.y;
    }
  }
}

// ---- E0: sort charges into tree order ----------------------------------------
// Points at or after n_charges (targets of a separate target tree) get q = 0.
// dup: FP32 near-field records (FP32C); df: charges of the double-float
// records (FP64DF), whose coordinates are set at build.
// It also clears the evaluation's work counters (8) and the n_ready
// readiness flags of the one-launch M2M (the kernels that use them run after
// it on the same stream).
__global__ void gather_kernel(int64_t n, int64_t n_charges, const int32_t* __restrict__ perm,
                              const double* __restrict__ q, const vec4* __restrict__ pos,
                              vec4* __restrict__ src, DupRec* __restrict__ dup, DFRec* __restrict__ df,
                              int* __restrict__ counters, int* __restrict__ ready, int64_t n_ready) {
  const int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (counters && tid < 8) counters[tid] = 0;
  if (ready)
    for (int64_t b = tid; b < n_ready; b += (int64_t)gridDim.x * blockDim.x) ready[b] = 0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    vec4 p = pos[i];
    const double qi = i < n_charges ? q[perm[i]] : 0.0;
    p.w = (real)qi;
    src[i] = p;
    if (dup) {
      const float x = (float)p.x, y = (float)p.y, z = (float)p.z, w = (float)p.w;
      dup[i] = DupRec{x, x, y, y, z, z, w, w};
    }
    if (df) {
      const float qh = (float)qi;
      df[i].qh = qh;
      df[i].ql = (float)(qi - (double)qh);
    }
  }
}

// ---- E1: P2M, a group of kP2MGroup lanes per leaf ---------------------------
// M^m_n = sum_i q_i Rt^m_n((x_i - c) / rho)   (Sec. II.C in the scaled basis)
// Lane j of a group accumulates the points j, j + G, ... of its leaf; the
// group's sums are combined by an xor butterfly (log2 G shuffle stages per
// coefficient, against 5 for a whole warp) and lane j stores coefficients
// c = j (mod G).
constexpr int kP2MGroup = 4;

template <int P>
__global__ void __launch_bounds__(128) p2m_kernel(int64_t n_leaves, const int32_t* __restrict__ leaf_box,
                                                  const int64_t* __restrict__ box_start,
                                                  const int32_t* __restrict__ box_count,
                                                  const double* __restrict__ center,
                                                  const vec4* __restrict__ src,
                                                  const real* __restrict__ inv_rho,
                                                  real* __restrict__ M) {
  constexpr int G = kP2MGroup;
  constexpr int NC = ncoef(P);
  const int64_t leaf = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) / G;
  if (leaf >= n_leaves) return;  // whole groups leave together
  const int j = threadIdx.x % G;
  const unsigned gmask = ((1u << G) - 1u) << ((threadIdx.x & 31) & ~(G - 1));
  const int64_t g = leaf_box[leaf];
  const int64_t start = box_start[g];
  const int cnt = box_count[g];
  const real ir = inv_rho[g];
  real cx = 0, cy = 0, cz = 0;
  if (!kF32) {
    cx = (real)center[3 * g];
    cy = (real)center[3 * g + 1];
    cz = (real)center[3 * g + 2];
  }
  real acc[NC];
#pragma unroll
  for (int c = 0; c < NC; c++) acc[c] = real(0);
  for (int i = j; i < cnt; i += G) {
    const vec4 s = src[start + i];
    const real x = ((real)s.x - cx) * ir, y = ((real)s.y - cy) * ir, z = ((real)s.z - cz) * ir;
    const real q = (real)s.w;
    real R[NC];
    regular_basis<P>(x, y, z, R, [&](auto nn) {
      constexpr int n = decltype(nn)::value;
#pragma unroll
      for (int c = n * n; c < (n + 1) * (n + 1); c++) acc[c] = fmar(q, R[c], acc[c]);
    });
  }
#pragma unroll
  for (int c = 0; c < NC; c++) {
    real v = acc[c];
#pragma unroll
    for (int o = 1; o < G; o <<= 1) v += __shfl_xor_sync(gmask, v, o);
    acc[c] = v;
  }
  real* out = M + g * ncoef_pad(P);
#pragma unroll
  for (int c = 0; c < NC; c++)
    if (c % G == j) out[c] = acc[c];
}

// ---- E2: M2M, one thread per child box of level l+1 -------------------------
template <int P>
__global__ void __launch_bounds__(128) m2m_kernel(int64_t n_child, const int32_t* __restrict__ child,
                                                  const int32_t* __restrict__ parent, int nch,
                                                  const real* __restrict__ edge,
                                                  int64_t edge_stride, real* __restrict__ M) {
  constexpr int NC = ncoef(P);
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const bool active = t < n_child;
  real v[NC];
  int64_t g = 0;
  if (active) {
    g = child[t];
    load_coef<P>(M + g * ncoef_pad(P), v);
    const real a = edge[0 * edge_stride + g], b = edge[1 * edge_stride + g];
    real cp[P], sp[P], ct[P], st[P];
    load_trig<P>(edge, edge_stride, g, 2, cp, sp, ct, st);
    translate_rotated<P>(v, cp, sp, ct, st, [&](real (&w)[ncoef(P)]) { axial_m2m<P>(w, a, b); });
  } else {
#pragma unroll
    for (int c = 0; c < NC; c++) v[c] = real(0);
  }
  // sum the 2^s children (consecutive lanes) of each parent
#pragma unroll
  for (int c = 0; c < NC; c++) {
    real x = v[c];
    for (int o = 1; o < nch; o <<= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    v[c] = x;
  }
  if (active && (t % nch) == 0) {
    real* out = M + (int64_t)parent[g] * ncoef_pad(P);
#pragma unroll
    for (int c = 0; c < NC; c++) out[c] = v[c];
  }
}

// ---- E2 in one launch: the M2M rounds of every tree of a batch ---------------
// The work list is the rounds' child boxes concatenated (round r: the boxes r
// levels above each tree's leaves; the 2^s children of a parent consecutive,
// rounds and parent groups aligned to multiples of 2^s).  Warps take chunks
// of 32 items in list order; a child that is not a leaf (round >= 1) is
// used once its own M2M sum is written: the warp that wrote it set
// ready[child] after a memory fence, and the reader waits for the flag (a
// bounded wait: on timeout ST_TIMEOUT is latched and the evaluation is
// incomplete).  Chunks are taken in order and only wait for earlier items,
// which running warps hold, so the waits always end.  Each child's
// translation and the sum over the 2^s children are the round kernel's, so
// the result is the same bit for bit.
constexpr int kMaxRounds = 40;
struct RoundTab {
  int64_t pad[kMaxRounds + 1];  // round r occupies chunk slots pad[r] .. pad[r + 1] - 1 (multiples of 32)
  int64_t off[kMaxRounds + 1];  // and items off[r] .. off[r + 1] - 1 of the work list
  int n;
};
template <int P>
__global__ void __launch_bounds__(128) m2m_persistent_kernel(RoundTab rt, const int32_t* __restrict__ child,
                                                             const int32_t* __restrict__ parent, int nch,
                                                             const real* __restrict__ edge, int64_t edge_stride,
                                                             real* M, int* ready, int* __restrict__ counter,
                                                             int* __restrict__ status, long long wait_cycles) {
  constexpr int NC = ncoef(P);
  const int lane = lane_id();
  for (;;) {
    int64_t base = 0;
    if (lane == 0) base = atomicAdd(counter, 32);
    base = __shfl_sync(0xffffffffu, base, 0);
    if (base >= rt.pad[rt.n]) break;
    // each round starts on a chunk boundary, so a chunk holds one round
    int r = 0;
    while (rt.pad[r + 1] <= base) r++;
    const int64_t k = base - rt.pad[r] + lane;
    const bool active = k < rt.off[r + 1] - rt.off[r];
    const int64_t t = rt.off[r] + k;
    real v[NC];
    int64_t g = 0;
    if (active) {
      g = child[t];
      if (r > 0) {
        // the child's own sum (written in the previous round) must be complete
        const long long t0 = clock64();
        while (atomicAdd(&ready[g], 0) == 0) {
          if (clock64() - t0 >= wait_cycles) {
            atomicOr(status, ST_TIMEOUT);
            break;
          }
          __nanosleep(100);  // leave the issue slots to the stages running beside
        }
        __threadfence();
      }
      const real* row = M + g * ncoef_pad(P);
#pragma unroll
      for (int c = 0; c < NC; c++) v[c] = __ldcg(row + c);
      const real a = edge[0 * edge_stride + g], b = edge[1 * edge_stride + g];
      real cp[P], sp[P], ct[P], st[P];
      load_trig<P>(edge, edge_stride, g, 2, cp, sp, ct, st);
      translate_rotated<P>(v, cp, sp, ct, st, [&](real (&w)[ncoef(P)]) { axial_m2m<P>(w, a, b); });
    } else {
#pragma unroll
      for (int c = 0; c < NC; c++) v[c] = real(0);
    }
#pragma unroll
    for (int c = 0; c < NC; c++) {
      real x = v[c];
      for (int o = 1; o < nch; o <<= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
      v[c] = x;
    }
    if (active && (k % nch) == 0) {
      const int64_t pg = parent[g];
      real* out = M + pg * ncoef_pad(P);
#pragma unroll
      for (int c = 0; c < NC; c++) __stcg(out + c, v[c]);
      __threadfence();
      atomicExch(&ready[pg], 1);
    }
  }
}

// ---- E3: M2L, persistent; one warp per target box, lanes over its list ------
// Each lane accumulates its interactions in a shared-memory row of m2l_chunks
// 16-byte chunks (4 FP32 or 2 FP64 values; an odd count, so the 8 lanes of a
// quarter-warp hit distinct banks); the warp then sums the 32 rows per
// coefficient in lane order.
template <int P>
constexpr int m2l_chunks() {
  constexpr int per = 16 / (int)sizeof(real);
  return ((ncoef(P) + per - 1) / per) | 1;
}

// row += v (ADD) or row = v, in 16-byte chunks
template <int P, bool ADD = true>
__device__ __forceinline__ void m2l_acc_add(real* row, const real (&v)[ncoef(P)]) {
  constexpr int NC = ncoef(P);
  sfor<0, m2l_chunks<P>()>([&](auto kk) {
    constexpr int k = decltype(kk)::value;
    if constexpr (kF32) {
      constexpr int i = 4 * k;
      if constexpr (i < NC) {
        float4* p4 = reinterpret_cast<float4*>(row) + k;
        float4 a = ADD ? *p4 : make_float4(0.f, 0.f, 0.f, 0.f);
        a.x += v[i];
        if constexpr (i + 1 < NC) a.y += v[i + 1];
        if constexpr (i + 2 < NC) a.z += v[i + 2];
        if constexpr (i + 3 < NC) a.w += v[i + 3];
        *p4 = a;
      }
    } else {
      constexpr int i = 2 * k;
      if constexpr (i < NC) {
        double2* p2 = reinterpret_cast<double2*>(row) + k;
        double2 a = ADD ? *p2 : make_double2(0.0, 0.0);
        a.x += v[i];
        if constexpr (i + 1 < NC) a.y += v[i + 1];
        *p2 = a;
      }
    }
  });
}

template <int P>
__global__ void __launch_bounds__(128) m2l_kernel(int64_t n_items, const M2LItem* __restrict__ items,
                                                  const int32_t* __restrict__ src,
                                                  const real* __restrict__ geo, int64_t n_m2l,
                                                  const real* __restrict__ M,
                                                  real* __restrict__ Lam, real* __restrict__ partial,
                                                  int* __restrict__ counter) {
  constexpr int NC = ncoef(P);
  constexpr int NCP = ncoef_pad(P);
  constexpr int ROW = m2l_chunks<P>() * (16 / (int)sizeof(real));  // reals per lane row
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int lane = lane_id();
  const int warp = threadIdx.x >> 5;
  real* rows = reinterpret_cast<real*>(smem_raw) + (size_t)warp * 32 * ROW;
  real* mine = rows + lane * ROW;
  for (;;) {
    int t = 0;
    if (lane == 0) t = atomicAdd(counter, 1);
    t = __shfl_sync(0xffffffffu, t, 0);
    if (t >= n_items) break;
    const M2LItem it = items[t];
    const int64_t g = it.g;
    const int64_t b = it.b, e = it.e;
#pragma unroll
    for (int c = 0; c < ROW; c++) mine[c] = real(0);
    for (int64_t i = b + lane; i < e; i += 32) {
      const int64_t s = src[i];
      real v[NC];
      load_coef<P>(M + s * NCP, v);
      const real rinv = geo[i], uS = geo[n_m2l + i], uT = geo[2 * n_m2l + i];
      real cp[P], sp[P], ct[P], st[P];
      trig_multiples<P>(geo[3 * n_m2l + i], geo[4 * n_m2l + i], cp, sp);
      trig_multiples<P>(geo[5 * n_m2l + i], geo[6 * n_m2l + i], ct, st);
      translate_rotated<P>(v, cp, sp, ct, st, [&](real (&w)[ncoef(P)]) { axial_m2l<P>(w, uS, uT, rinv); });
      m2l_acc_add<P>(mine, v);
    }
    __syncwarp();
    real* out = it.prow < 0 ? Lam + g * NCP : partial + (int64_t)it.prow * NCP;
    for (int c = lane; c < NCP; c += 32) {
      real s = real(0);
      if (c < NC) {
        // the 32 lane rows summed as a balanced tree (rounding error grows
        // with log2 32 = 5 levels, not with 32 terms), in a fixed order
        real x[32];
#pragma unroll
        for (int j = 0; j < 32; j++) x[j] = rows[j * ROW + c];
#pragma unroll
        for (int w = 16; w >= 1; w >>= 1)
#pragma unroll
          for (int j = 0; j < w; j++) x[j] += x[j + w];
        s = x[0];
      }
      out[c] = s;
    }
    __syncwarp();
  }
}

// ---- E3 (FP64DF): M2L in double-float arithmetic -----------------------------
// The FP64-accurate path's M2L on the FP32 pipes: as m2l_kernel, with the
// source multipoles, the rotation records and all arithmetic as double-float
// values (about 48 significant bits; FP64 runs at 1/64 of the FP32 rate on
// GB300).  Each lane keeps its sums in a shared-memory row of float pairs (an
// odd row length: conflict-free 8-byte accesses); the warp adds the 32 rows
// per coefficient in lane order and writes the FP64 locals.
template <int P>
__global__ void __launch_bounds__(128) m2l_kernel_df(int64_t n_items, const M2LItem* __restrict__ items,
                                                     const int32_t* __restrict__ src,
                                                     const float* __restrict__ geo_h,
                                                     const float* __restrict__ geo_l, int64_t n_m2l,
                                                     const float2* __restrict__ Mdf, double* __restrict__ Lam,
                                                     double* __restrict__ partial, int* __restrict__ counter) {
  constexpr int NC = ncoef(P);
  constexpr int NCP = ncoef_pad(P);
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int lane = lane_id();
  const int warp = threadIdx.x >> 5;
  float2* rows = reinterpret_cast<float2*>(smem_raw) + (size_t)warp * 32 * NC;
  float2* mine = rows + lane * NC;
  auto geo = [&](int f, int64_t i) { return dff(geo_h[(int64_t)f * n_m2l + i], geo_l[(int64_t)f * n_m2l + i]); };
  for (;;) {
    int t = 0;
    if (lane == 0) t = atomicAdd(counter, 1);
    t = __shfl_sync(0xffffffffu, t, 0);
    if (t >= n_items) break;
    const M2LItem it = items[t];
    const int64_t g = it.g;
    const int64_t b = it.b, e = it.e;
    for (int c = 0; c < NC; c++) mine[c] = make_float2(0.f, 0.f);
    for (int64_t i = b + lane; i < e; i += 32) {
      const float2* ms = Mdf + (int64_t)src[i] * NCP;
      dff v[NC];
#pragma unroll
      for (int c = 0; c < NC; c++) {
        const float2 x = ms[c];
        v[c] = dff(x.x, x.y);
      }
      const dff rinv = geo(0, i), uS = geo(1, i), uT = geo(2, i);
      dff cp[P], sp[P], ct[P], st[P];
      trig_multiples<P>(geo(3, i), geo(4, i), cp, sp);
      trig_multiples<P>(geo(5, i), geo(6, i), ct, st);
      translate_rotated<P>(v, cp, sp, ct, st, [&](dff (&w)[NC]) { axial_m2l<P>(w, uS, uT, rinv); });
#pragma unroll
      for (int c = 0; c < NC; c++) {
        const float2 a = mine[c];
        const dff s = dff(a.x, a.y) + v[c];
        mine[c] = make_float2(s.h, s.l);
      }
    }
    __syncwarp();
    double* out = it.prow < 0 ? Lam + g * NCP : partial + (int64_t)it.prow * NCP;
    for (int c = lane; c < NCP; c += 32) {
      dff s(0.f, 0.f);
      if (c < NC) {
        for (int j = 0; j < 32; j++) {
          const float2 a = rows[j * NC + c];
          s = s + dff(a.x, a.y);
        }
      }
      out[c] = to_double(s);
    }
    __syncwarp();
  }
}

// Locals of the targets whose M2L list was split into several work items:
// the items' partial rows added in item order (compensated in FP32).  One
// warp per target, lanes over coefficients.
template <class T>
__global__ void m2l_combine_kernel(int64_t n_split, const int32_t* __restrict__ split_g,
                                   const int64_t* __restrict__ split_row, int ncp, const T* __restrict__ partial,
                                   T* __restrict__ Lam) {
  const int64_t warps = (int64_t)gridDim.x * blockDim.x / 32;
  for (int64_t k = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) / 32; k < n_split; k += warps) {
    const int64_t g = split_g[k];
    for (int c = threadIdx.x & 31; c < ncp; c += 32) {
      T s = T(0), err = T(0);
      for (int64_t r = split_row[k]; r < split_row[k + 1]; r++) {
        if (std::is_same<T, float>::value) two_sum(s, err, partial[r * ncp + c]);
        else s += partial[r * ncp + c];
      }
      Lam[g * ncp + c] = s + err;
    }
  }
}

// FP64 values as double-float pairs (the multipoles before the M2L above)
__global__ void to_dff_kernel(int64_t n, const double* __restrict__ x, float2* __restrict__ y) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const dff d(x[i]);
    y[i] = make_float2(d.h, d.l);
  }
}

// ---- E4: L2L in direct form, a group of kL2LGroup lanes per target leaf ----
// The local expansion of a leaf is the chain of Sec. II.C: its own M2L sum
// plus L2L of its parent's complete local.  Unrolled, that is the leaf's M2L
// sum plus, over every ancestor a, L2L(a -> leaf) of a's own M2L sum: a local
// expansion of degree p is a polynomial of degree p, which a translation maps
// exactly onto the same degrees, so translations compose without truncation
// and the two forms differ by rounding only.  The direct form needs one
// launch instead of one round per level; only ancestors with a non-empty M2L
// list have records.  Lanes of a group translate the leaf's records in turn
// into shared-memory rows (as M2L), then lane j adds the group's rows, in lane
// order, to coefficients c = j (mod the group size) of the leaf's own M2L
// sum.  Internal boxes keep their M2L sums.
constexpr int kL2LGroup = 8;

template <int P>
__global__ void __launch_bounds__(128) l2l_direct_kernel(int64_t n_leaves, const int32_t* __restrict__ leaf_box,
                                                         const int64_t* __restrict__ off,
                                                         const int32_t* __restrict__ anc,
                                                         const real* __restrict__ edge, int64_t n_rec,
                                                         real* __restrict__ Lam) {
  constexpr int G = kL2LGroup;
  constexpr int NC = ncoef(P);
  constexpr int NCP = ncoef_pad(P);
  constexpr int ROW = m2l_chunks<P>() * (16 / (int)sizeof(real));
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int64_t leaf = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) / G;
  if (leaf >= n_leaves) return;  // whole groups leave together
  const int j = threadIdx.x % G;
  const unsigned gmask = ((1u << G) - 1u) << ((threadIdx.x & 31) & ~(G - 1));
  real* rows = reinterpret_cast<real*>(smem_raw) + (size_t)(threadIdx.x - j) * ROW;
  const int64_t b = off[leaf], e = off[leaf + 1];
  real* out = Lam + (int64_t)leaf_box[leaf] * NCP;
  for (int64_t r0 = b; r0 < e; r0 += G) {
    const int64_t i = r0 + j;
    if (i < e) {
      real v[NC];
      load_coef<P>(Lam + (int64_t)anc[i] * NCP, v);
      const real a = edge[i], bb = edge[n_rec + i];
      real cp[P], sp[P], ct[P], st[P];
      load_trig<P>(edge, n_rec, i, 2, cp, sp, ct, st);
      translate_rotated<P>(v, cp, sp, ct, st, [&](real (&w)[ncoef(P)]) { axial_l2l<P>(w, a, bb); });
      m2l_acc_add<P, false>(rows + j * ROW, v);
    }
    __syncwarp(gmask);
    const int nv = (int)((e - r0) < G ? (e - r0) : G);
    for (int c = j; c < NC; c += G) {
      real x = out[c];
      for (int q = 0; q < nv; q++) x += rows[q * ROW + c];
      out[c] = x;
    }
    __syncwarp(gmask);
  }
}

// ---- E6: P2P, persistent; one warp per target leaf ---------------------------
// Source leaves are staged in shared memory by 1D TMA bulk copies
// (cp.async.bulk) completing on per-warp mbarriers, double buffered.
__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t* bar) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(bar)) : "memory");
}
__device__ __forceinline__ void fence_barrier_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void fence_proxy_async() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
// cp.async.bulk of `bytes` completing on `bar` (the expected transaction
// count is registered by the caller)
__device__ __forceinline__ void bulk_copy(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_addr(dst)),
      "l"(src), "r"(bytes), "r"(smem_addr(bar))
      : "memory");
}

__device__ __forceinline__ void tma_load_1d(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
               : "memory");
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_addr(dst)),
      "l"(src), "r"(bytes), "r"(smem_addr(bar))
      : "memory");
}
// Waits for phase `parity` of the barrier; gives up and returns false once
// `limit` clock cycles have passed (limit 0: gives up before the first
// poll, which is how the timeout path is exercised without a fault).
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, long long limit) {
  const long long t0 = clock64();
  for (;;) {
    if (clock64() - t0 >= limit) return false;
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
        : "=r"(done)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    if (done) return true;
  }
}

// 1/sqrt(r2) in FP64: the hardware's FP64 reciprocal square root
// approximation (rsqrt.approx.f64; no conversions to and from FP32) with one
// third-order correction y (1 + rho / 2 + 3 rho^2 / 8), rho = 1 - r2 y^2, the
// first terms of (1 - rho)^(-1/2).  A seed error e leaves about 2.5 e^3 (e
// near 4.5e-7, inferred from a one-step Newton refinement: 2e-19, below FP64
// rounding).  r2 <= 0 (a point paired with itself, or a phantom target on a
// source) gives 0.
__device__ __forceinline__ double rsqrt_f64(double r2) {
  double y;
  asm("rsqrt.approx.ftz.f64 %0, %1;" : "=d"(y) : "d"(r2));
  const double rho = fma(-(r2 * y), y, 1.0);
  y = fma(y * rho, fma(0.375, rho, 0.5), y);
  return r2 > 0.0 ? y : 0.0;
}

template <bool MASK, bool FIELD, int TPL>
__device__ __forceinline__ void p2p_tile(const vec4* sb, int scount, const real (&tx)[TPL],
                                         const real (&ty)[TPL], const real (&tz)[TPL],
                                         real (&pu)[TPL], real (&fx)[TPL], real (&fy)[TPL],
                                         real (&fz)[TPL]) {
#pragma unroll 2
  for (int j = 0; j < scount; j++) {
    const vec4 s = sb[j];
#pragma unroll
    for (int k = 0; k < TPL; k++) {
      const real dx = tx[k] - (real)s.x, dy = ty[k] - (real)s.y, dz = tz[k] - (real)s.z;
      const real r2 = fmar(dz, dz, fmar(dy, dy, dx * dx));
      real ri;
      if (kF32) {
        ri = rsqrtf((float)r2);
      } else {
        ri = (real)rsqrt_f64((double)r2);
      }
      if (MASK) ri = (r2 > real(0)) ? ri : real(0);
      pu[k] = fmar((real)s.w, ri, pu[k]);
      if (FIELD) {
        const real w = (real)s.w * ri * ri * ri;
        fx[k] = fmar(w, dx, fx[k]);
        fy[k] = fmar(w, dy, fy[k]);
        fz[k] = fmar(w, dz, fz[k]);
      }
    }
  }
}

// Packed FP32 pairs (f32x2 arithmetic of sm_100-family GPUs): a 64-bit
// register holds two FP32 lanes, one instruction updates both.
typedef unsigned long long f2;
__device__ __forceinline__ f2 f2pack(float a, float b) {
  f2 r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
  return r;
}
__device__ __forceinline__ void f2unpack(f2 v, float& a, float& b) {
  asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(v));
}
__device__ __forceinline__ f2 f2add(f2 a, f2 b) {
  f2 r;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
  return r;
}
__device__ __forceinline__ f2 f2sub(f2 a, f2 b) {
  f2 r;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
  return r;
}
__device__ __forceinline__ f2 f2mul(f2 a, f2 b) {
  f2 r;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
  return r;
}
__device__ __forceinline__ f2 f2fma(f2 a, f2 b, f2 c) {
  f2 r;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(a), "l"(b), "l"(c));
  return r;
}
// MUFU reciprocal square root (denormal inputs flush to zero)
__device__ __forceinline__ float rsqrt_mufu(float x) {
  float y;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// FP32 near-field tile: sources staged as (x, x, y, y, z, z, q, q) so that
// each 128-bit shared load yields two packed operands; every lane updates its
// NP packed target pairs.
template <bool MASK, bool FIELD, int NP>
__device__ __forceinline__ void p2p_tile_f32(const DupRec* sb, int scount, const f2 (&tx)[NP], const f2 (&ty)[NP],
                                             const f2 (&tz)[NP], f2 (&pu)[NP], f2 (&fx)[NP], f2 (&fy)[NP],
                                             f2 (&fz)[NP], float thr) {
  const ulonglong2* s2 = reinterpret_cast<const ulonglong2*>(sb);
#pragma unroll 4
  for (int j = 0; j < scount; j++) {
    const ulonglong2 a = s2[2 * j];
    const ulonglong2 b = s2[2 * j + 1];
#pragma unroll
    for (int k = 0; k < NP; k++) {
      const f2 dx = f2sub(tx[k], a.x), dy = f2sub(ty[k], a.y), dz = f2sub(tz[k], b.x);
      const f2 r2 = f2fma(dz, dz, f2fma(dy, dy, f2mul(dx, dx)));
      float r0, r1;
      f2unpack(r2, r0, r1);
      float i0 = rsqrt_mufu(r0), i1 = rsqrt_mufu(r1);
      if (MASK) {
        i0 = (r0 > thr) ? i0 : 0.f;
        i1 = (r1 > thr) ? i1 : 0.f;
      }
      const f2 ri = f2pack(i0, i1);
      pu[k] = f2fma(b.y, ri, pu[k]);
      if (FIELD) {
        const f2 w = f2mul(f2mul(f2mul(ri, ri), ri), b.y);
        fx[k] = f2fma(w, dx, fx[k]);
        fy[k] = f2fma(w, dy, fy[k]);
        fz[k] = f2fma(w, dz, fz[k]);
      }
    }
  }
}

// FP32 near-field tile, half-warp split: lanes 0-15 take the even and lanes
// 16-31 the odd sources of the staged tile, each lane updating NPH packed
// target pairs (two independent accumulation chains per source for NPH = 2).
template <bool MASK, bool FIELD, int NPH>
__device__ __forceinline__ void p2p_pair_f32(const ulonglong2 a, const ulonglong2 b, const f2 (&tx)[NPH],
                                             const f2 (&ty)[NPH], const f2 (&tz)[NPH], f2 (&pu)[NPH],
                                             f2 (&fx)[NPH], f2 (&fy)[NPH], f2 (&fz)[NPH], float thr) {
#pragma unroll
  for (int k = 0; k < NPH; k++) {
    const f2 dx = f2sub(tx[k], a.x), dy = f2sub(ty[k], a.y), dz = f2sub(tz[k], b.x);
    const f2 r2 = f2fma(dz, dz, f2fma(dy, dy, f2mul(dx, dx)));
    float r0, r1;
    f2unpack(r2, r0, r1);
    float i0 = rsqrt_mufu(r0), i1 = rsqrt_mufu(r1);
    if (MASK) {
      i0 = (r0 > thr) ? i0 : 0.f;
      i1 = (r1 > thr) ? i1 : 0.f;
    }
    const f2 ri = f2pack(i0, i1);
    pu[k] = f2fma(b.y, ri, pu[k]);
    if (FIELD) {
      const f2 w = f2mul(f2mul(f2mul(ri, ri), ri), b.y);
      fx[k] = f2fma(w, dx, fx[k]);
      fy[k] = f2fma(w, dy, fy[k]);
      fz[k] = f2fma(w, dz, fz[k]);
    }
  }
}

// FP32 near-field tile, half-warp split: lanes 0-15 take the even and lanes
// 16-31 the odd sources of the staged tile, each lane updating NPH packed
// target pairs.  For the potential with up to two packed pairs, two
// accumulator sets (alternate sources) keep independent chains in flight.
template <bool MASK, bool FIELD, int NPH>
__device__ __forceinline__ void p2p_tile_f32h(const DupRec* sb, int scount, int half, const f2 (&tx)[NPH],
                                              const f2 (&ty)[NPH], const f2 (&tz)[NPH], f2 (&pu)[NPH],
                                              f2 (&fx)[NPH], f2 (&fy)[NPH], f2 (&fz)[NPH], float thr) {
  const ulonglong2* s2 = reinterpret_cast<const ulonglong2*>(sb);
  if constexpr (FIELD || NPH > 2) {
    // one accumulator set (register budget of the field and large tiles)
#pragma unroll 2
    for (int j = half; j < scount; j += 2)
      p2p_pair_f32<MASK, FIELD, NPH>(s2[2 * j], s2[2 * j + 1], tx, ty, tz, pu, fx, fy, fz, thr);
  } else {
    f2 pu2[NPH], fx2[NPH], fy2[NPH], fz2[NPH];
#pragma unroll
    for (int k = 0; k < NPH; k++) pu2[k] = fx2[k] = fy2[k] = fz2[k] = 0ull;
    int j = half;
#pragma unroll 2
    for (; j + 2 < scount; j += 4) {
      const ulonglong2 a0 = s2[2 * j], b0 = s2[2 * j + 1];
      const ulonglong2 a1 = s2[2 * j + 4], b1 = s2[2 * j + 5];
      p2p_pair_f32<MASK, FIELD, NPH>(a0, b0, tx, ty, tz, pu, fx, fy, fz, thr);
      p2p_pair_f32<MASK, FIELD, NPH>(a1, b1, tx, ty, tz, pu2, fx2, fy2, fz2, thr);
    }
    if (j < scount) p2p_pair_f32<MASK, FIELD, NPH>(s2[2 * j], s2[2 * j + 1], tx, ty, tz, pu, fx, fy, fz, thr);
#pragma unroll
    for (int k = 0; k < NPH; k++) {
      pu[k] = f2add(pu[k], pu2[k]);
      if (FIELD) {
        fx[k] = f2add(fx[k], fx2[k]);
        fy[k] = f2add(fy[k], fy2[k]);
        fz[k] = f2add(fz[k], fz2[k]);
      }
    }
  }
}

struct P2PArgs {
  int64_t n_leaves;
  const int32_t* leaf_box;      // global box id of each target leaf
  const int32_t* src_leaf_box;  // global box id of each source leaf
  int self_pairs;               // target leaf l and source leaf l are the same box
  const int32_t* order;
  const int64_t* off;
  const P2PEntry* ent32;
  const float* thr;  // per entry: squared FP32 distance at or below which points coincide
  // symmetric near field (one point set): per-leaf work entries as records
  // and the slots' sums
  const int64_t* work_off;
  const SymRec* rec;
  void* partial;  // float (FP32C) or double (FP64) slot sums
  int stride;
  // FP64DF: double-float point records and per-entry source frames
  const DFRec* df_tile;
  const SymFrame* frame;
  // backward pass: records of the second charge vector, its near sums
  const DupRec* tile_g;
  float* near_u2;
  float* near_f2;
  const int32_t* ent_src;
  const int64_t* box_start;
  const int32_t* box_count;
  const vec4* src;       // targets: (x_local, q) FP32 or (x, q) FP64
  const void* tile;      // sources staged by the bulk copies, 32 bytes per point:
                         // DupRec (FP32) or dvec4 (FP64)
  real* near_u;   // 2 per point (FP32: hi, lo) or 1 (FP64)
  real* near_f;   // 3 per point (FIELD)
  int* counter;
  int* status;
  long long wait_cycles;  // limit of a warp's wait for a staged tile (clock cycles)
};

template <int TPL, bool FIELD>
__global__ void __launch_bounds__(128) p2p_kernel(P2PArgs a) {
  constexpr int CAP = TPL * 32;
  constexpr int WARPS = 4;
  constexpr int NP = TPL >= 2 ? TPL / 2 : 1;  // packed target pairs per lane (FP32)
  using rec = typename std::conditional<kF32, DupRec, dvec4>::type;
  extern __shared__ __align__(128) unsigned char p2p_smem[];
  rec (*sbuf)[2][CAP] = reinterpret_cast<rec (*)[2][CAP]>(p2p_smem);  // [WARPS][2][CAP]
  const rec* tile = reinterpret_cast<const rec*>(a.tile);
  __shared__ __align__(8) uint64_t bars[WARPS][2];
  const int lane = lane_id();
  const int warp = threadIdx.x >> 5;
  uint64_t* bar = bars[warp];
  if (lane == 0) {
    mbar_init(&bar[0]);
    mbar_init(&bar[1]);
    fence_barrier_init();
  }
  __syncwarp();
  uint32_t phase = 0;  // bit b: parity of the next completion of barrier b
  bool ok = true;
  for (;;) {
    int t = 0;
    if (lane == 0) t = atomicAdd(a.counter, 1);
    t = __shfl_sync(0xffffffffu, t, 0);
    if (t >= a.n_leaves || !ok) break;
    const int64_t leaf = a.order[t];
    const int64_t g = a.leaf_box[leaf];
    const int64_t tstart = a.box_start[g];
    const int tcnt = a.box_count[g];
    real tx0[TPL], ty0[TPL], tz0[TPL];
#pragma unroll
    for (int k = 0; k < TPL; k++) {
      const int i = lane + 32 * k;
      if (i < tcnt) {
        const vec4 p = a.src[tstart + i];
        tx0[k] = (real)p.x;
        ty0[k] = (real)p.y;
        tz0[k] = (real)p.z;
      } else {
        tx0[k] = ty0[k] = tz0[k] = real(0);
      }
    }
    real hi[TPL], lo[TPL], fx[TPL], fy[TPL], fz[TPL];
#pragma unroll
    for (int k = 0; k < TPL; k++) hi[k] = lo[k] = fx[k] = fy[k] = fz[k] = real(0);
    const int64_t eb = a.off[leaf], ee = a.off[leaf + 1];
    auto src_leaf = [&](int64_t e) -> int {
      return kF32 ? (a.ent32[e].src & 0x7fffffff) : a.ent_src[e];
    };
    auto issue = [&](int64_t e, int buf) {
      const int64_t gs = a.src_leaf_box[src_leaf(e)];
      if (lane == 0) {
        fence_proxy_async();
        tma_load_1d(sbuf[warp][buf], tile + a.box_start[gs], (uint32_t)(a.box_count[gs] * sizeof(rec)),
                    &bar[buf]);
      }
    };
    if (eb < ee) issue(eb, 0);
    for (int64_t e = eb; e < ee; e++) {
      const int buf = (int)((e - eb) & 1);
      if (e + 1 < ee) issue(e + 1, buf ^ 1);
      const bool got = mbar_wait(&bar[buf], (phase >> buf) & 1u, a.wait_cycles);
      if (!got) {
        if (lane == 0) atomicOr(a.status, ST_TIMEOUT);
        // copies still in flight into this warp's buffers must land first
        mbar_wait(&bar[buf], (phase >> buf) & 1u, kDrainWaitCycles);
        if (e + 1 < ee) mbar_wait(&bar[buf ^ 1], (phase >> (buf ^ 1)) & 1u, kDrainWaitCycles);
        ok = false;
        break;
      }
      phase ^= 1u << buf;
      const int ls = src_leaf(e);
      const int scount = a.box_count[a.src_leaf_box[ls]];
      if constexpr (kF32) {
        const P2PEntry en = a.ent32[e];
        const bool mask = (en.src < 0) || (a.self_pairs && ls == (int)leaf);
        const f2 ddx = f2pack(en.dx, en.dx), ddy = f2pack(en.dy, en.dy), ddz = f2pack(en.dz, en.dz);
        f2 tx[NP], ty[NP], tz[NP], pu[NP], px[NP], py[NP], pz[NP];
#pragma unroll
        for (int k = 0; k < NP; k++) {
          const int k1 = (2 * k + 1 < TPL) ? 2 * k + 1 : 2 * k;
          tx[k] = f2add(f2pack(tx0[2 * k], tx0[k1]), ddx);
          ty[k] = f2add(f2pack(ty0[2 * k], ty0[k1]), ddy);
          tz[k] = f2add(f2pack(tz0[2 * k], tz0[k1]), ddz);
          pu[k] = px[k] = py[k] = pz[k] = 0ull;
        }
        const float thr = mask ? a.thr[e] : 0.f;
        if (mask) p2p_tile_f32<true, FIELD, NP>(sbuf[warp][buf], scount, tx, ty, tz, pu, px, py, pz, thr);
        else p2p_tile_f32<false, FIELD, NP>(sbuf[warp][buf], scount, tx, ty, tz, pu, px, py, pz, thr);
#pragma unroll
        for (int k = 0; k < NP; k++) {
          float u0, u1, x0, x1, y0, y1, z0, z1;
          f2unpack(pu[k], u0, u1);
          f2unpack(px[k], x0, x1);
          f2unpack(py[k], y0, y1);
          f2unpack(pz[k], z0, z1);
          two_sum(hi[2 * k], lo[2 * k], (real)u0);
          fx[2 * k] += (real)x0;
          fy[2 * k] += (real)y0;
          fz[2 * k] += (real)z0;
          if (2 * k + 1 < TPL) {
            two_sum(hi[2 * k + 1], lo[2 * k + 1], (real)u1);
            fx[2 * k + 1] += (real)x1;
            fy[2 * k + 1] += (real)y1;
            fz[2 * k + 1] += (real)z1;
          }
        }
      } else {
        real pu[TPL], px[TPL], py[TPL], pz[TPL];
#pragma unroll
        for (int k = 0; k < TPL; k++) pu[k] = px[k] = py[k] = pz[k] = real(0);
        p2p_tile<true, FIELD, TPL>(reinterpret_cast<const vec4*>(sbuf[warp][buf]), scount, tx0, ty0, tz0, pu, px,
                                   py, pz);
#pragma unroll
        for (int k = 0; k < TPL; k++) {
          hi[k] += pu[k];
          fx[k] += px[k];
          fy[k] += py[k];
          fz[k] += pz[k];
        }
      }
      __syncwarp();
    }
    if (!ok) break;
#pragma unroll
    for (int k = 0; k < TPL; k++) {
      const int i = lane + 32 * k;
      if (i < tcnt) {
        const int64_t pidx = tstart + i;
        if (kF32) {
          a.near_u[2 * pidx] = hi[k];
          a.near_u[2 * pidx + 1] = lo[k];
        } else {
          a.near_u[pidx] = hi[k];
        }
        if (FIELD) {
          a.near_f[3 * pidx] = fx[k];
          a.near_f[3 * pidx + 1] = fy[k];
          a.near_f[3 * pidx + 2] = fz[k];
        }
      }
    }
  }
}


// ---- E6 (FP32): near field, one warp per target leaf, one block of four
// leaves; each lane holds 2*TPL targets i = (lane & 15) + 16 k as TPL packed
// pairs and sums over half of every source tile; the halves are combined by
// a two-sum at the end.  Source leaves arrive by double-buffered 1D TMA bulk
// copies completing on per-warp mbarriers.
template <int TPL, bool FIELD>
__global__ void __launch_bounds__(128, (TPL <= 2 && !FIELD) ? 8 : ((TPL >= 8 || (FIELD && TPL >= 4)) ? 2 : (TPL <= 2 ? 5 : 4)))
    p2p_kernel_f32h(P2PArgs a) {
  constexpr int CAP = TPL * 32;
  constexpr int WARPS = 4;
  constexpr int NT = 2 * TPL;
  constexpr int NPH = TPL;
  extern __shared__ __align__(128) unsigned char p2p_smem[];
  DupRec (*sbuf)[2][CAP] = reinterpret_cast<DupRec (*)[2][CAP]>(p2p_smem);
  __shared__ __align__(8) uint64_t bars[WARPS][2];
  const DupRec* tile = reinterpret_cast<const DupRec*>(a.tile);
  const int lane = lane_id();
  const int warp = threadIdx.x >> 5;
  const int half = lane >> 4, l16 = lane & 15;
  uint64_t* bar = bars[warp];
  if (lane == 0) {
    mbar_init(&bar[0]);
    mbar_init(&bar[1]);
    fence_barrier_init();
  }
  __syncwarp();
  const int64_t t = (int64_t)blockIdx.x * WARPS + warp;
  if (t >= a.n_leaves) return;
  const int64_t leaf = a.order[t];
  const int64_t g = a.leaf_box[leaf];
  const int64_t tstart = a.box_start[g];
  const int tcnt = a.box_count[g];
  float tx0[NT], ty0[NT], tz0[NT];
#pragma unroll
  for (int k = 0; k < NT; k++) {
    const int i = l16 + 16 * k;
    if (i < tcnt) {
      const float4 p = reinterpret_cast<const float4*>(a.src)[tstart + i];
      tx0[k] = p.x;
      ty0[k] = p.y;
      tz0[k] = p.z;
    } else {
      tx0[k] = ty0[k] = tz0[k] = 0.f;
    }
  }
  float hi[NT], lo[NT], fx[NT], fy[NT], fz[NT];
#pragma unroll
  for (int k = 0; k < NT; k++) hi[k] = lo[k] = fx[k] = fy[k] = fz[k] = 0.f;
  const int64_t eb = a.off[leaf], ee = a.off[leaf + 1];
  auto issue = [&](int64_t e, int buf) {
    const int64_t gs = a.src_leaf_box[a.ent32[e].src & 0x7fffffff];
    if (lane == 0) {
      fence_proxy_async();
      tma_load_1d(sbuf[warp][buf], tile + a.box_start[gs], (uint32_t)(a.box_count[gs] * sizeof(DupRec)), &bar[buf]);
    }
  };
  uint32_t phase = 0;
  if (eb < ee) issue(eb, 0);
  for (int64_t e = eb; e < ee; e++) {
    const int buf = (int)((e - eb) & 1);
    if (e + 1 < ee) issue(e + 1, buf ^ 1);
    if (!mbar_wait(&bar[buf], (phase >> buf) & 1u, a.wait_cycles)) {
      if (lane == 0) atomicOr(a.status, ST_TIMEOUT);
      // copies still in flight into this warp's buffers must land first
      mbar_wait(&bar[buf], (phase >> buf) & 1u, kDrainWaitCycles);
      if (e + 1 < ee) mbar_wait(&bar[buf ^ 1], (phase >> (buf ^ 1)) & 1u, kDrainWaitCycles);
      return;
    }
    phase ^= 1u << buf;
    const P2PEntry en = a.ent32[e];
    const int ls = en.src & 0x7fffffff;
    const int scount = a.box_count[a.src_leaf_box[ls]];
    const bool mask = (en.src < 0) || (a.self_pairs && ls == (int)leaf);
    const f2 ddx = f2pack(en.dx, en.dx), ddy = f2pack(en.dy, en.dy), ddz = f2pack(en.dz, en.dz);
    f2 tx[NPH], ty[NPH], tz[NPH], pu[NPH], px[NPH], py[NPH], pz[NPH];
#pragma unroll
    for (int k = 0; k < NPH; k++) {
      tx[k] = f2add(f2pack(tx0[2 * k], tx0[2 * k + 1]), ddx);
      ty[k] = f2add(f2pack(ty0[2 * k], ty0[2 * k + 1]), ddy);
      tz[k] = f2add(f2pack(tz0[2 * k], tz0[2 * k + 1]), ddz);
      pu[k] = px[k] = py[k] = pz[k] = 0ull;
    }
    const float thr = mask ? a.thr[e] : 0.f;
    if (mask) p2p_tile_f32h<true, FIELD, NPH>(sbuf[warp][buf], scount, half, tx, ty, tz, pu, px, py, pz, thr);
    else p2p_tile_f32h<false, FIELD, NPH>(sbuf[warp][buf], scount, half, tx, ty, tz, pu, px, py, pz, thr);
#pragma unroll
    for (int k = 0; k < NPH; k++) {
      float u0, u1, x0, x1, y0, y1, z0, z1;
      f2unpack(pu[k], u0, u1);
      f2unpack(px[k], x0, x1);
      f2unpack(py[k], y0, y1);
      f2unpack(pz[k], z0, z1);
      two_sum(hi[2 * k], lo[2 * k], u0);
      two_sum(hi[2 * k + 1], lo[2 * k + 1], u1);
      fx[2 * k] += x0;
      fx[2 * k + 1] += x1;
      fy[2 * k] += y0;
      fy[2 * k + 1] += y1;
      fz[2 * k] += z0;
      fz[2 * k + 1] += z1;
    }
    __syncwarp();
  }
  // combine the two halves
#pragma unroll
  for (int k = 0; k < NT; k++) {
    const float oh = __shfl_xor_sync(0xffffffffu, hi[k], 16);
    const float ol = __shfl_xor_sync(0xffffffffu, lo[k], 16);
    two_sum(hi[k], lo[k], oh);
    lo[k] += ol;
    if (FIELD) {
      fx[k] += __shfl_xor_sync(0xffffffffu, fx[k], 16);
      fy[k] += __shfl_xor_sync(0xffffffffu, fy[k], 16);
      fz[k] += __shfl_xor_sync(0xffffffffu, fz[k], 16);
    }
  }
  if (half == 0) {
#pragma unroll
    for (int k = 0; k < NT; k++) {
      const int i = l16 + 16 * k;
      if (i < tcnt) {
        const int64_t pidx = tstart + i;
        a.near_u[2 * pidx] = hi[k];
        a.near_u[2 * pidx + 1] = lo[k];
        if (FIELD) {
          a.near_f[3 * pidx] = fx[k];
          a.near_f[3 * pidx + 1] = fy[k];
          a.near_f[3 * pidx + 2] = fz[k];
        }
      }
    }
  }
}

// ---- E6 for the backward pass (FP32C): both charge vectors in one sweep ------
// The backward pass needs the field of the charges q and the potential and
// field of dL/du (g) at every point.  One pass over the near-field list
// shares the distance and 1/r of every pair between the two: per ordered
// pair, field of q (w = q_j / r^3), potential and field of g.  Lane layout and
// staging as in p2p_kernel_f32h, with the q and g records of a source leaf
// copied side by side.
template <bool MASK, int NPH>
__device__ __forceinline__ void bwd_pair(const ulonglong2 a, const ulonglong2 b, const ulonglong2 gb,
                                         const f2 (&tx)[NPH], const f2 (&ty)[NPH], const f2 (&tz)[NPH],
                                         f2 (&fqx)[NPH], f2 (&fqy)[NPH], f2 (&fqz)[NPH], f2 (&ug)[NPH],
                                         f2 (&fgx)[NPH], f2 (&fgy)[NPH], f2 (&fgz)[NPH], float thr) {
#pragma unroll
  for (int k = 0; k < NPH; k++) {
    const f2 dx = f2sub(tx[k], a.x), dy = f2sub(ty[k], a.y), dz = f2sub(tz[k], b.x);
    const f2 r2 = f2fma(dz, dz, f2fma(dy, dy, f2mul(dx, dx)));
    float r0, r1;
    f2unpack(r2, r0, r1);
    float i0 = rsqrt_mufu(r0), i1 = rsqrt_mufu(r1);
    if (MASK) {
      i0 = (r0 > thr) ? i0 : 0.f;
      i1 = (r1 > thr) ? i1 : 0.f;
    }
    const f2 ri = f2pack(i0, i1);
    const f2 ri3 = f2mul(f2mul(ri, ri), ri);
    ug[k] = f2fma(gb.y, ri, ug[k]);
    const f2 wq = f2mul(b.y, ri3), wg = f2mul(gb.y, ri3);
    fqx[k] = f2fma(wq, dx, fqx[k]);
    fqy[k] = f2fma(wq, dy, fqy[k]);
    fqz[k] = f2fma(wq, dz, fqz[k]);
    fgx[k] = f2fma(wg, dx, fgx[k]);
    fgy[k] = f2fma(wg, dy, fgy[k]);
    fgz[k] = f2fma(wg, dz, fgz[k]);
  }
}

template <int TPL>
__global__ void __launch_bounds__(128, TPL <= 2 ? 4 : 2) p2p_kernel_bwd(P2PArgs a) {  // TPL <= 4
  constexpr int CAP = TPL * 32;
  constexpr int WARPS = 4;
  constexpr int NT = 2 * TPL;
  constexpr int NPH = TPL;
  extern __shared__ __align__(128) unsigned char p2p_smem[];
  DupRec (*sbuf)[2][2][CAP] = reinterpret_cast<DupRec (*)[2][2][CAP]>(p2p_smem);  // [warp][buf][q, g]
  __shared__ __align__(8) uint64_t bars[WARPS][2];
  const DupRec* tile = reinterpret_cast<const DupRec*>(a.tile);
  const DupRec* tile_g = a.tile_g;
  const int lane = lane_id();
  const int warp = threadIdx.x >> 5;
  const int half = lane >> 4, l16 = lane & 15;
  uint64_t* bar = bars[warp];
  if (lane == 0) {
    mbar_init(&bar[0]);
    mbar_init(&bar[1]);
    fence_barrier_init();
  }
  __syncwarp();
  const int64_t t = (int64_t)blockIdx.x * WARPS + warp;
  if (t >= a.n_leaves) return;
  const int64_t leaf = a.order[t];
  const int64_t g = a.leaf_box[leaf];
  const int64_t tstart = a.box_start[g];
  const int tcnt = a.box_count[g];
  float tx0[NT], ty0[NT], tz0[NT];
#pragma unroll
  for (int k = 0; k < NT; k++) {
    const int i = l16 + 16 * k;
    if (i < tcnt) {
      const float4 p = reinterpret_cast<const float4*>(a.src)[tstart + i];
      tx0[k] = p.x;
      ty0[k] = p.y;
      tz0[k] = p.z;
    } else {
      tx0[k] = ty0[k] = tz0[k] = 0.f;
    }
  }
  float uh[NT], ul[NT], qx[NT], qy[NT], qz[NT], gx[NT], gy[NT], gz[NT];
#pragma unroll
  for (int k = 0; k < NT; k++) uh[k] = ul[k] = qx[k] = qy[k] = qz[k] = gx[k] = gy[k] = gz[k] = 0.f;
  const int64_t eb = a.off[leaf], ee = a.off[leaf + 1];
  auto issue = [&](int64_t e, int buf) {
    const int64_t gs = a.src_leaf_box[a.ent32[e].src & 0x7fffffff];
    if (lane == 0) {
      const uint32_t bytes = (uint32_t)(a.box_count[gs] * sizeof(DupRec));
      fence_proxy_async();
      asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(&bar[buf])),
                   "r"(2 * bytes)
                   : "memory");
      bulk_copy(sbuf[warp][buf][0], tile + a.box_start[gs], bytes, &bar[buf]);
      bulk_copy(sbuf[warp][buf][1], tile_g + a.box_start[gs], bytes, &bar[buf]);
    }
  };
  uint32_t phase = 0;
  if (eb < ee) issue(eb, 0);
  for (int64_t e = eb; e < ee; e++) {
    const int buf = (int)((e - eb) & 1);
    if (e + 1 < ee) issue(e + 1, buf ^ 1);
    if (!mbar_wait(&bar[buf], (phase >> buf) & 1u, a.wait_cycles)) {
      if (lane == 0) atomicOr(a.status, ST_TIMEOUT);
      // copies still in flight into this warp's buffers must land first
      mbar_wait(&bar[buf], (phase >> buf) & 1u, kDrainWaitCycles);
      if (e + 1 < ee) mbar_wait(&bar[buf ^ 1], (phase >> (buf ^ 1)) & 1u, kDrainWaitCycles);
      return;
    }
    phase ^= 1u << buf;
    const P2PEntry en = a.ent32[e];
    const int ls = en.src & 0x7fffffff;
    const int scount = a.box_count[a.src_leaf_box[ls]];
    const bool mask = (en.src < 0) || ls == (int)leaf;
    const float thr = mask ? a.thr[e] : 0.f;
    const f2 ddx = f2pack(en.dx, en.dx), ddy = f2pack(en.dy, en.dy), ddz = f2pack(en.dz, en.dz);
    f2 tx[NPH], ty[NPH], tz[NPH], fqx[NPH], fqy[NPH], fqz[NPH], ug[NPH], fgx[NPH], fgy[NPH], fgz[NPH];
#pragma unroll
    for (int k = 0; k < NPH; k++) {
      tx[k] = f2add(f2pack(tx0[2 * k], tx0[2 * k + 1]), ddx);
      ty[k] = f2add(f2pack(ty0[2 * k], ty0[2 * k + 1]), ddy);
      tz[k] = f2add(f2pack(tz0[2 * k], tz0[2 * k + 1]), ddz);
      fqx[k] = fqy[k] = fqz[k] = ug[k] = fgx[k] = fgy[k] = fgz[k] = 0ull;
    }
    const ulonglong2* s2 = reinterpret_cast<const ulonglong2*>(sbuf[warp][buf][0]);
    const ulonglong2* g2 = reinterpret_cast<const ulonglong2*>(sbuf[warp][buf][1]);
    if (mask) {
#pragma unroll 2
      for (int j = half; j < scount; j += 2)
        bwd_pair<true, NPH>(s2[2 * j], s2[2 * j + 1], g2[2 * j + 1], tx, ty, tz, fqx, fqy, fqz, ug, fgx, fgy, fgz,
                            thr);
    } else {
#pragma unroll 2
      for (int j = half; j < scount; j += 2)
        bwd_pair<false, NPH>(s2[2 * j], s2[2 * j + 1], g2[2 * j + 1], tx, ty, tz, fqx, fqy, fqz, ug, fgx, fgy, fgz,
                             thr);
    }
#pragma unroll
    for (int k = 0; k < NPH; k++) {
      float a0, a1;
      f2unpack(ug[k], a0, a1);
      two_sum(uh[2 * k], ul[2 * k], a0);
      two_sum(uh[2 * k + 1], ul[2 * k + 1], a1);
      f2unpack(fqx[k], a0, a1), qx[2 * k] += a0, qx[2 * k + 1] += a1;
      f2unpack(fqy[k], a0, a1), qy[2 * k] += a0, qy[2 * k + 1] += a1;
      f2unpack(fqz[k], a0, a1), qz[2 * k] += a0, qz[2 * k + 1] += a1;
      f2unpack(fgx[k], a0, a1), gx[2 * k] += a0, gx[2 * k + 1] += a1;
      f2unpack(fgy[k], a0, a1), gy[2 * k] += a0, gy[2 * k + 1] += a1;
      f2unpack(fgz[k], a0, a1), gz[2 * k] += a0, gz[2 * k + 1] += a1;
    }
    __syncwarp();
  }
  // combine the two halves
#pragma unroll
  for (int k = 0; k < NT; k++) {
    const float oh = __shfl_xor_sync(0xffffffffu, uh[k], 16);
    const float ol = __shfl_xor_sync(0xffffffffu, ul[k], 16);
    two_sum(uh[k], ul[k], oh);
    ul[k] += ol;
    qx[k] += __shfl_xor_sync(0xffffffffu, qx[k], 16);
    qy[k] += __shfl_xor_sync(0xffffffffu, qy[k], 16);
    qz[k] += __shfl_xor_sync(0xffffffffu, qz[k], 16);
    gx[k] += __shfl_xor_sync(0xffffffffu, gx[k], 16);
    gy[k] += __shfl_xor_sync(0xffffffffu, gy[k], 16);
    gz[k] += __shfl_xor_sync(0xffffffffu, gz[k], 16);
  }
  if (half == 0) {
#pragma unroll
    for (int k = 0; k < NT; k++) {
      const int i = l16 + 16 * k;
      if (i < tcnt) {
        const int64_t pidx = tstart + i;
        a.near_f[3 * pidx] = qx[k];
        a.near_f[3 * pidx + 1] = qy[k];
        a.near_f[3 * pidx + 2] = qz[k];
        a.near_u2[2 * pidx] = uh[k];
        a.near_u2[2 * pidx + 1] = ul[k];
        a.near_f2[3 * pidx] = gx[k];
        a.near_f2[3 * pidx + 1] = gy[k];
        a.near_f2[3 * pidx + 2] = gz[k];
      }
    }
  }
}

// ---- E6 (FP32, potential, one point set): symmetric near field ----------------
// A leaf pair {A, B} listed in both directions is evaluated once, by the warp
// of the smaller leaf A: every 1/r serves both q_B / r (A's potentials,
// accumulated in registers) and q_A / r (B's potentials).  The second sums,
// per source point of B, are reduced across the half-warp by a reduce-scatter
// butterfly over chunks of 16 sources and stored to the pair's slot; the
// local evaluation of leaf B adds its slots in list order.  The self pair and
// pairs listed in one direction only are evaluated one-sided.  Lane layout
// and staging as in p2p_kernel_f32h.
//
// Source order inside a chunk of 32: lane l16 of half h takes, at step jj,
// record c0 + 4 (jj mod 8) + h + 2 w with w = (jj >= 8) xor (bit 3 of l16)
// (records c0 + 4 k + h for steps k, then c0 + 4 k + 2 + h, or the reverse in
// the upper eight lanes).  A lane's step jj and its partner's (lane xor 8)
// step jj xor 8 then hold the same source, so the butterfly's first stage
// needs no selects; at every step a warp reads four records whose
// 16-byte halves fall in distinct banks.
__device__ __forceinline__ float butterfly_sum(float (&P)[16], int l16) {
#pragma unroll
  for (int i = 0; i < 8; i++) P[i] += __shfl_xor_sync(0xffffffffu, P[i + 8], 8);
  // after the stages with masks 4, 2, 1 lane l16 holds the half-warp sum of
  // its step (l16 mod 8)
#pragma unroll
  for (int m = 4; m >= 1; m >>= 1) {
    const bool up = (l16 & m) != 0;
#pragma unroll
    for (int i = 0; i < m; i++) {
      const float keep = up ? P[i + m] : P[i];
      const float send = up ? P[i] : P[i + m];
      P[i] = keep + __shfl_xor_sync(0xffffffffu, send, m);
    }
  }
  return P[0];
}
template <int NPH>
__device__ __forceinline__ void butterfly_store(float (&P)[16], int l16, float* dst, int j, int scount) {
  const float v = butterfly_sum(P, l16);
  if (j < scount) dst[j] = v;
}

// One chunk of 32 sources (16 per half-warp): u of the lane's targets in pu,
// and per source the lane's share of sum_i q_i / r in P (step order above;
// sw = bit 3 of l16).  FULL: all 32 sources of the chunk exist.
template <bool MASK, bool FULL, int NPH>
__device__ __forceinline__ void sym_chunk(const ulonglong2* s2, int c0, int half, int sw, int scount,
                                          const f2 (&tx)[NPH], const f2 (&ty)[NPH], const f2 (&tz)[NPH],
                                          const f2 (&tq)[NPH], f2 (&pu)[NPH], float (&P)[16], float thr) {
  const int r_lo = c0 + half + 2 * sw, r_hi = c0 + half + 2 - 2 * sw;
  const ulonglong2* p_lo = s2 + 2 * r_lo;
  const ulonglong2* p_hi = s2 + 2 * r_hi;
#pragma unroll
  for (int jj = 0; jj < 16; jj++) {
    const int k = jj & 7;
    const int j = (jj < 8 ? r_lo : r_hi) + 4 * k;
    P[jj] = 0.f;
    if (FULL || j < scount) {
      const ulonglong2* pr = (jj < 8 ? p_lo : p_hi) + 8 * k;
      const ulonglong2 sa = pr[0], sb = pr[1];
      f2 acc = 0ull;
#pragma unroll
      for (int kk = 0; kk < NPH; kk++) {
        const f2 dx = f2sub(tx[kk], sa.x), dy = f2sub(ty[kk], sa.y), dz = f2sub(tz[kk], sb.x);
        const f2 r2 = f2fma(dz, dz, f2fma(dy, dy, f2mul(dx, dx)));
        float r0, r1;
        f2unpack(r2, r0, r1);
        float i0 = rsqrt_mufu(r0), i1 = rsqrt_mufu(r1);
        if (MASK) {
          i0 = (r0 > thr) ? i0 : 0.f;
          i1 = (r1 > thr) ? i1 : 0.f;
        }
        const f2 ri = f2pack(i0, i1);
        pu[kk] = f2fma(sb.y, ri, pu[kk]);
        acc = f2fma(tq[kk], ri, acc);
      }
      float a0, a1;
      f2unpack(acc, a0, a1);
      P[jj] = a0 + a1;
    }
  }
}

// One target leaf of the symmetric near field with NPH packed target pairs
// per lane (2 NPH targets, 32 NPH per warp); the staging buffers hold
// CAP-record source tiles.
template <int NPH, int CAP>
__device__ __forceinline__ void sym_leaf_f32(const P2PArgs& a, DupRec (&sb)[2][CAP], uint64_t* bar, int64_t leaf,
                                             int64_t tstart, int tcnt) {
  constexpr int NT = 2 * NPH;
  const DupRec* tile = reinterpret_cast<const DupRec*>(a.tile);
  const int lane = lane_id();
  const int half = lane >> 4, l16 = lane & 15;
  float tx0[NT], ty0[NT], tz0[NT], tq0[NT];
#pragma unroll
  for (int k = 0; k < NT; k++) {
    const int i = l16 + 16 * k;
    if (i < tcnt) {
      const float4 p = reinterpret_cast<const float4*>(a.src)[tstart + i];
      tx0[k] = p.x;
      ty0[k] = p.y;
      tz0[k] = p.z;
      tq0[k] = p.w;
    } else {
      // absent targets far from every source (finite 1/r, zero charge): they
      // must not add 0 * inf to the sources' sums
      tx0[k] = 1e18f;
      ty0[k] = tz0[k] = tq0[k] = 0.f;
    }
  }
  f2 tq[NPH];
#pragma unroll
  for (int k = 0; k < NPH; k++) tq[k] = f2pack(tq0[2 * k], tq0[2 * k + 1]);
  float hi[NT], lo[NT];
#pragma unroll
  for (int k = 0; k < NT; k++) hi[k] = lo[k] = 0.f;
  const int64_t kb = a.work_off[leaf];
  const int nwk = (int)(a.work_off[leaf + 1] - kb);
  // work records: lane l holds the record of entry base + l of the current
  // batch of 32; fields are broadcast per entry
  SymRec mine{};
  auto load_batch = [&](int base) {
    if (base + lane < nwk) mine = a.rec[kb + base + lane];
  };
  auto bcast = [&](int src_lane) {
    SymRec r;
    r.start = __shfl_sync(0xffffffffu, mine.start, src_lane);
    r.count = __shfl_sync(0xffffffffu, mine.count, src_lane);
    r.slot = __shfl_sync(0xffffffffu, mine.slot, src_lane);
    r.dx = __shfl_sync(0xffffffffu, mine.dx, src_lane);
    r.dy = __shfl_sync(0xffffffffu, mine.dy, src_lane);
    r.dz = __shfl_sync(0xffffffffu, mine.dz, src_lane);
    r.thr = __shfl_sync(0xffffffffu, mine.thr, src_lane);
    return r;
  };
  auto issue = [&](const SymRec& r, int buf) {
    if (lane == 0) {
      fence_proxy_async();
      tma_load_1d(sb[buf], tile + r.start, (uint32_t)(r.count * sizeof(DupRec)), &bar[buf]);
    }
  };
  uint32_t phase = 0;
  if (nwk > 0) {
    load_batch(0);
    issue(bcast(0), 0);
  }
  for (int w = 0; w < nwk; w++) {
    const int buf = w & 1;
    if (w > 0 && (w & 31) == 0) load_batch(w);  // warp-uniform
    const SymRec en = bcast(w & 31);
    if (w + 1 < nwk) {
      const SymRec nx = ((w + 1) & 31) ? bcast((w + 1) & 31) : a.rec[kb + w + 1];
      issue(nx, buf ^ 1);
    }
    if (!mbar_wait(&bar[buf], (phase >> buf) & 1u, a.wait_cycles)) {
      if (lane == 0) atomicOr(a.status, ST_TIMEOUT);
      // copies still in flight into this warp's buffers must land first
      mbar_wait(&bar[buf], (phase >> buf) & 1u, kDrainWaitCycles);
      if (w + 1 < nwk) mbar_wait(&bar[buf ^ 1], (phase >> (buf ^ 1)) & 1u, kDrainWaitCycles);
      return;
    }
    phase ^= 1u << buf;
    const int scount = en.count;
    const bool mask = en.thr >= 0.f;
    const float thr = en.thr;
    const int slot = en.slot;
    const f2 ddx = f2pack(en.dx, en.dx), ddy = f2pack(en.dy, en.dy), ddz = f2pack(en.dz, en.dz);
    f2 tx[NPH], ty[NPH], tz[NPH], pu[NPH];
#pragma unroll
    for (int k = 0; k < NPH; k++) {
      tx[k] = f2add(f2pack(tx0[2 * k], tx0[2 * k + 1]), ddx);
      ty[k] = f2add(f2pack(ty0[2 * k], ty0[2 * k + 1]), ddy);
      tz[k] = f2add(f2pack(tz0[2 * k], tz0[2 * k + 1]), ddz);
      pu[k] = 0ull;
    }
    const ulonglong2* s2 = reinterpret_cast<const ulonglong2*>(sb[buf]);
    if (slot < 0) {
      // one-sided: the self pair and pairs listed in one direction only
      f2 px[NPH], py[NPH], pz[NPH];
      if (mask) p2p_tile_f32h<true, false, NPH>(sb[buf], scount, half, tx, ty, tz, pu, px, py, pz, thr);
      else p2p_tile_f32h<false, false, NPH>(sb[buf], scount, half, tx, ty, tz, pu, px, py, pz, thr);
    } else {
      float* dst = reinterpret_cast<float*>(a.partial) + (int64_t)slot * a.stride;
      float P[16];
      int c0 = 0;
      const int sw = (l16 >> 3) & 1;
      const int jmine = half + 4 * (l16 & 7) + 2 * sw;  // source of this lane after the butterfly
      for (; c0 + 32 <= scount; c0 += 32) {
        if (mask) sym_chunk<true, true, NPH>(s2, c0, half, sw, scount, tx, ty, tz, tq, pu, P, thr);
        else sym_chunk<false, true, NPH>(s2, c0, half, sw, scount, tx, ty, tz, tq, pu, P, thr);
        butterfly_store<NPH>(P, l16, dst, c0 + jmine, scount);
      }
      if (c0 < scount) {
        if (mask) sym_chunk<true, false, NPH>(s2, c0, half, sw, scount, tx, ty, tz, tq, pu, P, thr);
        else sym_chunk<false, false, NPH>(s2, c0, half, sw, scount, tx, ty, tz, tq, pu, P, thr);
        butterfly_store<NPH>(P, l16, dst, c0 + jmine, scount);
      }
    }
#pragma unroll
    for (int k = 0; k < NPH; k++) {
      float u0, u1;
      f2unpack(pu[k], u0, u1);
      two_sum(hi[2 * k], lo[2 * k], u0);
      two_sum(hi[2 * k + 1], lo[2 * k + 1], u1);
    }
    __syncwarp();
  }
  // combine the two halves
#pragma unroll
  for (int k = 0; k < NT; k++) {
    const float oh = __shfl_xor_sync(0xffffffffu, hi[k], 16);
    const float ol = __shfl_xor_sync(0xffffffffu, lo[k], 16);
    two_sum(hi[k], lo[k], oh);
    lo[k] += ol;
  }
  if (half == 0) {
#pragma unroll
    for (int k = 0; k < NT; k++) {
      const int i = l16 + 16 * k;
      if (i < tcnt) {
        const int64_t pidx = tstart + i;
        a.near_u[2 * pidx] = hi[k];
        a.near_u[2 * pidx + 1] = lo[k];
      }
    }
  }
}

// Quarter-warp layout for target leaves of at most 32 points: four groups
// of 8 lanes take every fourth source record of a chunk of 32, and each lane
// holds 4 targets i = l8 + 8 k as two packed pairs, so every record loaded
// serves 4 targets (the half-warp layout serves 2 with such leaves).  The
// sources' sums of a group's 8 records are reduced by a 3-stage
// reduce-scatter over the group (lane l8 ends with its step l8's record).
// Every leaf of at most 32 points takes this layout in every kernel, so a
// batch evaluates its small leaves as the single trees do, bit for bit.
template <bool MASK, bool FULL>
__device__ __forceinline__ void symq_chunk(const ulonglong2* s2, int c0, int grp, int scount, const f2 (&tx)[2],
                                           const f2 (&ty)[2], const f2 (&tz)[2], const f2 (&tq)[2], f2 (&pu)[2],
                                           float (&P)[8], float thr) {
#pragma unroll
  for (int jj = 0; jj < 8; jj++) {
    const int j = c0 + 4 * jj + grp;
    P[jj] = 0.f;
    if (FULL || j < scount) {
      const ulonglong2 sa = s2[2 * j], sb = s2[2 * j + 1];
      f2 acc = 0ull;
#pragma unroll
      for (int kk = 0; kk < 2; kk++) {
        const f2 dx = f2sub(tx[kk], sa.x), dy = f2sub(ty[kk], sa.y), dz = f2sub(tz[kk], sb.x);
        const f2 r2 = f2fma(dz, dz, f2fma(dy, dy, f2mul(dx, dx)));
        float r0, r1;
        f2unpack(r2, r0, r1);
        float i0 = rsqrt_mufu(r0), i1 = rsqrt_mufu(r1);
        if (MASK) {
          i0 = (r0 > thr) ? i0 : 0.f;
          i1 = (r1 > thr) ? i1 : 0.f;
        }
        const f2 ri = f2pack(i0, i1);
        pu[kk] = f2fma(sb.y, ri, pu[kk]);
        acc = f2fma(tq[kk], ri, acc);
      }
      float a0, a1;
      f2unpack(acc, a0, a1);
      P[jj] = a0 + a1;
    }
  }
}

__device__ __forceinline__ float butterfly8_sum(float (&P)[8], int l8) {
#pragma unroll
  for (int m = 4; m >= 1; m >>= 1) {
    const bool up = (l8 & m) != 0;
#pragma unroll
    for (int i = 0; i < m; i++) {
      const float keep = up ? P[i + m] : P[i];
      const float send = up ? P[i] : P[i + m];
      P[i] = keep + __shfl_xor_sync(0xffffffffu, send, m);
    }
  }
  return P[0];
}

template <int CAP>
__device__ __forceinline__ void symq_leaf_f32(const P2PArgs& a, DupRec (&sb)[2][CAP], uint64_t* bar, int64_t leaf,
                                              int64_t tstart, int tcnt) {
  const DupRec* tile = reinterpret_cast<const DupRec*>(a.tile);
  const int lane = lane_id();
  const int grp = lane >> 3, l8 = lane & 7;
  float tx0[4], ty0[4], tz0[4], tq0[4];
#pragma unroll
  for (int k = 0; k < 4; k++) {
    const int i = l8 + 8 * k;
    if (i < tcnt) {
      const float4 p = reinterpret_cast<const float4*>(a.src)[tstart + i];
      tx0[k] = p.x;
      ty0[k] = p.y;
      tz0[k] = p.z;
      tq0[k] = p.w;
    } else {
      // absent targets far from every source, with zero charge
      tx0[k] = 1e18f;
      ty0[k] = tz0[k] = tq0[k] = 0.f;
    }
  }
  f2 tq[2];
#pragma unroll
  for (int k = 0; k < 2; k++) tq[k] = f2pack(tq0[2 * k], tq0[2 * k + 1]);
  float hi[4], lo[4];
#pragma unroll
  for (int k = 0; k < 4; k++) hi[k] = lo[k] = 0.f;
  const int64_t kb = a.work_off[leaf];
  const int nwk = (int)(a.work_off[leaf + 1] - kb);
  SymRec mine{};
  auto load_batch = [&](int base) {
    if (base + lane < nwk) mine = a.rec[kb + base + lane];
  };
  auto bcast = [&](int src_lane) {
    SymRec r;
    r.start = __shfl_sync(0xffffffffu, mine.start, src_lane);
    r.count = __shfl_sync(0xffffffffu, mine.count, src_lane);
    r.slot = __shfl_sync(0xffffffffu, mine.slot, src_lane);
    r.dx = __shfl_sync(0xffffffffu, mine.dx, src_lane);
    r.dy = __shfl_sync(0xffffffffu, mine.dy, src_lane);
    r.dz = __shfl_sync(0xffffffffu, mine.dz, src_lane);
    r.thr = __shfl_sync(0xffffffffu, mine.thr, src_lane);
    return r;
  };
  auto issue = [&](const SymRec& r, int buf) {
    if (lane == 0) {
      fence_proxy_async();
      tma_load_1d(sb[buf], tile + r.start, (uint32_t)(r.count * sizeof(DupRec)), &bar[buf]);
    }
  };
  uint32_t phase = 0;
  if (nwk > 0) {
    load_batch(0);
    issue(bcast(0), 0);
  }
  for (int w = 0; w < nwk; w++) {
    const int buf = w & 1;
    if (w > 0 && (w & 31) == 0) load_batch(w);  // warp-uniform
    const SymRec en = bcast(w & 31);
    if (w + 1 < nwk) {
      const SymRec nx = ((w + 1) & 31) ? bcast((w + 1) & 31) : a.rec[kb + w + 1];
      issue(nx, buf ^ 1);
    }
    if (!mbar_wait(&bar[buf], (phase >> buf) & 1u, a.wait_cycles)) {
      if (lane == 0) atomicOr(a.status, ST_TIMEOUT);
      // copies still in flight into this warp's buffers must land first
      mbar_wait(&bar[buf], (phase >> buf) & 1u, kDrainWaitCycles);
      if (w + 1 < nwk) mbar_wait(&bar[buf ^ 1], (phase >> (buf ^ 1)) & 1u, kDrainWaitCycles);
      return;
    }
    phase ^= 1u << buf;
    const int scount = en.count;
    const bool mask = en.thr >= 0.f;
    const float thr = en.thr;
    const int slot = en.slot;
    const f2 ddx = f2pack(en.dx, en.dx), ddy = f2pack(en.dy, en.dy), ddz = f2pack(en.dz, en.dz);
    f2 tx[2], ty[2], tz[2], pu[2];
#pragma unroll
    for (int k = 0; k < 2; k++) {
      tx[k] = f2add(f2pack(tx0[2 * k], tx0[2 * k + 1]), ddx);
      ty[k] = f2add(f2pack(ty0[2 * k], ty0[2 * k + 1]), ddy);
      tz[k] = f2add(f2pack(tz0[2 * k], tz0[2 * k + 1]), ddz);
      pu[k] = 0ull;
    }
    const ulonglong2* s2 = reinterpret_cast<const ulonglong2*>(sb[buf]);
    if (slot < 0) {
      // one-sided: the self pair and pairs listed in one direction only
      f2 px[2], py[2], pz[2];
      for (int j = grp; j < scount; j += 4) {
        if (mask) p2p_pair_f32<true, false, 2>(s2[2 * j], s2[2 * j + 1], tx, ty, tz, pu, px, py, pz, thr);
        else p2p_pair_f32<false, false, 2>(s2[2 * j], s2[2 * j + 1], tx, ty, tz, pu, px, py, pz, thr);
      }
    } else {
      float* dst = reinterpret_cast<float*>(a.partial) + (int64_t)slot * a.stride;
      float P[8];
      int c0 = 0;
      for (; c0 + 32 <= scount; c0 += 32) {
        if (mask) symq_chunk<true, true>(s2, c0, grp, scount, tx, ty, tz, tq, pu, P, thr);
        else symq_chunk<false, true>(s2, c0, grp, scount, tx, ty, tz, tq, pu, P, thr);
        const float v = butterfly8_sum(P, l8);
        dst[c0 + 4 * l8 + grp] = v;
      }
      if (c0 < scount) {
        if (mask) symq_chunk<true, false>(s2, c0, grp, scount, tx, ty, tz, tq, pu, P, thr);
        else symq_chunk<false, false>(s2, c0, grp, scount, tx, ty, tz, tq, pu, P, thr);
        const float v = butterfly8_sum(P, l8);
        const int j = c0 + 4 * l8 + grp;
        if (j < scount) dst[j] = v;
      }
    }
#pragma unroll
    for (int k = 0; k < 2; k++) {
      float u0, u1;
      f2unpack(pu[k], u0, u1);
      two_sum(hi[2 * k], lo[2 * k], u0);
      two_sum(hi[2 * k + 1], lo[2 * k + 1], u1);
    }
    __syncwarp();
  }
  // combine the four groups (lanes l8, l8 + 8, l8 + 16, l8 + 24)
#pragma unroll
  for (int m = 8; m <= 16; m <<= 1) {
#pragma unroll
    for (int k = 0; k < 4; k++) {
      const float oh = __shfl_xor_sync(0xffffffffu, hi[k], m);
      const float ol = __shfl_xor_sync(0xffffffffu, lo[k], m);
      two_sum(hi[k], lo[k], oh);
      lo[k] += ol;
    }
  }
  if (grp == 0) {
#pragma unroll
    for (int k = 0; k < 4; k++) {
      const int i = l8 + 8 * k;
      if (i < tcnt) {
        const int64_t pidx = tstart + i;
        a.near_u[2 * pidx] = hi[k];
        a.near_u[2 * pidx + 1] = lo[k];
      }
    }
  }
}

// Symmetric near field kernel for trees whose smallest leaf fills at most
// half of the warp's target slots (such as a batch of sets of different
// sizes): such leaves take the half-width layout, so no lane computes for
// absent targets in the second packed pair.  Trees of full leaves launch
// p2p_kernel_f32s (the same per-leaf code written out in the kernel, which
// keeps its register allocation).
template <int TPL>
__global__ void __launch_bounds__(128, TPL <= 2 ? 5 : (TPL == 4 ? 3 : 2)) p2p_kernel_f32s_half(P2PArgs a) {
  constexpr int CAP = TPL * 32;
  constexpr int WARPS = 4;
  extern __shared__ __align__(128) unsigned char p2p_smem[];
  DupRec (*sbuf)[2][CAP] = reinterpret_cast<DupRec (*)[2][CAP]>(p2p_smem);
  __shared__ __align__(8) uint64_t bars[WARPS][2];
  const int lane = lane_id();
  const int warp = threadIdx.x >> 5;
  uint64_t* bar = bars[warp];
  if (lane == 0) {
    mbar_init(&bar[0]);
    mbar_init(&bar[1]);
    fence_barrier_init();
  }
  __syncwarp();
  const int64_t t = (int64_t)blockIdx.x * WARPS + warp;
  if (t >= a.n_leaves) return;
  const int64_t leaf = a.order[t];
  const int64_t g = a.leaf_box[leaf];
  const int64_t tstart = a.box_start[g];
  const int tcnt = a.box_count[g];
  if (tcnt <= 32) symq_leaf_f32<CAP>(a, sbuf[warp], bar, leaf, tstart, tcnt);
  else if (tcnt <= 16 * TPL) sym_leaf_f32<TPL / 2, CAP>(a, sbuf[warp], bar, leaf, tstart, tcnt);
  else sym_leaf_f32<TPL, CAP>(a, sbuf[warp], bar, leaf, tstart, tcnt);
}

template <int TPL>
__global__ void __launch_bounds__(128, TPL <= 2 ? 5 : (TPL == 4 ? 3 : 2)) p2p_kernel_f32s(P2PArgs a) {
  constexpr int CAP = TPL * 32;
  constexpr int WARPS = 4;
  constexpr int NT = 2 * TPL;
  constexpr int NPH = TPL;
  extern __shared__ __align__(128) unsigned char p2p_smem[];
  DupRec (*sbuf)[2][CAP] = reinterpret_cast<DupRec (*)[2][CAP]>(p2p_smem);
  __shared__ __align__(8) uint64_t bars[WARPS][2];
  const DupRec* tile = reinterpret_cast<const DupRec*>(a.tile);
  const int lane = lane_id();
  const int warp = threadIdx.x >> 5;
  const int half = lane >> 4, l16 = lane & 15;
  uint64_t* bar = bars[warp];
  if (lane == 0) {
    mbar_init(&bar[0]);
    mbar_init(&bar[1]);
    fence_barrier_init();
  }
  __syncwarp();
  const int64_t t = (int64_t)blockIdx.x * WARPS + warp;
  if (t >= a.n_leaves) return;
  const int64_t leaf = a.order[t];
  const int64_t g = a.leaf_box[leaf];
  const int64_t tstart = a.box_start[g];
  const int tcnt = a.box_count[g];
  if constexpr (TPL == 1) {
    // leaves of at most 32 points: the quarter-warp layout
    symq_leaf_f32<CAP>(a, sbuf[warp], bar, leaf, tstart, tcnt);
    return;
  }
  float tx0[NT], ty0[NT], tz0[NT], tq0[NT];
#pragma unroll
  for (int k = 0; k < NT; k++) {
    const int i = l16 + 16 * k;
    if (i < tcnt) {
      const float4 p = reinterpret_cast<const float4*>(a.src)[tstart + i];
      tx0[k] = p.x;
      ty0[k] = p.y;
      tz0[k] = p.z;
      tq0[k] = p.w;
    } else {
      // absent targets far from every source (finite 1/r, zero charge): they
      // must not add 0 * inf to the sources' sums
      tx0[k] = 1e18f;
      ty0[k] = tz0[k] = tq0[k] = 0.f;
    }
  }
  f2 tq[NPH];
#pragma unroll
  for (int k = 0; k < NPH; k++) tq[k] = f2pack(tq0[2 * k], tq0[2 * k + 1]);
  float hi[NT], lo[NT];
#pragma unroll
  for (int k = 0; k < NT; k++) hi[k] = lo[k] = 0.f;
  const int64_t kb = a.work_off[leaf];
  const int nwk = (int)(a.work_off[leaf + 1] - kb);
  // work records: lane l holds the record of entry base + l of the current
  // batch of 32; fields are broadcast per entry
  SymRec mine{};
  auto load_batch = [&](int base) {
    if (base + lane < nwk) mine = a.rec[kb + base + lane];
  };
  auto bcast = [&](int src_lane) {
    SymRec r;
    r.start = __shfl_sync(0xffffffffu, mine.start, src_lane);
    r.count = __shfl_sync(0xffffffffu, mine.count, src_lane);
    r.slot = __shfl_sync(0xffffffffu, mine.slot, src_lane);
    r.dx = __shfl_sync(0xffffffffu, mine.dx, src_lane);
    r.dy = __shfl_sync(0xffffffffu, mine.dy, src_lane);
    r.dz = __shfl_sync(0xffffffffu, mine.dz, src_lane);
    r.thr = __shfl_sync(0xffffffffu, mine.thr, src_lane);
    return r;
  };
  auto issue = [&](const SymRec& r, int buf) {
    if (lane == 0) {
      fence_proxy_async();
      tma_load_1d(sbuf[warp][buf], tile + r.start, (uint32_t)(r.count * sizeof(DupRec)), &bar[buf]);
    }
  };
  uint32_t phase = 0;
  if (nwk > 0) {
    load_batch(0);
    issue(bcast(0), 0);
  }
  for (int w = 0; w < nwk; w++) {
    const int buf = w & 1;
    if (w > 0 && (w & 31) == 0) load_batch(w);  // warp-uniform
    const SymRec en = bcast(w & 31);
    if (w + 1 < nwk) {
      const SymRec nx = ((w + 1) & 31) ? bcast((w + 1) & 31) : a.rec[kb + w + 1];
      issue(nx, buf ^ 1);
    }
    if (!mbar_wait(&bar[buf], (phase >> buf) & 1u, a.wait_cycles)) {
      if (lane == 0) atomicOr(a.status, ST_TIMEOUT);
      // copies still in flight into this warp's buffers must land first
      mbar_wait(&bar[buf], (phase >> buf) & 1u, kDrainWaitCycles);
      if (w + 1 < nwk) mbar_wait(&bar[buf ^ 1], (phase >> (buf ^ 1)) & 1u, kDrainWaitCycles);
      return;
    }
    phase ^= 1u << buf;
    const int scount = en.count;
    const bool mask = en.thr >= 0.f;
    const float thr = en.thr;
    const int slot = en.slot;
    const f2 ddx = f2pack(en.dx, en.dx), ddy = f2pack(en.dy, en.dy), ddz = f2pack(en.dz, en.dz);
    f2 tx[NPH], ty[NPH], tz[NPH], pu[NPH];
#pragma unroll
    for (int k = 0; k < NPH; k++) {
      tx[k] = f2add(f2pack(tx0[2 * k], tx0[2 * k + 1]), ddx);
      ty[k] = f2add(f2pack(ty0[2 * k], ty0[2 * k + 1]), ddy);
      tz[k] = f2add(f2pack(tz0[2 * k], tz0[2 * k + 1]), ddz);
      pu[k] = 0ull;
    }
    const ulonglong2* s2 = reinterpret_cast<const ulonglong2*>(sbuf[warp][buf]);
    if (slot < 0) {
      // one-sided: the self pair and pairs listed in one direction only
      f2 px[NPH], py[NPH], pz[NPH];
      if (mask) p2p_tile_f32h<true, false, NPH>(sbuf[warp][buf], scount, half, tx, ty, tz, pu, px, py, pz, thr);
      else p2p_tile_f32h<false, false, NPH>(sbuf[warp][buf], scount, half, tx, ty, tz, pu, px, py, pz, thr);
    } else {
      float* dst = reinterpret_cast<float*>(a.partial) + (int64_t)slot * a.stride;
      float P[16];
      int c0 = 0;
      const int sw = (l16 >> 3) & 1;
      const int jmine = half + 4 * (l16 & 7) + 2 * sw;  // source of this lane after the butterfly
      for (; c0 + 32 <= scount; c0 += 32) {
        if (mask) sym_chunk<true, true, NPH>(s2, c0, half, sw, scount, tx, ty, tz, tq, pu, P, thr);
        else sym_chunk<false, true, NPH>(s2, c0, half, sw, scount, tx, ty, tz, tq, pu, P, thr);
        butterfly_store<NPH>(P, l16, dst, c0 + jmine, scount);
      }
      if (c0 < scount) {
        if (mask) sym_chunk<true, false, NPH>(s2, c0, half, sw, scount, tx, ty, tz, tq, pu, P, thr);
        else sym_chunk<false, false, NPH>(s2, c0, half, sw, scount, tx, ty, tz, tq, pu, P, thr);
        butterfly_store<NPH>(P, l16, dst, c0 + jmine, scount);
      }
    }
#pragma unroll
    for (int k = 0; k < NPH; k++) {
      float u0, u1;
      f2unpack(pu[k], u0, u1);
      two_sum(hi[2 * k], lo[2 * k], u0);
      two_sum(hi[2 * k + 1], lo[2 * k + 1], u1);
    }
    __syncwarp();
  }
  // combine the two halves
#pragma unroll
  for (int k = 0; k < NT; k++) {
    const float oh = __shfl_xor_sync(0xffffffffu, hi[k], 16);
    const float ol = __shfl_xor_sync(0xffffffffu, lo[k], 16);
    two_sum(hi[k], lo[k], oh);
    lo[k] += ol;
  }
  if (half == 0) {
#pragma unroll
    for (int k = 0; k < NT; k++) {
      const int i = l16 + 16 * k;
      if (i < tcnt) {
        const int64_t pidx = tstart + i;
        a.near_u[2 * pidx] = hi[k];
        a.near_u[2 * pidx + 1] = lo[k];
      }
    }
  }
}

// Symmetric near field, second half: every leaf adds the slots it received
// (sums computed by the warps of its partners; contiguous, in list order) to
// its near-field sums.  Warp per leaf, each lane two points, eight slots'
// loads in flight per point.
// Chunks of at most kGatherChunk slots, one warp each: a leaf with one
// chunk adds it to its sums directly; a leaf with several writes each
// chunk's sums (hi, lo per point) to a partial row, and sym_combine_kernel
// adds the rows in chunk order.
__global__ void __launch_bounds__(128) sym_gather_kernel(int64_t n_chunks, const int32_t* __restrict__ gch_leaf,
                                                         const int64_t* __restrict__ gch_r0,
                                                         const int64_t* __restrict__ gch_first,
                                                         const int32_t* __restrict__ leaf_box,
                                                         const int64_t* __restrict__ box_start,
                                                         const int32_t* __restrict__ box_count,
                                                         const int64_t* __restrict__ recv_off,
                                                         const float* __restrict__ partial, int64_t stride,
                                                         float* __restrict__ near_u, float* __restrict__ gpart) {
  const int lane = lane_id();
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x / 32);
  for (int64_t ch = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) / 32; ch < n_chunks; ch += warps) {
    const int64_t leaf = gch_leaf[ch];
    const int64_t r0 = gch_r0[ch], r1 = min(r0 + kGatherChunk, recv_off[leaf + 1]);
    const bool single = gch_first[leaf + 1] - gch_first[leaf] == 1;
    const int64_t g = leaf_box[leaf];
    const int64_t start = box_start[g];
    const int cnt = box_count[g];
    for (int base = 0; base < cnt; base += 64) {
      const int i0 = base + lane, i1 = base + 32 + lane;
      const bool ok0 = i0 < cnt, ok1 = i1 < cnt;
      float h0 = 0.f, l0 = 0.f, h1 = 0.f, l1 = 0.f;
      if (single) {
        h0 = ok0 ? near_u[2 * (start + i0)] : 0.f;
        l0 = ok0 ? near_u[2 * (start + i0) + 1] : 0.f;
        h1 = ok1 ? near_u[2 * (start + i1)] : 0.f;
        l1 = ok1 ? near_u[2 * (start + i1) + 1] : 0.f;
      }
      for (int64_t r = r0; r < r1; r += 8) {
        float v0[8], v1[8];
#pragma unroll
        for (int k = 0; k < 8; k++) {
          const bool in = r + k < r1;
          const float* row = partial + (r + k) * stride;
          v0[k] = (in && ok0) ? row[i0] : 0.f;
          v1[k] = (in && ok1) ? row[i1] : 0.f;
        }
#pragma unroll
        for (int k = 0; k < 8; k++) {
          if (r + k < r1) {
            two_sum(h0, l0, v0[k]);
            two_sum(h1, l1, v1[k]);
          }
        }
      }
      float* dst = single ? near_u + 2 * start : gpart + 2 * ch * stride;
      if (ok0) {
        dst[2 * i0] = h0;
        dst[2 * i0 + 1] = l0;
      }
      if (ok1) {
        dst[2 * i1] = h1;
        dst[2 * i1 + 1] = l1;
      }
    }
  }
}

// Leaves gathered in several chunks: the chunks' sums added in chunk order.
__global__ void __launch_bounds__(128) sym_combine_kernel(int64_t n_multi, const int32_t* __restrict__ mleaf,
                                                          const int64_t* __restrict__ gch_first,
                                                          const int32_t* __restrict__ leaf_box,
                                                          const int64_t* __restrict__ box_start,
                                                          const int32_t* __restrict__ box_count, int64_t stride,
                                                          const float* __restrict__ gpart, float* __restrict__ near_u) {
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x / 32);
  for (int64_t k = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) / 32; k < n_multi; k += warps) {
    const int64_t leaf = mleaf[k];
    const int64_t g = leaf_box[leaf];
    const int64_t start = box_start[g];
    const int cnt = box_count[g];
    for (int i = threadIdx.x & 31; i < cnt; i += 32) {
      float h = near_u[2 * (start + i)], l = near_u[2 * (start + i) + 1];
      for (int64_t ch = gch_first[leaf]; ch < gch_first[leaf + 1]; ch++) {
        two_sum(h, l, gpart[2 * (ch * stride + i)]);
        l += gpart[2 * (ch * stride + i) + 1];
      }
      near_u[2 * (start + i)] = h;
      near_u[2 * (start + i) + 1] = l;
    }
  }
}

// ---- E6 (FP32C, one point set): symmetric near field of a vector quantity ------
// The symmetric scheme of p2p_kernel_f32s for evaluations that need, besides
// 1/r, the vector d / r^3 (d = x_t - x_s) at both points of a pair.  Each
// point ends with a potential-like sum U (compensated, as the potential) and a
// vector sum V:
//   kSvField (the field of the charges q):
//     U_t = sum_s q_s / r,  V_t = sum_s q_s d_ts / r^3   (the source side of a
//     pair gets q_t / r and q_t d_st / r^3 = -q_t d_ts / r^3);
//   kSvBackward (the near-field part of the backward pass, charges q and
//   cotangents g = dL/du):
//     U_t = sum_s g_s / r  (the potential of g, for dL/dq), and
//     V_t = sum_s (g_t q_s + q_t g_s) d_ts / r^3, whose coefficient is the
//     same for both points of a pair, so the source side gets -V's term; up to
//     the factor 1/(4 pi) it is the near part of dL/dx_t (the gradient of
//     sum_ij g_i K_ij q_j with K = -1/(4 pi r)).
// The source side of a pair is summed over the lane's targets in registers,
// then over the half-warp by four reduce-scatter butterflies, and stored as
// (U, V) float4 records to the pair's slot row; sv_gather_kernel adds the
// received rows.  Targets and sources are both read from the DupRec tiles
// (positions relative to their leaf's centre; q from `tile`, g from
// `tile_g`), so the far field may rewrite the FP32 point records meanwhile.
constexpr int kSvField = 0;
constexpr int kSvBackward = 1;

// One ordered pair, one-sided (self pairs and pairs listed one way): the
// target side only.
template <int MODE, bool MASK, int NPH>
__device__ __forceinline__ void sv_pair_one(const ulonglong2 a, const ulonglong2 b, const f2 sg, const f2 (&tx)[NPH],
                                            const f2 (&ty)[NPH], const f2 (&tz)[NPH], const f2 (&tq)[NPH],
                                            const f2 (&tg)[NPH], f2 (&pu)[NPH], f2 (&vx)[NPH], f2 (&vy)[NPH],
                                            f2 (&vz)[NPH], float thr) {
#pragma unroll
  for (int k = 0; k < NPH; k++) {
    const f2 dx = f2sub(tx[k], a.x), dy = f2sub(ty[k], a.y), dz = f2sub(tz[k], b.x);
    const f2 r2 = f2fma(dz, dz, f2fma(dy, dy, f2mul(dx, dx)));
    float r0, r1;
    f2unpack(r2, r0, r1);
    float i0 = rsqrt_mufu(r0), i1 = rsqrt_mufu(r1);
    if (MASK) {
      i0 = (r0 > thr) ? i0 : 0.f;
      i1 = (r1 > thr) ? i1 : 0.f;
    }
    const f2 ri = f2pack(i0, i1);
    const f2 ri3 = f2mul(f2mul(ri, ri), ri);
    f2 w;
    if (MODE == kSvField) {
      pu[k] = f2fma(b.y, ri, pu[k]);
      w = f2mul(b.y, ri3);
    } else {
      pu[k] = f2fma(sg, ri, pu[k]);
      const f2 c = f2fma(tg[k], b.y, f2mul(tq[k], sg));
      w = f2mul(c, ri3);
    }
    vx[k] = f2fma(w, dx, vx[k]);
    vy[k] = f2fma(w, dy, vy[k]);
    vz[k] = f2fma(w, dz, vz[k]);
  }
}

// One chunk of 32 sources of a pair evaluated for both sides (source order
// and butterfly as in sym_chunk): the target sums in pu, vx, vy, vz; the
// lane's share of each source's sums in PU, PX, PY, PZ (V's source-side terms
// with the sign of d_ts: negated when stored).
template <int MODE, bool MASK, bool FULL, int NPH>
__device__ __forceinline__ void sv_chunk(const ulonglong2* s2, const ulonglong2* g2, int c0, int half, int sw,
                                         int scount, const f2 (&tx)[NPH], const f2 (&ty)[NPH],
                                         const f2 (&tz)[NPH], const f2 (&tq)[NPH], const f2 (&tg)[NPH],
                                         f2 (&pu)[NPH], f2 (&vx)[NPH], f2 (&vy)[NPH], f2 (&vz)[NPH],
                                         float (&PU)[16], float (&PX)[16], float (&PY)[16], float (&PZ)[16],
                                         float thr) {
  const int r_lo = c0 + half + 2 * sw, r_hi = c0 + half + 2 - 2 * sw;
#pragma unroll
  for (int jj = 0; jj < 16; jj++) {
    const int k = jj & 7;
    const int j = (jj < 8 ? r_lo : r_hi) + 4 * k;
    PU[jj] = PX[jj] = PY[jj] = PZ[jj] = 0.f;
    if (FULL || j < scount) {
      const ulonglong2 sa = s2[2 * j], sb = s2[2 * j + 1];
      const f2 sg = (MODE == kSvBackward) ? g2[2 * j + 1].y : 0ull;
      f2 au = 0ull, ax = 0ull, ay = 0ull, az = 0ull;
#pragma unroll
      for (int kk = 0; kk < NPH; kk++) {
        const f2 dx = f2sub(tx[kk], sa.x), dy = f2sub(ty[kk], sa.y), dz = f2sub(tz[kk], sb.x);
        const f2 r2 = f2fma(dz, dz, f2fma(dy, dy, f2mul(dx, dx)));
        float r0, r1;
        f2unpack(r2, r0, r1);
        float i0 = rsqrt_mufu(r0), i1 = rsqrt_mufu(r1);
        if (MASK) {
          i0 = (r0 > thr) ? i0 : 0.f;
          i1 = (r1 > thr) ? i1 : 0.f;
        }
        const f2 ri = f2pack(i0, i1);
        const f2 ri3 = f2mul(f2mul(ri, ri), ri);
        if (MODE == kSvField) {
          pu[kk] = f2fma(sb.y, ri, pu[kk]);
          const f2 ws = f2mul(sb.y, ri3);  // q_s / r^3
          vx[kk] = f2fma(ws, dx, vx[kk]);
          vy[kk] = f2fma(ws, dy, vy[kk]);
          vz[kk] = f2fma(ws, dz, vz[kk]);
          au = f2fma(tq[kk], ri, au);
          const f2 wt = f2mul(tq[kk], ri3);  // q_t / r^3
          ax = f2fma(wt, dx, ax);
          ay = f2fma(wt, dy, ay);
          az = f2fma(wt, dz, az);
        } else {
          pu[kk] = f2fma(sg, ri, pu[kk]);
          au = f2fma(tg[kk], ri, au);
          const f2 c = f2fma(tg[kk], sb.y, f2mul(tq[kk], sg));
          const f2 w = f2mul(c, ri3);
          vx[kk] = f2fma(w, dx, vx[kk]);
          vy[kk] = f2fma(w, dy, vy[kk]);
          vz[kk] = f2fma(w, dz, vz[kk]);
          ax = f2fma(w, dx, ax);
          ay = f2fma(w, dy, ay);
          az = f2fma(w, dz, az);
        }
      }
      float a0, a1;
      f2unpack(au, a0, a1);
      PU[jj] = a0 + a1;
      f2unpack(ax, a0, a1);
      PX[jj] = a0 + a1;
      f2unpack(ay, a0, a1);
      PY[jj] = a0 + a1;
      f2unpack(az, a0, a1);
      PZ[jj] = a0 + a1;
    }
  }
}

template <int TPL, int MODE>
__global__ void __launch_bounds__(128, TPL <= 2 ? 3 : 2) p2p_kernel_f32sv(P2PArgs a) {
  constexpr bool BWD = MODE == kSvBackward;
  constexpr int CAP = TPL * 32;
  constexpr int WARPS = 4;
  constexpr int NT = 2 * TPL;
  constexpr int NPH = TPL;
  constexpr int NTILE = BWD ? 2 : 1;  // staged tiles per source leaf: q (and g)
  extern __shared__ __align__(128) unsigned char p2p_smem[];
  DupRec (*sbuf)[2][NTILE][CAP] = reinterpret_cast<DupRec (*)[2][NTILE][CAP]>(p2p_smem);
  __shared__ __align__(8) uint64_t bars[WARPS][2];
  const DupRec* tile = reinterpret_cast<const DupRec*>(a.tile);
  const DupRec* tile_g = a.tile_g;
  const int lane = lane_id();
  const int warp = threadIdx.x >> 5;
  const int half = lane >> 4, l16 = lane & 15;
  uint64_t* bar = bars[warp];
  if (lane == 0) {
    mbar_init(&bar[0]);
    mbar_init(&bar[1]);
    fence_barrier_init();
  }
  __syncwarp();
  const int64_t t = (int64_t)blockIdx.x * WARPS + warp;
  if (t >= a.n_leaves) return;
  const int64_t leaf = a.order[t];
  const int64_t g = a.leaf_box[leaf];
  const int64_t tstart = a.box_start[g];
  const int tcnt = a.box_count[g];
  float tx0[NT], ty0[NT], tz0[NT], tq0[NT], tg0[NT];
#pragma unroll
  for (int k = 0; k < NT; k++) {
    const int i = l16 + 16 * k;
    if (i < tcnt) {
      const DupRec p = tile[tstart + i];
      tx0[k] = p.x0;
      ty0[k] = p.y0;
      tz0[k] = p.z0;
      tq0[k] = p.q0;
      tg0[k] = BWD ? tile_g[tstart + i].q0 : 0.f;
    } else {
      // absent targets far from every source, with zero charges: finite
      // terms that add nothing to the sources' sums
      tx0[k] = 1e18f;
      ty0[k] = tz0[k] = tq0[k] = tg0[k] = 0.f;
    }
  }
  f2 tq[NPH], tg[NPH], vx[NPH], vy[NPH], vz[NPH];
#pragma unroll
  for (int k = 0; k < NPH; k++) {
    tq[k] = f2pack(tq0[2 * k], tq0[2 * k + 1]);
    tg[k] = f2pack(tg0[2 * k], tg0[2 * k + 1]);
    vx[k] = vy[k] = vz[k] = 0ull;
  }
  float hi[NT], lo[NT];
#pragma unroll
  for (int k = 0; k < NT; k++) hi[k] = lo[k] = 0.f;
  const int64_t kb = a.work_off[leaf];
  const int nwk = (int)(a.work_off[leaf + 1] - kb);
  SymRec mine{};
  auto load_batch = [&](int base) {
    if (base + lane < nwk) mine = a.rec[kb + base + lane];
  };
  auto bcast = [&](int src_lane) {
    SymRec r;
    r.start = __shfl_sync(0xffffffffu, mine.start, src_lane);
    r.count = __shfl_sync(0xffffffffu, mine.count, src_lane);
    r.slot = __shfl_sync(0xffffffffu, mine.slot, src_lane);
    r.dx = __shfl_sync(0xffffffffu, mine.dx, src_lane);
    r.dy = __shfl_sync(0xffffffffu, mine.dy, src_lane);
    r.dz = __shfl_sync(0xffffffffu, mine.dz, src_lane);
    r.thr = __shfl_sync(0xffffffffu, mine.thr, src_lane);
    return r;
  };
  auto issue = [&](const SymRec& r, int buf) {
    if (lane == 0) {
      const uint32_t bytes = (uint32_t)(r.count * sizeof(DupRec));
      fence_proxy_async();
      asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(&bar[buf])),
                   "r"(NTILE * bytes)
                   : "memory");
      bulk_copy(sbuf[warp][buf][0], tile + r.start, bytes, &bar[buf]);
      if (BWD) bulk_copy(sbuf[warp][buf][NTILE - 1], tile_g + r.start, bytes, &bar[buf]);
    }
  };
  uint32_t phase = 0;
  if (nwk > 0) {
    load_batch(0);
    issue(bcast(0), 0);
  }
  for (int w = 0; w < nwk; w++) {
    const int buf = w & 1;
    if (w > 0 && (w & 31) == 0) load_batch(w);  // warp-uniform
    const SymRec en = bcast(w & 31);
    if (w + 1 < nwk) {
      const SymRec nx = ((w + 1) & 31) ? bcast((w + 1) & 31) : a.rec[kb + w + 1];
      issue(nx, buf ^ 1);
    }
    if (!mbar_wait(&bar[buf], (phase >> buf) & 1u, a.wait_cycles)) {
      if (lane == 0) atomicOr(a.status, ST_TIMEOUT);
      // copies still in flight into this warp's buffers must land first
      mbar_wait(&bar[buf], (phase >> buf) & 1u, kDrainWaitCycles);
      if (w + 1 < nwk) mbar_wait(&bar[buf ^ 1], (phase >> (buf ^ 1)) & 1u, kDrainWaitCycles);
      return;
    }
    phase ^= 1u << buf;
    const int scount = en.count;
    const bool mask = en.thr >= 0.f;
    const float thr = en.thr;
    const int slot = en.slot;
    const f2 ddx = f2pack(en.dx, en.dx), ddy = f2pack(en.dy, en.dy), ddz = f2pack(en.dz, en.dz);
    f2 tx[NPH], ty[NPH], tz[NPH], pu[NPH];
#pragma unroll
    for (int k = 0; k < NPH; k++) {
      tx[k] = f2add(f2pack(tx0[2 * k], tx0[2 * k + 1]), ddx);
      ty[k] = f2add(f2pack(ty0[2 * k], ty0[2 * k + 1]), ddy);
      tz[k] = f2add(f2pack(tz0[2 * k], tz0[2 * k + 1]), ddz);
      pu[k] = 0ull;
    }
    const ulonglong2* s2 = reinterpret_cast<const ulonglong2*>(sbuf[warp][buf][0]);
    const ulonglong2* g2 = reinterpret_cast<const ulonglong2*>(sbuf[warp][buf][NTILE - 1]);
    if (slot < 0) {
      // one-sided: the self pair and pairs listed in one direction only
      if (mask) {
#pragma unroll 2
        for (int j = half; j < scount; j += 2)
          sv_pair_one<MODE, true, NPH>(s2[2 * j], s2[2 * j + 1], BWD ? g2[2 * j + 1].y : 0ull, tx, ty, tz, tq, tg,
                                       pu, vx, vy, vz, thr);
      } else {
#pragma unroll 2
        for (int j = half; j < scount; j += 2)
          sv_pair_one<MODE, false, NPH>(s2[2 * j], s2[2 * j + 1], BWD ? g2[2 * j + 1].y : 0ull, tx, ty, tz, tq, tg,
                                        pu, vx, vy, vz, thr);
      }
    } else {
      float4* dst = reinterpret_cast<float4*>(a.partial) + (int64_t)slot * a.stride;
      float PU[16], PX[16], PY[16], PZ[16];
      const int sw = (l16 >> 3) & 1;
      const int jmine = half + 4 * (l16 & 7) + 2 * sw;  // source of this lane after the butterflies
      auto finish = [&](int c0) {
        const float su = butterfly_sum(PU, l16);
        const float sx = butterfly_sum(PX, l16);
        const float sy = butterfly_sum(PY, l16);
        const float sz = butterfly_sum(PZ, l16);
        if (c0 + jmine < scount) dst[c0 + jmine] = make_float4(su, -sx, -sy, -sz);
      };
      int c0 = 0;
      for (; c0 + 32 <= scount; c0 += 32) {
        if (mask)
          sv_chunk<MODE, true, true, NPH>(s2, g2, c0, half, sw, scount, tx, ty, tz, tq, tg, pu, vx, vy, vz, PU, PX,
                                          PY, PZ, thr);
        else
          sv_chunk<MODE, false, true, NPH>(s2, g2, c0, half, sw, scount, tx, ty, tz, tq, tg, pu, vx, vy, vz, PU, PX,
                                           PY, PZ, thr);
        finish(c0);
      }
      if (c0 < scount) {
        if (mask)
          sv_chunk<MODE, true, false, NPH>(s2, g2, c0, half, sw, scount, tx, ty, tz, tq, tg, pu, vx, vy, vz, PU, PX,
                                           PY, PZ, thr);
        else
          sv_chunk<MODE, false, false, NPH>(s2, g2, c0, half, sw, scount, tx, ty, tz, tq, tg, pu, vx, vy, vz, PU,
                                            PX, PY, PZ, thr);
        finish(c0);
      }
    }
#pragma unroll
    for (int k = 0; k < NPH; k++) {
      float u0, u1;
      f2unpack(pu[k], u0, u1);
      two_sum(hi[2 * k], lo[2 * k], u0);
      two_sum(hi[2 * k + 1], lo[2 * k + 1], u1);
    }
    __syncwarp();
  }
  // combine the two halves
  float fx[NT], fy[NT], fz[NT];
#pragma unroll
  for (int k = 0; k < NPH; k++) {
    f2unpack(vx[k], fx[2 * k], fx[2 * k + 1]);
    f2unpack(vy[k], fy[2 * k], fy[2 * k + 1]);
    f2unpack(vz[k], fz[2 * k], fz[2 * k + 1]);
  }
#pragma unroll
  for (int k = 0; k < NT; k++) {
    const float oh = __shfl_xor_sync(0xffffffffu, hi[k], 16);
    const float ol = __shfl_xor_sync(0xffffffffu, lo[k], 16);
    two_sum(hi[k], lo[k], oh);
    lo[k] += ol;
    fx[k] += __shfl_xor_sync(0xffffffffu, fx[k], 16);
    fy[k] += __shfl_xor_sync(0xffffffffu, fy[k], 16);
    fz[k] += __shfl_xor_sync(0xffffffffu, fz[k], 16);
  }
  if (half == 0) {
#pragma unroll
    for (int k = 0; k < NT; k++) {
      const int i = l16 + 16 * k;
      if (i < tcnt) {
        const int64_t pidx = tstart + i;
        a.near_u[2 * pidx] = hi[k];
        a.near_u[2 * pidx + 1] = lo[k];
        a.near_f[3 * pidx] = fx[k];
        a.near_f[3 * pidx + 1] = fy[k];
        a.near_f[3 * pidx + 2] = fz[k];
      }
    }
  }
}

// Gather of the vector variants: every leaf adds the (U, V) rows it received
// (list order) to its sums; chunking as in sym_gather_kernel, partial sums of
// a leaf with several chunks in gpart rows of 8 floats per point
// (U hi, U lo, Vx, Vy, Vz, unused).
__global__ void __launch_bounds__(128) sv_gather_kernel(int64_t n_chunks, const int32_t* __restrict__ gch_leaf,
                                                        const int64_t* __restrict__ gch_r0,
                                                        const int64_t* __restrict__ gch_first,
                                                        const int32_t* __restrict__ leaf_box,
                                                        const int64_t* __restrict__ box_start,
                                                        const int32_t* __restrict__ box_count,
                                                        const int64_t* __restrict__ recv_off,
                                                        const float4* __restrict__ partial, int64_t stride,
                                                        float* __restrict__ near_u, float* __restrict__ near_v,
                                                        float* __restrict__ gpart) {
  const int lane = lane_id();
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x / 32);
  for (int64_t ch = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) / 32; ch < n_chunks; ch += warps) {
    const int64_t leaf = gch_leaf[ch];
    const int64_t r0 = gch_r0[ch], r1 = min(r0 + kGatherChunk, recv_off[leaf + 1]);
    const bool single = gch_first[leaf + 1] - gch_first[leaf] == 1;
    const int64_t g = leaf_box[leaf];
    const int64_t start = box_start[g];
    const int cnt = box_count[g];
    for (int i = lane; i < cnt; i += 32) {
      float h = 0.f, l = 0.f, vx = 0.f, vy = 0.f, vz = 0.f;
      if (single) {
        const int64_t p = start + i;
        h = near_u[2 * p];
        l = near_u[2 * p + 1];
        vx = near_v[3 * p];
        vy = near_v[3 * p + 1];
        vz = near_v[3 * p + 2];
      }
      for (int64_t r = r0; r < r1; r += 8) {
        float4 v[8];
#pragma unroll
        for (int k = 0; k < 8; k++) v[k] = (r + k < r1) ? partial[(r + k) * stride + i] : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
        for (int k = 0; k < 8; k++) {
          if (r + k < r1) {
            two_sum(h, l, v[k].x);
            vx += v[k].y;
            vy += v[k].z;
            vz += v[k].w;
          }
        }
      }
      if (single) {
        const int64_t p = start + i;
        near_u[2 * p] = h;
        near_u[2 * p + 1] = l;
        near_v[3 * p] = vx;
        near_v[3 * p + 1] = vy;
        near_v[3 * p + 2] = vz;
      } else {
        float4* row = reinterpret_cast<float4*>(gpart) + 2 * (ch * stride + i);
        row[0] = make_float4(h, l, vx, vy);
        row[1] = make_float4(vz, 0.f, 0.f, 0.f);
      }
    }
  }
}

// Leaves gathered in several chunks: the chunks' (U, V) sums added in chunk
// order.
__global__ void __launch_bounds__(128) sv_combine_kernel(int64_t n_multi, const int32_t* __restrict__ mleaf,
                                                         const int64_t* __restrict__ gch_first,
                                                         const int32_t* __restrict__ leaf_box,
                                                         const int64_t* __restrict__ box_start,
                                                         const int32_t* __restrict__ box_count, int64_t stride,
                                                         const float* __restrict__ gpart, float* __restrict__ near_u,
                                                         float* __restrict__ near_v) {
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x / 32);
  for (int64_t k = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) / 32; k < n_multi; k += warps) {
    const int64_t leaf = mleaf[k];
    const int64_t g = leaf_box[leaf];
    const int64_t start = box_start[g];
    const int cnt = box_count[g];
    for (int i = threadIdx.x & 31; i < cnt; i += 32) {
      const int64_t p = start + i;
      float h = near_u[2 * p], l = near_u[2 * p + 1];
      float vx = near_v[3 * p], vy = near_v[3 * p + 1], vz = near_v[3 * p + 2];
      for (int64_t ch = gch_first[leaf]; ch < gch_first[leaf + 1]; ch++) {
        const float4* row = reinterpret_cast<const float4*>(gpart) + 2 * (ch * stride + i);
        const float4 a0 = row[0], a1 = row[1];
        two_sum(h, l, a0.x);
        l += a0.y;
        vx += a0.z;
        vy += a0.w;
        vz += a1.x;
      }
      near_u[2 * p] = h;
      near_u[2 * p + 1] = l;
      near_v[3 * p] = vx;
      near_v[3 * p + 1] = vy;
      near_v[3 * p + 2] = vz;
    }
  }
}

template <int TPL>
__global__ void __launch_bounds__(128) p2p_kernel_f64s(P2PArgs a) {
  constexpr int CAP = TPL * 32;
  constexpr int WARPS = 4;
  extern __shared__ __align__(128) unsigned char p2p_smem[];
  dvec4 (*sbuf)[2][CAP] = reinterpret_cast<dvec4 (*)[2][CAP]>(p2p_smem);
  __shared__ __align__(8) uint64_t bars[WARPS][2];
  const dvec4* tile = reinterpret_cast<const dvec4*>(a.tile);
  const int lane = lane_id();
  const int warp = threadIdx.x >> 5;
  uint64_t* bar = bars[warp];
  if (lane == 0) {
    mbar_init(&bar[0]);
    mbar_init(&bar[1]);
    fence_barrier_init();
  }
  __syncwarp();
  const int64_t t = (int64_t)blockIdx.x * WARPS + warp;
  if (t >= a.n_leaves) return;
  const int64_t leaf = a.order[t];
  const int64_t g = a.leaf_box[leaf];
  const int64_t tstart = a.box_start[g];
  const int tcnt = a.box_count[g];
  const dvec4* tsrc = reinterpret_cast<const dvec4*>(a.src);
  double tx[TPL], ty[TPL], tz[TPL], tq[TPL], u[TPL];
#pragma unroll
  for (int k = 0; k < TPL; k++) {
    const int i = lane + 32 * k;
    if (i < tcnt) {
      const dvec4 p = tsrc[tstart + i];
      tx[k] = p.x;
      ty[k] = p.y;
      tz[k] = p.z;
      tq[k] = p.w;
    } else {
      tx[k] = ty[k] = tz[k] = tq[k] = 0.0;
    }
    u[k] = 0.0;
  }
  const int64_t kb = a.work_off[leaf];
  const int nwk = (int)(a.work_off[leaf + 1] - kb);
  SymRec mine{};
  auto load_batch = [&](int base) {
    if (base + lane < nwk) mine = a.rec[kb + base + lane];
  };
  auto bcast = [&](int src_lane) {
    SymRec r;
    r.start = __shfl_sync(0xffffffffu, mine.start, src_lane);
    r.count = __shfl_sync(0xffffffffu, mine.count, src_lane);
    r.slot = __shfl_sync(0xffffffffu, mine.slot, src_lane);
    r.thr = __shfl_sync(0xffffffffu, mine.thr, src_lane);
    return r;
  };
  auto issue = [&](const SymRec& r, int buf) {
    if (lane == 0) {
      fence_proxy_async();
      tma_load_1d(sbuf[warp][buf], tile + r.start, (uint32_t)(r.count * sizeof(dvec4)), &bar[buf]);
    }
  };
  uint32_t phase = 0;
  if (nwk > 0) {
    load_batch(0);
    issue(bcast(0), 0);
  }
  for (int w = 0; w < nwk; w++) {
    const int buf = w & 1;
    if (w > 0 && (w & 31) == 0) load_batch(w);  // warp-uniform
    const SymRec en = bcast(w & 31);
    if (w + 1 < nwk) {
      const SymRec nx = ((w + 1) & 31) ? bcast((w + 1) & 31) : a.rec[kb + w + 1];
      issue(nx, buf ^ 1);
    }
    if (!mbar_wait(&bar[buf], (phase >> buf) & 1u, a.wait_cycles)) {
      if (lane == 0) atomicOr(a.status, ST_TIMEOUT);
      // copies still in flight into this warp's buffers must land first
      mbar_wait(&bar[buf], (phase >> buf) & 1u, kDrainWaitCycles);
      if (w + 1 < nwk) mbar_wait(&bar[buf ^ 1], (phase >> (buf ^ 1)) & 1u, kDrainWaitCycles);
      return;
    }
    phase ^= 1u << buf;
    const int scount = en.count;
    const bool mask = en.thr >= 0.f;  // coincident points possible: exact zero test
    const dvec4* sb = sbuf[warp][buf];
    if (en.slot < 0) {
      // one-sided: the self pair and pairs listed in one direction only
#pragma unroll 2
      for (int j = 0; j < scount; j++) {
        const dvec4 s = sb[j];
#pragma unroll
        for (int k = 0; k < TPL; k++) {
          const double dx = tx[k] - s.x, dy = ty[k] - s.y, dz = tz[k] - s.z;
          const double r2 = fma(dz, dz, fma(dy, dy, dx * dx));
          double ri = rsqrt_f64(r2);
          if (mask) ri = (r2 > 0.0) ? ri : 0.0;
          u[k] = fma(s.w, ri, u[k]);
        }
      }
    } else {
      double* dst = reinterpret_cast<double*>(a.partial) + (int64_t)en.slot * a.stride;
      for (int c0 = 0; c0 < scount; c0 += 16) {
        double P[16];
#pragma unroll
        for (int jj = 0; jj < 16; jj++) {
          const int j = c0 + jj;
          P[jj] = 0.0;
          if (j < scount) {
            const dvec4 s = sb[j];
            double acc = 0.0;
#pragma unroll
            for (int k = 0; k < TPL; k++) {
              const double dx = tx[k] - s.x, dy = ty[k] - s.y, dz = tz[k] - s.z;
              const double r2 = fma(dz, dz, fma(dy, dy, dx * dx));
              double ri = rsqrt_f64(r2);
              if (mask) ri = (r2 > 0.0) ? ri : 0.0;
              u[k] = fma(s.w, ri, u[k]);
              acc = fma(tq[k], ri, acc);
            }
            P[jj] = acc;
          }
        }
        // reduce-scatter over lane bits 4..1: lane l ends with P[l >> 1]
#pragma unroll
        for (int m = 16, h = 8; h >= 1; m >>= 1, h >>= 1) {
          const bool up = (lane & m) != 0;
#pragma unroll
          for (int i = 0; i < h; i++) {
            const double keep = up ? P[i + h] : P[i];
            const double send = up ? P[i] : P[i + h];
            P[i] = keep + __shfl_xor_sync(0xffffffffu, send, m);
          }
        }
        P[0] += __shfl_xor_sync(0xffffffffu, P[0], 1);
        const int j = c0 + (lane >> 1);
        if ((lane & 1) == 0 && j < scount) dst[j] = P[0];
      }
    }
    __syncwarp();
  }
  double* near = reinterpret_cast<double*>(a.near_u);
#pragma unroll
  for (int k = 0; k < TPL; k++) {
    const int i = lane + 32 * k;
    if (i < tcnt) near[tstart + i] = u[k];
  }
}

// FP64 counterpart of sym_gather_kernel: plain FP64 sums in list order.
// FP64: as sym_gather_kernel / sym_combine_kernel with FP64 sums
__global__ void __launch_bounds__(128) sym_gather_f64_kernel(int64_t n_chunks, const int32_t* __restrict__ gch_leaf,
                                                             const int64_t* __restrict__ gch_r0,
                                                             const int64_t* __restrict__ gch_first,
                                                             const int32_t* __restrict__ leaf_box,
                                                             const int64_t* __restrict__ box_start,
                                                             const int32_t* __restrict__ box_count,
                                                             const int64_t* __restrict__ recv_off,
                                                             const double* __restrict__ partial, int64_t stride,
                                                             double* __restrict__ near_u, double* __restrict__ gpart) {
  const int lane = lane_id();
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x / 32);
  for (int64_t ch = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) / 32; ch < n_chunks; ch += warps) {
    const int64_t leaf = gch_leaf[ch];
    const int64_t r0 = gch_r0[ch], r1 = min(r0 + kGatherChunk, recv_off[leaf + 1]);
    const bool single = gch_first[leaf + 1] - gch_first[leaf] == 1;
    const int64_t g = leaf_box[leaf];
    const int64_t start = box_start[g];
    const int cnt = box_count[g];
    for (int i = lane; i < cnt; i += 32) {
      double acc = single ? near_u[start + i] : 0.0;
      for (int64_t r = r0; r < r1; r += 8) {
        double v[8];
#pragma unroll
        for (int k = 0; k < 8; k++) v[k] = (r + k < r1) ? partial[(r + k) * stride + i] : 0.0;
#pragma unroll
        for (int k = 0; k < 8; k++)
          if (r + k < r1) acc += v[k];
      }
      if (single) near_u[start + i] = acc;
      else gpart[ch * stride + i] = acc;
    }
  }
}

__global__ void __launch_bounds__(128) sym_combine_f64_kernel(int64_t n_multi, const int32_t* __restrict__ mleaf,
                                                              const int64_t* __restrict__ gch_first,
                                                              const int32_t* __restrict__ leaf_box,
                                                              const int64_t* __restrict__ box_start,
                                                              const int32_t* __restrict__ box_count, int64_t stride,
                                                              const double* __restrict__ gpart,
                                                              double* __restrict__ near_u) {
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x / 32);
  for (int64_t k = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) / 32; k < n_multi; k += warps) {
    const int64_t leaf = mleaf[k];
    const int64_t g = leaf_box[leaf];
    const int64_t start = box_start[g];
    const int cnt = box_count[g];
    for (int i = threadIdx.x & 31; i < cnt; i += 32) {
      double acc = near_u[start + i];
      for (int64_t ch = gch_first[leaf]; ch < gch_first[leaf + 1]; ch++) acc += gpart[ch * stride + i];
      near_u[start + i] = acc;
    }
  }
}

// ---- E6 (FP64DF, potential, one point set): double-float symmetric near field --
// FP64 accuracy on the FP32 pipes (GB300 runs FP64 at 1/64 of the FP32 rate).
// Values are unevaluated sums h + l of two FP32 numbers.  Positions live in
// the frame of the source leaf (offsets from its centre, FP64, split h + l);
// differences of hi parts are taken exactly by two-sum (Knuth), so the
// difference carries about 2^-48 of the larger offset.  r^2 is summed with
// two-sum error terms, 1/r is the MUFU seed y refined by y (1 + rho / 2) with
// rho = 1 - r^2 y^2 evaluated from FMA product errors, and the sums are
// accumulated as renormalised (h, l) pairs.  Lane and slot layout as in
// p2p_kernel_f64s (lane l holds targets l + 32 k).
struct dfl {
  float h, l;
};

__device__ __forceinline__ dfl df_two_sum(float a, float b) {
  const float s = a + b;
  const float bb = s - a;
  return dfl{s, (a - (s - bb)) + (b - bb)};
}

// acc += p + pe, renormalised (|l| <= ulp(h) / 2) so that the rounding of
// later additions to l stays at 2^-48 of the sum
__device__ __forceinline__ void df_acc(dfl& acc, float p, float pe) {
  const dfl s = df_two_sum(acc.h, p);
  const float l = acc.l + s.l + pe;
  acc.h = s.h + l;
  acc.l = l - (acc.h - s.h);
}

// 1/|t - s| as y + yl for target (th, tl) and source (sh, sl) in one frame;
// zero for coincident points when MASK.
template <bool MASK>
__device__ __forceinline__ void df_rinv(const float (&th)[3], const float (&tl)[3], const float4& sh,
                                        const float4& sl, float& y, float& yl) {
  const dfl dx = df_two_sum(th[0], -sh.x), dy = df_two_sum(th[1], -sh.y), dz = df_two_sum(th[2], -sh.z);
  const float ax = dx.h, ay = dy.h, az = dz.h;
  const float bx = dx.l + (tl[0] - sl.x), by = dy.l + (tl[1] - sl.y), bz = dz.l + (tl[2] - sl.z);
  const float px = ax * ax, py = ay * ay, pz = az * az;
  float ex = fmaf(ax, ax, -px), ey = fmaf(ay, ay, -py), ez = fmaf(az, az, -pz);
  ex = fmaf(bx, bx, fmaf(ax + ax, bx, ex));
  ey = fmaf(by, by, fmaf(ay + ay, by, ey));
  ez = fmaf(bz, bz, fmaf(az + az, bz, ez));
  const dfl s1 = df_two_sum(px, py);
  const dfl s2 = df_two_sum(s1.h, pz);
  const float e = ((ex + ey) + ez) + (s1.l + s2.l);
  const float rh = s2.h + e;
  const float rl = e - (rh - s2.h);
  y = rsqrt_mufu(rh);
  const float w = y * y, we = fmaf(y, y, -w);
  const float t1 = rh * w;
  const float t1e = fmaf(rh, we, fmaf(rl, w, fmaf(rh, w, -t1)));
  const float rho = (1.f - t1) - t1e;
  yl = y * (0.5f * rho);
  if (MASK && !(rh > 0.f)) y = yl = 0.f;
}

template <int TPL>
__global__ void __launch_bounds__(128, TPL <= 2 ? 5 : 1) p2p_kernel_dfs(P2PArgs a) {
  constexpr int CAP = TPL * 32;
  constexpr int WARPS = 4;
  extern __shared__ __align__(128) unsigned char p2p_smem[];
  DFRec (*sbuf)[2][CAP] = reinterpret_cast<DFRec (*)[2][CAP]>(p2p_smem);
  __shared__ __align__(8) uint64_t bars[WARPS][2];
  const DFRec* tile = a.df_tile;
  const int lane = lane_id();
  const int warp = threadIdx.x >> 5;
  uint64_t* bar = bars[warp];
  if (lane == 0) {
    mbar_init(&bar[0]);
    mbar_init(&bar[1]);
    fence_barrier_init();
  }
  __syncwarp();
  const int64_t t = (int64_t)blockIdx.x * WARPS + warp;
  if (t >= a.n_leaves) return;
  const int64_t leaf = a.order[t];
  const int64_t g = a.leaf_box[leaf];
  const int64_t tstart = a.box_start[g];
  const int tcnt = a.box_count[g];
  // FP64 target positions are re-read per entry (L1/L2 hits) to keep
  // registers for the double-float state
  const dvec4* tsrc = reinterpret_cast<const dvec4*>(a.src) + tstart;
  dfl tq[TPL], u[TPL];
#pragma unroll
  for (int k = 0; k < TPL; k++) {
    const int i = lane + 32 * k;
    tq[k] = dfl{0.f, 0.f};
    if (i < tcnt) {
      const DFRec r = a.df_tile[tstart + i];
      tq[k] = dfl{r.qh, r.ql};
    }
    u[k] = dfl{0.f, 0.f};
  }
  const int64_t kb = a.work_off[leaf];
  const int nwk = (int)(a.work_off[leaf + 1] - kb);
  SymRec mine{};
  SymFrame mframe{};
  auto load_batch = [&](int base) {
    if (base + lane < nwk) {
      mine = a.rec[kb + base + lane];
      mframe = a.frame[kb + base + lane];
    }
  };
  auto issue = [&](int64_t start, int count, int buf) {
    if (lane == 0) {
      fence_proxy_async();
      tma_load_1d(sbuf[warp][buf], tile + start, (uint32_t)(count * sizeof(DFRec)), &bar[buf]);
    }
  };
  uint32_t phase = 0;
  if (nwk > 0) {
    load_batch(0);
    issue(__shfl_sync(0xffffffffu, mine.start, 0), __shfl_sync(0xffffffffu, mine.count, 0), 0);
  }
  for (int w = 0; w < nwk; w++) {
    const int buf = w & 1;
    if (w > 0 && (w & 31) == 0) load_batch(w);  // warp-uniform
    const int sl = w & 31;
    const int scount = __shfl_sync(0xffffffffu, mine.count, sl);
    const int slot = __shfl_sync(0xffffffffu, mine.slot, sl);
    const bool mask = __shfl_sync(0xffffffffu, mine.thr, sl) >= 0.f;
    const double cx = __shfl_sync(0xffffffffu, mframe.cx, sl), cy = __shfl_sync(0xffffffffu, mframe.cy, sl),
                 cz = __shfl_sync(0xffffffffu, mframe.cz, sl);
    if (w + 1 < nwk) {
      int64_t ns;
      int nc;
      if ((w + 1) & 31) {
        ns = __shfl_sync(0xffffffffu, mine.start, (w + 1) & 31);
        nc = __shfl_sync(0xffffffffu, mine.count, (w + 1) & 31);
      } else {
        const SymRec nx = a.rec[kb + w + 1];
        ns = nx.start;
        nc = nx.count;
      }
      issue(ns, nc, buf ^ 1);
    }
    // targets in the source leaf's frame, split as the source records were
    // (coincident points get identical splits); absent targets far away
    float th[TPL][3], tl[TPL][3];
#pragma unroll
    for (int k = 0; k < TPL; k++) {
      const int i = lane + 32 * k;
      const dvec4 p = i < tcnt ? tsrc[i] : dvec4{cx + 1e18, cy, cz, 0.0};
      const double d[3] = {p.x - cx, p.y - cy, p.z - cz};
#pragma unroll
      for (int c = 0; c < 3; c++) {
        const float h = (float)d[c];
        th[k][c] = h;
        tl[k][c] = (float)(d[c] - (double)h);
      }
    }
    if (!mbar_wait(&bar[buf], (phase >> buf) & 1u, a.wait_cycles)) {
      if (lane == 0) atomicOr(a.status, ST_TIMEOUT);
      // copies still in flight into this warp's buffers must land first
      mbar_wait(&bar[buf], (phase >> buf) & 1u, kDrainWaitCycles);
      if (w + 1 < nwk) mbar_wait(&bar[buf ^ 1], (phase >> (buf ^ 1)) & 1u, kDrainWaitCycles);
      return;
    }
    phase ^= 1u << buf;
    const float4* sb = reinterpret_cast<const float4*>(sbuf[warp][buf]);
    if (slot < 0) {
      // one-sided: the self pair and pairs listed in one direction only
      for (int j = 0; j < scount; j++) {
        const float4 sh = sb[2 * j], slo = sb[2 * j + 1];  // (xh, yh, zh, qh), (xl, yl, zl, ql)
#pragma unroll
        for (int k = 0; k < TPL; k++) {
          float y, yl;
          if (mask) df_rinv<true>(th[k], tl[k], sh, slo, y, yl);
          else df_rinv<false>(th[k], tl[k], sh, slo, y, yl);
          const float p = sh.w * y;
          df_acc(u[k], p, fmaf(sh.w, yl, fmaf(slo.w, y, fmaf(sh.w, y, -p))));
        }
      }
    } else {
      double* dst = reinterpret_cast<double*>(a.partial) + (int64_t)slot * a.stride;
      if constexpr (TPL >= 4) {
        // many targets per lane: one source at a time (compact code), its sum
        // over the warp by a butterfly all-reduce
#pragma unroll 1
        for (int j = 0; j < scount; j++) {
          const float4 sh = sb[2 * j], slo = sb[2 * j + 1];
          dfl acc{0.f, 0.f};
#pragma unroll
          for (int k = 0; k < TPL; k++) {
            float y, yl;
            if (mask) df_rinv<true>(th[k], tl[k], sh, slo, y, yl);
            else df_rinv<false>(th[k], tl[k], sh, slo, y, yl);
            const float p = sh.w * y;
            df_acc(u[k], p, fmaf(sh.w, yl, fmaf(slo.w, y, fmaf(sh.w, y, -p))));
            const float pq = tq[k].h * y;
            df_acc(acc, pq, fmaf(tq[k].h, yl, fmaf(tq[k].l, y, fmaf(tq[k].h, y, -pq))));
          }
#pragma unroll
          for (int m = 16; m >= 1; m >>= 1) {
            const float rh = __shfl_xor_sync(0xffffffffu, acc.h, m);
            const float rl = __shfl_xor_sync(0xffffffffu, acc.l, m);
            df_acc(acc, rh, rl);
          }
          if (lane == 0) dst[j] = (double)acc.h + (double)acc.l;
        }
      } else {
        // the mask decided once per entry: each variant's unrolled chunk
        // loop is one contiguous stretch of code (instruction-cache footprint)
        auto chunks = [&](auto mk) {
          constexpr bool MK = decltype(mk)::value;
          for (int c0 = 0; c0 < scount; c0 += 16) {
            dfl P[16];
#pragma unroll
            for (int jj = 0; jj < 16; jj++) {
              const int j = c0 + jj;
              P[jj] = dfl{0.f, 0.f};
              if (j < scount) {
                const float4 sh = sb[2 * j], slo = sb[2 * j + 1];
#pragma unroll
                for (int k = 0; k < TPL; k++) {
                  float y, yl;
                  df_rinv<MK>(th[k], tl[k], sh, slo, y, yl);
                  const float p = sh.w * y;
                  df_acc(u[k], p, fmaf(sh.w, yl, fmaf(slo.w, y, fmaf(sh.w, y, -p))));
                  const float pq = tq[k].h * y;
                  df_acc(P[jj], pq, fmaf(tq[k].h, yl, fmaf(tq[k].l, y, fmaf(tq[k].h, y, -pq))));
                }
              }
            }
            // reduce-scatter over lane bits 4..1 (lane l ends with P[l >> 1]), then the lane pair
#pragma unroll
            for (int m = 16, hh = 8; hh >= 1; m >>= 1, hh >>= 1) {
              const bool up = (lane & m) != 0;
#pragma unroll
              for (int i = 0; i < hh; i++) {
                const dfl keep = up ? P[i + hh] : P[i];
                const dfl send = up ? P[i] : P[i + hh];
                const float rh = __shfl_xor_sync(0xffffffffu, send.h, m);
                const float rl = __shfl_xor_sync(0xffffffffu, send.l, m);
                P[i] = keep;
                df_acc(P[i], rh, rl);
              }
            }
            {
              const float rh = __shfl_xor_sync(0xffffffffu, P[0].h, 1);
              const float rl = __shfl_xor_sync(0xffffffffu, P[0].l, 1);
              df_acc(P[0], rh, rl);
            }
            const int j = c0 + (lane >> 1);
            if ((lane & 1) == 0 && j < scount) dst[j] = (double)P[0].h + (double)P[0].l;
          }
        };
        if (mask) chunks(std::true_type{});
        else chunks(std::false_type{});
      }
    }
    __syncwarp();
  }
  double* near = reinterpret_cast<double*>(a.near_u);
#pragma unroll
  for (int k = 0; k < TPL; k++) {
    const int i = lane + 32 * k;
    if (i < tcnt) near[tstart + i] = (double)u[k].h + (double)u[k].l;
  }
}

// Inputs of one point of the local evaluation (position and charge record,
// near-field sum, output index, near field), zero beyond the leaf's count.
struct PointIn {
  vec4 s;
  double nearv;
  real nf[3];
  int32_t o;
};
template <bool FIELD>
__device__ __forceinline__ PointIn l2p_point_in(const vec4* __restrict__ src, const real* __restrict__ near_u,
                                                const real* __restrict__ near_f, const int32_t* __restrict__ perm,
                                                int64_t start, int i, int cnt) {
  PointIn r{};
  if (i < cnt) {
    const int64_t pidx = start + i;
    r.s = src[pidx];
    // no near sums (NULL): the far field alone
    if (near_u) r.nearv = kF32 ? (double)near_u[2 * pidx] + (double)near_u[2 * pidx + 1] : (double)near_u[pidx];
    r.o = perm[pidx];
    if (FIELD && near_f) {
      r.nf[0] = near_f[3 * pidx];
      r.nf[1] = near_f[3 * pidx + 1];
      r.nf[2] = near_f[3 * pidx + 2];
    }
  }
  return r;
}

// ---- E5 + E7: L2P, near + far combination and inverse sort --------------------
// u = -1/(4 pi) (far + near);  E = -grad u = 1/(4 pi) (grad far - sum q d / r^3).
template <int P, bool FIELD>
__global__ void __launch_bounds__(128) l2p_kernel(int64_t n_leaves, const int32_t* __restrict__ leaf_box,
                                                  const int64_t* __restrict__ box_start,
                                                  const int32_t* __restrict__ box_count,
                                                  const double* __restrict__ center,
                                                  const int32_t* __restrict__ perm, int64_t out_base,
                                                  const vec4* __restrict__ src,
                                                  const real* __restrict__ inv_rho,
                                                  const real* __restrict__ Lam,
                                                  const real* __restrict__ near_u,
                                                  const real* __restrict__ near_f,
                                                  double* __restrict__ u_out,
                                                  double* __restrict__ f_out) {
  constexpr int NC = ncoef(P);
  constexpr int NG = P * P;  // gradient coefficients reach degree P-1
  __shared__ real sL[4][NC];
  __shared__ real sG[4][FIELD ? 3 * NG : 1];
  const int lane = lane_id();
  const int warp = threadIdx.x >> 5;
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x / 32);
  for (int64_t leaf = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) / 32; leaf < n_leaves;
       leaf += warps) {
    const int64_t g = leaf_box[leaf];
    // box data (and in the field variant the lane's first point) are
    // requested before the shared copy of the local expansion completes
    const int64_t start = box_start[g];
    const int cnt = box_count[g];
    const real ir = inv_rho[g];
    real cx = 0, cy = 0, cz = 0;
    if (!kF32) {
      cx = (real)center[3 * g];
      cy = (real)center[3 * g + 1];
      cz = (real)center[3 * g + 2];
    }
    // the field variant keeps the next point's inputs in flight during the
    // current one (measured: field 4.92 -> 4.87 ms at 2^20); the potential
    // variant is register-limited and loads each point when it starts
    constexpr bool kAhead = FIELD;
    PointIn nxt{};
    if (kAhead) nxt = l2p_point_in<FIELD>(src, near_u, near_f, perm, start, lane, cnt);
    const real* L = Lam + g * ncoef_pad(P);
    for (int c = lane; c < NC; c += 32) sL[warp][c] = L[c];
    __syncwarp();
    if (FIELD) {
      // per-leaf differentiated locals: d/dx, d/dy, d/dz of sum w L Rt as
      // sums of G Rt over degrees < P (ladder relations of the regular basis)
      for (int id = lane; id < NG; id += 32) {
        int n1 = 0;
        while ((n1 + 1) * (n1 + 1) <= id) n1++;
        const int m = id - n1 * n1 - n1;
        const int n = n1 + 1;
        const int mp = m < 0 ? -m : m;
        const real kp = sqrt((real)((n + mp + 1) * (n + mp)));
        const real km = sqrt((real)((n - mp + 1) * (n - mp)));
        const real kz = sqrt((real)((n - mp) * (n + mp)));
        auto Lv = [&](int mm) -> real { return sL[warp][n * n + n + mm]; };
        real gx, gy, gz;
        if (m >= 0) {
          gx = kp * Lv(mp + 1) - (mp >= 1 ? km * Lv(mp - 1) : real(0));
          gy = -(kp * Lv(-(mp + 1)) + (mp >= 2 ? km * Lv(-(mp - 1)) : real(0)));
          gz = (mp == 0 ? real(1) : real(2)) * kz * Lv(mp);
        } else {
          gx = kp * Lv(-(mp + 1)) - (mp >= 2 ? km * Lv(-(mp - 1)) : real(0));
          gy = kp * Lv(mp + 1) + km * Lv(mp - 1);
          gz = real(2) * kz * Lv(-mp);
        }
        sG[warp][id] = gx;
        sG[warp][NG + id] = gy;
        sG[warp][2 * NG + id] = gz;
      }
      __syncwarp();
    }
    for (int i = lane; i < cnt; i += 32) {
      PointIn cur;
      if (kAhead) {
        cur = nxt;
        nxt = l2p_point_in<FIELD>(src, near_u, near_f, perm, start, i + 32, cnt);  // next point, in flight
      } else {
        cur = l2p_point_in<FIELD>(src, near_u, near_f, perm, start, i, cnt);
      }
      const vec4 s = cur.s;
      const real x = ((real)s.x - cx) * ir, y = ((real)s.y - cy) * ir, z = ((real)s.z - cz) * ir;
      real u0 = real(0), um = real(0), gx = real(0), gy = real(0), gz = real(0);
      real R[NC];
      regular_basis<P>(x, y, z, R, [&](auto nn) {
        constexpr int n = decltype(nn)::value;
        u0 = fmar(sL[warp][n * n + n], R[n * n + n], u0);
#pragma unroll
        for (int c = n * n; c < (n + 1) * (n + 1); c++)
          if (c != n * n + n) um = fmar(sL[warp][c], R[c], um);
        if (FIELD && n < P) {
#pragma unroll
          for (int c = n * n; c < (n + 1) * (n + 1); c++) {
            gx = fmar(sG[warp][c], R[c], gx);
            gy = fmar(sG[warp][NG + c], R[c], gy);
            gz = fmar(sG[warp][2 * NG + c], R[c], gz);
          }
        }
      });
      const double far = (double)u0 + 2.0 * (double)um;
      const int64_t o = cur.o - out_base;
      if (u_out) u_out[o] = -kInv4Pi * (far + cur.nearv);
      if (FIELD) {
        const double irr = (double)ir;
        f_out[3 * o] = kInv4Pi * ((double)gx * irr - (double)cur.nf[0]);
        f_out[3 * o + 1] = kInv4Pi * ((double)gy * irr - (double)cur.nf[1]);
        f_out[3 * o + 2] = kInv4Pi * ((double)gz * irr - (double)cur.nf[2]);
      }
    }
    __syncwarp();
  }
}

// ---- host side ----------------------------------------------------------------
struct Ptrs {
  vec4* pos;
  vec4* src;
  const real* inv_rho;
  const real* geo;
  const real* m2m;
  const real* l2d;  // direct L2L records
  real* M;
  real* Lam;
};

Ptrs ptrs(const fmm_tree* t);

// Upward pass: P2M on the leaves, then M2M round by round (round r holds
// the child boxes r levels above the leaves of every tree in the batch).
template <int P>
void run_upward(const fmm_tree* t, const Ptrs& pp, cudaStream_t st) {
  const int nch = 1 << t->s;
  stage_event(t, FMM_STAGE_P2M, false, st);
  p2m_kernel<P><<<grid_for(t->n_src_leaves * kP2MGroup, 128, 1 << 30), 128, 0, st>>>(
      t->n_src_leaves, t->src_leaf_box, t->box_start, t->box_count, t->center, pp.src, pp.inv_rho, pp.M);
  FMM_LAUNCH_CHECK();
  t->launches += 1 + t->n_up;
  stage_event(t, FMM_STAGE_P2M, true, st);
  stage_event(t, FMM_STAGE_M2M, false, st);
  if (t->m2m_ready && t->opt_m2m_one_launch && t->n_up > 1 && t->n_up <= kMaxRounds) {
    // every round in one launch (readiness flags cleared by the gather)
    RoundTab rt{};
    rt.n = t->n_up;
    rt.pad[0] = 0;
    for (int r = 0; r < t->n_up; r++) {
      rt.off[r] = t->up_off_h[r];
      rt.pad[r + 1] = rt.pad[r] + (t->up_off_h[r + 1] - t->up_off_h[r] + 31) / 32 * 32;
    }
    rt.off[t->n_up] = t->up_off_h[t->n_up];
    int dev = 0, nsm = 0, occ = 0;
    FMM_CUDA_TRY(cudaGetDevice(&dev));
    FMM_CUDA_TRY(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    // one block per SM: the rounds are short and the near field runs beside
    int64_t blocks = std::min<int64_t>(nsm, (rt.pad[rt.n] + 127) / 128);
    m2m_persistent_kernel<P><<<(int)std::max<int64_t>(blocks, 1), 128, 0, st>>>(
        rt, t->up_ids, t->box_parent, nch, pp.m2m, t->n_boxes, pp.M, t->m2m_ready, t->counters + 2, t->status,
        t->wait_cycles);
    FMM_LAUNCH_CHECK();
    t->launches += 1 - t->n_up;
  } else {
    for (int r = 0; r < t->n_up; r++) {
      const int64_t nchild = t->up_off_h[r + 1] - t->up_off_h[r];
      m2m_kernel<P><<<grid_for(nchild, 128, 1 << 30), 128, 0, st>>>(nchild, t->up_ids + t->up_off_h[r],
                                                                   t->box_parent, nch, pp.m2m, t->n_boxes, pp.M);
      FMM_LAUNCH_CHECK();
    }
  }
  stage_event(t, FMM_STAGE_M2M, true, st);
}

// Order of the stages.  The near field and the far field are independent
// until the local evaluation.  All heavy stages (near field, M2L) are FP32
// issue bound, so they run alone at full occupancy; what runs beside the near
// field (on the tree's second, higher-priority stream) is only latency-bound
// work that cannot fill the GPU by itself:
//   kSerial:     P2M, M2M, M2L, L2L, near field, L2P on the caller's stream
//   kUpwardSide: P2M and M2M rounds beside the near field, then M2L, L2L, L2P
//   kFarSide:    P2M, M2M, then M2L and L2L beside the near field (M2L capped at
//                kM2LBlocksPerSM blocks per SM)
// Measured beside the symmetric near field with the level-by-level L2L
// (ms per evaluation, 2^20-point cube / 2^18-point cube / 2^22-point
// Plummer): kFarSide 2.53-2.70 / - / -, kSerial 2.29 / 0.650 / 54.5,
// kUpwardSide 2.20 / 0.622 / 46.7, kSplitNear 2.25 / 0.588 / 55.9.
//   kSplitNear:  the near field in two launches (heaviest leaves first): P2M
//                and M2M beside the first, M2L alone, L2L beside the second,
//                then the slot gather and L2P
enum { kSerial = 0, kUpwardSide = 1, kFarSide = 2, kSplitNear = 3 };
// The order is a tree option (fmm_tree_set_option, FMM_OPT_SCHEDULE; the
// enumerators match its values), kUpwardSide by default.
constexpr int kM2LBlocksPerSM = 1;

// Downward pass: M2L over the whole list, then L2L in direct form.
// FP64DF: the multipoles as double-float pairs, then the double-float M2L
template <int P>
void run_m2l_df(const fmm_tree* t, const Ptrs& pp, cudaStream_t st) {
  const size_t smem = (size_t)4 * 32 * ncoef(P) * sizeof(float2);
  static bool attr_set = false;
  if (!attr_set) {
    FMM_CUDA_TRY(cudaFuncSetAttribute(m2l_kernel_df<P>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    attr_set = true;
  }
  stage_event(t, FMM_STAGE_M2L, false, st);
  const int64_t nm = t->n_boxes * (int64_t)ncoef_pad(P);
  to_dff_kernel<<<grid_for(nm, 256), 256, 0, st>>>(nm, reinterpret_cast<const double*>(pp.M), t->m_df);
  FMM_LAUNCH_CHECK();
  int dev = 0, nsm = 0, occ = 0;
  FMM_CUDA_TRY(cudaGetDevice(&dev));
  FMM_CUDA_TRY(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  FMM_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, m2l_kernel_df<P>, 128, smem));
  if (occ < 1) occ = 1;
  int64_t blocks = (int64_t)nsm * occ;
  const int64_t need = (t->n_m2l_items + 3) / 4;
  if (blocks > need) blocks = need;
  m2l_kernel_df<P><<<(int)blocks, 128, smem, st>>>(t->n_m2l_items, t->m2l_items, t->m2l_src, t->geo32,
                                                   t->geo_lo, t->n_m2l, t->m_df,
                                                   reinterpret_cast<double*>(pp.Lam), t->m2l_partial, t->counters);
  FMM_LAUNCH_CHECK();
  t->launches += 2;
  if (t->n_m2l_split > 0) {
    m2l_combine_kernel<double><<<grid_for(t->n_m2l_split * 32, 128), 128, 0, st>>>(
        t->n_m2l_split, t->m2l_split_g, t->m2l_split_row, ncoef_pad(P), t->m2l_partial,
        reinterpret_cast<double*>(pp.Lam));
    FMM_LAUNCH_CHECK();
    t->launches += 1;
  }
  stage_event(t, FMM_STAGE_M2L, true, st);
}

template <int P>
void run_m2l(const fmm_tree* t, const Ptrs& pp, cudaStream_t st, bool df_far = false) {
  // the double-float M2L up to p = 8 (2^20 cube, p = 8: 11.1 ms against
  // 18.8 ms in FP64); at p = 10 its register spills make it slower (24.7 ms
  // against 20.1 ms on the paper's set 3), so FP64 from p = 9 on
  if constexpr (!kF32 && P <= 8) {
    if (df_far && t->geo_lo && t->m_df) {
      run_m2l_df<P>(t, pp, st);
      return;
    }
  }
  const size_t smem = (size_t)4 * 32 * m2l_chunks<P>() * 16;
  static bool attr_set = false;
  if (!attr_set) {
    FMM_CUDA_TRY(cudaFuncSetAttribute(m2l_kernel<P>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    attr_set = true;
  }
  stage_event(t, FMM_STAGE_M2L, false, st);
  int dev = 0, nsm = 0, occ = 0;
  FMM_CUDA_TRY(cudaGetDevice(&dev));
  FMM_CUDA_TRY(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  FMM_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, m2l_kernel<P>, 128, smem));
  if (occ < 1) occ = 1;
  if (t->opt_schedule == kFarSide && occ > kM2LBlocksPerSM) occ = kM2LBlocksPerSM;
  if (t->opt_m2l_blocks_per_sm > 0 && occ > t->opt_m2l_blocks_per_sm) occ = t->opt_m2l_blocks_per_sm;
  int64_t blocks = (int64_t)nsm * occ;
  const int64_t need = (t->n_m2l_items + 3) / 4;
  if (blocks > need) blocks = need;
  real* partial = reinterpret_cast<real*>(t->m2l_partial);
  m2l_kernel<P><<<(int)blocks, 128, smem, st>>>(t->n_m2l_items, t->m2l_items, t->m2l_src, pp.geo, t->n_m2l, pp.M,
                                                pp.Lam, partial, t->counters);
  FMM_LAUNCH_CHECK();
  t->launches += 1;
  if (t->n_m2l_split > 0) {
    m2l_combine_kernel<real><<<grid_for(t->n_m2l_split * 32, 128), 128, 0, st>>>(
        t->n_m2l_split, t->m2l_split_g, t->m2l_split_row, ncoef_pad(P), partial, pp.Lam);
    FMM_LAUNCH_CHECK();
    t->launches += 1;
  }
  stage_event(t, FMM_STAGE_M2L, true, st);
}

// L2L in direct form: one launch over the target leaves
template <int P>
void run_l2l(const fmm_tree* t, const Ptrs& pp, cudaStream_t st) {
  stage_event(t, FMM_STAGE_L2L, false, st);
  const size_t l2l_smem = (size_t)128 * m2l_chunks<P>() * 16;
  static bool attr_set = false;
  if (!attr_set) {
    FMM_CUDA_TRY(
        cudaFuncSetAttribute(l2l_direct_kernel<P>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)l2l_smem));
    attr_set = true;
  }
  if (t->n_l2d > 0) {
    l2l_direct_kernel<P><<<grid_for(t->n_leaves * kL2LGroup, 128, 1 << 30), 128, l2l_smem, st>>>(
        t->n_leaves, t->leaf_box, t->l2d_off, t->l2d_anc, pp.l2d, t->n_l2d, pp.Lam);
    FMM_LAUNCH_CHECK();
    t->launches += 1;
  }
  stage_event(t, FMM_STAGE_L2L, true, st);
}

template <int P>
void run_downward(const fmm_tree* t, const Ptrs& pp, cudaStream_t st, bool df_far = false) {
  run_m2l<P>(t, pp, st, df_far);
  run_l2l<P>(t, pp, st);
}

// Does this evaluation use the symmetric near field (whose received slots a
// gather adds before the local evaluation)?  Fields: the FP32C vector variant,
// once its slot buffers exist (leaves of at most 128 points).
bool uses_sym(const fmm_tree* t, bool field) {
  if (!t->sym || !t->opt_near_sym) return false;
  if (!field) return true;
  return kF32 && t->sym_partial4 != nullptr && t->max_leaf <= 128;
}

template <int P>
void run_l2p(const fmm_tree* t, const Ptrs& pp, const real* near_u, const real* near_f, double* u,
             double* field, cudaStream_t st) {
  t->launches += 1;
  if (field)
    l2p_kernel<P, true><<<grid_for(t->n_leaves * 32, 128), 128, 0, st>>>(
        t->n_leaves, t->leaf_box, t->box_start, t->box_count, t->center, t->perm, t->out_base, pp.src, pp.inv_rho,
        pp.Lam, near_u, near_f, u, field);
  else
    l2p_kernel<P, false><<<grid_for(t->n_leaves * 32, 128), 128, 0, st>>>(
        t->n_leaves, t->leaf_box, t->box_start, t->box_count, t->center, t->perm, t->out_base, pp.src, pp.inv_rho,
        pp.Lam, near_u, near_f, u, field);
  FMM_LAUNCH_CHECK();
}

template <int TPL>
void run_p2p_tpl(const fmm_tree* t, const Ptrs& pp, real* near_u, real* near_f, bool field, int64_t lb,
                 int64_t le, cudaStream_t st) {
  P2PArgs a{};
  a.n_leaves = le - lb;  // positions lb .. le - 1 of the work order
  a.leaf_box = t->leaf_box;
  a.src_leaf_box = t->src_leaf_box;
  a.self_pairs = t->two_trees ? 0 : 1;
  a.order = t->leaf_order + lb;
  a.off = t->p2p_off;
  a.ent32 = t->p2p32;
  a.thr = t->p2p_thr;
  a.ent_src = t->p2p_src;
  a.box_start = t->box_start;
  a.box_count = t->box_count;
  a.src = pp.src;
  a.tile = kF32 ? (const void*)t->src_dup : (const void*)pp.src;
  a.near_u = near_u;
  a.near_f = near_f;
  a.counter = t->counters + 1;
  a.status = t->status;
  a.wait_cycles = t->wait_cycles;
  const size_t smem = (size_t)4 * 2 * TPL * 32 * 32;  // 32-byte records
  t->launches += 1;
  if constexpr (kF32) {
    static bool attr_set = false;
    if (!attr_set) {
      FMM_CUDA_TRY(cudaFuncSetAttribute(p2p_kernel_f32h<TPL, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
      FMM_CUDA_TRY(cudaFuncSetAttribute(p2p_kernel_f32h<TPL, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
      FMM_CUDA_TRY(cudaFuncSetAttribute(p2p_kernel_f32h<TPL, true>, cudaFuncAttributePreferredSharedMemoryCarveout,
                                        (int)cudaSharedmemCarveoutMaxShared));
      FMM_CUDA_TRY(cudaFuncSetAttribute(p2p_kernel_f32h<TPL, false>, cudaFuncAttributePreferredSharedMemoryCarveout,
                                        (int)cudaSharedmemCarveoutMaxShared));
      attr_set = true;
    }
    const int64_t blocks = (a.n_leaves + 3) / 4;
    if (!field && t->sym && t->opt_near_sym) {
      static bool sym_attr = false;
      if (!sym_attr) {
        FMM_CUDA_TRY(cudaFuncSetAttribute(p2p_kernel_f32s<TPL>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          (int)smem));
        FMM_CUDA_TRY(cudaFuncSetAttribute(p2p_kernel_f32s<TPL>, cudaFuncAttributePreferredSharedMemoryCarveout,
                                          (int)cudaSharedmemCarveoutMaxShared));
        if constexpr (TPL >= 2) {
          FMM_CUDA_TRY(cudaFuncSetAttribute(p2p_kernel_f32s_half<TPL>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                            (int)smem));
          FMM_CUDA_TRY(cudaFuncSetAttribute(p2p_kernel_f32s_half<TPL>,
                                            cudaFuncAttributePreferredSharedMemoryCarveout,
                                            (int)cudaSharedmemCarveoutMaxShared));
        }
        sym_attr = true;
      }
      a.order = t->leaf_order_sym + lb;
      a.work_off = t->sym_work_off;
      a.rec = t->sym_rec;
      a.partial = t->sym_partial;
      a.stride = t->sym_stride;
      // leaves that fill at most half of the target slots exist
      bool half_launched = false;
      if constexpr (TPL >= 2) {
        if (t->min_leaf <= 16 * TPL) {
          p2p_kernel_f32s_half<TPL><<<(unsigned)blocks, 128, smem, st>>>(a);
          half_launched = true;
        }
      }
      if (!half_launched) p2p_kernel_f32s<TPL><<<(unsigned)blocks, 128, smem, st>>>(a);
      FMM_LAUNCH_CHECK();
      return;
    }
    if constexpr (TPL <= 4) {
      if (field && uses_sym(t, true)) {
        static bool sv_attr = false;
        if (!sv_attr) {
          FMM_CUDA_TRY(cudaFuncSetAttribute(p2p_kernel_f32sv<TPL, kSvField>,
                                            cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
          FMM_CUDA_TRY(cudaFuncSetAttribute(p2p_kernel_f32sv<TPL, kSvField>,
                                            cudaFuncAttributePreferredSharedMemoryCarveout,
                                            (int)cudaSharedmemCarveoutMaxShared));
          sv_attr = true;
        }
        a.order = t->leaf_order_sym + lb;
        a.work_off = t->sym_work_off;
        a.rec = t->sym_rec;
        a.partial = t->sym_partial4;
        a.stride = t->sym_stride;
        p2p_kernel_f32sv<TPL, kSvField><<<(unsigned)blocks, 128, smem, st>>>(a);
        FMM_LAUNCH_CHECK();
        return;
      }
    }
    if (field) p2p_kernel_f32h<TPL, true><<<(unsigned)blocks, 128, smem, st>>>(a);
    else p2p_kernel_f32h<TPL, false><<<(unsigned)blocks, 128, smem, st>>>(a);
    FMM_LAUNCH_CHECK();
    return;
  } else {
    if (!field && t->sym && t->opt_near_sym && t->prm.precision == FMM_FP64DF) {
      static bool df_attr = false;
      if (!df_attr) {
        FMM_CUDA_TRY(cudaFuncSetAttribute(p2p_kernel_dfs<TPL>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        df_attr = true;
      }
      a.order = t->leaf_order_sym + lb;
      a.work_off = t->sym_work_off;
      a.rec = t->sym_rec;
      a.frame = t->sym_frame;
      a.df_tile = t->src_df;
      a.partial = t->sym_partial;
      a.stride = t->sym_stride;
      p2p_kernel_dfs<TPL><<<(unsigned)((a.n_leaves + 3) / 4), 128, smem, st>>>(a);
      FMM_LAUNCH_CHECK();
      return;
    }
    if (!field && t->sym && t->opt_near_sym) {
      static bool sym_attr = false;
      if (!sym_attr) {
        FMM_CUDA_TRY(cudaFuncSetAttribute(p2p_kernel_f64s<TPL>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        sym_attr = true;
      }
      a.order = t->leaf_order_sym + lb;
      a.work_off = t->sym_work_off;
      a.rec = t->sym_rec;
      a.partial = t->sym_partial;
      a.stride = t->sym_stride;
      p2p_kernel_f64s<TPL><<<(unsigned)((a.n_leaves + 3) / 4), 128, smem, st>>>(a);
      FMM_LAUNCH_CHECK();
      return;
    }
    // FP64 fields and two-tree evaluations: the one-sided kernel (its work
    // counter was cleared by the gather)
    static bool attr_set = false;
    if (!attr_set) {
      FMM_CUDA_TRY(cudaFuncSetAttribute(p2p_kernel<TPL, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
      FMM_CUDA_TRY(cudaFuncSetAttribute(p2p_kernel<TPL, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
      attr_set = true;
    }
    int dev = 0, nsm = 0, occ = 0;
    FMM_CUDA_TRY(cudaGetDevice(&dev));
    FMM_CUDA_TRY(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    if (field) FMM_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, p2p_kernel<TPL, true>, 128, smem));
    else FMM_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, p2p_kernel<TPL, false>, 128, smem));
    if (occ < 1) occ = 1;
    int64_t blocks = (int64_t)nsm * occ;
    const int64_t need = (a.n_leaves + 3) / 4;
    if (blocks > need) blocks = need;
    if (field) p2p_kernel<TPL, true><<<(int)blocks, 128, smem, st>>>(a);
    else p2p_kernel<TPL, false><<<(int)blocks, 128, smem, st>>>(a);
    FMM_LAUNCH_CHECK();
  }
}

// Near field of the leaves at positions lb .. le - 1 of the work order.
void run_p2p(const fmm_tree* t, const Ptrs& pp, real* near_u, real* near_f, bool field, int64_t lb, int64_t le,
             cudaStream_t st) {
  if (le <= lb) return;
  if (t->max_leaf <= 32) run_p2p_tpl<1>(t, pp, near_u, near_f, field, lb, le, st);
  else if (t->max_leaf <= 64) run_p2p_tpl<2>(t, pp, near_u, near_f, field, lb, le, st);
  else if (t->max_leaf <= 128) run_p2p_tpl<4>(t, pp, near_u, near_f, field, lb, le, st);
  else run_p2p_tpl<8>(t, pp, near_u, near_f, field, lb, le, st);
}

// The slot gather of the symmetric near field's vector variants: (U, V)
// rows into near_u (hi, lo) and near_v (3 floats per point).
void run_sv_gather(const fmm_tree* t, float* near_u, float* near_v, cudaStream_t st) {
  sv_gather_kernel<<<grid_for(t->n_gchunks * 32, 128), 128, 0, st>>>(
      t->n_gchunks, t->gch_leaf, t->gch_r0, t->gch_first, t->leaf_box, t->box_start, t->box_count, t->sym_recv_off,
      reinterpret_cast<const float4*>(t->sym_partial4), (int64_t)t->sym_stride, near_u, near_v, t->gpart4);
  FMM_LAUNCH_CHECK();
  if (t->n_gmulti > 0) {
    sv_combine_kernel<<<grid_for(t->n_gmulti * 32, 128), 128, 0, st>>>(
        t->n_gmulti, t->gmulti_leaf, t->gch_first, t->leaf_box, t->box_start, t->box_count, (int64_t)t->sym_stride,
        t->gpart4, near_u, near_v);
    FMM_LAUNCH_CHECK();
  }
  t->launches += 1 + (t->n_gmulti > 0 ? 1 : 0);
}

// The slot gather of the symmetric near field (after the near-field kernel).
void run_sym_gather(const fmm_tree* t, real* near_u, real* near_f, bool field, cudaStream_t st) {
  if constexpr (kF32) {
    if (field) {
      run_sv_gather(t, reinterpret_cast<float*>(near_u), reinterpret_cast<float*>(near_f), st);
      return;
    }
    sym_gather_kernel<<<grid_for(t->n_gchunks * 32, 128), 128, 0, st>>>(
        t->n_gchunks, t->gch_leaf, t->gch_r0, t->gch_first, t->leaf_box, t->box_start, t->box_count,
        t->sym_recv_off, reinterpret_cast<const float*>(t->sym_partial), (int64_t)t->sym_stride,
        reinterpret_cast<float*>(near_u), reinterpret_cast<float*>(t->gpart));
    FMM_LAUNCH_CHECK();
    if (t->n_gmulti > 0) {
      sym_combine_kernel<<<grid_for(t->n_gmulti * 32, 128), 128, 0, st>>>(
          t->n_gmulti, t->gmulti_leaf, t->gch_first, t->leaf_box, t->box_start, t->box_count, (int64_t)t->sym_stride,
          reinterpret_cast<const float*>(t->gpart), reinterpret_cast<float*>(near_u));
      FMM_LAUNCH_CHECK();
    }
  } else {
    sym_gather_f64_kernel<<<grid_for(t->n_gchunks * 32, 128), 128, 0, st>>>(
        t->n_gchunks, t->gch_leaf, t->gch_r0, t->gch_first, t->leaf_box, t->box_start, t->box_count,
        t->sym_recv_off, t->sym_partial, (int64_t)t->sym_stride, reinterpret_cast<double*>(near_u), t->gpart);
    FMM_LAUNCH_CHECK();
    if (t->n_gmulti > 0) {
      sym_combine_f64_kernel<<<grid_for(t->n_gmulti * 32, 128), 128, 0, st>>>(
          t->n_gmulti, t->gmulti_leaf, t->gch_first, t->leaf_box, t->box_start, t->box_count, (int64_t)t->sym_stride,
          t->gpart, reinterpret_cast<double*>(near_u));
      FMM_LAUNCH_CHECK();
    }
  }
  t->launches += 1 + (t->n_gmulti > 0 ? 1 : 0);
}

template <class F>
void dispatch_p(int p, F&& f) {
  switch (p) {
    case 1: f(std::integral_constant<int, 1>{}); break;
    case 2: f(std::integral_constant<int, 2>{}); break;
    case 3: f(std::integral_constant<int, 3>{}); break;
    case 4: f(std::integral_constant<int, 4>{}); break;
    case 5: f(std::integral_constant<int, 5>{}); break;
    case 6: f(std::integral_constant<int, 6>{}); break;
    case 7: f(std::integral_constant<int, 7>{}); break;
    case 8: f(std::integral_constant<int, 8>{}); break;
    case 9: f(std::integral_constant<int, 9>{}); break;
    case 10: f(std::integral_constant<int, 10>{}); break;
    default: set_error("unsupported expansion order %d", p); throw Fail{FMM_ERR_INVALID_ARG};
  }
}

void eval_impl(const fmm_tree* t, const double* q, double* u, double* field, cudaStream_t st) {
  Ptrs pp = ptrs(t);
  stage_event(t, FMM_STAGE_SORT, false, st);
  const bool df = !kF32 && t->prm.precision == FMM_FP64DF && t->sym && t->opt_near_sym && t->src_df && field == nullptr;
  gather_kernel<<<grid_for(t->n, 256), 256, 0, st>>>(t->n, t->n_charges, t->perm, q, pp.pos, pp.src,
                                                     kF32 ? t->src_dup : nullptr, df ? t->src_df : nullptr,
                                                     t->counters, t->m2m_ready, t->m2m_ready ? t->n_boxes : 0);
  FMM_LAUNCH_CHECK();
  t->launches += 1;
  stage_event(t, FMM_STAGE_SORT, true, st);
  // the slot of a second near-field launch is recorded empty unless used
  stage_event(t, fmm_tree::kStageP2P2, false, st);
  stage_event(t, fmm_tree::kStageP2P2, true, st);
  real* near_u = reinterpret_cast<real*>(t->near_u);
  real* near_f = reinterpret_cast<real*>(t->near_f);
  auto upward = [&](cudaStream_t ss) {
    dispatch_p(t->prm.p, [&](auto pc) {
      constexpr int P = decltype(pc)::value;
      run_upward<P>(t, pp, ss);
    });
  };
  auto downward = [&](cudaStream_t ss) {
    dispatch_p(t->prm.p, [&](auto pc) {
      constexpr int P = decltype(pc)::value;
      run_downward<P>(t, pp, ss, df);
    });
  };
  const bool sym = uses_sym(t, field != nullptr);
  auto near_range = [&](int64_t lb, int64_t le, int stage) {
    stage_event(t, stage, false, st);
    run_p2p(t, pp, near_u, near_f, field != nullptr, lb, le, st);
    stage_event(t, stage, true, st);
  };
  auto near = [&] { near_range(0, t->n_leaves, FMM_STAGE_P2P); };
  auto m2l = [&](cudaStream_t ss) {
    dispatch_p(t->prm.p, [&](auto pc) {
      constexpr int P = decltype(pc)::value;
      run_m2l<P>(t, pp, ss, df);
    });
  };
  auto l2l = [&](cudaStream_t ss) {
    dispatch_p(t->prm.p, [&](auto pc) {
      constexpr int P = decltype(pc)::value;
      run_l2l<P>(t, pp, ss);
    });
  };
  auto fork = [&] {
    FMM_CUDA_TRY(cudaEventRecord(t->ev_fork, st));
    FMM_CUDA_TRY(cudaStreamWaitEvent(t->far_stream, t->ev_fork, 0));
  };
  auto join = [&] {
    FMM_CUDA_TRY(cudaEventRecord(t->ev_join, t->far_stream));
    FMM_CUDA_TRY(cudaStreamWaitEvent(st, t->ev_join, 0));
  };
  const int schedule = t->opt_schedule;
  if (schedule == kSplitNear) {
    const int64_t half = t->n_leaves / 2;
    fork();
    upward(t->far_stream);
    near_range(0, half, FMM_STAGE_P2P);
    join();
    m2l(st);
    fork();
    l2l(t->far_stream);
    near_range(half, t->n_leaves, fmm_tree::kStageP2P2);
    if (sym) run_sym_gather(t, near_u, near_f, field != nullptr, st);
    join();
  } else if (schedule == kUpwardSide) {
    // P2M, M2M beside the near field; then the slot gather (memory bound)
    // beside M2L and L2L on the higher-priority stream (beside L2L alone:
    // 2.08 / 0.511 / 53.7 ms on the three workloads below, against 2.08 /
    // 0.503 / 43.1; on the caller's stream with M2L and L2L on the
    // higher-priority one: 2.061 / 0.505 / 52.8, against 2.058 / 0.506 / 42.6;
    // the gather on a grid of 2 blocks per SM: 2.130 / - / 61.8)
    fork();
    upward(t->far_stream);
    near();
    join();
    if (sym) {
      fork();
      run_sym_gather(t, near_u, near_f, field != nullptr, t->far_stream);
      downward(st);
      join();
    } else {
      downward(st);
    }
  } else if (schedule == kFarSide) {
    upward(st);
    fork();
    downward(t->far_stream);
    near();
    if (sym) run_sym_gather(t, near_u, near_f, field != nullptr, st);
    join();
  } else {
    upward(st);
    downward(st);
    near();
    if (sym) run_sym_gather(t, near_u, near_f, field != nullptr, st);
  }
  stage_event(t, FMM_STAGE_L2P, false, st);
  dispatch_p(t->prm.p, [&](auto pc) {
    constexpr int P = decltype(pc)::value;
    run_l2p<P>(t, pp, near_u, near_f, u, field, st);
  });
  stage_event(t, FMM_STAGE_L2P, true, st);
}

// Backward pass (FP32C): near field of both charge vectors in one sweep, then
// the far field of each, local evaluations into the field of q (fq) and the
// potential and field of g (ug, fg), all in the caller's point order.
template <int TPL>
void run_p2p_bwd_tpl(const fmm_tree* t, const Ptrs& pp, cudaStream_t st) {
  P2PArgs a{};
  a.n_leaves = t->n_leaves;
  a.leaf_box = t->leaf_box;
  a.src_leaf_box = t->src_leaf_box;
  a.order = t->leaf_order;
  a.off = t->p2p_off;
  a.ent32 = t->p2p32;
  a.thr = t->p2p_thr;
  a.box_start = t->box_start;
  a.box_count = t->box_count;
  a.src = pp.src;
  a.tile = t->src_dup;
  a.tile_g = t->src_dup2;
  a.near_f = reinterpret_cast<real*>(t->near_f);
  a.near_u2 = t->near_u2;
  a.near_f2 = t->near_f2;
  a.status = t->status;
  a.wait_cycles = t->wait_cycles;
  const size_t smem = (size_t)4 * 2 * 2 * TPL * 32 * 32;  // [warp][buf][q, g] 32-byte records
  static bool attr_set = false;
  if (!attr_set) {
    FMM_CUDA_TRY(cudaFuncSetAttribute(p2p_kernel_bwd<TPL>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    FMM_CUDA_TRY(cudaFuncSetAttribute(p2p_kernel_bwd<TPL>, cudaFuncAttributePreferredSharedMemoryCarveout,
                                      (int)cudaSharedmemCarveoutMaxShared));
    attr_set = true;
  }
  p2p_kernel_bwd<TPL><<<(unsigned)((t->n_leaves + 3) / 4), 128, smem, st>>>(a);
  FMM_LAUNCH_CHECK();
  t->launches += 1;
}

template <int Unused = 0>
void backward_impl(const fmm_tree* t, const double* q, const double* g, double* ug, double* fq, double* fg,
                   cudaStream_t st) {
  Ptrs pp = ptrs(t);
  real* near_u = reinterpret_cast<real*>(t->near_u);
  real* near_f = reinterpret_cast<real*>(t->near_f);
  // near-field records of g, then of q (src32 ends up holding q)
  gather_kernel<<<grid_for(t->n, 256), 256, 0, st>>>(t->n, t->n_charges, t->perm, g, pp.pos, pp.src, t->src_dup2,
                                                     nullptr, t->counters, t->m2m_ready,
                                                     t->m2m_ready ? t->n_boxes : 0);
  FMM_LAUNCH_CHECK();
  gather_kernel<<<grid_for(t->n, 256), 256, 0, st>>>(t->n, t->n_charges, t->perm, q, pp.pos, pp.src, t->src_dup,
                                                     nullptr, t->counters, t->m2m_ready,
                                                     t->m2m_ready ? t->n_boxes : 0);
  FMM_LAUNCH_CHECK();
  t->launches += 2;
  require(t->max_leaf <= 128, "fused backward sweep needs leaves of at most 128 points");
  if (t->max_leaf <= 32) run_p2p_bwd_tpl<1>(t, pp, st);
  else if (t->max_leaf <= 64) run_p2p_bwd_tpl<2>(t, pp, st);
  else run_p2p_bwd_tpl<4>(t, pp, st);
  // far field of q and its local evaluation: the field of q
  dispatch_p(t->prm.p, [&](auto pc) {
    constexpr int P = decltype(pc)::value;
    run_upward<P>(t, pp, st);
    run_downward<P>(t, pp, st);
    run_l2p<P>(t, pp, near_u, near_f, nullptr, fq, st);
  });
  // far field of g: potential and field
  gather_kernel<<<grid_for(t->n, 256), 256, 0, st>>>(t->n, t->n_charges, t->perm, g, pp.pos, pp.src, nullptr,
                                                     nullptr, t->counters, t->m2m_ready,
                                                     t->m2m_ready ? t->n_boxes : 0);
  FMM_LAUNCH_CHECK();
  t->launches += 1;
  dispatch_p(t->prm.p, [&](auto pc) {
    constexpr int P = decltype(pc)::value;
    run_upward<P>(t, pp, st);
    run_downward<P>(t, pp, st);
    run_l2p<P>(t, pp, reinterpret_cast<real*>(t->near_u2), reinterpret_cast<real*>(t->near_f2), ug, fg, st);
  });
}


// Backward pass with the symmetric near field (FP32C, one point set, leaves of
// at most 128 points, vector slot buffers present): one symmetric sweep gives
// U = the near potential sums of g and the pair-symmetric vector C
// (p2p_kernel_f32sv, kSvBackward); the far fields of q and then of g run
// meanwhile on the tree's second stream (far parts only: L2P without near
// sums), and a combine in tree order adds the near parts:
//   dL/dq_i = (K g)_i = (far part) - U_i / (4 pi),
//   dL/dx_i = -(g_i E^far_q,i + q_i E^far_g,i) + C_i / (4 pi).
__global__ void backward_sym_combine_kernel(int64_t n, const int32_t* __restrict__ perm, int64_t out_base,
                                            const double* __restrict__ q, const double* __restrict__ g,
                                            const double* __restrict__ fq, const double* __restrict__ fg,
                                            const float* __restrict__ near_u, const float* __restrict__ near_v,
                                            double* __restrict__ grad_q, double* __restrict__ grad_pos) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t o = perm[i] - out_base;
    if (grad_q) grad_q[o] -= kInv4Pi * ((double)near_u[2 * i] + (double)near_u[2 * i + 1]);
    if (grad_pos) {
      const double qi = q[o], gi = g[o];
      for (int c = 0; c < 3; c++)
        grad_pos[3 * o + c] = -(gi * fq[3 * o + c] + qi * fg[3 * o + c]) + kInv4Pi * (double)near_v[3 * i + c];
    }
  }
}

template <int TPL>
void run_p2p_bwd_sym_tpl(const fmm_tree* t, cudaStream_t st) {
  P2PArgs a{};
  a.n_leaves = t->n_leaves;
  a.leaf_box = t->leaf_box;
  a.order = t->leaf_order_sym;
  a.work_off = t->sym_work_off;
  a.rec = t->sym_rec;
  a.partial = t->sym_partial4;
  a.stride = t->sym_stride;
  a.box_start = t->box_start;
  a.box_count = t->box_count;
  a.tile = t->src_dup;
  a.tile_g = t->src_dup2;
  a.near_u = reinterpret_cast<real*>(t->near_u2);
  a.near_f = reinterpret_cast<real*>(t->near_f2);
  a.status = t->status;
  a.wait_cycles = t->wait_cycles;
  const size_t smem = (size_t)4 * 2 * 2 * TPL * 32 * 32;  // [warp][buf][q, g] 32-byte records
  static bool attr_set = false;
  if (!attr_set) {
    FMM_CUDA_TRY(cudaFuncSetAttribute(p2p_kernel_f32sv<TPL, kSvBackward>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)smem));
    FMM_CUDA_TRY(cudaFuncSetAttribute(p2p_kernel_f32sv<TPL, kSvBackward>,
                                      cudaFuncAttributePreferredSharedMemoryCarveout,
                                      (int)cudaSharedmemCarveoutMaxShared));
    attr_set = true;
  }
  p2p_kernel_f32sv<TPL, kSvBackward><<<(unsigned)((t->n_leaves + 3) / 4), 128, smem, st>>>(a);
  FMM_LAUNCH_CHECK();
  t->launches += 1;
}

template <int Unused = 0>
void backward_sym_impl(const fmm_tree* t, const double* q, const double* g, double* grad_q, double* grad_pos,
                       cudaStream_t st) {
  Ptrs pp = ptrs(t);
  // near-field records of g, then of q (the FP32 point records end up
  // holding q for the far field of q)
  gather_kernel<<<grid_for(t->n, 256), 256, 0, st>>>(t->n, t->n_charges, t->perm, g, pp.pos, pp.src, t->src_dup2,
                                                     nullptr, t->counters, t->m2m_ready,
                                                     t->m2m_ready ? t->n_boxes : 0);
  FMM_LAUNCH_CHECK();
  gather_kernel<<<grid_for(t->n, 256), 256, 0, st>>>(t->n, t->n_charges, t->perm, q, pp.pos, pp.src, t->src_dup,
                                                     nullptr, t->counters, t->m2m_ready,
                                                     t->m2m_ready ? t->n_boxes : 0);
  FMM_LAUNCH_CHECK();
  t->launches += 2;
  FMM_CUDA_TRY(cudaEventRecord(t->ev_fork, st));
  FMM_CUDA_TRY(cudaStreamWaitEvent(t->far_stream, t->ev_fork, 0));
  // far fields on the second stream: q, then g (whose gather rewrites the
  // FP32 point records only after q's local evaluation has read them)
  cudaStream_t fs = t->far_stream;
  dispatch_p(t->prm.p, [&](auto pc) {
    constexpr int P = decltype(pc)::value;
    run_upward<P>(t, pp, fs);
    run_downward<P>(t, pp, fs);
    run_l2p<P>(t, pp, nullptr, nullptr, nullptr, t->f_stage, fs);
  });
  gather_kernel<<<grid_for(t->n, 256), 256, 0, fs>>>(t->n, t->n_charges, t->perm, g, pp.pos, pp.src, nullptr,
                                                     nullptr, t->counters, t->m2m_ready,
                                                     t->m2m_ready ? t->n_boxes : 0);
  FMM_LAUNCH_CHECK();
  t->launches += 1;
  dispatch_p(t->prm.p, [&](auto pc) {
    constexpr int P = decltype(pc)::value;
    run_upward<P>(t, pp, fs);
    run_downward<P>(t, pp, fs);
    run_l2p<P>(t, pp, nullptr, nullptr, grad_q, t->g_stage, fs);
  });
  // the near field on the caller's stream meanwhile
  if (t->max_leaf <= 32) run_p2p_bwd_sym_tpl<1>(t, st);
  else if (t->max_leaf <= 64) run_p2p_bwd_sym_tpl<2>(t, st);
  else run_p2p_bwd_sym_tpl<4>(t, st);
  run_sv_gather(t, t->near_u2, t->near_f2, st);
  FMM_CUDA_TRY(cudaEventRecord(t->ev_join, fs));
  FMM_CUDA_TRY(cudaStreamWaitEvent(st, t->ev_join, 0));
  backward_sym_combine_kernel<<<grid_for(t->n, 256), 256, 0, st>>>(t->n, t->perm, t->out_base, q, g, t->f_stage,
                                                                   t->g_stage, t->near_u2, t->near_f2, grad_q,
                                                                   grad_pos);
  FMM_LAUNCH_CHECK();
  t->launches += 1;
}

}  // namespace
}  // namespace fmm
