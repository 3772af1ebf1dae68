// Device construction of the FMM hierarchy (Sec. II.A, II.B, Listing 2):
// median-split 2^s-tree, box geometry, level-marching interaction lists and
// the rotation coefficients of every translation.
//
// Tree.  Each bisection round splits every segment of the current tree order
// in two: the axis of largest extent of the segment's bounding box (ties to
// the lowest axis), then the ceil(n/2) points smallest in (coordinate, original
// index) form the lower child.  The split point is found by radix selection
// on 96-bit keys (order-preserving 64-bit image of the FP64 coordinate, then
// the 32-bit index), 8 bits per pass with early exit once the bin holding the
// pivot is a single point; points are then partitioned around it.  Segments
// small enough for one CTA (kSmallCap points) finish all their remaining
// rounds inside that CTA with bitonic sorts in shared memory, and every leaf
// is finally sorted by original index.  The result depends only on the point
// sets, never on the order inside a segment, so it is deterministic.
//
// Geometry.  Bounding boxes are exact min/max; centre = (lo + hi) * 0.5 and
// radius = sqrt((ex^2 + ey^2) + ez^2) * 0.5 with every FP64 operation rounded
// separately (no contraction), as is the well-separation test
// R + theta r <= theta d (Eq. 4, with d > 0 required).
//
// Lists.  Level march (Sec. II.B): start from (root, root); each step moves
// well-separated candidate pairs to the M2L list and replaces the others by
// the children of the side whose level has the larger average radius (ties:
// source, or target with FMM_TIE_TARGET); pairs left when both sides reach
// the leaf level form the near field.  Average radii are adjacent-pair sums
// repeated down to one value, divided by the box count.  FMM_SAME_LEVEL
// replaces the march by the same-level lists of Sec. II.B steps 1-3: both
// sides descend together, so only boxes of one level are compared.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <vector>

#include "common.cuh"

namespace fmm {
namespace {

constexpr int kThreads = 256;
constexpr int kItems = 8;
constexpr int kChunk = kThreads * kItems;

__host__ __device__ inline int64_t level_offset(int l, int s) {
  int64_t o = 0;
  for (int i = 0; i < l; i++) o += (int64_t)1 << (s * i);
  return o;
}

__device__ __forceinline__ unsigned long long okey(double d) {
  unsigned long long b = (unsigned long long)__double_as_longlong(d);
  return (b >> 63) ? ~b : (b | 0x8000000000000000ull);
}
__device__ __forceinline__ double okey_inv(unsigned long long k) {
  unsigned long long b = (k >> 63) ? (k & 0x7fffffffffffffffull) : ~k;
  return __longlong_as_double((long long)b);
}

// index of the segment containing position i: largest j with starts[j] <= i
__device__ __forceinline__ int seg_of(const int64_t* starts, int nseg, int64_t i) {
  int lo = 0, hi = nseg - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (starts[mid] <= i) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

// ---- input: SoA copy with -0.0 -> +0.0, finiteness check ----------------------
// soa: positions given as three arrays of n (x, then y, then z) instead of
// n rows of (x, y, z)
__global__ void canon_kernel(const double* __restrict__ pos, int64_t n, int soa, double* __restrict__ X,
                             int32_t* __restrict__ idx, int* __restrict__ bad) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    for (int a = 0; a < 3; a++) {
      double v = __dadd_rn(soa ? pos[a * n + i] : pos[3 * i + a], 0.0);
      if (!isfinite(v)) atomicOr(bad, 1);
      X[a * n + i] = v;
    }
    idx[i] = (int32_t)i;
  }
}

// ---- segment boundaries of round r+1 from round r (closed form) --------------
__global__ void split_starts_kernel(const int64_t* __restrict__ st, int nseg, int64_t* __restrict__ nx) {
  int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j < nseg) {
    int64_t a = st[j], b = st[j + 1];
    nx[2 * j] = a;
    nx[2 * j + 1] = a + (b - a + 1) / 2;
    if (j == nseg - 1) nx[2 * nseg] = b;
  }
}

// ---- bounding boxes of segments (large rounds) ---------------------------------
__global__ void __launch_bounds__(kThreads) seg_bbox_kernel(const double* __restrict__ X, int64_t n,
                                                            const int64_t* __restrict__ starts, int nseg,
                                                            unsigned long long* __restrict__ bmin,
                                                            unsigned long long* __restrict__ bmax) {
  const int64_t c0 = (int64_t)blockIdx.x * kChunk;
  const int64_t c1 = min(c0 + kChunk, n);
  if (c0 >= n) return;
  const int s0 = seg_of(starts, nseg, c0), s1 = seg_of(starts, nseg, c1 - 1);
  if (s0 == s1) {
    unsigned long long mn[3] = {~0ull, ~0ull, ~0ull}, mx[3] = {0, 0, 0};
    for (int64_t i = c0 + threadIdx.x; i < c1; i += kThreads)
      for (int a = 0; a < 3; a++) {
        unsigned long long k = okey(X[a * n + i]);
        mn[a] = min(mn[a], k);
        mx[a] = max(mx[a], k);
      }
    __shared__ unsigned long long sm[6][kThreads / 32];
    for (int a = 0; a < 3; a++) {
      for (int o = 16; o > 0; o >>= 1) {
        mn[a] = min(mn[a], __shfl_xor_sync(0xffffffffu, mn[a], o));
        mx[a] = max(mx[a], __shfl_xor_sync(0xffffffffu, mx[a], o));
      }
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0)
      for (int a = 0; a < 3; a++) {
        sm[a][warp] = mn[a];
        sm[3 + a][warp] = mx[a];
      }
    __syncthreads();
    if (threadIdx.x < 3) {
      int a = threadIdx.x;
      unsigned long long m0 = ~0ull, m1 = 0;
      for (int w = 0; w < kThreads / 32; w++) {
        m0 = min(m0, sm[a][w]);
        m1 = max(m1, sm[3 + a][w]);
      }
      atomicMin(&bmin[3 * s0 + a], m0);
      atomicMax(&bmax[3 * s0 + a], m1);
    }
  } else {
    for (int64_t i = c0 + threadIdx.x; i < c1; i += kThreads) {
      int sg = seg_of(starts, nseg, i);
      for (int a = 0; a < 3; a++) {
        unsigned long long k = okey(X[a * n + i]);
        atomicMin(&bmin[3 * sg + a], k);
        atomicMax(&bmax[3 * sg + a], k);
      }
    }
  }
}

// Radix-select state of one segment.
struct Sel {
  unsigned long long phi;  // prefix of the 96-bit key (left aligned), high word
  unsigned int plo;        // low word
  int bits;                // prefix bits fixed so far
  long long krem;          // rank of the pivot among keys with this prefix
  int resolved;            // 1 once the prefix names exactly one point
  int axis;
};

__global__ void seg_axis_kernel(const unsigned long long* __restrict__ bmin,
                                const unsigned long long* __restrict__ bmax,
                                const int64_t* __restrict__ starts, int nseg, Sel* __restrict__ sel) {
  int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= nseg) return;
  double e[3];
  for (int a = 0; a < 3; a++) e[a] = __dsub_rn(okey_inv(bmax[3 * j + a]), okey_inv(bmin[3 * j + a]));
  int ax = 0;
  if (e[1] > e[ax]) ax = 1;
  if (e[2] > e[ax]) ax = 2;
  const int64_t cnt = starts[j + 1] - starts[j];
  Sel s;
  s.phi = 0;
  s.plo = 0;
  s.bits = 0;
  s.krem = (cnt + 1) / 2 - 1;
  s.resolved = (cnt <= 1);
  s.axis = ax;
  sel[j] = s;
}

__device__ __forceinline__ unsigned digit_of(unsigned long long hi, unsigned lo, int d) {
  return d < 8 ? (unsigned)((hi >> (56 - 8 * d)) & 0xffu) : ((lo >> (24 - 8 * (d - 8))) & 0xffu);
}
// -1, 0, 1: top `bits` bits of (hi, lo) below, equal to, above the prefix
__device__ __forceinline__ int cmp_prefix(unsigned long long hi, unsigned lo, const Sel& s) {
  const int b = s.bits;
  if (b <= 64) {
    unsigned long long m = (b == 0) ? 0ull : (~0ull << (64 - b));
    unsigned long long kh = hi & m;
    return kh < s.phi ? -1 : (kh > s.phi ? 1 : 0);
  }
  if (hi != s.phi) return hi < s.phi ? -1 : 1;
  unsigned m = (b >= 96) ? ~0u : (~0u << (96 - b));
  unsigned kl = lo & m;
  return kl < s.plo ? -1 : (kl > s.plo ? 1 : 0);
}

__global__ void __launch_bounds__(kThreads) radix_hist_kernel(const double* __restrict__ X,
                                                              const int32_t* __restrict__ idx, int64_t n,
                                                              const int64_t* __restrict__ starts, int nseg,
                                                              const Sel* __restrict__ sel, int d,
                                                              unsigned* __restrict__ hist,
                                                              const int* __restrict__ prev_unresolved) {
  const int64_t c0 = (int64_t)blockIdx.x * kChunk;
  const int64_t c1 = min(c0 + kChunk, n);
  if (c0 >= n) return;
  // every segment's pivot was settled by an earlier digit: nothing to count
  if (prev_unresolved && *prev_unresolved == 0) return;
  const int s0 = seg_of(starts, nseg, c0), s1 = seg_of(starts, nseg, c1 - 1);
  __shared__ unsigned sh[256];
  if (s0 == s1) {
    const Sel s = sel[s0];
    if (s.resolved) return;
    for (int i = threadIdx.x; i < 256; i += kThreads) sh[i] = 0;
    __syncthreads();
    for (int64_t i = c0 + threadIdx.x; i < c1; i += kThreads) {
      unsigned long long hi = okey(X[s.axis * n + i]);
      unsigned lo = (unsigned)idx[i];
      if (cmp_prefix(hi, lo, s) == 0) atomicAdd(&sh[digit_of(hi, lo, d)], 1u);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < 256; i += kThreads)
      if (sh[i]) atomicAdd(&hist[(size_t)s0 * 256 + i], sh[i]);
  } else {
    for (int64_t i = c0 + threadIdx.x; i < c1; i += kThreads) {
      int sg = seg_of(starts, nseg, i);
      const Sel s = sel[sg];
      if (s.resolved) continue;
      unsigned long long hi = okey(X[s.axis * n + i]);
      unsigned lo = (unsigned)idx[i];
      if (cmp_prefix(hi, lo, s) == 0) atomicAdd(&hist[(size_t)sg * 256 + digit_of(hi, lo, d)], 1u);
    }
  }
}

// One warp per segment: lane j holds bins 8j .. 8j + 7 of the segment's
// histogram; a warp prefix sum over the lanes' totals finds the bin holding
// the pivot (the first bin whose cumulative count exceeds its rank), and the
// bins are cleared for the next digit.
__global__ void radix_select_kernel(Sel* __restrict__ sel, int nseg, int d, unsigned* __restrict__ hist,
                                    const int* __restrict__ prev_unresolved, int* __restrict__ unresolved) {
  const int j = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5);
  const int lane = threadIdx.x & 31;
  if (j >= nseg) return;  // whole warps leave together
  if (prev_unresolved && *prev_unresolved == 0) return;  // all settled; the bins are clear
  unsigned* h = hist + (size_t)j * 256 + 8 * lane;
  Sel s = sel[j];
  if (!s.resolved) {
    unsigned b[8];
    unsigned tot = 0;
#pragma unroll
    for (int k = 0; k < 8; k++) {
      b[k] = h[k];
      tot += b[k];
    }
    // exclusive prefix of the lanes' totals
    unsigned inc = tot;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned y = __shfl_up_sync(0xffffffffu, inc, o);
      if (lane >= o) inc += y;
    }
    const long long before = (long long)(inc - tot);
    // the lane whose range holds rank krem
    bool mine = before <= s.krem && s.krem < before + (long long)tot;
    // no bin holds the rank (cannot happen for a segment with points left):
    // the last bin, as a resolved prefix
    if (__ballot_sync(0xffffffffu, mine) == 0u && lane == 31) mine = true;
    if (mine) {
      long long cum = before;
      int dig = 8 * lane + 7;
      unsigned cnt = 0;
#pragma unroll
      for (int k = 0; k < 8; k++) {
        if (cnt == 0 && cum + (long long)b[k] > s.krem) {
          dig = 8 * lane + k;
          cnt = b[k];
        } else if (cnt == 0) {
          cum += b[k];
        }
      }
      s.krem -= cum;
      if (d < 8) s.phi |= (unsigned long long)dig << (56 - 8 * d);
      else s.plo |= (unsigned)dig << (24 - 8 * (d - 8));
      s.bits += 8;
      if (cnt <= 1) s.resolved = 1;
      else atomicOr(unresolved, 1);
      sel[j] = s;
    }
  }
#pragma unroll
  for (int k = 0; k < 8; k++) h[k] = 0;
}

// Points with key prefix <= the pivot's go to the lower child.
__global__ void __launch_bounds__(kThreads) partition_kernel(const double* __restrict__ X,
                                                             const int32_t* __restrict__ idx, int64_t n,
                                                             const int64_t* __restrict__ starts, int nseg,
                                                             const Sel* __restrict__ sel,
                                                             unsigned long long* __restrict__ ctr,
                                                             double* __restrict__ Xo,
                                                             int32_t* __restrict__ idxo) {
  const int64_t c0 = (int64_t)blockIdx.x * kChunk;
  const int64_t c1 = min(c0 + kChunk, n);
  if (c0 >= n) return;
  const int s0 = seg_of(starts, nseg, c0), s1 = seg_of(starts, nseg, c1 - 1);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (s0 == s1) {
    const Sel s = sel[s0];
    const int64_t a = starts[s0], b = starts[s0 + 1];
    const int64_t half = (b - a + 1) / 2;
    __shared__ unsigned wl[kThreads / 32], wu[kThreads / 32];
    __shared__ unsigned long long base_lo, base_hi;
    for (int64_t it = c0; it < c1; it += kThreads) {
      const int64_t i = it + threadIdx.x;
      const bool valid = i < c1;
      bool lower = false;
      if (valid) {
        unsigned long long hi = okey(X[s.axis * n + i]);
        lower = cmp_prefix(hi, (unsigned)idx[i], s) <= 0;
      }
      const unsigned bl = __ballot_sync(0xffffffffu, valid && lower);
      const unsigned bu = __ballot_sync(0xffffffffu, valid && !lower);
      if (lane == 0) {
        wl[warp] = __popc(bl);
        wu[warp] = __popc(bu);
      }
      __syncthreads();
      if (threadIdx.x == 0) {
        unsigned tl = 0, tu = 0;
        for (int w = 0; w < kThreads / 32; w++) {
          unsigned x = wl[w], y = wu[w];
          wl[w] = tl;
          wu[w] = tu;
          tl += x;
          tu += y;
        }
        base_lo = atomicAdd(&ctr[2 * s0], (unsigned long long)tl);
        base_hi = atomicAdd(&ctr[2 * s0 + 1], (unsigned long long)tu);
      }
      __syncthreads();
      if (valid) {
        const unsigned mask_lt = (1u << lane) - 1u;
        int64_t dst = lower ? a + (int64_t)base_lo + wl[warp] + __popc(bl & mask_lt)
                            : a + half + (int64_t)base_hi + wu[warp] + __popc(bu & mask_lt);
        for (int ax = 0; ax < 3; ax++) Xo[ax * n + dst] = X[ax * n + i];
        idxo[dst] = idx[i];
      }
      __syncthreads();
    }
  } else {
    for (int64_t i = c0 + threadIdx.x; i < c1; i += kThreads) {
      const int sg = seg_of(starts, nseg, i);
      const Sel s = sel[sg];
      const int64_t a = starts[sg], b = starts[sg + 1];
      const int64_t half = (b - a + 1) / 2;
      unsigned long long hi = okey(X[s.axis * n + i]);
      const bool lower = cmp_prefix(hi, (unsigned)idx[i], s) <= 0;
      int64_t dst = lower ? a + (int64_t)atomicAdd(&ctr[2 * sg], 1ull)
                          : a + half + (int64_t)atomicAdd(&ctr[2 * sg + 1], 1ull);
      for (int ax = 0; ax < 3; ax++) Xo[ax * n + dst] = X[ax * n + i];
      idxo[dst] = idx[i];
    }
  }
}

// ---- small segments: all remaining rounds and the leaf sort in one CTA ---------
constexpr int kSmallThreads = 256;

// Bitonic sort of the `total / sub` consecutive blocks of `sub` keys (sub a
// power of two dividing total), each ascending in (kh, kl).
__device__ void bitonic_sort_blocks(unsigned long long* kh, unsigned long long* kl, int total, int sub) {
  for (int k = 2; k <= sub; k <<= 1) {
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int i = threadIdx.x; i < total; i += blockDim.x) {
        const int ixj = i ^ j;
        if (ixj > i) {
          const bool asc = k == sub || (i & k) == 0;
          const bool gt = (kh[i] > kh[ixj]) || (kh[i] == kh[ixj] && kl[i] > kl[ixj]);
          if (gt == asc) {
            unsigned long long t = kh[i];
            kh[i] = kh[ixj];
            kh[ixj] = t;
            t = kl[i];
            kl[i] = kl[ixj];
            kl[ixj] = t;
          }
        }
      }
      __syncthreads();
    }
  }
}

// One CTA per segment of at most kSmallCap points: every remaining round and
// the leaf sort.  Shared memory holds only the sort keys and the points'
// current order (local slot numbers); coordinates and original indices are
// read through that order from global memory (the segment's 48 KB stay in
// L1/L2), so four CTAs fit on an SM and all segments of a 2^20-point build
// are resident at once.
__global__ void __launch_bounds__(kSmallThreads, 4) small_segment_kernel(
    const double* __restrict__ X, const int32_t* __restrict__ idx, int64_t n,
    const int64_t* __restrict__ starts, int rounds, double* __restrict__ Xo, int32_t* __restrict__ perm) {
  extern __shared__ __align__(16) unsigned char sm[];
  const int64_t g0 = starts[blockIdx.x], g1 = starts[blockIdx.x + 1];
  const int cnt = (int)(g1 - g0);
  const int nsub_max = 1 << rounds;
  const double* Xs = X + g0;      // this segment's coordinates: Xs[a * n + l]
  const int32_t* Is = idx + g0;   // and original indices
  // 8-byte items first, then 4-byte ones
  unsigned long long* kh = reinterpret_cast<unsigned long long*>(sm);
  unsigned long long* kl = kh + kSmallCap;
  unsigned long long* bb = kl + kSmallCap;                 // 6 x nsub_max
  int32_t* ia = reinterpret_cast<int32_t*>(bb + 6 * nsub_max);  // current order: local slots
  int32_t* ib = ia + kSmallCap;
  int* st = ib + kSmallCap;                                // nsub_max + 2
  int* axis = st + nsub_max + 2;                           // nsub_max
  for (int i = threadIdx.x; i < cnt; i += blockDim.x) ia[i] = i;
  if (threadIdx.x == 0) {
    st[0] = 0;
    st[1] = cnt;
  }
  __syncthreads();
  for (int r = 0; r < rounds; r++) {
    const int nsub = 1 << r;
    for (int j = threadIdx.x; j < nsub; j += blockDim.x)
      for (int a = 0; a < 3; a++) {
        bb[6 * j + a] = ~0ull;
        bb[6 * j + 3 + a] = 0ull;
      }
    __syncthreads();
    for (int i = threadIdx.x; i < cnt; i += blockDim.x) {
      int lo = 0, hi = nsub - 1;
      while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (st[mid] <= i) lo = mid;
        else hi = mid - 1;
      }
      const int l = ia[i];
      for (int a = 0; a < 3; a++) {
        unsigned long long k = okey(Xs[a * n + l]);
        atomicMin(&bb[6 * lo + a], k);
        atomicMax(&bb[6 * lo + 3 + a], k);
      }
    }
    __syncthreads();
    for (int j = threadIdx.x; j < nsub; j += blockDim.x) {
      double e[3];
      for (int a = 0; a < 3; a++) e[a] = __dsub_rn(okey_inv(bb[6 * j + 3 + a]), okey_inv(bb[6 * j + a]));
      int ax = 0;
      if (e[1] > e[ax]) ax = 1;
      if (e[2] > e[ax]) ax = 2;
      axis[j] = ax;
    }
    __syncthreads();
    // each sub-segment sorted on its own: (key on its axis, original index,
    // position), in blocks of `sub` slots (the largest sub-segment, rounded
    // up to a power of two; nsub * sub <= kSmallCap)
    int sub = 1;
    while (sub < (cnt + nsub - 1) / nsub) sub <<= 1;
    for (int i = threadIdx.x; i < nsub * sub; i += blockDim.x) {
      kh[i] = ~0ull;
      kl[i] = ~0ull;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < cnt; i += blockDim.x) {
      int lo = 0, hi = nsub - 1;
      while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (st[mid] <= i) lo = mid;
        else hi = mid - 1;
      }
      const int slot = lo * sub + (i - st[lo]);
      const int l = ia[i];
      kh[slot] = okey(Xs[axis[lo] * n + l]);
      kl[slot] = ((unsigned long long)(uint32_t)Is[l] << 12) | (unsigned long long)i;
    }
    __syncthreads();
    bitonic_sort_blocks(kh, kl, nsub * sub, sub);
    for (int i = threadIdx.x; i < nsub * sub; i += blockDim.x) {
      const int j = i / sub, k = i - j * sub;
      if (k < st[j + 1] - st[j]) ib[st[j] + k] = ia[(int)(kl[i] & 0xfffull)];
    }
    __syncthreads();
    {
      int32_t* u = ia;
      ia = ib;
      ib = u;
    }
    // next round's boundaries: ceil half to the lower child
    if (threadIdx.x == 0) {
      for (int j = nsub - 1; j >= 0; j--) {
        const int a = st[j], b = st[j + 1];
        st[2 * j + 2] = b;
        st[2 * j + 1] = a + (b - a + 1) / 2;
        st[2 * j] = a;
      }
    }
    __syncthreads();
  }
  // leaves in ascending original index (Listing 2, last line), each leaf
  // sorted on its own in a block of `sub` slots
  const int nleaf = 1 << rounds;
  int sub = 1;
  while (sub < (cnt + nleaf - 1) / nleaf) sub <<= 1;
  for (int i = threadIdx.x; i < nleaf * sub; i += blockDim.x) {
    kh[i] = ~0ull;
    kl[i] = ~0ull;
  }
  __syncthreads();
  for (int i = threadIdx.x; i < cnt; i += blockDim.x) {
    int lo = 0, hi = nleaf - 1;
    while (lo < hi) {
      int mid = (lo + hi + 1) >> 1;
      if (st[mid] <= i) lo = mid;
      else hi = mid - 1;
    }
    const int slot = lo * sub + (i - st[lo]);
    kh[slot] = (unsigned long long)(uint32_t)Is[ia[i]];
    kl[slot] = (unsigned long long)i;
  }
  __syncthreads();
  bitonic_sort_blocks(kh, kl, nleaf * sub, sub);
  for (int i = threadIdx.x; i < nleaf * sub; i += blockDim.x) {
    const int j = i / sub, k = i - j * sub;
    if (k < st[j + 1] - st[j]) {
      const int l = ia[(int)kl[i]], to = st[j] + k;
      for (int ax = 0; ax < 3; ax++) Xo[ax * n + g0 + to] = Xs[ax * n + l];
      perm[g0 + to] = Is[l];
    }
  }
}

// segments of at most kSmallCap = 2048 points split at most 11 more times
constexpr int kSmallMaxRounds = 11;
size_t small_smem_bytes(int rounds) {
  const size_t nsub = (size_t)1 << rounds;
  return (size_t)kSmallCap * (8 + 8 + 4 + 4) + nsub * 48 + sizeof(int) * (2 * nsub + 2);
}

// ---- geometry --------------------------------------------------------------------
// leaf bounding boxes: one warp per leaf
__global__ void leaf_bbox_kernel(const double* __restrict__ X, int64_t n, const int64_t* __restrict__ bs,
                                 const int32_t* __restrict__ bc, int64_t leaf_off, int64_t n_leaves,
                                 double* __restrict__ lo, double* __restrict__ hi) {
  const int lane = threadIdx.x & 31;
  const int64_t w = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  if (w >= n_leaves) return;
  const int64_t g = leaf_off + w;
  const int64_t a = bs[g];
  const int c = bc[g];
  for (int ax = 0; ax < 3; ax++) {
    double mn = INFINITY, mx = -INFINITY;
    for (int i = lane; i < c; i += 32) {
      double v = X[ax * n + a + i];
      mn = fmin(mn, v);
      mx = fmax(mx, v);
    }
    for (int o = 16; o > 0; o >>= 1) {
      mn = fmin(mn, __shfl_xor_sync(0xffffffffu, mn, o));
      mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    }
    if (lane == 0) {
      lo[3 * g + ax] = mn;
      hi[3 * g + ax] = mx;
    }
  }
}

// parent boxes: union of the 2^s children (exact)
__global__ void parent_bbox_kernel(int64_t nb, int64_t off, int64_t coff, int nch, double* __restrict__ lo,
                                   double* __restrict__ hi) {
  const int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (b >= nb) return;
  const int64_t g = off + b;
  for (int ax = 0; ax < 3; ax++) {
    double mn = INFINITY, mx = -INFINITY;
    for (int c = 0; c < nch; c++) {
      const int64_t gc = coff + b * nch + c;
      mn = fmin(mn, lo[3 * gc + ax]);
      mx = fmax(mx, hi[3 * gc + ax]);
    }
    lo[3 * g + ax] = mn;
    hi[3 * g + ax] = mx;
  }
}

__global__ void centre_radius_kernel(int64_t nbox, const double* __restrict__ lo, const double* __restrict__ hi,
                                     double* __restrict__ center, double* __restrict__ radius,
                                     float* __restrict__ ir32, double* __restrict__ ir64) {
  const int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (g >= nbox) return;
  double e[3];
  for (int a = 0; a < 3; a++) {
    center[3 * g + a] = __dmul_rn(__dadd_rn(lo[3 * g + a], hi[3 * g + a]), 0.5);
    e[a] = __dsub_rn(hi[3 * g + a], lo[3 * g + a]);
  }
  double d2 = __dadd_rn(__dmul_rn(e[0], e[0]), __dmul_rn(e[1], e[1]));
  d2 = __dadd_rn(d2, __dmul_rn(e[2], e[2]));
  const double r = __dmul_rn(__dsqrt_rn(d2), 0.5);
  radius[g] = r;
  ir64[g] = (r > 0.0) ? 1.0 / r : 0.0;
  ir32[g] = (r > 1e-30) ? (float)(1.0 / r) : 0.0f;
}

// boxes' start offsets for one level from the segment boundaries of its round
__global__ void box_range_kernel(const int64_t* __restrict__ st, int64_t nb, int64_t off,
                                 int64_t* __restrict__ bs, int32_t* __restrict__ bc) {
  const int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (b >= nb) return;
  bs[off + b] = st[b];
  bc[off + b] = (int32_t)(st[b + 1] - st[b]);
}

// leaf box ids, parents and per-level box ids of one tree
__global__ void index_lists_kernel(int64_t nbox, int s, int L, int32_t* __restrict__ leaf_box,
                                   int32_t* __restrict__ parent) {
  const int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (g >= nbox) return;
  int l = 0;
  while (level_offset(l + 1, s) <= g) l++;
  const int64_t b = g - level_offset(l, s);
  parent[g] = (l == 0) ? -1 : (int32_t)(level_offset(l - 1, s) + (b >> s));
  if (l == L) leaf_box[b] = (int32_t)g;
}

// adjacent-pair sums, one stage
// Sum of the radii of every level (block l: level l, 2^(s l) boxes from
// offset level_offset(l, s)), as adjacent-pair sums repeated down to one
// value: each thread first sums a contiguous power-of-two chunk with the same
// pairing (a binary counter: a partial sum is combined with its left
// neighbour of equal size as soon as one exists), then the block pairs the
// threads' partials in shared memory.
constexpr int kLevelSumThreads = 256;
__global__ void __launch_bounds__(kLevelSumThreads) level_sum_kernel(const double* __restrict__ radius, int s,
                                                                    double* __restrict__ out) {
  const int l = blockIdx.x;
  const int64_t m = (int64_t)1 << (s * l);
  int64_t off = 0;
  for (int i = 0; i < l; i++) off += (int64_t)1 << (s * i);
  const int nt = m < kLevelSumThreads ? (int)m : kLevelSumThreads;  // a power of two
  const int64_t chunk = m / nt;
  __shared__ double part[kLevelSumThreads];
  if (threadIdx.x < nt) {
    double stack[64];
    int64_t size[64];
    int top = 0;
    const double* v = radius + off + (int64_t)threadIdx.x * chunk;
    for (int64_t k = 0; k < chunk; k++) {
      double x = v[k];
      int64_t sz = 1;
      while (top > 0 && size[top - 1] == sz) {
        x = __dadd_rn(stack[top - 1], x);
        sz *= 2;
        top--;
      }
      stack[top] = x;
      size[top] = sz;
      top++;
    }
    part[threadIdx.x] = stack[0];
  }
  __syncthreads();
  for (int w = nt / 2; w >= 1; w /= 2) {
    double x = 0.0;
    if (threadIdx.x < w) x = __dadd_rn(part[2 * threadIdx.x], part[2 * threadIdx.x + 1]);
    __syncthreads();
    if (threadIdx.x < w) part[threadIdx.x] = x;
    __syncthreads();
  }
  if (threadIdx.x == 0) out[l] = part[0];
}

// ---- lists -----------------------------------------------------------------------
__device__ __forceinline__ bool well_separated(const double* __restrict__ c, const double* __restrict__ rad,
                                               int64_t gs, int64_t gt, double theta) {
  const double dx = __dsub_rn(c[3 * gs], c[3 * gt]);
  const double dy = __dsub_rn(c[3 * gs + 1], c[3 * gt + 1]);
  const double dz = __dsub_rn(c[3 * gs + 2], c[3 * gt + 2]);
  double d2 = __dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy));
  d2 = __dadd_rn(d2, __dmul_rn(dz, dz));
  const double d = __dsqrt_rn(d2);
  const double rs = rad[gs], rt = rad[gt];
  const double R = rs > rt ? rs : rt;
  const double r = rs > rt ? rt : rs;
  const double lhs = __dadd_rn(R, __dmul_rn(theta, r));
  const double rhs = __dmul_rn(theta, d);
  return d > 0.0 && lhs <= rhs;
}

// Box centres as double-float pairs (hi, lo per coordinate) and radii in
// FP32, for the FP32 pre-test of Eq. 4 below.
__global__ void centre_pairs_kernel(int64_t nb, const double* __restrict__ center, const double* __restrict__ radius,
                                    float* __restrict__ cf, float* __restrict__ rf) {
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < nb; g += (int64_t)gridDim.x * blockDim.x) {
    for (int a = 0; a < 3; a++) {
      const double c = center[3 * g + a];
      const float h = (float)c;
      cf[6 * g + a] = h;
      cf[6 * g + 3 + a] = (float)(c - (double)h);
    }
    rf[g] = (float)radius[g];
  }
}

// Eq. 4 on every candidate pair; the two flags (well separated, kept) are
// packed as ws + (keep << 32) so that one scan yields both prefix counts
// (each stays below 2^32).  The test is decided in FP32 when its two sides
// differ by far more than the FP32 evaluation can be off (relative 1e-5
// against a bound of about 1e-6, plus the double-float centres' absolute
// error); the remaining near-ties, zero distances and huge coordinate
// ranges take the FP64 sequence that the oracle uses, so every decision is
// the FP64 one.
__global__ void ws_kernel(const int32_t* __restrict__ ct, const int32_t* __restrict__ cs, int64_t nc,
                          int64_t offt, int64_t offs, const double* __restrict__ center,
                          const double* __restrict__ radius, const float* __restrict__ cf,
                          const float* __restrict__ rf, double theta, int64_t* __restrict__ flags) {
  const float thf = (float)theta;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nc; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t gs = offs + cs[e], gt = offt + ct[e];
    const float* a = cf + 6 * gs;
    const float* b = cf + 6 * gt;
    const float dx = (a[0] - b[0]) + (a[3] - b[3]);
    const float dy = (a[1] - b[1]) + (a[4] - b[4]);
    const float dz = (a[2] - b[2]) + (a[5] - b[5]);
    const float d = sqrtf(fmaf(dx, dx, fmaf(dy, dy, dz * dz)));
    const float ra = rf[gs], rb = rf[gt];
    const float R = fmaxf(ra, rb), r = fminf(ra, rb);
    const float lhs = fmaf(thf, r, R), rhs = thf * d;
    const float mag = fabsf(a[0]) + fabsf(a[1]) + fabsf(a[2]) + fabsf(b[0]) + fabsf(b[1]) + fabsf(b[2]);
    const float guard = 1e-5f * (lhs + rhs) + 1e-12f * mag;
    bool w;
    if (d > 0.f && lhs + guard < rhs) w = true;
    else if (d > 0.f && lhs > rhs + guard) w = false;
    else w = well_separated(center, radius, gs, gt, theta);
    flags[e] = w ? 1 : ((int64_t)1 << 32);
  }
}

__global__ void emit_kernel(const int32_t* __restrict__ ct, const int32_t* __restrict__ cs, int64_t nc,
                            int64_t offt, int64_t offs, const int64_t* __restrict__ flags,
                            const int64_t* __restrict__ pref, int32_t* __restrict__ mt, int32_t* __restrict__ ms,
                            int32_t* __restrict__ kt, int32_t* __restrict__ ks) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nc; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t p = pref[e];
    if (flags[e] & 1) {
      const int64_t o = p & 0xffffffffll;
      mt[o] = (int32_t)(offt + ct[e]);
      ms[o] = (int32_t)(offs + cs[e]);
    } else {
      const int64_t o = p >> 32;
      kt[o] = ct[e];
      ks[o] = cs[e];
    }
  }
}

__device__ __forceinline__ int64_t lower_bound32(const int32_t* a, int64_t n, int32_t v) {
  int64_t lo = 0, hi = n;
  while (lo < hi) {
    int64_t mid = (lo + hi) >> 1;
    if (a[mid] < v) lo = mid + 1;
    else hi = mid;
  }
  return lo;
}

// children of the advanced side (adv: 1 source, 0 target, 2 both); the result
// stays sorted by (target, source)
__global__ void expand_kernel(const int32_t* __restrict__ kt, const int32_t* __restrict__ ks, int64_t nk,
                              int nch, int adv, int32_t* __restrict__ ct, int32_t* __restrict__ cs) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nk; e += (int64_t)gridDim.x * blockDim.x) {
    const int32_t t = kt[e], s = ks[e];
    if (adv == 2) {
      const int64_t first = lower_bound32(kt, nk, t);
      const int64_t last = lower_bound32(kt, nk, t + 1);
      const int64_t k = last - first;
      for (int c = 0; c < nch; c++)
        for (int d = 0; d < nch; d++) {
          const int64_t o = (int64_t)nch * nch * first + (int64_t)c * nch * k + (e - first) * nch + d;
          ct[o] = nch * t + c;
          cs[o] = nch * s + d;
        }
    } else if (adv == 1) {
      for (int c = 0; c < nch; c++) {
        ct[nch * e + c] = t;
        cs[nch * e + c] = nch * s + c;
      }
    } else {
      const int64_t first = lower_bound32(kt, nk, t);
      const int64_t last = lower_bound32(kt, nk, t + 1);
      const int64_t k = last - first;
      for (int c = 0; c < nch; c++) {
        const int64_t o = nch * first + c * k + (e - first);
        ct[o] = nch * t + c;
        cs[o] = s;
      }
    }
  }
}


// Lists of one march step are sorted by target, so each target forms one run
// of consecutive entries.  run_start_kernel records where each target's run
// begins; m2l_scatter_kernel places entry e of the run of g at off[g] +
// fill[g] + (e - start of the run); m2l_fill_kernel adds each run's length to
// fill[g] (also used to count the entries per target).
__global__ void run_start_kernel(const int32_t* __restrict__ mt, int64_t nm, int64_t* __restrict__ rs) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nm; e += (int64_t)gridDim.x * blockDim.x) {
    const int32_t g = mt[e];
    if (e == 0 || mt[e - 1] != g) rs[g] = e;
  }
}

__global__ void m2l_scatter_kernel(const int32_t* __restrict__ mt, const int32_t* __restrict__ ms, int64_t nm,
                                   const int64_t* __restrict__ off, const int64_t* __restrict__ fill,
                                   const int64_t* __restrict__ rs, int32_t* __restrict__ out_t,
                                   int32_t* __restrict__ out_s) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nm; e += (int64_t)gridDim.x * blockDim.x) {
    const int32_t g = mt[e];
    const int64_t pos = off[g] + fill[g] + (e - rs[g]);
    out_t[pos] = g;
    out_s[pos] = ms[e];
  }
}

__global__ void m2l_fill_kernel(const int32_t* __restrict__ mt, int64_t nm, int64_t* __restrict__ fill) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nm; e += (int64_t)gridDim.x * blockDim.x) {
    const int32_t g = mt[e];
    if (e == 0 || mt[e - 1] != g) fill[g] += lower_bound32(mt, nm, g + 1) - e;
  }
}

// ---- rotation coefficients -----------------------------------------------------------
// For t = c_old - c_new: 1/r and cos/sin of the multiples of the polar angle
// theta and azimuth phi of t, in FP64 by angle addition, stored in FP64
// (g64) and rounded to FP32 (g32); either may be NULL (the FP64 copies are
// made only once a tree's precision needs them).
__device__ void trig_rows(const double t[3], int p, int64_t e, int64_t stride, int f0, double* g64, float* g32,
                          double* rout) {
  const double rxy = sqrt(t[0] * t[0] + t[1] * t[1]);
  const double r = sqrt(rxy * rxy + t[2] * t[2]);
  double ct = 1.0, st = 0.0, cp = 1.0, sp = 0.0;
  if (r > 0.0) {
    ct = t[2] / r;
    st = rxy / r;
  }
  if (rxy > 0.0) {
    cp = t[0] / rxy;
    sp = t[1] / rxy;
  }
  double cpm = 1.0, spm = 0.0, ctm = 1.0, stm = 0.0;
  for (int m = 1; m <= p; m++) {
    double a = cpm * cp - spm * sp, b = spm * cp + cpm * sp;
    cpm = a;
    spm = b;
    a = ctm * ct - stm * st;
    b = stm * ct + ctm * st;
    ctm = a;
    stm = b;
    const int64_t rows[4] = {f0 + m - 1, f0 + p + m - 1, f0 + 2 * p + m - 1, f0 + 3 * p + m - 1};
    const double vals[4] = {cpm, spm, ctm, stm};
    for (int k = 0; k < 4; k++) {
      if (g64) g64[rows[k] * stride + e] = vals[k];
      if (g32) g32[rows[k] * stride + e] = (float)vals[k];
    }
  }
  *rout = r;
}

// M2L records: 1/r, rho_S/r, rho_T/r and the cosines and sines of the polar
// angle theta and azimuth phi of t = c_S - c_T, in FP64 (g64) and rounded to
// FP32 (g32); either may be NULL.
__global__ void m2l_geo_kernel(const int32_t* __restrict__ mt, const int32_t* __restrict__ ms, int64_t nm,
                               const double* __restrict__ center, const double* __restrict__ radius, int p,
                               double* __restrict__ g64, float* __restrict__ g32) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nm; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t gt = mt[e], gs = ms[e];
    const double t[3] = {center[3 * gs] - center[3 * gt], center[3 * gs + 1] - center[3 * gt + 1],
                         center[3 * gs + 2] - center[3 * gt + 2]};
    if (!g64) {
      // FP32 records only: t in FP64 (a difference of nearby centres), the
      // rest in FP32 (a few roundings, like the records' own rounding)
      const float tx = (float)t[0], ty = (float)t[1], tz = (float)t[2];
      const float rxy = sqrtf(fmaf(tx, tx, ty * ty));
      const float r = sqrtf(fmaf(rxy, rxy, tz * tz));
      const float ri = 1.0f / r;
      const float rxyi = rxy > 0.f ? 1.0f / rxy : 0.f;
      const float vals[7] = {ri, (float)radius[gs] * ri, (float)radius[gt] * ri, rxy > 0.f ? tx * rxyi : 1.f,
                             rxy > 0.f ? ty * rxyi : 0.f, r > 0.f ? tz * ri : 1.f, r > 0.f ? rxy * ri : 0.f};
      for (int k = 0; k < 7; k++) g32[k * nm + e] = vals[k];
      continue;
    }
    const double rxy = sqrt(t[0] * t[0] + t[1] * t[1]);
    const double r = sqrt(rxy * rxy + t[2] * t[2]);
    double ct = 1.0, st = 0.0, cp = 1.0, sp = 0.0;
    if (r > 0.0) {
      ct = t[2] / r;
      st = rxy / r;
    }
    if (rxy > 0.0) {
      cp = t[0] / rxy;
      sp = t[1] / rxy;
    }
    const double vals[7] = {1.0 / r, radius[gs] / r, radius[gt] / r, cp, sp, ct, st};
    for (int k = 0; k < 7; k++) {
      if (g64) g64[k * nm + e] = vals[k];
      if (g32) g32[k * nm + e] = (float)vals[k];
    }
  }
  (void)p;
}

// M2M (t = c_child - c_parent) per child box; boxes without a parent (the
// roots) get zero rows.  m64 / m32 may be NULL.
__global__ void edge_geo_kernel(int64_t nbox, const int32_t* __restrict__ parent, const double* __restrict__ center,
                                const double* __restrict__ radius, int p, double* __restrict__ m64,
                                float* __restrict__ m32) {
  const int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (g >= nbox) return;
  const int64_t gp = parent[g];
  if (gp < 0) {
    for (int f = 0; f < 2 + 4 * p; f++) {
      if (m64) m64[f * nbox + g] = 0;
      if (m32) m32[f * nbox + g] = 0;
    }
    return;
  }
  const double t[3] = {center[3 * g] - center[3 * gp], center[3 * g + 1] - center[3 * gp + 1],
                       center[3 * g + 2] - center[3 * gp + 2]};
  double r;
  trig_rows(t, p, g, nbox, 2, m64, m32, &r);
  const double rp = radius[gp];
  const double a = rp > 0.0 ? r / rp : 0.0, bb = rp > 0.0 ? radius[g] / rp : 0.0;
  if (m64) {
    m64[g] = a;
    m64[nbox + g] = bb;
  }
  if (m32) {
    m32[g] = (float)a;
    m32[nbox + g] = (float)bb;
  }
}

// Direct L2L records (one per target leaf and ancestor with a non-empty M2L
// list, nearest ancestor first): t = c_ancestor - c_leaf, the axial
// parameters |t| / rho_a and rho_leaf / rho_a, and the rotation angles.
__device__ __forceinline__ bool has_m2l(const int64_t* __restrict__ m2l_off, int64_t a) {
  return m2l_off[a + 1] > m2l_off[a];
}
__global__ void l2d_count_kernel(int64_t nl, const int32_t* __restrict__ leaf_box, const int32_t* __restrict__ parent,
                                 const int64_t* __restrict__ m2l_off, int64_t* __restrict__ cnt) {
  const int64_t leaf = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (leaf >= nl) return;
  int64_t c = 0;
  for (int64_t a = parent[leaf_box[leaf]]; a >= 0; a = parent[a]) c += has_m2l(m2l_off, a) ? 1 : 0;
  cnt[leaf] = c;
}
__global__ void l2d_fill_kernel(int64_t nl, const int32_t* __restrict__ leaf_box, const int32_t* __restrict__ parent,
                                const int64_t* __restrict__ m2l_off, const int64_t* __restrict__ off,
                                const double* __restrict__ center, const double* __restrict__ radius, int p,
                                int64_t n_rec, int32_t* __restrict__ anc, double* __restrict__ e64,
                                float* __restrict__ e32) {
  const int64_t leaf = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (leaf >= nl) return;
  const int64_t g = leaf_box[leaf];
  int64_t e = off[leaf];
  for (int64_t a = parent[g]; a >= 0; a = parent[a]) {
    if (!has_m2l(m2l_off, a)) continue;
    if (anc) anc[e] = (int32_t)a;
    const double t[3] = {center[3 * a] - center[3 * g], center[3 * a + 1] - center[3 * g + 1],
                         center[3 * a + 2] - center[3 * g + 2]};
    double r;
    trig_rows(t, p, e, n_rec, 2, e64, e32, &r);
    const double ra = radius[a];
    const double va = ra > 0.0 ? r / ra : 0.0, vb = ra > 0.0 ? radius[g] / ra : 0.0;
    if (e64) {
      e64[e] = va;
      e64[n_rec + e] = vb;
    }
    if (e32) {
      e32[e] = (float)va;
      e32[n_rec + e] = (float)vb;
    }
    e++;
  }
}

// Are two distinct points at exactly the same position?  Open-addressing
// hash table over the coordinate bits (splitmix64 finaliser), load factor
// <= 1/2, probing bounded by the table size.
__device__ __forceinline__ unsigned long long mix64(unsigned long long z) {
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
  return z ^ (z >> 31);
}
__global__ void duplicate_kernel(const double* __restrict__ X, int64_t n, int* __restrict__ tab, int64_t mask,
                                 int* __restrict__ found) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const double x = X[i], y = X[n + i], z = X[2 * n + i];
    unsigned long long h = mix64((unsigned long long)__double_as_longlong(x));
    h = mix64(h ^ (unsigned long long)__double_as_longlong(y));
    h = mix64(h ^ (unsigned long long)__double_as_longlong(z));
    int64_t slot = (int64_t)(h & (unsigned long long)mask);
    for (int64_t probe = 0; probe <= mask; probe++) {
      const int prev = atomicCAS(&tab[slot], -1, (int)i);
      if (prev == -1) break;
      if (X[prev] == x && X[n + prev] == y && X[2 * n + prev] == z) {
        atomicOr(found, 1);
        break;
      }
      slot = (slot + 1) & mask;
    }
  }
}

// near-field entries: source leaf, FP32 centre offset, the flag that zero
// distances are possible (coincident points may exist and the leaves'
// bounding boxes touch; without boxes (lo == NULL) the bounding spheres of
// radius `radius` are tested instead) and the FP32 coincidence threshold
__global__ void p2p_entry_kernel(const int32_t* __restrict__ pt, const int32_t* __restrict__ ps, int64_t np,
                                 int64_t trg_base, int64_t src_base, const double* __restrict__ center,
                                 const double* __restrict__ radius, const double* __restrict__ lo,
                                 const double* __restrict__ hi, const int32_t* __restrict__ bc, int has_dup,
                                 P2PEntry* __restrict__ ent, float* __restrict__ thr,
                                 unsigned long long* __restrict__ pairs) {
  for (int64_t e0 = (blockIdx.x * (int64_t)blockDim.x) & ~31ll; e0 < np; e0 += (int64_t)gridDim.x * blockDim.x) {
    const int64_t e = e0 + (threadIdx.x & 31) + (threadIdx.x & ~31);
    unsigned long long w = 0;
    if (e < np) {
      const int64_t gt = trg_base + pt[e], gs = src_base + ps[e];
      bool touch = has_dup != 0;
      if (lo) {
        for (int a = 0; a < 3; a++)
          touch = touch && lo[3 * gt + a] <= hi[3 * gs + a] && lo[3 * gs + a] <= hi[3 * gt + a];
      } else {
        const double dx = center[3 * gt] - center[3 * gs], dy = center[3 * gt + 1] - center[3 * gs + 1],
                     dz = center[3 * gt + 2] - center[3 * gs + 2];
        const double rr = radius[gt] + radius[gs];
        touch = touch && (dx * dx + dy * dy + dz * dz) <= 1.0000001 * rr * rr;
      }
      P2PEntry en;
      en.src = ps[e] | (touch ? (int)0x80000000 : 0);
      en.dx = (float)(center[3 * gt] - center[3 * gs]);
      en.dy = (float)(center[3 * gt + 1] - center[3 * gs + 1]);
      en.dz = (float)(center[3 * gt + 2] - center[3 * gs + 2]);
      ent[e] = en;
      // FP32 leaf-local coordinates of coincident points differ by at most a
      // few units in the last place of the leaves' extent: squared distances
      // below (1e-5 max radius)^2 are taken as zero distances
      const double rm = 1e-5 * fmax(radius[gt], radius[gs]);
      thr[e] = (float)(rm * rm);
      w = (unsigned long long)bc[gt] * (unsigned long long)bc[gs];
    }
    for (int o = 16; o > 0; o >>= 1) w += __shfl_xor_sync(0xffffffffu, w, o);
    if ((threadIdx.x & 31) == 0 && w) atomicAdd(pairs, w);
  }
}

// tree-ordered point records: FP64 position and FP32 offset from the leaf centre
__global__ void point_records_kernel(const double* __restrict__ X, int64_t n, const int64_t* __restrict__ bs,
                                     const int32_t* __restrict__ bc, int64_t leaf_off, int64_t n_leaves,
                                     const double* __restrict__ center, float4* __restrict__ loc,
                                     dvec4* __restrict__ p64) {
  const int lane = threadIdx.x & 31;
  const int64_t w = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  if (w >= n_leaves) return;
  const int64_t g = leaf_off + w;
  const int64_t a = bs[g];
  const int c = bc[g];
  for (int i = lane; i < c; i += 32) {
    const int64_t k = a + i;
    const double x = X[k], y = X[n + k], z = X[2 * n + k];
    p64[k] = dvec4{x, y, z, 0.0};
    loc[k] = make_float4((float)(x - center[3 * g]), (float)(y - center[3 * g + 1]),
                         (float)(z - center[3 * g + 2]), 0.0f);
  }
}

template <class T>
void dfree(T*& p) {
  if (p) dev_free(p);
  p = nullptr;
}

template <class T>
std::vector<T> to_host(const T* d, int64_t n, cudaStream_t st) {
  std::vector<T> h((size_t)std::max<int64_t>(n, 0));
  if (n > 0) FMM_CUDA_TRY(cudaMemcpyAsync(h.data(), d, sizeof(T) * n, cudaMemcpyDeviceToHost, st));
  FMM_CUDA_TRY(cudaStreamSynchronize(st));
  return h;
}

// Hierarchy of one point set (Sec. II.A): tree order, box ranges, geometry,
// index lists, level averages, point records and M2M/L2L edge coefficients.
// The leaf bounding boxes (3 n_boxes lo and hi) are handed to the caller.
void build_hierarchy(fmm_tree* t, const double* pos, cudaStream_t st, double** blo_out, double** bhi_out) {
  const int64_t n = t->n;
  const int s = t->prm.splits;
  const int nch = 1 << s;
  const int L = t->L;
  const int R = L * s;
  t->s = s;
  t->n_boxes = level_offset(L + 1, s);
  t->n_leaves = (int64_t)1 << (s * L);
  const int64_t NB = t->n_boxes, NL = t->n_leaves;
  const int64_t leaf_off = level_offset(L, s);
  t->max_leaf = (int)((n + NL - 1) / NL);
  t->min_leaf = (int)(n / NL);  // median splits: every leaf holds floor or ceil of n / NL

  // ---- canonical SoA copy, validation ----
  double* Xa = scratch_alloc<double>(3 * (size_t)n);
  double* Xb = scratch_alloc<double>(3 * (size_t)n);
  int32_t* Ia = scratch_alloc<int32_t>(n);
  int32_t* Ib = scratch_alloc<int32_t>(n);
  int* flag = scratch_alloc<int>(4);
  FMM_CUDA_TRY(cudaMemsetAsync(flag, 0, 4 * sizeof(int), st));
  canon_kernel<<<grid_for(n, 256), 256, 0, st>>>(pos, n, (t->prm.flags & FMM_POS_SOA) ? 1 : 0, Xa, Ia, flag);
  FMM_LAUNCH_CHECK();
  // the duplicate test runs on whatever was read (a non-finite position
  // makes its answer meaningless, not unsafe), so that one round trip
  // returns both flags
  int hflag[2] = {0, 0};
  {
    int64_t tsize = 1;
    while (tsize < 2 * n) tsize <<= 1;
    int* tab = scratch_alloc<int>(tsize);
    FMM_CUDA_TRY(cudaMemsetAsync(tab, 0xff, sizeof(int) * tsize, st));
    duplicate_kernel<<<grid_for(n, 256), 256, 0, st>>>(Xa, n, tab, tsize - 1, flag + 1);
    FMM_LAUNCH_CHECK();
    FMM_CUDA_TRY(cudaMemcpyAsync(hflag, flag, 2 * sizeof(int), cudaMemcpyDeviceToHost, st));
    FMM_CUDA_TRY(cudaStreamSynchronize(st));
    dev_free(tab);
  }
  if (hflag[0]) {
    dev_free(Xa), dev_free(Xb), dev_free(Ia), dev_free(Ib), dev_free(flag);
    require(false, "positions must be finite");
  }
  const int has_dup = hflag[1];
  t->has_duplicates = has_dup;
  trace_mark("canon + duplicates");

  // ---- segment boundaries of every round (closed form) ----
  std::vector<int64_t> round_off(R + 2);
  int64_t tot = 0;
  for (int r = 0; r <= R; r++) {
    round_off[r] = tot;
    tot += ((int64_t)1 << r) + 1;
  }
  int64_t* starts = dev_alloc<int64_t>(nullptr, tot);
  {
    int64_t h0[2] = {0, n};
    FMM_CUDA_TRY(cudaMemcpyAsync(starts, h0, sizeof(h0), cudaMemcpyHostToDevice, st));
    for (int r = 0; r < R; r++) {
      const int ns = 1 << r;
      split_starts_kernel<<<(ns + 255) / 256, 256, 0, st>>>(starts + round_off[r], ns, starts + round_off[r + 1]);
      FMM_LAUNCH_CHECK();
    }
  }

  // ---- large rounds ----
  int r0 = 0;
  while (r0 < R && (n + ((int64_t)1 << r0) - 1) / ((int64_t)1 << r0) > kSmallCap) r0++;
  if (r0 > 0) {
    const int maxseg = 1 << (r0 - 1);
    unsigned long long* bmin = scratch_alloc<unsigned long long>(3 * (size_t)maxseg);
    unsigned long long* bmax = scratch_alloc<unsigned long long>(3 * (size_t)maxseg);
    unsigned long long* ctr = scratch_alloc<unsigned long long>(2 * (size_t)maxseg);
    unsigned* hist = scratch_alloc<unsigned>(256 * (size_t)maxseg);
    Sel* sel = scratch_alloc<Sel>(maxseg);
    int* uflag = scratch_alloc<int>(12);  // per digit: some segment still unresolved
    FMM_CUDA_TRY(cudaMemsetAsync(hist, 0, sizeof(unsigned) * 256 * (size_t)maxseg, st));
    const int nblk = (int)((n + kChunk - 1) / kChunk);
    int guess = 5;  // digits queued before the first look (random keys of ~2^20 points)
    for (int r = 0; r < r0; r++) {
      const int ns = 1 << r;
      const int64_t* stt = starts + round_off[r];
      FMM_CUDA_TRY(cudaMemsetAsync(bmin, 0xff, sizeof(unsigned long long) * 3 * ns, st));
      FMM_CUDA_TRY(cudaMemsetAsync(bmax, 0, sizeof(unsigned long long) * 3 * ns, st));
      seg_bbox_kernel<<<nblk, kThreads, 0, st>>>(Xa, n, stt, ns, bmin, bmax);
      FMM_LAUNCH_CHECK();
      seg_axis_kernel<<<(ns + 255) / 256, 256, 0, st>>>(bmin, bmax, stt, ns, sel);
      FMM_LAUNCH_CHECK();
      // 8-bit digits of the 96-bit key.  As many digits as the previous
      // round needed are queued at once (a resolved segment skips the later
      // passes, and once every segment is resolved the remaining launches
      // return at once); one host round trip reads the per-digit flags, and
      // more digits follow only if some segment is still unresolved
      FMM_CUDA_TRY(cudaMemsetAsync(uflag, 0, sizeof(int) * 12, st));
      int queued = 0, need = 12;
      while (queued < 12) {
        const int upto = std::min(12, queued == 0 ? guess : queued + 1);
        for (int d = queued; d < upto; d++) {
          const int* prev = d > 0 ? uflag + d - 1 : nullptr;
          radix_hist_kernel<<<nblk, kThreads, 0, st>>>(Xa, Ia, n, stt, ns, sel, d, hist, prev);
          FMM_LAUNCH_CHECK();
          radix_select_kernel<<<(ns + 3) / 4, 128, 0, st>>>(sel, ns, d, hist, prev, uflag + d);
          FMM_LAUNCH_CHECK();
        }
        queued = upto;
        int hf[12];
        FMM_CUDA_TRY(cudaMemcpyAsync(hf, uflag, sizeof(int) * queued, cudaMemcpyDeviceToHost, st));
        FMM_CUDA_TRY(cudaStreamSynchronize(st));
        int d = 0;
        while (d < queued && hf[d]) d++;
        if (d < queued) {
          need = d + 1;  // digit d left every segment resolved
          break;
        }
      }
      guess = std::max(need, 2);
      FMM_CUDA_TRY(cudaMemsetAsync(ctr, 0, sizeof(unsigned long long) * 2 * ns, st));
      partition_kernel<<<nblk, kThreads, 0, st>>>(Xa, Ia, n, stt, ns, sel, ctr, Xb, Ib);
      FMM_LAUNCH_CHECK();
      std::swap(Xa, Xb);
      std::swap(Ia, Ib);
    }
    FMM_CUDA_TRY(cudaStreamSynchronize(st));
    dev_free(bmin), dev_free(bmax), dev_free(ctr), dev_free(hist), dev_free(sel), dev_free(uflag);
  }
  trace_mark("large bisection rounds");

  // ---- remaining rounds and the leaf sort, one CTA per segment ----
  t->perm = dev_alloc<int32_t>(t, n);
  {
    const int rounds = R - r0;
    require(rounds <= kSmallMaxRounds, "segment rounds beyond the small-segment kernel's tables");
    const size_t smem = small_smem_bytes(rounds);
    // one constant limit for every build (builds on other threads launch
    // this kernel concurrently; a per-launch value could undercut theirs)
    FMM_CUDA_TRY(cudaFuncSetAttribute(small_segment_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)small_smem_bytes(kSmallMaxRounds)));
    FMM_CUDA_TRY(cudaFuncSetAttribute(small_segment_kernel, cudaFuncAttributePreferredSharedMemoryCarveout,
                                      (int)cudaSharedmemCarveoutMaxShared));
    small_segment_kernel<<<1 << r0, kSmallThreads, smem, st>>>(Xa, Ia, n, starts + round_off[r0], rounds, Xb,
                                                               t->perm);
    FMM_LAUNCH_CHECK();
    std::swap(Xa, Xb);  // Xa: positions in tree order
  }
  trace_mark("small segments + leaf order");

  // ---- box ranges and geometry ----
  t->box_start = dev_alloc<int64_t>(t, NB);
  t->box_count = dev_alloc<int32_t>(t, NB);
  t->center = dev_alloc<double>(t, 3 * NB);
  t->radius = dev_alloc<double>(t, NB);
  t->inv_rho32 = dev_alloc<float>(t, NB);
  t->inv_rho64 = dev_alloc<double>(t, NB);
  double* blo = dev_alloc<double>(t, 3 * NB);
  double* bhi = dev_alloc<double>(t, 3 * NB);
  for (int l = 0; l <= L; l++) {
    const int64_t nb = (int64_t)1 << (s * l);
    box_range_kernel<<<grid_for(nb, 256, 1 << 30), 256, 0, st>>>(starts + round_off[l * s], nb, level_offset(l, s),
                                                                 t->box_start, t->box_count);
    FMM_LAUNCH_CHECK();
  }
  leaf_bbox_kernel<<<grid_for(NL * 32, 256, 1 << 30), 256, 0, st>>>(Xa, n, t->box_start, t->box_count, leaf_off, NL,
                                                                    blo, bhi);
  FMM_LAUNCH_CHECK();
  for (int l = L - 1; l >= 0; l--) {
    const int64_t nb = (int64_t)1 << (s * l);
    parent_bbox_kernel<<<grid_for(nb, 256, 1 << 30), 256, 0, st>>>(nb, level_offset(l, s), level_offset(l + 1, s), nch,
                                                                   blo, bhi);
    FMM_LAUNCH_CHECK();
  }
  centre_radius_kernel<<<grid_for(NB, 256, 1 << 30), 256, 0, st>>>(NB, blo, bhi, t->center, t->radius, t->inv_rho32,
                                                                   t->inv_rho64);
  FMM_LAUNCH_CHECK();
  trace_mark("box ranges + geometry");
  // index lists: a single tree's M2M round r holds level L - r (children of
  // a parent consecutive)
  t->leaf_box = dev_alloc<int32_t>(t, NL);
  t->box_parent = dev_alloc<int32_t>(t, NB);
  t->up_ids = dev_alloc<int32_t>(t, NB);
  index_lists_kernel<<<grid_for(NB, 256, 1 << 30), 256, 0, st>>>(NB, s, L, t->leaf_box, t->box_parent);
  FMM_LAUNCH_CHECK();
  t->n_up = L;
  t->up_off_h = new int64_t[L + 1];
  {
    std::vector<int32_t> up;
    up.reserve((size_t)NB);
    for (int r = 0; r < L; r++) {
      t->up_off_h[r] = (int64_t)up.size();
      for (int64_t g = level_offset(L - r, s); g < level_offset(L - r + 1, s); g++) up.push_back((int32_t)g);
    }
    t->up_off_h[L] = (int64_t)up.size();
    if (!up.empty())
      FMM_CUDA_TRY(cudaMemcpyAsync(t->up_ids, up.data(), sizeof(int32_t) * up.size(), cudaMemcpyHostToDevice, st));
    FMM_CUDA_TRY(cudaStreamSynchronize(st));
  }

  // ---- average radius per level ----
  t->level_avg_host = new double[L + 1];
  {
    double* sums = scratch_alloc<double>(L + 1);
    level_sum_kernel<<<L + 1, kLevelSumThreads, 0, st>>>(t->radius, s, sums);
    FMM_LAUNCH_CHECK();
    std::vector<double> h(L + 1);
    FMM_CUDA_TRY(cudaMemcpyAsync(h.data(), sums, sizeof(double) * (L + 1), cudaMemcpyDeviceToHost, st));
    FMM_CUDA_TRY(cudaStreamSynchronize(st));
    dev_free(sums);
    for (int l = 0; l <= L; l++) t->level_avg_host[l] = h[l] / (double)((int64_t)1 << (s * l));
  }
  trace_mark("index lists + level averages");

  // ---- point records and M2M edge coefficients ----
  const int p = t->prm.p;
  t->pos_local = dev_alloc<float4>(t, n);
  t->pos64 = dev_alloc<dvec4>(t, n);
  point_records_kernel<<<grid_for(NL * 32, 256, 1 << 30), 256, 0, st>>>(Xa, n, t->box_start, t->box_count, leaf_off,
                                                                        NL, t->center, t->pos_local, t->pos64);
  FMM_LAUNCH_CHECK();
  t->m2m32 = dev_alloc<float>(t, (size_t)edge_fields(p) * NB);
  edge_geo_kernel<<<grid_for(NB, 128, 1 << 30), 128, 0, st>>>(NB, t->box_parent, t->center, t->radius, p, nullptr,
                                                              t->m2m32);
  FMM_LAUNCH_CHECK();
  FMM_CUDA_TRY(cudaStreamSynchronize(st));
  t->device_bytes -= sizeof(double) * 6 * NB;  // bounding boxes leave with the caller
  *blo_out = blo;
  *bhi_out = bhi;
  dev_free(starts);
  dev_free(Xa), dev_free(Xb), dev_free(Ia), dev_free(Ib), dev_free(flag);
  trace_mark("point records + edges");
}

// One side of the list construction: the combined id of the side's root and
// its depth and level averages.
struct Side {
  int64_t base;
  int L;
  const double* avg;
};
struct Step {
  int32_t *t, *s;
  int64_t n;
};

// Interaction lists between the boxes of a source side and a target side
// (Sec. II.B): level march, or same-level lists with FMM_SAME_LEVEL.  M2L
// pairs (combined ids) per step; the pairs left at both leaf levels are the
// near field (target leaf, source leaf), sorted by (target, source).
void march(const fmm_tree* t, Side S, Side T, cudaStream_t st, std::vector<Step>& steps, int32_t** p2p_t_out,
           int32_t** p2p_s_out, int64_t* np_out) {
  const int s = t->prm.splits;
  const int nch = 1 << s;
  int32_t* ct = dev_alloc<int32_t>(nullptr, 1);
  int32_t* cs = dev_alloc<int32_t>(nullptr, 1);
  FMM_CUDA_TRY(cudaMemsetAsync(ct, 0, sizeof(int32_t), st));
  FMM_CUDA_TRY(cudaMemsetAsync(cs, 0, sizeof(int32_t), st));
  int64_t nc = 1;
  int ls = 0, lt = 0;
  int32_t *p2p_t = nullptr, *p2p_s = nullptr;
  int64_t np = 0;
  const bool tie_target = (t->prm.flags & FMM_TIE_TARGET) != 0;
  const bool same_level = (t->prm.flags & FMM_SAME_LEVEL) != 0;
  float* cf = scratch_alloc<float>(6 * (size_t)t->n_boxes);
  float* rf = scratch_alloc<float>(t->n_boxes);
  centre_pairs_kernel<<<grid_for(t->n_boxes, 256), 256, 0, st>>>(t->n_boxes, t->center, t->radius, cf, rf);
  FMM_LAUNCH_CHECK();
  for (;;) {
    require(nc < ((int64_t)1 << 32), "too many candidate pairs in one level-march step");
    int64_t* flags = scratch_alloc<int64_t>(nc);
    int64_t* pref = scratch_alloc<int64_t>(nc);
    const int64_t offt = T.base + level_offset(lt, s), offs = S.base + level_offset(ls, s);
    ws_kernel<<<grid_for(nc, 256), 256, 0, st>>>(ct, cs, nc, offt, offs, t->center, t->radius, cf, rf,
                                                 t->prm.theta, flags);
    FMM_LAUNCH_CHECK();
    const int64_t both = exclusive_scan(flags, pref, nc, st);
    const int64_t nws = both & 0xffffffffll, nkeep = both >> 32;
    Step stp{dev_alloc<int32_t>(nullptr, nws), dev_alloc<int32_t>(nullptr, nws), nws};
    int32_t* kt = dev_alloc<int32_t>(nullptr, nkeep);
    int32_t* ks = dev_alloc<int32_t>(nullptr, nkeep);
    emit_kernel<<<grid_for(nc, 256), 256, 0, st>>>(ct, cs, nc, offt, offs, flags, pref, stp.t, stp.s, kt, ks);
    FMM_LAUNCH_CHECK();
    dev_free(flags), dev_free(pref), dev_free(ct), dev_free(cs);
    if (nws > 0) steps.push_back(stp);
    else dev_free(stp.t), dev_free(stp.s);
    if (nkeep == 0) {
      dev_free(kt), dev_free(ks);
      ct = cs = nullptr;
      break;
    }
    const bool can_s = ls < S.L, can_t = lt < T.L;
    if (!can_s && !can_t) {
      p2p_t = kt;
      p2p_s = ks;
      np = nkeep;
      ct = cs = nullptr;
      break;
    }
    int adv;  // 1 source, 0 target, 2 both (same-level lists)
    if (same_level) {
      adv = 2;
    } else if (can_s && can_t) {
      const double as = S.avg[ls], at = T.avg[lt];
      adv = (as > at) || (as == at && !tie_target) ? 1 : 0;
    } else {
      adv = can_s ? 1 : 0;
    }
    nc = nkeep * (adv == 2 ? nch * nch : nch);
    ct = dev_alloc<int32_t>(nullptr, nc);
    cs = dev_alloc<int32_t>(nullptr, nc);
    expand_kernel<<<grid_for(nkeep, 256), 256, 0, st>>>(kt, ks, nkeep, nch, adv, ct, cs);
    FMM_LAUNCH_CHECK();
    dev_free(kt), dev_free(ks);
    if (adv != 0) ls++;
    if (adv != 1) lt++;
  }
  dev_free(cf), dev_free(rf);
  *p2p_t_out = p2p_t;
  *p2p_s_out = p2p_s;
  *np_out = np;
  trace_mark("level march");
}

// Lists into their device form, per-interaction coefficients, near-field
// entries, work orders and the evaluation workspace.  Target leaves are the
// boxes trg_leaf_base .. + n_leaves - 1, source leaves src_leaf_base .. +
// n_src_leaves - 1 (combined ids).  blo/bhi: leaf bounding boxes for the
// coincident-point test, or NULL for the bounding-sphere test.
void finish_tree(fmm_tree* t, std::vector<Step>& steps, int32_t* p2p_t, int32_t* p2p_s, int64_t np,
                 int64_t trg_leaf_base, int64_t src_leaf_base, const double* blo, const double* bhi, int has_dup,
                 cudaStream_t st) {
  const int64_t NB = t->n_boxes, NL = t->n_leaves, NLS = t->n_src_leaves, n = t->n;
  const int p = t->prm.p;

  // ---- M2L lists as CSR by target, sources ascending ----
  int64_t nm = 0;
  for (auto& x : steps) nm += x.n;
  t->n_m2l = nm;
  t->m2l_off = dev_alloc<int64_t>(t, NB + 1);
  t->m2l_src = dev_alloc<int32_t>(t, nm);
  t->m2l_trg = dev_alloc<int32_t>(t, nm);
  {
    int64_t* cnt = scratch_alloc<int64_t>(NB + 1);
    int64_t* fill = scratch_alloc<int64_t>(NB + 1);
    int64_t* rs = scratch_alloc<int64_t>(NB + 1);
    FMM_CUDA_TRY(cudaMemsetAsync(cnt, 0, sizeof(int64_t) * (NB + 1), st));
    FMM_CUDA_TRY(cudaMemsetAsync(fill, 0, sizeof(int64_t) * (NB + 1), st));
    for (auto& x : steps) {
      m2l_fill_kernel<<<grid_for(x.n, 256), 256, 0, st>>>(x.t, x.n, cnt);
      FMM_LAUNCH_CHECK();
    }
    exclusive_scan(cnt, t->m2l_off, NB + 1, st);
    for (auto& x : steps) {
      run_start_kernel<<<grid_for(x.n, 256), 256, 0, st>>>(x.t, x.n, rs);
      FMM_LAUNCH_CHECK();
      m2l_scatter_kernel<<<grid_for(x.n, 256), 256, 0, st>>>(x.t, x.s, x.n, t->m2l_off, fill, rs, t->m2l_trg,
                                                             t->m2l_src);
      FMM_LAUNCH_CHECK();
      m2l_fill_kernel<<<grid_for(x.n, 256), 256, 0, st>>>(x.t, x.n, fill);
      FMM_LAUNCH_CHECK();
    }
    FMM_CUDA_TRY(cudaStreamSynchronize(st));
    dev_free(cnt), dev_free(fill), dev_free(rs);
    for (auto& x : steps) dev_free(x.t), dev_free(x.s);
    steps.clear();
  }
  trace_mark("M2L lists (CSR)");

  // ---- near-field lists as CSR by target leaf ----
  t->n_p2p = np;
  t->p2p_off = dev_alloc<int64_t>(t, NL + 1);
  t->p2p_src = dev_alloc<int32_t>(t, np);
  t->p2p32 = dev_alloc<P2PEntry>(t, np);
  t->p2p_thr = dev_alloc<float>(t, np);
  int32_t* p2p_trg = dev_alloc<int32_t>(nullptr, np);
  {
    int64_t* cnt = scratch_alloc<int64_t>(NL + 1);
    FMM_CUDA_TRY(cudaMemsetAsync(cnt, 0, sizeof(int64_t) * (NL + 1), st));
    if (np > 0) {
      m2l_fill_kernel<<<grid_for(np, 256), 256, 0, st>>>(p2p_t, np, cnt);  // runs by target leaf
      FMM_LAUNCH_CHECK();
      FMM_CUDA_TRY(cudaMemcpyAsync(t->p2p_src, p2p_s, sizeof(int32_t) * np, cudaMemcpyDeviceToDevice, st));
      FMM_CUDA_TRY(cudaMemcpyAsync(p2p_trg, p2p_t, sizeof(int32_t) * np, cudaMemcpyDeviceToDevice, st));
    }
    exclusive_scan(cnt, t->p2p_off, NL + 1, st);
    FMM_CUDA_TRY(cudaStreamSynchronize(st));
    dev_free(cnt);
    if (p2p_t) dev_free(p2p_t), dev_free(p2p_s);
  }
  trace_mark("near-field lists (CSR)");

  // ---- rotation coefficients and near-field entries ----
  t->geo32 = dev_alloc<float>(t, (size_t)m2l_fields(p) * std::max<int64_t>(nm, 1));
  trace_mark("  M2L records: allocation");
  if (nm > 0) {
    m2l_geo_kernel<<<grid_for(nm, 256), 256, 0, st>>>(t->m2l_trg, t->m2l_src, nm, t->center, t->radius, p, nullptr,
                                                      t->geo32);
    FMM_LAUNCH_CHECK();
  }
  trace_mark("M2L rotation records");
  build_l2l_direct(t, st);
  trace_mark("direct L2L records");
  {
    unsigned long long* pairs = scratch_alloc<unsigned long long>(1);
    FMM_CUDA_TRY(cudaMemsetAsync(pairs, 0, sizeof(unsigned long long), st));
    if (np > 0) {
      p2p_entry_kernel<<<grid_for(np, 256), 256, 0, st>>>(p2p_trg, t->p2p_src, np, trg_leaf_base, src_leaf_base,
                                                          t->center, t->radius, blo, bhi, t->box_count, has_dup,
                                                          t->p2p32, t->p2p_thr, pairs);
      FMM_LAUNCH_CHECK();
    }
    unsigned long long hp = 0;
    FMM_CUDA_TRY(cudaMemcpyAsync(&hp, pairs, sizeof(hp), cudaMemcpyDeviceToHost, st));
    FMM_CUDA_TRY(cudaStreamSynchronize(st));
    t->n_p2p_pairs = (int64_t)hp;
    dev_free(pairs);
  }
  dev_free(p2p_trg);

  trace_mark("near-field entries");
  // ---- work orders: longest M2L lists and heaviest near fields first ----
  build_work_orders(t, st);
  trace_mark("work orders");

  // ---- evaluation workspace ----
  const int NCP = ncoef_pad(p);
  t->src32 = dev_alloc<float4>(t, n);
  t->src_dup = dev_alloc<DupRec>(t, n);
  t->M32 = dev_alloc<float>(t, (size_t)NB * NCP);
  t->Lam32 = dev_alloc<float>(t, (size_t)NB * NCP);
  FMM_CUDA_TRY(cudaMemsetAsync(t->M32, 0, sizeof(float) * NB * NCP, st));
  FMM_CUDA_TRY(cudaMemsetAsync(t->Lam32, 0, sizeof(float) * NB * NCP, st));
  t->near_u = dev_alloc<double>(t, n);
  t->near_f = dev_alloc<double>(t, 3 * (size_t)n);
  if (!t->two_trees) {
    t->src_dup2 = dev_alloc<DupRec>(t, n);
    t->near_u2 = dev_alloc<float>(t, 2 * (size_t)n);
    t->near_f2 = dev_alloc<float>(t, 3 * (size_t)n);
  }
  t->q_stage = dev_alloc<double>(t, n);
  t->u_stage = dev_alloc<double>(t, n);
  t->f_stage = dev_alloc<double>(t, 3 * (size_t)n);
  t->g_stage = dev_alloc<double>(t, 3 * (size_t)n);
  {
    int lo_prio = 0, hi_prio = 0;
    FMM_CUDA_TRY(cudaDeviceGetStreamPriorityRange(&lo_prio, &hi_prio));
    FMM_CUDA_TRY(cudaStreamCreateWithPriority(&t->far_stream, cudaStreamNonBlocking, hi_prio));
    FMM_CUDA_TRY(cudaEventCreateWithFlags(&t->ev_fork, cudaEventDisableTiming));
    FMM_CUDA_TRY(cudaEventCreateWithFlags(&t->ev_join, cudaEventDisableTiming));
  }
  t->counters = dev_alloc<int>(t, 8);
  t->m2m_ready = dev_alloc<int>(t, NB);
  t->status = dev_alloc<int>(t, 1);
  FMM_CUDA_TRY(cudaMemsetAsync(t->status, 0, sizeof(int), st));
  FMM_CUDA_TRY(cudaStreamSynchronize(st));
  trace_mark("evaluation workspace");
}

template <class T>
void copy_d2d(T* dst, const T* src, int64_t n, cudaStream_t st) {
  if (n > 0) FMM_CUDA_TRY(cudaMemcpyAsync(dst, src, sizeof(T) * n, cudaMemcpyDeviceToDevice, st));
}

// field-major rows of `width` entries into rows of `total` entries at `col`
template <class T>
void copy_rows(T* dst, int64_t total, int64_t col, const T* src, int64_t width, int rows, cudaStream_t st) {
  if (width > 0)
    FMM_CUDA_TRY(cudaMemcpy2DAsync(dst + col, sizeof(T) * total, src, sizeof(T) * width, sizeof(T) * width, rows,
                                   cudaMemcpyDeviceToDevice, st));
}

// FP64 tree-order records into x[], y[], z[] rows
__global__ void soa_kernel(const dvec4* __restrict__ p, int64_t n, double* __restrict__ X) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const dvec4 v = p[i];
    X[i] = v.x;
    X[n + i] = v.y;
    X[2 * n + i] = v.z;
  }
}

__global__ void offset_i32_kernel(int32_t* __restrict__ dst, const int32_t* __restrict__ src, int64_t n, int32_t add,
                                  int keep_negative) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int32_t v = src[i];
    dst[i] = (keep_negative && v < 0) ? v : v + add;
  }
}
__global__ void offset_i64_kernel(int64_t* __restrict__ dst, const int64_t* __restrict__ src, int64_t n,
                                  int64_t add) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    dst[i] = src[i] + add;
}

}  // namespace

namespace {
__global__ void geo_lo_kernel(int64_t n, const double* __restrict__ g64, const float* __restrict__ g32,
                              float* __restrict__ lo) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    lo[i] = (float)(g64[i] - (double)g32[i]);
}
}  // namespace

// The FP64 data of a tree, made the first time its precision needs them:
// FP64 rotation records of every M2L, M2M and direct L2L translation (the
// build stores only their FP32 roundings), FP64 expansions and point records,
// and near-field slots wide enough for doubles.  Synchronous.
void ensure_fp64(fmm_tree* t, cudaStream_t st) {
  const int p = t->prm.p;
  const int64_t NB = t->n_boxes, nm = t->n_m2l;
  const int NCP = ncoef_pad(p);
  if (!t->geo64) {
    t->geo64 = dev_alloc<double>(t, (size_t)m2l_fields(p) * std::max<int64_t>(nm, 1));
    if (nm > 0) {
      m2l_geo_kernel<<<grid_for(nm, 256), 256, 0, st>>>(t->m2l_trg, t->m2l_src, nm, t->center, t->radius, p,
                                                        t->geo64, nullptr);
      FMM_LAUNCH_CHECK();
    }
  }
  if (!t->m2m64) {
    t->m2m64 = dev_alloc<double>(t, (size_t)edge_fields(p) * NB);
    edge_geo_kernel<<<grid_for(NB, 128, 1 << 30), 128, 0, st>>>(NB, t->box_parent, t->center, t->radius, p,
                                                                t->m2m64, nullptr);
    FMM_LAUNCH_CHECK();
  }
  if (!t->l2d64) {
    const int64_t nr = t->n_l2d;
    t->l2d64 = dev_alloc<double>(t, (size_t)edge_fields(p) * std::max<int64_t>(nr, 1));
    if (nr > 0) {
      l2d_fill_kernel<<<grid_for(t->n_leaves, 128), 128, 0, st>>>(t->n_leaves, t->leaf_box, t->box_parent,
                                                                  t->m2l_off, t->l2d_off, t->center, t->radius, p,
                                                                  nr, nullptr, t->l2d64, nullptr);
      FMM_LAUNCH_CHECK();
    }
  }
  const bool more_ws = !t->M64 || !t->src64 || (t->sym && !t->sym_partial_f64);
  require(!(more_ws && t->ws_external),
          "this precision needs a larger evaluation workspace: detach the caller's workspace "
          "(fmm_tree_set_workspace with NULL) before selecting it, then attach a new one");
  if (!t->M64) {
    t->M64 = dev_alloc<double>(t, (size_t)NB * NCP);
    t->Lam64 = dev_alloc<double>(t, (size_t)NB * NCP);
    FMM_CUDA_TRY(cudaMemsetAsync(t->M64, 0, sizeof(double) * NB * NCP, st));
    FMM_CUDA_TRY(cudaMemsetAsync(t->Lam64, 0, sizeof(double) * NB * NCP, st));
  }
  if (!t->src64) t->src64 = dev_alloc<dvec4>(t, t->n);
  if (t->sym && !t->sym_partial_f64) {
    dev_free(t->sym_partial);
    t->device_bytes -= sizeof(float) * (size_t)std::max<int64_t>(t->n_slots, 1) * t->sym_stride;
    t->sym_partial = dev_alloc<double>(t, (size_t)std::max<int64_t>(t->n_slots, 1) * t->sym_stride);
    t->sym_partial_f64 = 1;
  }
  FMM_CUDA_TRY(cudaStreamSynchronize(st));
}

void prepare_df_far(fmm_tree* t, cudaStream_t st) {
  if (t->geo_lo || t->two_trees) return;
  require(!t->ws_external,
          "FMM_FP64DF needs a larger evaluation workspace: detach the caller's workspace "
          "(fmm_tree_set_workspace with NULL) before selecting it, then attach a new one");
  ensure_fp64(t, st);
  const int p = t->prm.p;
  const int64_t ng = (int64_t)m2l_fields(p) * std::max<int64_t>(t->n_m2l, 1);
  t->geo_lo = dev_alloc<float>(t, ng);
  geo_lo_kernel<<<grid_for(ng, 256), 256, 0, st>>>(ng, t->geo64, t->geo32, t->geo_lo);
  FMM_LAUNCH_CHECK();
  t->m_df = dev_alloc<float2>(t, (size_t)t->n_boxes * ncoef_pad(p));
  if (t->sym) build_df_near(t, st);
  FMM_CUDA_TRY(cudaStreamSynchronize(st));
}

namespace {
// near-field work of every target leaf: its point count times the points of
// its list's source leaves (one warp per leaf)
__global__ void leaf_work_kernel(int64_t nl, const int64_t* __restrict__ off, const int32_t* __restrict__ src,
                                 const int32_t* __restrict__ leaf_box, const int32_t* __restrict__ src_leaf_box,
                                 const int32_t* __restrict__ box_count, int64_t* __restrict__ key) {
  const int64_t warps = (int64_t)gridDim.x * blockDim.x / 32;
  for (int64_t l = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) / 32; l < nl; l += warps) {
    int64_t w = 0;
    for (int64_t e = off[l] + (threadIdx.x & 31); e < off[l + 1]; e += 32) w += box_count[src_leaf_box[src[e]]];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) w += __shfl_xor_sync(0xffffffffu, w, o);
    if ((threadIdx.x & 31) == 0) key[l] = w * box_count[leaf_box[l]];
  }
}
}  // namespace

namespace {
// items of every target (kM2LItem interactions at most), in target order
__global__ void m2l_item_count_kernel(int64_t nb, const int64_t* __restrict__ off, int64_t* __restrict__ nit,
                                      int64_t* __restrict__ nrow, int64_t* __restrict__ split) {
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < nb; g += (int64_t)gridDim.x * blockDim.x) {
    const int64_t len = off[g + 1] - off[g];
    const int64_t k = len > kM2LItem ? (len + kM2LItem - 1) / kM2LItem : 1;
    nit[g] = k;
    nrow[g] = k > 1 ? k : 0;
    split[g] = k > 1 ? 1 : 0;
  }
}
__global__ void m2l_item_fill_kernel(int64_t nb, const int64_t* __restrict__ off, const int64_t* __restrict__ item_off,
                                     const int64_t* __restrict__ row_off, const int64_t* __restrict__ split_off,
                                     M2LItem* __restrict__ items, int64_t* __restrict__ len_out,
                                     int32_t* __restrict__ split_g, int64_t* __restrict__ split_row) {
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < nb; g += (int64_t)gridDim.x * blockDim.x) {
    const int64_t b = off[g], e = off[g + 1];
    const int64_t k = item_off[g + 1] - item_off[g];
    for (int64_t j = 0; j < k; j++) {
      const int64_t ib = b + j * kM2LItem, ie = ib + kM2LItem < e ? ib + kM2LItem : e;
      items[item_off[g] + j] = M2LItem{ib, ie, (int32_t)g, k > 1 ? (int32_t)(row_off[g] + j) : -1};
      len_out[item_off[g] + j] = ie - ib;
    }
    if (k > 1) {
      split_g[split_off[g]] = (int32_t)g;
      split_row[split_off[g]] = row_off[g];
    }
  }
}
__global__ void gather_items_kernel(int64_t n, const int32_t* __restrict__ perm, const M2LItem* __restrict__ in,
                                    M2LItem* __restrict__ out) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = in[perm[i]];
}
}  // namespace

// M2L work items: every target's list, split into items of at most
// kM2LItem interactions (a list of tens of thousands of interactions, as
// outlier boxes of a Plummer sphere have, would otherwise keep one warp busy
// for milliseconds), ordered longest first; and the near-field work order.
void build_work_orders(fmm_tree* t, cudaStream_t st) {
  const int64_t NB = t->n_boxes, NL = t->n_leaves;
  int64_t* nit = scratch_alloc<int64_t>(NB + 1);
  int64_t* nrow = scratch_alloc<int64_t>(NB + 1);
  int64_t* split = scratch_alloc<int64_t>(NB + 1);
  int64_t* item_off = scratch_alloc<int64_t>(NB + 1);
  int64_t* row_off = scratch_alloc<int64_t>(NB + 1);
  int64_t* split_off = scratch_alloc<int64_t>(NB + 1);
  FMM_CUDA_TRY(cudaMemsetAsync(nit + NB, 0, sizeof(int64_t), st));
  FMM_CUDA_TRY(cudaMemsetAsync(nrow + NB, 0, sizeof(int64_t), st));
  FMM_CUDA_TRY(cudaMemsetAsync(split + NB, 0, sizeof(int64_t), st));
  m2l_item_count_kernel<<<grid_for(NB, 256), 256, 0, st>>>(NB, t->m2l_off, nit, nrow, split);
  FMM_LAUNCH_CHECK();
  const int64_t NI = exclusive_scan(nit, item_off, NB + 1, st);
  const int64_t NR = exclusive_scan(nrow, row_off, NB + 1, st);
  const int64_t NS = exclusive_scan(split, split_off, NB + 1, st);
  M2LItem* items = scratch_alloc<M2LItem>(NI);
  int64_t* len = scratch_alloc<int64_t>(NI);
  int32_t* perm = scratch_alloc<int32_t>(NI);
  t->n_m2l_items = NI;
  t->n_m2l_split = NS;
  t->m2l_items = dev_alloc<M2LItem>(t, NI);
  t->m2l_split_g = dev_alloc<int32_t>(t, std::max<int64_t>(NS, 1));
  t->m2l_split_row = dev_alloc<int64_t>(t, NS + 1);
  t->m2l_partial_rows = NR;
  t->m2l_partial = dev_alloc<double>(t, (size_t)std::max<int64_t>(NR, 1) * ncoef_pad(t->prm.p));
  m2l_item_fill_kernel<<<grid_for(NB, 256), 256, 0, st>>>(NB, t->m2l_off, item_off, row_off, split_off, items, len,
                                                          t->m2l_split_g, t->m2l_split_row);
  FMM_LAUNCH_CHECK();
  FMM_CUDA_TRY(cudaMemcpyAsync(t->m2l_split_row + NS, &NR, sizeof(int64_t), cudaMemcpyHostToDevice, st));
  order_desc(len, NI, perm, st);
  gather_items_kernel<<<grid_for(NI, 256), 256, 0, st>>>(NI, perm, items, t->m2l_items);
  FMM_LAUNCH_CHECK();
  dev_free(nit), dev_free(nrow), dev_free(split), dev_free(item_off), dev_free(row_off), dev_free(split_off);
  dev_free(items), dev_free(len), dev_free(perm);

  int64_t* key = scratch_alloc<int64_t>(std::max<int64_t>(NL, 1));
  t->leaf_order = dev_alloc<int32_t>(t, NL);
  leaf_work_kernel<<<grid_for(NL * 32, 256), 256, 0, st>>>(NL, t->p2p_off, t->p2p_src, t->leaf_box,
                                                          t->src_leaf_box, t->box_count, key);
  FMM_LAUNCH_CHECK();
  order_desc(key, NL, t->leaf_order, st);
  dev_free(key);
  FMM_CUDA_TRY(cudaStreamSynchronize(st));
}

// Direct L2L records of a tree whose lists, geometry and parents are set
// (single trees, separate hierarchies and merged batches alike).
void build_l2l_direct(fmm_tree* t, cudaStream_t st) {
  const int64_t NL = t->n_leaves;
  const int p = t->prm.p;
  int64_t* cnt = scratch_alloc<int64_t>(NL + 1);
  FMM_CUDA_TRY(cudaMemsetAsync(cnt, 0, sizeof(int64_t) * (NL + 1), st));
  if (NL > 0) {
    l2d_count_kernel<<<grid_for(NL, 128), 128, 0, st>>>(NL, t->leaf_box, t->box_parent, t->m2l_off, cnt);
    FMM_LAUNCH_CHECK();
  }
  t->l2d_off = dev_alloc<int64_t>(t, NL + 1);
  const int64_t nr = exclusive_scan(cnt, t->l2d_off, NL + 1, st);
  dev_free(cnt);
  t->n_l2d = nr;
  t->l2d_anc = dev_alloc<int32_t>(t, std::max<int64_t>(nr, 1));
  t->l2d32 = dev_alloc<float>(t, (size_t)edge_fields(p) * std::max<int64_t>(nr, 1));
  if (nr > 0) {
    l2d_fill_kernel<<<grid_for(NL, 128), 128, 0, st>>>(NL, t->leaf_box, t->box_parent, t->m2l_off, t->l2d_off,
                                                       t->center, t->radius, p, nr, t->l2d_anc, nullptr, t->l2d32);
    FMM_LAUNCH_CHECK();
  }
  FMM_CUDA_TRY(cudaStreamSynchronize(st));
}

void build_tree(fmm_tree* t, const double* pos, cudaStream_t st) {
  double *blo = nullptr, *bhi = nullptr;
  build_hierarchy(t, pos, st, &blo, &bhi);
  t->n_charges = t->n;
  t->out_base = 0;
  t->n_src_leaves = t->n_leaves;
  t->src_leaf_box = t->leaf_box;
  const int64_t leaf_off = level_offset(t->L, t->s);
  std::vector<Step> steps;
  int32_t *p2p_t = nullptr, *p2p_s = nullptr;
  int64_t np = 0;
  const Side side{0, t->L, t->level_avg_host};
  try {
    march(t, side, side, st, steps, &p2p_t, &p2p_s, &np);
    finish_tree(t, steps, p2p_t, p2p_s, np, leaf_off, leaf_off, blo, bhi, t->has_duplicates, st);
    build_symmetric(t, st);
    trace_mark("symmetric near field");
  } catch (...) {
    dev_free(blo), dev_free(bhi);
    throw;
  }
  dev_free(blo), dev_free(bhi);
}

// Two hierarchies (Sec. II.B, final part): the source tree's boxes come first
// (ids 0 .. NB_s - 1), the target tree's follow; points likewise (sources
// 0 .. n_s - 1 carry the charges, targets n_s .. n - 1 are evaluated).
void build_tree2(fmm_tree* m, const double* src, int64_t n_s, const double* trg, int64_t n_t, cudaStream_t st) {
  const fmm_params prm = m->prm;
  const int s = prm.splits, p = prm.p;
  fmm_tree* S = new fmm_tree();
  fmm_tree* T = new fmm_tree();
  double *blo_s = nullptr, *bhi_s = nullptr, *blo_t = nullptr, *bhi_t = nullptr;
  auto cleanup = [&] {
    dev_free(blo_s), dev_free(bhi_s), dev_free(blo_t), dev_free(bhi_t);
    S->src_leaf_box = T->src_leaf_box = nullptr;
    free_tree(S);
    free_tree(T);
  };
  try {
    S->prm = prm;
    S->n = n_s;
    S->L = fmm_num_levels(n_s, prm.leaf_size, s);
    T->prm = prm;
    T->n = n_t;
    T->L = fmm_num_levels(n_t, prm.leaf_size, s);
    build_hierarchy(S, src, st, &blo_s, &bhi_s);
    build_hierarchy(T, trg, st, &blo_t, &bhi_t);
    const int64_t NBs = S->n_boxes, NBt = T->n_boxes, NB = NBs + NBt, N = n_s + n_t;
    require(NB < ((int64_t)1 << 31) && N < ((int64_t)1 << 31), "source and target sets too large");
    m->n = N;
    m->s = s;
    m->L = T->L;
    m->L_src = S->L;
    m->two_trees = 1;
    m->n_charges = n_s;
    m->out_base = n_s;
    m->n_boxes = NB;
    m->n_leaves = T->n_leaves;
    m->n_src_leaves = S->n_leaves;
    m->max_leaf = std::max(S->max_leaf, T->max_leaf);
    m->min_leaf = T->min_leaf;
    m->level_avg_host = new double[S->L + T->L + 2];
    for (int l = 0; l <= S->L; l++) m->level_avg_host[l] = S->level_avg_host[l];
    for (int l = 0; l <= T->L; l++) m->level_avg_host[S->L + 1 + l] = T->level_avg_host[l];

    m->perm = dev_alloc<int32_t>(m, N);
    m->box_start = dev_alloc<int64_t>(m, NB);
    m->box_count = dev_alloc<int32_t>(m, NB);
    m->center = dev_alloc<double>(m, 3 * NB);
    m->radius = dev_alloc<double>(m, NB);
    m->inv_rho32 = dev_alloc<float>(m, NB);
    m->inv_rho64 = dev_alloc<double>(m, NB);
    m->leaf_box = dev_alloc<int32_t>(m, T->n_leaves);
    m->src_leaf_box = dev_alloc<int32_t>(m, S->n_leaves);
    m->box_parent = dev_alloc<int32_t>(m, NB);
    m->pos_local = dev_alloc<float4>(m, N);
    m->pos64 = dev_alloc<dvec4>(m, N);
    m->m2m32 = dev_alloc<float>(m, (size_t)edge_fields(p) * NB);
    FMM_CUDA_TRY(cudaMemsetAsync(m->m2m32, 0, sizeof(float) * edge_fields(p) * NB, st));

    copy_d2d(m->perm, S->perm, n_s, st);
    offset_i32_kernel<<<grid_for(n_t, 256), 256, 0, st>>>(m->perm + n_s, T->perm, n_t, (int32_t)n_s, 0);
    copy_d2d(m->box_start, S->box_start, NBs, st);
    offset_i64_kernel<<<grid_for(NBt, 256), 256, 0, st>>>(m->box_start + NBs, T->box_start, NBt, n_s);
    copy_d2d(m->box_count, S->box_count, NBs, st);
    copy_d2d(m->box_count + NBs, T->box_count, NBt, st);
    copy_d2d(m->center, S->center, 3 * NBs, st);
    copy_d2d(m->center + 3 * NBs, T->center, 3 * NBt, st);
    copy_d2d(m->radius, S->radius, NBs, st);
    copy_d2d(m->radius + NBs, T->radius, NBt, st);
    copy_d2d(m->inv_rho32, S->inv_rho32, NBs, st);
    copy_d2d(m->inv_rho32 + NBs, T->inv_rho32, NBt, st);
    copy_d2d(m->inv_rho64, S->inv_rho64, NBs, st);
    copy_d2d(m->inv_rho64 + NBs, T->inv_rho64, NBt, st);
    offset_i32_kernel<<<grid_for(T->n_leaves, 256), 256, 0, st>>>(m->leaf_box, T->leaf_box, T->n_leaves,
                                                                  (int32_t)NBs, 0);
    copy_d2d(m->src_leaf_box, S->leaf_box, S->n_leaves, st);
    copy_d2d(m->box_parent, S->box_parent, NBs, st);
    offset_i32_kernel<<<grid_for(NBt, 256), 256, 0, st>>>(m->box_parent + NBs, T->box_parent, NBt, (int32_t)NBs, 1);
    FMM_LAUNCH_CHECK();
    copy_d2d(m->pos_local, S->pos_local, n_s, st);
    copy_d2d(m->pos_local + n_s, T->pos_local, n_t, st);
    copy_d2d(m->pos64, S->pos64, n_s, st);
    copy_d2d(m->pos64 + n_s, T->pos64, n_t, st);
    // multipoles move up the source tree (M2M rounds); locals reach the
    // target leaves by the direct L2L records of the target tree
    copy_rows(m->m2m32, NB, 0, S->m2m32, NBs, edge_fields(p), st);
    m->n_up = S->L;
    m->up_off_h = new int64_t[S->L + 1];
    for (int r = 0; r <= S->L; r++) m->up_off_h[r] = S->up_off_h[r];
    m->up_ids = dev_alloc<int32_t>(m, std::max<int64_t>(NBs, 1));
    copy_d2d(m->up_ids, S->up_ids, NBs, st);
    FMM_CUDA_TRY(cudaStreamSynchronize(st));

    // can a target coincide with a source?  (duplicates among the union;
    // conservative when a set has duplicates of its own)
    int has_dup = S->has_duplicates | T->has_duplicates;
    if (!has_dup) {
      double* X = scratch_alloc<double>(3 * (size_t)N);
      soa_kernel<<<grid_for(N, 256), 256, 0, st>>>(m->pos64, N, X);
      FMM_LAUNCH_CHECK();
      int64_t tsize = 1;
      while (tsize < 2 * N) tsize <<= 1;
      int* tab = scratch_alloc<int>(tsize);
      int* flag = scratch_alloc<int>(1);
      FMM_CUDA_TRY(cudaMemsetAsync(tab, 0xff, sizeof(int) * tsize, st));
      FMM_CUDA_TRY(cudaMemsetAsync(flag, 0, sizeof(int), st));
      duplicate_kernel<<<grid_for(N, 256), 256, 0, st>>>(X, N, tab, tsize - 1, flag);
      FMM_LAUNCH_CHECK();
      FMM_CUDA_TRY(cudaMemcpyAsync(&has_dup, flag, sizeof(int), cudaMemcpyDeviceToHost, st));
      FMM_CUDA_TRY(cudaStreamSynchronize(st));
      dev_free(X), dev_free(tab), dev_free(flag);
    }
    m->has_duplicates = has_dup;
    double* blo = scratch_alloc<double>(3 * (size_t)NB);
    double* bhi = scratch_alloc<double>(3 * (size_t)NB);
    copy_d2d(blo, blo_s, 3 * NBs, st);
    copy_d2d(blo + 3 * NBs, blo_t, 3 * NBt, st);
    copy_d2d(bhi, bhi_s, 3 * NBs, st);
    copy_d2d(bhi + 3 * NBs, bhi_t, 3 * NBt, st);

    std::vector<Step> steps;
    int32_t *p2p_t = nullptr, *p2p_s = nullptr;
    int64_t np = 0;
    try {
      march(m, Side{0, S->L, S->level_avg_host}, Side{NBs, T->L, T->level_avg_host}, st, steps, &p2p_t, &p2p_s,
            &np);
      finish_tree(m, steps, p2p_t, p2p_s, np, NBs + level_offset(T->L, s), level_offset(S->L, s), blo, bhi,
                  has_dup, st);
    } catch (...) {
      dev_free(blo), dev_free(bhi);
      throw;
    }
    dev_free(blo), dev_free(bhi);
  } catch (...) {
    cleanup();
    throw;
  }
  cleanup();
}

}  // namespace fmm
