// Work lists of the symmetric near field of one point set (or of a batch of
// independent point sets).  Eq. 4 is symmetric in the two boxes, but the
// level march is not (ties advance one side), so a leaf pair can sit in the
// near field in one direction only.  Per entry (target leaf l, source leaf s)
// of the near-field list (sorted by source within each leaf):
//   * (s, l) is listed too and l owns the pair (see owner()): the warp of l
//     evaluates it once and leaves the sums q_l / r at s's points in a slot;
//   * (s, l) is listed and s owns the pair: received.  Leaf s's warp computes
//     it; the gather before the local evaluation of l adds the slot;
//   * anything else (the self pair, pairs listed in one direction only):
//     evaluated one-sided by the warp of l, as in the one-sided kernel.
// All orders are fixed, so results do not depend on scheduling.
#include <algorithm>
#include <vector>

#include "common.cuh"

namespace fmm {
namespace {

__device__ __forceinline__ int64_t find_src(const int32_t* __restrict__ src, int64_t lo, int64_t hi, int32_t v) {
  while (lo < hi) {
    const int64_t mid = (lo + hi) >> 1;
    if (src[mid] < v) lo = mid + 1;
    else hi = mid;
  }
  return lo;
}

// Which leaf evaluates a pair listed both ways: the one with the shorter
// list (ties: the smaller index), so leaves with very long lists (boxes
// around outliers, whose bounding boxes are large) hand their pairs to their
// partners and no single warp becomes the long pole.
__device__ __forceinline__ bool owner(const int64_t* __restrict__ off, int32_t l, int32_t s) {
  const int64_t nl = off[l + 1] - off[l], ns = off[s + 1] - off[s];
  return nl < ns || (nl == ns && l < s);
}

// mirror entry index of every entry (-1: not listed the other way), and the
// flag of the entries whose leaf owns the pair (and a slot)
__global__ void mirror_kernel(int64_t n_leaves, const int64_t* __restrict__ off, const int32_t* __restrict__ src,
                              int64_t* __restrict__ mirror, int64_t* __restrict__ owns) {
  const int64_t warps = (int64_t)gridDim.x * blockDim.x / 32;
  for (int64_t l = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) / 32; l < n_leaves; l += warps) {
    for (int64_t e = off[l] + (threadIdx.x & 31); e < off[l + 1]; e += 32) {
      const int32_t s = src[e];
      int64_t m = -1;
      if (s != (int32_t)l) {
        const int64_t f = find_src(src, off[s], off[s + 1], (int32_t)l);
        if (f < off[s + 1] && src[f] == (int32_t)l) m = f;
      }
      mirror[e] = m;
      owns[e] = (m >= 0 && owner(off, (int32_t)l, s)) ? 1 : 0;
    }
  }
}

// per leaf: entries its warp evaluates (owned pairs and one-sided entries)
// and entries it receives (pairs owned by the partner)
__global__ void count_kernel(int64_t n_leaves, const int64_t* __restrict__ off, const int64_t* __restrict__ mirror,
                             const int64_t* __restrict__ owns, int64_t* __restrict__ n_work,
                             int64_t* __restrict__ n_recv) {
  for (int64_t l = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; l < n_leaves;
       l += (int64_t)gridDim.x * blockDim.x) {
    int64_t w = 0, r = 0;
    for (int64_t e = off[l]; e < off[l + 1]; e++) {
      if (!owns[e] && mirror[e] >= 0) r++;
      else w++;
    }
    n_work[l] = w;
    n_recv[l] = r;
  }
}

// Work entries in list order, and slots: a received entry's slot is its
// position in the receivers' concatenated lists, so the slots a leaf adds are
// contiguous; the owning entry (its mirror) writes to the same slot.
__global__ void fill_kernel(int64_t n_leaves, const int64_t* __restrict__ off, const int64_t* __restrict__ mirror,
                            const int64_t* __restrict__ owns, const int64_t* __restrict__ work_off,
                            const int64_t* __restrict__ recv_off, int32_t* __restrict__ work,
                            int32_t* __restrict__ slot) {
  for (int64_t l = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; l < n_leaves;
       l += (int64_t)gridDim.x * blockDim.x) {
    int64_t w = work_off[l], r = recv_off[l];
    for (int64_t e = off[l]; e < off[l + 1]; e++) {
      if (!owns[e] && mirror[e] >= 0) {
        slot[e] = (int32_t)r;
        slot[mirror[e]] = (int32_t)r;
        r++;
      } else {
        if (!owns[e]) slot[e] = -1;
        work[w++] = (int32_t)e;
      }
    }
  }
}

// one record per work entry (see SymRec)
__global__ void rec_kernel(int64_t n_leaves, const int64_t* __restrict__ work_off, const int32_t* __restrict__ work,
                           const P2PEntry* __restrict__ ent, const float* __restrict__ thr,
                           const int32_t* __restrict__ slot, const int32_t* __restrict__ src_leaf_box,
                           const int64_t* __restrict__ box_start, const int32_t* __restrict__ box_count,
                           SymRec* __restrict__ rec) {
  const int64_t warps = (int64_t)gridDim.x * blockDim.x / 32;
  for (int64_t l = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) / 32; l < n_leaves; l += warps) {
    for (int64_t k = work_off[l] + (threadIdx.x & 31); k < work_off[l + 1]; k += 32) {
      const int64_t e = work[k];
      const P2PEntry en = ent[e];
      const int ls = en.src & 0x7fffffff;
      const int64_t gs = src_leaf_box[ls];
      const bool mask = en.src < 0 || ls == (int)l;
      rec[k] = SymRec{box_start[gs], box_count[gs], slot[e], en.dx, en.dy, en.dz, mask ? thr[e] : -1.f};
    }
  }
}

// ---- FP64DF point records and frames ----
// coordinates of every point in its leaf's frame (offset from the leaf
// centre in FP64), split h + l
__global__ void df_points_kernel(int64_t n_leaves, const int32_t* __restrict__ leaf_box,
                                 const int64_t* __restrict__ box_start, const int32_t* __restrict__ box_count,
                                 const double* __restrict__ center, const dvec4* __restrict__ pos,
                                 DFRec* __restrict__ rec) {
  const int64_t warps = (int64_t)gridDim.x * blockDim.x / 32;
  for (int64_t l = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) / 32; l < n_leaves; l += warps) {
    const int64_t g = leaf_box[l];
    const double cx = center[3 * g], cy = center[3 * g + 1], cz = center[3 * g + 2];
    for (int i = threadIdx.x & 31; i < box_count[g]; i += 32) {
      const int64_t k = box_start[g] + i;
      const dvec4 p = pos[k];
      const double x = p.x - cx, y = p.y - cy, z = p.z - cz;
      const float hx = (float)x, hy = (float)y, hz = (float)z;
      DFRec r;
      r.xh = hx;
      r.yh = hy;
      r.zh = hz;
      r.xl = (float)(x - (double)hx);
      r.yl = (float)(y - (double)hy);
      r.zl = (float)(z - (double)hz);
      r.qh = r.ql = 0.f;
      rec[k] = r;
    }
  }
}

// source frame of every work entry
__global__ void frame_rec_kernel(int64_t n_leaves, const int64_t* __restrict__ work_off,
                                 const int32_t* __restrict__ work, const int32_t* __restrict__ src,
                                 const int32_t* __restrict__ leaf_box, const double* __restrict__ center,
                                 SymFrame* __restrict__ frame) {
  const int64_t warps = (int64_t)gridDim.x * blockDim.x / 32;
  for (int64_t l = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) / 32; l < n_leaves; l += warps) {
    for (int64_t k = work_off[l] + (threadIdx.x & 31); k < work_off[l + 1]; k += 32) {
      const int s = src[work[k]];
      const int64_t gs = leaf_box[s];
      frame[k] = SymFrame{center[3 * gs], center[3 * gs + 1], center[3 * gs + 2], 0.f, 0.f};
    }
  }
}

template <class T>
std::vector<T> host_copy(const T* d, int64_t n, cudaStream_t st) {
  std::vector<T> h((size_t)std::max<int64_t>(n, 0));
  if (n > 0) FMM_CUDA_TRY(cudaMemcpyAsync(h.data(), d, sizeof(T) * n, cudaMemcpyDeviceToHost, st));
  FMM_CUDA_TRY(cudaStreamSynchronize(st));
  return h;
}

}  // namespace

void build_symmetric(fmm_tree* t, cudaStream_t st) {
  const int64_t NL = t->n_leaves, NE = t->n_p2p;
  require(NE < ((int64_t)1 << 31), "near-field list too long for the symmetric kernel");
  const int64_t NE1 = std::max<int64_t>(NE, 1);
  int64_t* mirror = scratch_alloc<int64_t>(NE1);
  int64_t* owns = scratch_alloc<int64_t>(NE1);
  int64_t* n_work = scratch_alloc<int64_t>(NL + 1);
  int64_t* n_recv = scratch_alloc<int64_t>(NL + 1);
  FMM_CUDA_TRY(cudaMemsetAsync(n_work + NL, 0, sizeof(int64_t), st));
  FMM_CUDA_TRY(cudaMemsetAsync(n_recv + NL, 0, sizeof(int64_t), st));
  mirror_kernel<<<grid_for(NL * 32, 256), 256, 0, st>>>(NL, t->p2p_off, t->p2p_src, mirror, owns);
  FMM_LAUNCH_CHECK();
  count_kernel<<<grid_for(NL, 128), 128, 0, st>>>(NL, t->p2p_off, mirror, owns, n_work, n_recv);
  FMM_LAUNCH_CHECK();
  t->sym_work_off = dev_alloc<int64_t>(t, NL + 1);
  t->sym_recv_off = dev_alloc<int64_t>(t, NL + 1);
  const int64_t nw = exclusive_scan(n_work, t->sym_work_off, NL + 1, st);
  t->n_slots = exclusive_scan(n_recv, t->sym_recv_off, NL + 1, st);
  require(t->n_slots < ((int64_t)1 << 31), "too many symmetric pairs");
  t->sym_slot = dev_alloc<int32_t>(t, NE1);
  t->sym_work = dev_alloc<int32_t>(t, std::max<int64_t>(nw, 1));
  fill_kernel<<<grid_for(NL, 128), 128, 0, st>>>(NL, t->p2p_off, mirror, owns, t->sym_work_off, t->sym_recv_off,
                                                 t->sym_work, t->sym_slot);
  FMM_LAUNCH_CHECK();
  t->sym_rec = dev_alloc<SymRec>(t, std::max<int64_t>(nw, 1));
  rec_kernel<<<grid_for(NL * 32, 256), 256, 0, st>>>(NL, t->sym_work_off, t->sym_work, t->p2p32, t->p2p_thr,
                                                     t->sym_slot, t->src_leaf_box, t->box_start, t->box_count,
                                                     t->sym_rec);
  FMM_LAUNCH_CHECK();
  // FP64DF point records and per-entry source frames
  t->src_df = dev_alloc<DFRec>(t, t->n);
  df_points_kernel<<<grid_for(NL * 32, 256), 256, 0, st>>>(NL, t->leaf_box, t->box_start, t->box_count, t->center,
                                                           t->pos64, t->src_df);
  FMM_LAUNCH_CHECK();
  t->sym_frame = dev_alloc<SymFrame>(t, std::max<int64_t>(nw, 1));
  frame_rec_kernel<<<grid_for(NL * 32, 256), 256, 0, st>>>(NL, t->sym_work_off, t->sym_work, t->p2p_src, t->leaf_box,
                                                           t->center, t->sym_frame);
  FMM_LAUNCH_CHECK();
  FMM_CUDA_TRY(cudaStreamSynchronize(st));
  dev_free(mirror), dev_free(owns), dev_free(n_work), dev_free(n_recv);
  t->sym_stride = std::max(t->max_leaf, 1);
  // slot sums in FP32 (FP32C path) or FP64 (FP64 path): room for doubles
  t->sym_partial = dev_alloc<double>(t, std::max<int64_t>(t->n_slots, 1) * t->sym_stride);

  // work order of the symmetric kernel: heaviest work list first
  std::vector<int64_t> woff = host_copy(t->sym_work_off, NL + 1, st);
  std::vector<int32_t> work = host_copy(t->sym_work, nw, st);
  std::vector<int32_t> src = host_copy(t->p2p_src, NE, st);
  std::vector<int32_t> lbox = host_copy(t->leaf_box, NL, st);
  std::vector<int32_t> cnt = host_copy(t->box_count, t->n_boxes, st);
  std::vector<int64_t> cost(NL, 0);
  for (int64_t l = 0; l < NL; l++)
    for (int64_t k = woff[l]; k < woff[l + 1]; k++) cost[l] += cnt[lbox[src[work[k]]]];
  std::vector<int32_t> ord(NL);
  for (int64_t l = 0; l < NL; l++) ord[l] = (int32_t)l;
  std::stable_sort(ord.begin(), ord.end(), [&](int32_t a, int32_t b) { return cost[a] > cost[b]; });
  t->leaf_order_sym = dev_alloc<int32_t>(t, NL);
  FMM_CUDA_TRY(cudaMemcpyAsync(t->leaf_order_sym, ord.data(), sizeof(int32_t) * NL, cudaMemcpyHostToDevice, st));
  FMM_CUDA_TRY(cudaStreamSynchronize(st));
  t->sym = 1;
}

}  // namespace fmm
