// Work lists of the symmetric near field of one point set (or of a batch of
// independent point sets).  Eq. 4 is symmetric in the two boxes, but the
// level march is not (ties advance one side), so a leaf pair can sit in the
// near field in one direction only.  Per entry (target leaf l, source leaf s)
// of the near-field list (sorted by source within each leaf):
//   * s > l and (s, l) is listed too: a symmetric pair.  The warp of l
//     evaluates it once and leaves the sums q_l / r at s's points in a slot;
//   * s < l and (s, l) is listed: received.  Leaf s's warp computes it; the
//     local evaluation of l adds the slot;
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

// mirror entry index of every entry (-1: not listed the other way), and the
// flag of the upper entries that own a slot
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
      owns[e] = (m >= 0 && s > (int32_t)l) ? 1 : 0;
    }
  }
}

// slot of every entry: owners get theirs from the scan, received entries the
// slot of their mirror, the rest -1; per-leaf counts of work and received
// entries
__global__ void slot_kernel(int64_t n_leaves, const int64_t* __restrict__ off, const int32_t* __restrict__ src,
                            const int64_t* __restrict__ mirror, const int64_t* __restrict__ owns,
                            const int64_t* __restrict__ slot_scan, int32_t* __restrict__ slot,
                            int64_t* __restrict__ n_work, int64_t* __restrict__ n_recv) {
  for (int64_t l = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; l < n_leaves;
       l += (int64_t)gridDim.x * blockDim.x) {
    int64_t w = 0, r = 0;
    for (int64_t e = off[l]; e < off[l + 1]; e++) {
      const int64_t m = mirror[e];
      if (owns[e]) {
        slot[e] = (int32_t)slot_scan[e];
        w++;
      } else if (m >= 0 && src[e] < (int32_t)l) {
        slot[e] = (int32_t)slot_scan[m];
        r++;
      } else {
        slot[e] = -1;
        w++;
      }
    }
    n_work[l] = w;
    n_recv[l] = r;
  }
}

// work entries (list order) and received slots (list order) per leaf
__global__ void fill_kernel(int64_t n_leaves, const int64_t* __restrict__ off, const int32_t* __restrict__ src,
                            const int32_t* __restrict__ slot, const int64_t* __restrict__ work_off,
                            const int64_t* __restrict__ recv_off, int32_t* __restrict__ work,
                            int32_t* __restrict__ recv) {
  for (int64_t l = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; l < n_leaves;
       l += (int64_t)gridDim.x * blockDim.x) {
    int64_t w = work_off[l], r = recv_off[l];
    for (int64_t e = off[l]; e < off[l + 1]; e++) {
      if (slot[e] >= 0 && src[e] < (int32_t)l) recv[r++] = slot[e];
      else work[w++] = (int32_t)e;
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
  int64_t* owns = scratch_alloc<int64_t>(NE1 + 1);
  int64_t* slot_scan = scratch_alloc<int64_t>(NE1 + 1);
  int64_t* n_work = scratch_alloc<int64_t>(NL + 1);
  int64_t* n_recv = scratch_alloc<int64_t>(NL + 1);
  FMM_CUDA_TRY(cudaMemsetAsync(owns, 0, sizeof(int64_t) * (NE1 + 1), st));
  FMM_CUDA_TRY(cudaMemsetAsync(n_work + NL, 0, sizeof(int64_t), st));
  FMM_CUDA_TRY(cudaMemsetAsync(n_recv + NL, 0, sizeof(int64_t), st));
  mirror_kernel<<<grid_for(NL * 32, 256), 256, 0, st>>>(NL, t->p2p_off, t->p2p_src, mirror, owns);
  FMM_LAUNCH_CHECK();
  t->n_slots = exclusive_scan(owns, slot_scan, NE + 1, st);
  t->sym_slot = dev_alloc<int32_t>(t, NE1);
  slot_kernel<<<grid_for(NL, 128), 128, 0, st>>>(NL, t->p2p_off, t->p2p_src, mirror, owns, slot_scan, t->sym_slot,
                                                 n_work, n_recv);
  FMM_LAUNCH_CHECK();
  t->sym_work_off = dev_alloc<int64_t>(t, NL + 1);
  t->sym_recv_off = dev_alloc<int64_t>(t, NL + 1);
  const int64_t nw = exclusive_scan(n_work, t->sym_work_off, NL + 1, st);
  const int64_t nr = exclusive_scan(n_recv, t->sym_recv_off, NL + 1, st);
  t->sym_work = dev_alloc<int32_t>(t, std::max<int64_t>(nw, 1));
  t->sym_recv = dev_alloc<int32_t>(t, std::max<int64_t>(nr, 1));
  fill_kernel<<<grid_for(NL, 128), 128, 0, st>>>(NL, t->p2p_off, t->p2p_src, t->sym_slot, t->sym_work_off,
                                                 t->sym_recv_off, t->sym_work, t->sym_recv);
  FMM_LAUNCH_CHECK();
  FMM_CUDA_TRY(cudaStreamSynchronize(st));
  cudaFree(mirror), cudaFree(owns), cudaFree(slot_scan), cudaFree(n_work), cudaFree(n_recv);
  t->sym_stride = std::max(t->max_leaf, 1);
  t->sym_partial = dev_alloc<float>(t, std::max<int64_t>(t->n_slots, 1) * t->sym_stride);

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
