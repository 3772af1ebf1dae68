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
// One warp per leaf (lanes over its entries): a received entry (the
// partner owns the pair) or an entry the leaf's warp evaluates.
__device__ __forceinline__ bool is_received(const int64_t* __restrict__ mirror, const int64_t* __restrict__ owns,
                                            int64_t e) {
  return !owns[e] && mirror[e] >= 0;
}

__global__ void count_kernel(int64_t n_leaves, const int64_t* __restrict__ off, const int64_t* __restrict__ mirror,
                             const int64_t* __restrict__ owns, int64_t* __restrict__ n_work,
                             int64_t* __restrict__ n_recv) {
  const int64_t warps = (int64_t)gridDim.x * blockDim.x / 32;
  const int lane = threadIdx.x & 31;
  for (int64_t l = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) / 32; l < n_leaves; l += warps) {
    int64_t r = 0;
    for (int64_t e = off[l] + lane; e < off[l + 1]; e += 32) r += is_received(mirror, owns, e) ? 1 : 0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) r += __shfl_xor_sync(0xffffffffu, r, o);
    if (lane == 0) {
      n_work[l] = (off[l + 1] - off[l]) - r;
      n_recv[l] = r;
    }
  }
}

// Work entries in list order, and slots: a received entry's slot is its
// position in the receivers' concatenated lists, so the slots a leaf adds are
// contiguous; the owning entry (its mirror) writes to the same slot.  The
// warp walks its leaf's list in chunks of 32 entries, in order, ranking
// each kind of entry by ballot.
__global__ void fill_kernel(int64_t n_leaves, const int64_t* __restrict__ off, const int64_t* __restrict__ mirror,
                            const int64_t* __restrict__ owns, const int64_t* __restrict__ work_off,
                            const int64_t* __restrict__ recv_off, int32_t* __restrict__ work,
                            int32_t* __restrict__ slot) {
  const int64_t warps = (int64_t)gridDim.x * blockDim.x / 32;
  const int lane = threadIdx.x & 31;
  const unsigned below = (1u << lane) - 1u;
  for (int64_t l = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) / 32; l < n_leaves; l += warps) {
    int64_t w = work_off[l], r = recv_off[l];
    for (int64_t e0 = off[l]; e0 < off[l + 1]; e0 += 32) {
      const int64_t e = e0 + lane;
      const bool valid = e < off[l + 1];
      const bool recv = valid && is_received(mirror, owns, e);
      const unsigned br = __ballot_sync(0xffffffffu, recv);
      const unsigned bw = __ballot_sync(0xffffffffu, valid && !recv);
      if (recv) {
        const int32_t sl = (int32_t)(r + __popc(br & below));
        slot[e] = sl;
        slot[mirror[e]] = sl;
      } else if (valid) {
        if (!owns[e]) slot[e] = -1;
        work[w + __popc(bw & below)] = (int32_t)e;
      }
      r += __popc(br);
      w += __popc(bw);
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

// chunks of the slot gather: leaf l's received slots in pieces of at most
// kGatherChunk (count, then fill in leaf order)
__global__ void gch_count_kernel(int64_t n_leaves, const int64_t* __restrict__ recv_off, int64_t* __restrict__ nch,
                                 int64_t* __restrict__ multi) {
  for (int64_t l = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; l < n_leaves; l += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = recv_off[l + 1] - recv_off[l];
    const int64_t k = (r + kGatherChunk - 1) / kGatherChunk;
    nch[l] = k;
    multi[l] = k > 1 ? 1 : 0;
  }
}
__global__ void gch_fill_kernel(int64_t n_leaves, const int64_t* __restrict__ recv_off,
                                const int64_t* __restrict__ first, const int64_t* __restrict__ multi_off,
                                int32_t* __restrict__ gleaf, int64_t* __restrict__ gr0, int32_t* __restrict__ mleaf) {
  for (int64_t l = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; l < n_leaves; l += (int64_t)gridDim.x * blockDim.x) {
    const int64_t k = first[l + 1] - first[l];
    for (int64_t j = 0; j < k; j++) {
      gleaf[first[l] + j] = (int32_t)l;
      gr0[first[l] + j] = recv_off[l] + j * kGatherChunk;
    }
    if (k > 1) mleaf[multi_off[l]] = (int32_t)l;
  }
}

// points of the source leaves a leaf's warp evaluates (its work list)
__global__ void sym_cost_kernel(int64_t n_leaves, const int64_t* __restrict__ work_off,
                                const int32_t* __restrict__ work, const int32_t* __restrict__ src,
                                const int32_t* __restrict__ src_leaf_box, const int32_t* __restrict__ box_count,
                                int64_t* __restrict__ cost) {
  const int64_t warps = (int64_t)gridDim.x * blockDim.x / 32;
  for (int64_t l = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) / 32; l < n_leaves; l += warps) {
    int64_t c = 0;
    for (int64_t k = work_off[l] + (threadIdx.x & 31); k < work_off[l + 1]; k += 32)
      c += box_count[src_leaf_box[src[work[k]]]];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
    if ((threadIdx.x & 31) == 0) cost[l] = c;
  }
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
  trace_mark("  sym: scratch");
  mirror_kernel<<<grid_for(NL * 32, 256), 256, 0, st>>>(NL, t->p2p_off, t->p2p_src, mirror, owns);
  FMM_LAUNCH_CHECK();
  trace_mark("  sym: mirror");
  count_kernel<<<grid_for(NL * 32, 256), 256, 0, st>>>(NL, t->p2p_off, mirror, owns, n_work, n_recv);
  FMM_LAUNCH_CHECK();
  t->sym_work_off = dev_alloc<int64_t>(t, NL + 1);
  t->sym_recv_off = dev_alloc<int64_t>(t, NL + 1);
  const int64_t nw = exclusive_scan(n_work, t->sym_work_off, NL + 1, st);
  t->n_slots = exclusive_scan(n_recv, t->sym_recv_off, NL + 1, st);
  require(t->n_slots < ((int64_t)1 << 31), "too many symmetric pairs");
  trace_mark("  sym: count + scans");
  t->sym_slot = dev_alloc<int32_t>(t, NE1);
  t->sym_work = dev_alloc<int32_t>(t, std::max<int64_t>(nw, 1));
  fill_kernel<<<grid_for(NL * 32, 256), 256, 0, st>>>(NL, t->p2p_off, mirror, owns, t->sym_work_off,
                                                       t->sym_recv_off, t->sym_work, t->sym_slot);
  FMM_LAUNCH_CHECK();
  trace_mark("  sym: fill");
  t->sym_rec = dev_alloc<SymRec>(t, std::max<int64_t>(nw, 1));
  rec_kernel<<<grid_for(NL * 32, 256), 256, 0, st>>>(NL, t->sym_work_off, t->sym_work, t->p2p32, t->p2p_thr,
                                                     t->sym_slot, t->src_leaf_box, t->box_start, t->box_count,
                                                     t->sym_rec);
  FMM_LAUNCH_CHECK();
  trace_mark("  sym: records");
  dev_free(mirror), dev_free(owns), dev_free(n_work), dev_free(n_recv);
  t->sym_stride = std::max(t->max_leaf, 1);
  // slot sums in FP32 for the FP32C path; ensure_fp64 widens them to doubles
  // when an FP64 precision is selected
  t->sym_partial = reinterpret_cast<double*>(
      dev_alloc<float>(t, (size_t)std::max<int64_t>(t->n_slots, 1) * t->sym_stride));
  t->sym_partial_f64 = 0;
  trace_mark("  sym: slots");

  // slot gather in chunks (a leaf that receives tens of thousands of slots,
  // such as an outlier leaf of a Plummer sphere paired with every other leaf,
  // is gathered by many warps)
  {
    int64_t* nchk = scratch_alloc<int64_t>(NL + 1);
    int64_t* multi = scratch_alloc<int64_t>(NL + 1);
    int64_t* multi_off = scratch_alloc<int64_t>(NL + 1);
    FMM_CUDA_TRY(cudaMemsetAsync(nchk + NL, 0, sizeof(int64_t), st));
    FMM_CUDA_TRY(cudaMemsetAsync(multi + NL, 0, sizeof(int64_t), st));
    gch_count_kernel<<<grid_for(NL, 256), 256, 0, st>>>(NL, t->sym_recv_off, nchk, multi);
    FMM_LAUNCH_CHECK();
    t->gch_first = dev_alloc<int64_t>(t, NL + 1);
    t->n_gchunks = exclusive_scan(nchk, t->gch_first, NL + 1, st);
    t->n_gmulti = exclusive_scan(multi, multi_off, NL + 1, st);
    t->gch_leaf = dev_alloc<int32_t>(t, std::max<int64_t>(t->n_gchunks, 1));
    t->gch_r0 = dev_alloc<int64_t>(t, std::max<int64_t>(t->n_gchunks, 1));
    t->gmulti_leaf = dev_alloc<int32_t>(t, std::max<int64_t>(t->n_gmulti, 1));
    gch_fill_kernel<<<grid_for(NL, 256), 256, 0, st>>>(NL, t->sym_recv_off, t->gch_first, multi_off, t->gch_leaf,
                                                       t->gch_r0, t->gmulti_leaf);
    FMM_LAUNCH_CHECK();
    t->gpart = dev_alloc<double>(t, (size_t)std::max<int64_t>(t->n_gchunks, 1) * t->sym_stride);
    dev_free(nchk), dev_free(multi), dev_free(multi_off);
  }

  // work order of the symmetric kernel: heaviest work list first
  int64_t* cost = scratch_alloc<int64_t>(std::max<int64_t>(NL, 1));
  sym_cost_kernel<<<grid_for(NL * 32, 256), 256, 0, st>>>(NL, t->sym_work_off, t->sym_work, t->p2p_src,
                                                          t->src_leaf_box, t->box_count, cost);
  FMM_LAUNCH_CHECK();
  t->leaf_order_sym = dev_alloc<int32_t>(t, NL);
  order_desc(cost, NL, t->leaf_order_sym, st);
  dev_free(cost);
  FMM_CUDA_TRY(cudaStreamSynchronize(st));
  t->sym = 1;
}

// FP64DF near field: double-float point records and the source frame of
// every work entry (made once, when FMM_FP64DF is first selected)
void build_df_near(fmm_tree* t, cudaStream_t st) {
  if (t->src_df || !t->sym) return;
  const int64_t NL = t->n_leaves;
  int64_t nw = 0;
  FMM_CUDA_TRY(cudaMemcpyAsync(&nw, t->sym_work_off + NL, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
  FMM_CUDA_TRY(cudaStreamSynchronize(st));
  t->src_df = dev_alloc<DFRec>(t, t->n);
  df_points_kernel<<<grid_for(NL * 32, 256), 256, 0, st>>>(NL, t->leaf_box, t->box_start, t->box_count, t->center,
                                                           t->pos64, t->src_df);
  FMM_LAUNCH_CHECK();
  t->sym_frame = dev_alloc<SymFrame>(t, std::max<int64_t>(nw, 1));
  frame_rec_kernel<<<grid_for(NL * 32, 256), 256, 0, st>>>(NL, t->sym_work_off, t->sym_work, t->p2p_src, t->leaf_box,
                                                           t->center, t->sym_frame);
  FMM_LAUNCH_CHECK();
  FMM_CUDA_TRY(cudaStreamSynchronize(st));
}

bool ensure_sym_vec(fmm_tree* t, cudaStream_t st) {
  if (!t->sym || t->max_leaf > 128) return false;
  if (t->sym_partial4) return true;
  if (t->ws_external) return false;  // evaluations allocate nothing beside a caller's workspace
  const size_t stride = (size_t)std::max(t->sym_stride, 1);
  t->sym_partial4 = dev_alloc<float>(t, 4 * (size_t)std::max<int64_t>(t->n_slots, 1) * stride);
  t->gpart4 = dev_alloc<float>(t, 8 * (size_t)std::max<int64_t>(t->n_gchunks, 1) * stride);
  FMM_CUDA_TRY(cudaStreamSynchronize(st));
  return true;
}

}  // namespace fmm
