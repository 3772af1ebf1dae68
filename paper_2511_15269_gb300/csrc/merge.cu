// fmm_tree_merge: one tree-shaped object holding several independent trees
// (a batch of charge sets), so that every evaluation stage runs as one launch
// over all of them.  Points, boxes, interaction lists and per-interaction
// coefficients are concatenated with offsets; leaf boxes and the M2M rounds
// become explicit index lists (M2M round r: the boxes r levels above each
// tree's leaves), and the direct L2L records are rebuilt over the batch.
#include <algorithm>
#include <chrono>
#include <vector>

#include <climits>

#include "common.cuh"

namespace fmm {
namespace {

__global__ void add_i32_kernel(int32_t* __restrict__ dst, const int32_t* __restrict__ src, int64_t n, int32_t add,
                               int keep_negative) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int32_t v = src[i];
    dst[i] = (keep_negative && v < 0) ? v : v + add;
  }
}
__global__ void add_i64_kernel(int64_t* __restrict__ dst, const int64_t* __restrict__ src, int64_t n, int64_t add) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    dst[i] = src[i] + add;
}
// near-field entries: shift the source leaf, keep the coincident-point flag
__global__ void shift_entries_kernel(P2PEntry* __restrict__ dst, const P2PEntry* __restrict__ src, int64_t n,
                                     int32_t add) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    P2PEntry e = src[i];
    const int flag = e.src & (int)0x80000000;
    e.src = ((e.src & 0x7fffffff) + add) | flag;
    dst[i] = e;
  }
}

template <class T>
void copy_d2d(T* dst, const T* src, int64_t n, cudaStream_t st) {
  if (n > 0) FMM_CUDA_TRY(cudaMemcpyAsync(dst, src, sizeof(T) * n, cudaMemcpyDeviceToDevice, st));
}

// field-major structure of arrays: rows of `width` entries into rows of
// `total` entries at column `col`
template <class T>
void copy_rows(T* dst, int64_t total, int64_t col, const T* src, int64_t width, int rows, cudaStream_t st) {
  if (width > 0)
    FMM_CUDA_TRY(cudaMemcpy2DAsync(dst + col, sizeof(T) * total, src, sizeof(T) * width, sizeof(T) * width, rows,
                                   cudaMemcpyDeviceToDevice, st));
}

}  // namespace

void merge_trees(fmm_tree* const* in, int nt, cudaStream_t st, fmm_tree* m) {
  const fmm_tree& t0 = *in[0];
  for (int k = 0; k < nt; k++) {
    require(in[k] != nullptr, "NULL tree");
    require(in[k]->n_trees == 1, "trees to merge must not be merged batches");
    require(!in[k]->two_trees, "trees with separate source and target sets cannot be merged");
    require(in[k]->prm.p == t0.prm.p && in[k]->prm.splits == t0.prm.splits, "trees must share p and splits");
  }
  const int p = t0.prm.p, s = t0.prm.splits;
  m->prm = t0.prm;
  m->s = s;
  m->n_trees = nt;
  std::vector<int64_t> po(nt + 1, 0), bo(nt + 1, 0), lo(nt + 1, 0), mo(nt + 1, 0), eo(nt + 1, 0);
  int Lmax = 0, max_leaf = 0, min_leaf = INT_MAX;
  int64_t pairs = 0;
  for (int k = 0; k < nt; k++) {
    const fmm_tree& t = *in[k];
    po[k + 1] = po[k] + t.n;
    bo[k + 1] = bo[k] + t.n_boxes;
    lo[k + 1] = lo[k] + t.n_leaves;
    mo[k + 1] = mo[k] + t.n_m2l;
    eo[k + 1] = eo[k] + t.n_p2p;
    Lmax = std::max(Lmax, t.L);
    max_leaf = std::max(max_leaf, t.max_leaf);
    min_leaf = std::min(min_leaf, t.min_leaf);
    pairs += t.n_p2p_pairs;
    m->prm.leaf_size = std::max(m->prm.leaf_size, t.prm.leaf_size);
    m->has_duplicates |= t.has_duplicates;
  }
  require(bo[nt] < ((int64_t)1 << 31) && po[nt] < ((int64_t)1 << 31), "merged batch too large");
  const int64_t N = po[nt], NB = bo[nt], NL = lo[nt], NM = mo[nt], NP = eo[nt];
  m->n = N;
  m->L = Lmax;
  m->n_boxes = NB;
  m->n_leaves = NL;
  m->n_m2l = NM;
  m->n_p2p = NP;
  m->n_p2p_pairs = pairs;
  m->max_leaf = max_leaf;
  m->min_leaf = nt > 0 ? min_leaf : 0;
  m->tree_point_off_h = new int64_t[nt + 1];
  for (int k = 0; k <= nt; k++) m->tree_point_off_h[k] = po[k];
  m->level_avg_host = new double[Lmax + 1]();

  m->perm = dev_alloc<int32_t>(m, N);
  m->box_start = dev_alloc<int64_t>(m, NB);
  m->box_count = dev_alloc<int32_t>(m, NB);
  m->center = dev_alloc<double>(m, 3 * NB);
  m->radius = dev_alloc<double>(m, NB);
  m->inv_rho32 = dev_alloc<float>(m, NB);
  m->inv_rho64 = dev_alloc<double>(m, NB);
  m->m2l_off = dev_alloc<int64_t>(m, NB + 1);
  m->m2l_src = dev_alloc<int32_t>(m, NM);
  m->m2l_trg = dev_alloc<int32_t>(m, NM);
  m->p2p_off = dev_alloc<int64_t>(m, NL + 1);
  m->p2p_src = dev_alloc<int32_t>(m, NP);
  m->p2p32 = dev_alloc<P2PEntry>(m, NP);
  m->p2p_thr = dev_alloc<float>(m, NP);
  m->leaf_box = dev_alloc<int32_t>(m, NL);
  m->box_parent = dev_alloc<int32_t>(m, NB);
  m->pos_local = dev_alloc<float4>(m, N);
  m->pos64 = dev_alloc<dvec4>(m, N);
  m->geo32 = dev_alloc<float>(m, (size_t)m2l_fields(p) * std::max<int64_t>(NM, 1));
  m->m2m32 = dev_alloc<float>(m, (size_t)edge_fields(p) * NB);

  for (int k = 0; k < nt; k++) {
    const fmm_tree& t = *in[k];
    add_i32_kernel<<<grid_for(t.n, 256), 256, 0, st>>>(m->perm + po[k], t.perm, t.n, (int32_t)po[k], 0);
    add_i64_kernel<<<grid_for(t.n_boxes, 256), 256, 0, st>>>(m->box_start + bo[k], t.box_start, t.n_boxes, po[k]);
    copy_d2d(m->box_count + bo[k], t.box_count, t.n_boxes, st);
    copy_d2d(m->center + 3 * bo[k], t.center, 3 * t.n_boxes, st);
    copy_d2d(m->radius + bo[k], t.radius, t.n_boxes, st);
    copy_d2d(m->inv_rho32 + bo[k], t.inv_rho32, t.n_boxes, st);
    copy_d2d(m->inv_rho64 + bo[k], t.inv_rho64, t.n_boxes, st);
    add_i64_kernel<<<grid_for(t.n_boxes, 256), 256, 0, st>>>(m->m2l_off + bo[k], t.m2l_off, t.n_boxes, mo[k]);
    add_i32_kernel<<<grid_for(t.n_m2l, 256), 256, 0, st>>>(m->m2l_src + mo[k], t.m2l_src, t.n_m2l, (int32_t)bo[k], 0);
    add_i32_kernel<<<grid_for(t.n_m2l, 256), 256, 0, st>>>(m->m2l_trg + mo[k], t.m2l_trg, t.n_m2l, (int32_t)bo[k], 0);
    add_i64_kernel<<<grid_for(t.n_leaves, 256), 256, 0, st>>>(m->p2p_off + lo[k], t.p2p_off, t.n_leaves, eo[k]);
    add_i32_kernel<<<grid_for(t.n_p2p, 256), 256, 0, st>>>(m->p2p_src + eo[k], t.p2p_src, t.n_p2p, (int32_t)lo[k], 0);
    shift_entries_kernel<<<grid_for(t.n_p2p, 256), 256, 0, st>>>(m->p2p32 + eo[k], t.p2p32, t.n_p2p, (int32_t)lo[k]);
    copy_d2d(m->p2p_thr + eo[k], t.p2p_thr, t.n_p2p, st);
    add_i32_kernel<<<grid_for(t.n_leaves, 256), 256, 0, st>>>(m->leaf_box + lo[k], t.leaf_box, t.n_leaves,
                                                              (int32_t)bo[k], 0);
    add_i32_kernel<<<grid_for(t.n_boxes, 256), 256, 0, st>>>(m->box_parent + bo[k], t.box_parent, t.n_boxes,
                                                             (int32_t)bo[k], 1);
    FMM_LAUNCH_CHECK();
    copy_d2d(m->pos_local + po[k], t.pos_local, t.n, st);
    copy_d2d(m->pos64 + po[k], t.pos64, t.n, st);
    copy_rows(m->geo32, NM, mo[k], t.geo32, t.n_m2l, m2l_fields(p), st);
    copy_rows(m->m2m32, NB, bo[k], t.m2m32, t.n_boxes, edge_fields(p), st);
  }
  {
    const int64_t tails[2] = {NM, NP};
    FMM_CUDA_TRY(cudaMemcpyAsync(m->m2l_off + NB, &tails[0], sizeof(int64_t), cudaMemcpyHostToDevice, st));
    FMM_CUDA_TRY(cudaMemcpyAsync(m->p2p_off + NL, &tails[1], sizeof(int64_t), cudaMemcpyHostToDevice, st));
    FMM_CUDA_TRY(cudaStreamSynchronize(st));
  }

  // rounds: M2M round r takes, from every tree with L > r, its level L - r
  auto loff = [&](int l) {
    int64_t o = 0;
    for (int i = 0; i < l; i++) o += (int64_t)1 << (s * i);
    return o;
  };
  std::vector<int32_t> up;
  m->n_up = Lmax;
  m->up_off_h = new int64_t[Lmax + 1];
  for (int r = 0; r < Lmax; r++) {
    m->up_off_h[r] = (int64_t)up.size();
    for (int k = 0; k < nt; k++) {
      const int L = in[k]->L;
      if (L > r)
        for (int64_t g = loff(L - r); g < loff(L - r + 1); g++) up.push_back((int32_t)(bo[k] + g));
    }
  }
  m->up_off_h[Lmax] = (int64_t)up.size();
  m->up_ids = dev_alloc<int32_t>(m, std::max<size_t>(up.size(), 1));
  if (!up.empty())
    FMM_CUDA_TRY(cudaMemcpyAsync(m->up_ids, up.data(), sizeof(int32_t) * up.size(), cudaMemcpyHostToDevice, st));
  // locals reach the leaves of every tree by direct L2L records
  build_l2l_direct(m, st);

  // work orders over the whole batch: longest M2L lists and heaviest near
  // fields first
  m->src_leaf_box = m->leaf_box;
  build_work_orders(m, st);

  // evaluation workspace
  const int NCP = ncoef_pad(p);
  m->src32 = dev_alloc<float4>(m, N);
  m->src_dup = dev_alloc<DupRec>(m, N);
  m->M32 = dev_alloc<float>(m, (size_t)NB * NCP);
  m->Lam32 = dev_alloc<float>(m, (size_t)NB * NCP);
  m->near_u = dev_alloc<double>(m, N);
  m->near_f = dev_alloc<double>(m, 3 * (size_t)N);
  m->src_dup2 = dev_alloc<DupRec>(m, N);
  m->near_u2 = dev_alloc<float>(m, 2 * (size_t)N);
  m->near_f2 = dev_alloc<float>(m, 3 * (size_t)N);
  m->q_stage = dev_alloc<double>(m, N);
  m->u_stage = dev_alloc<double>(m, N);
  m->f_stage = dev_alloc<double>(m, 3 * (size_t)N);
  m->g_stage = dev_alloc<double>(m, 3 * (size_t)N);
  int lo_prio = 0, hi_prio = 0;
  FMM_CUDA_TRY(cudaDeviceGetStreamPriorityRange(&lo_prio, &hi_prio));
  FMM_CUDA_TRY(cudaStreamCreateWithPriority(&m->far_stream, cudaStreamNonBlocking, hi_prio));
  FMM_CUDA_TRY(cudaEventCreateWithFlags(&m->ev_fork, cudaEventDisableTiming));
  FMM_CUDA_TRY(cudaEventCreateWithFlags(&m->ev_join, cudaEventDisableTiming));
  m->n_charges = N;
  m->out_base = 0;
  m->n_src_leaves = NL;
  m->src_leaf_box = m->leaf_box;
  build_symmetric(m, st);
  m->counters = dev_alloc<int>(m, 8);
  m->m2m_ready = dev_alloc<int>(m, NB);
  m->status = dev_alloc<int>(m, 1);
  FMM_CUDA_TRY(cudaMemsetAsync(m->status, 0, sizeof(int), st));
  FMM_CUDA_TRY(cudaStreamSynchronize(st));
}

}  // namespace fmm
