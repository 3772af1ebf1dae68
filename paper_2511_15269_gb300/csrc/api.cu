// C ABI of the FMM library (declarations and contracts in include/fmm.h).
#include <cstdarg>
#include <chrono>
#include <cstring>
#include <mutex>
#include <unordered_map>
#include <vector>

#include "common.cuh"

namespace fmm {

namespace {
thread_local char g_err[1024] = "";
std::mutex g_init_mu;
bool g_tables_ready[64] = {};

void ensure_tables() {
  int dev = 0;
  FMM_CUDA_TRY(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> lk(g_init_mu);
  if (dev >= 0 && dev < 64 && g_tables_ready[dev]) return;
  init_tables_fp32();
  init_tables_fp64();
  if (dev >= 0 && dev < 64) g_tables_ready[dev] = true;
}

// grad_pos = g grad u + q grad v = -(g E_q + q E_g)
__global__ void backward_combine_kernel(int64_t n, const double* __restrict__ q, const double* __restrict__ g,
                                        const double* __restrict__ eq, const double* __restrict__ eg,
                                        double* __restrict__ out) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    for (int a = 0; a < 3; a++) out[3 * i + a] = -(g[i] * eq[3 * i + a] + q[i] * eg[3 * i + a]);
}

// Evaluation workspace of a tree: the buffers every evaluation overwrites
// (point records, near-field sums and slots, expansions, staging buffers,
// work counters), for the precisions prepared so far.
struct WsItem {
  void** ptr;
  size_t bytes;
};
std::vector<WsItem> ws_items(fmm_tree* t) {
  const int64_t n = t->n, NB = t->n_boxes;
  const size_t NCP = (size_t)ncoef_pad(t->prm.p);
  std::vector<WsItem> v;
  auto add = [&](void* field_addr, size_t bytes) {
    void** f = reinterpret_cast<void**>(field_addr);
    if (*f) v.push_back(WsItem{f, bytes});
  };
  add(&t->src32, sizeof(float4) * n);
  add(&t->src_dup, sizeof(DupRec) * n);
  add(&t->src64, sizeof(dvec4) * n);
  add(&t->near_u, sizeof(double) * n);
  add(&t->near_f, sizeof(double) * 3 * n);
  add(&t->M32, sizeof(float) * NB * NCP);
  add(&t->Lam32, sizeof(float) * NB * NCP);
  add(&t->M64, sizeof(double) * NB * NCP);
  add(&t->Lam64, sizeof(double) * NB * NCP);
  add(&t->m_df, sizeof(float2) * NB * NCP);
  add(&t->sym_partial, (t->sym_partial_f64 ? sizeof(double) : sizeof(float)) *
                           (size_t)std::max<int64_t>(t->n_slots, 1) * std::max(t->sym_stride, 1));
  add(&t->src_dup2, sizeof(DupRec) * n);
  add(&t->near_u2, sizeof(float) * 2 * n);
  add(&t->near_f2, sizeof(float) * 3 * n);
  add(&t->q_stage, sizeof(double) * n);
  add(&t->u_stage, sizeof(double) * n);
  add(&t->f_stage, sizeof(double) * 3 * n);
  add(&t->g_stage, sizeof(double) * 3 * n);
  add(&t->counters, sizeof(int) * 8);
  add(&t->m2m_ready, sizeof(int) * NB);
  add(&t->m2l_partial, sizeof(double) * NCP * (size_t)std::max<int64_t>(t->m2l_partial_rows, 1));
  add(&t->gpart, sizeof(double) * (size_t)std::max<int64_t>(t->n_gchunks, 1) * std::max(t->sym_stride, 1));
  add(&t->sym_partial4, 4 * sizeof(float) * (size_t)std::max<int64_t>(t->n_slots, 1) * std::max(t->sym_stride, 1));
  add(&t->gpart4, 8 * sizeof(float) * (size_t)std::max<int64_t>(t->n_gchunks, 1) * std::max(t->sym_stride, 1));
  return v;
}
size_t ws_bytes(const std::vector<WsItem>& v) {
  size_t b = 0;
  for (auto& w : v) b += (w.bytes + 255) & ~(size_t)255;
  return b;
}

// Batched charge sets: per-set pointers passed by value (up to kBatchPtrs
// sets per launch).
constexpr int kBatchPtrs = 256;
struct SetPtrs {
  const double* p[kBatchPtrs];
  int64_t off[kBatchPtrs + 1];  // set k: points off[k] .. off[k + 1] - 1 of the batch
};
__global__ void batch_gather_kernel(SetPtrs sp, int nsets, double* __restrict__ dst) {
  const int64_t base = sp.off[0];
  const int64_t total = sp.off[nsets] - base;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    int lo = 0, hi = nsets - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (sp.off[mid] - base <= i) lo = mid;
      else hi = mid - 1;
    }
    dst[base + i] = sp.p[lo][base + i - sp.off[lo]];
  }
}
__global__ void batch_scatter_kernel(SetPtrs sp, int nsets, const double* __restrict__ src) {
  const int64_t base = sp.off[0];
  const int64_t total = sp.off[nsets] - base;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    int lo = 0, hi = nsets - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (sp.off[mid] - base <= i) lo = mid;
      else hi = mid - 1;
    }
    const_cast<double*>(sp.p[lo])[base + i - sp.off[lo]] = src[base + i];
  }
}

void eval_any(const fmm_tree* t, const double* q, double* u, double* field, cudaStream_t st) {
  if (t->prm.precision == FMM_FP32C) eval_fp32(t, q, u, field, st);
  else eval_fp64(t, q, u, field, st);
}

template <class F>
int guarded(F&& f) {
  try {
    f();
    return FMM_OK;
  } catch (const Fail& e) {
    return e.code;
  } catch (...) {
    set_error("unexpected C++ exception");
    return FMM_ERR_CUDA;
  }
}

}  // namespace

void free_tree(fmm_tree* t) {
  if (!t) return;
  cudaDeviceSynchronize();
  void* ptrs[] = {t->perm,     t->box_start, t->box_count, t->center,   t->radius,   t->m2l_off,  t->m2l_src,
                  t->m2l_trg,  t->m2l_items, t->m2l_split_g, t->m2l_split_row, t->m2l_partial,
                  t->gch_leaf, t->gch_r0, t->gch_first, t->gmulti_leaf, t->gpart, t->p2p_off,   t->p2p_src,  t->p2p32,    t->leaf_order, t->pos_local,
                  t->pos64,    t->inv_rho32, t->inv_rho64, t->geo32,    t->geo64,    t->m2m32,    t->m2m64,
                  t->l2d32,    t->l2d64,     t->geo_lo,    t->m_df,     t->src32,     t->src64,    t->M32,      t->Lam32,    t->M64,
                  t->Lam64,    t->src_dup,   t->near_u,    t->near_f,    t->q_stage,  t->u_stage,  t->f_stage,  t->g_stage,
                  t->counters, t->status,   t->leaf_box,  t->box_parent, t->up_ids,  t->l2d_off, t->l2d_anc,
                  t->two_trees ? t->src_leaf_box : nullptr, t->p2p_thr, t->sym_slot, t->sym_work_off,
                  t->sym_work, t->sym_recv_off, t->sym_partial, t->leaf_order_sym, t->sym_rec, t->src_df, t->sym_frame, t->src_dup2, t->near_u2, t->near_f2,
                  t->m2m_ready, t->sym_partial4, t->gpart4};
  for (void* p : ptrs)
    if (p) dev_free(p);
  if (t->prof_ev) {
    for (int i = 0; i < fmm_tree::kProfCalls * fmm_tree::kProfSlots * 2; i++) cudaEventDestroy(t->prof_ev[i]);
    delete[] t->prof_ev;
  }
  if (t->ev_fork) cudaEventDestroy(t->ev_fork);
  if (t->ev_join) cudaEventDestroy(t->ev_join);
  if (t->far_stream) cudaStreamDestroy(t->far_stream);
  delete[] t->level_avg_host;
  delete[] t->up_off_h;
  delete[] t->tree_point_off_h;
  delete t;
  trim_pool();
}

namespace {
struct LiveAlloc {
  size_t bytes;
  bool pooled;  // from the library's stream-ordered pool (cudaMallocFromPoolAsync)
};
std::mutex g_mem_mu;
std::unordered_map<void*, LiveAlloc> g_live;  // library allocation -> size, origin
size_t g_live_bytes = 0;
size_t g_mem_limit = 0;  // 0: no cap
size_t g_pool_keep = (size_t)2 << 30;  // unused pool memory kept for later builds
cudaMemPool_t g_pool[64] = {};

// The library's memory pool on the current device, created on first use;
// it keeps freed memory for reuse until the end of the build that freed it
// (AllocScope trims it then), so the many short-lived scratch buffers of a
// build cost neither cudaMalloc nor an implicit synchronisation of cudaFree.
cudaMemPool_t pool_for_device() {
  int dev = 0;
  FMM_CUDA_TRY(cudaGetDevice(&dev));
  require(dev >= 0 && dev < 64, "device ordinal out of range");
  std::lock_guard<std::mutex> lk(g_mem_mu);
  if (!g_pool[dev]) {
    cudaMemPoolProps props = {};
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = dev;
    cudaMemPool_t pool = nullptr;
    FMM_CUDA_TRY(cudaMemPoolCreate(&pool, &props));
    uint64_t keep = UINT64_MAX;
    FMM_CUDA_TRY(cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep));
    g_pool[dev] = pool;
  }
  return g_pool[dev];
}
}  // namespace

namespace {
thread_local cudaStream_t tl_build_stream_end = nullptr;  // the outermost scope's stream

// Unused pool memory to keep: the retention, within the headroom under a cap.
size_t pool_keep_bytes() {
  std::lock_guard<std::mutex> lk(g_mem_mu);
  size_t keep = g_pool_keep;
  if (g_mem_limit) keep = std::min(keep, g_mem_limit > g_live_bytes ? g_mem_limit - g_live_bytes : (size_t)0);
  return keep;
}
}  // namespace

void trim_pool() {
  if (tl_alloc_pool) return;  // inside a build: its scope trims at the end
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return;
  cudaMemPool_t pool = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_mem_mu);
    pool = g_pool[dev];
  }
  if (pool) {
    cudaDeviceSynchronize();
    cudaMemPoolTrimTo(pool, pool_keep_bytes());
  }
}

AllocScope::AllocScope(cudaStream_t s)
    : prev(tl_alloc_stream), prev_pool(tl_alloc_pool), pool(pool_for_device()) {
  tl_alloc_stream = s;
  tl_alloc_pool = pool;
  if (!prev_pool) tl_build_stream_end = s;
}
AllocScope::~AllocScope() {
  tl_alloc_stream = prev;
  tl_alloc_pool = prev_pool;
  if (!prev_pool) {
    // the outermost scope gives the memory freed during the build back
    // (builds on other threads and streams keep theirs)
    cudaStreamSynchronize(tl_build_stream_end);
    cudaMemPoolTrimTo(pool, pool_keep_bytes());
  }
}

void* tracked_malloc(size_t bytes) {
  {
    std::lock_guard<std::mutex> lk(g_mem_mu);
    if (g_mem_limit && g_live_bytes + bytes > g_mem_limit) {
      set_error("device allocation of %zu bytes refused: the library holds %zu bytes and its limit is %zu "
                "(fmm_set_device_memory_limit)",
                bytes, g_live_bytes, g_mem_limit);
      throw Fail{FMM_ERR_OOM};
    }
  }
  void* p = nullptr;
  const bool pooled = tl_alloc_pool != nullptr;
  const cudaError_t e = pooled ? cudaMallocFromPoolAsync(&p, bytes, tl_alloc_pool, tl_alloc_stream)
                               : cudaMalloc(&p, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();  // clear the allocation error
    set_error("device allocation of %zu bytes failed: %s", bytes, cudaGetErrorString(e));
    throw Fail{FMM_ERR_OOM};
  }
  std::lock_guard<std::mutex> lk(g_mem_mu);
  g_live[p] = LiveAlloc{bytes, pooled};
  g_live_bytes += bytes;
  return p;
}

void dev_free(void* p) {
  if (!p) return;
  bool pooled = false, tracked = false;
  {
    std::lock_guard<std::mutex> lk(g_mem_mu);
    auto it = g_live.find(p);
    if (it != g_live.end()) {
      g_live_bytes -= it->second.bytes;
      pooled = it->second.pooled;
      tracked = true;
      g_live.erase(it);
    }
  }
  if (!tracked) return;  // not the library's (a caller's workspace)
  // stream-ordered inside a build (the memory is reused once the work queued
  // before the free has run); otherwise after the device is idle
  if (pooled) cudaFreeAsync(p, tl_alloc_pool ? tl_alloc_stream : nullptr);
  else cudaFree(p);
}

void set_error(const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
}
const char* last_error() { return g_err; }

}  // namespace fmm

using namespace fmm;

extern "C" {

const char* fmm_last_error(void) { return fmm::last_error(); }

int fmm_set_device_memory_limit(size_t bytes) {
  std::lock_guard<std::mutex> lk(g_mem_mu);
  g_mem_limit = bytes;
  return FMM_OK;
}

int fmm_set_pool_retention(size_t bytes) {
  {
    std::lock_guard<std::mutex> lk(g_mem_mu);
    g_pool_keep = bytes;
  }
  trim_pool();
  return FMM_OK;
}

int fmm_device_memory_in_use(size_t* bytes) {
  if (!bytes) {
    set_error("invalid argument: bytes is NULL");
    return FMM_ERR_INVALID_ARG;
  }
  std::lock_guard<std::mutex> lk(g_mem_mu);
  *bytes = g_live_bytes;
  return FMM_OK;
}

int fmm_tree_set_option(fmm_tree* tree, int option, int value) {
  return guarded([&] {
    require(tree != nullptr, "tree is NULL");
    switch (option) {
      case FMM_OPT_SCHEDULE:
        require(value >= 0 && value <= 3, "FMM_OPT_SCHEDULE takes 0 .. 3");
        tree->opt_schedule = value;
        break;
      case FMM_OPT_M2M_ONE_LAUNCH:
        require(value == 0 || value == 1, "FMM_OPT_M2M_ONE_LAUNCH takes 0 or 1");
        tree->opt_m2m_one_launch = value;
        break;
      case FMM_OPT_NEAR_SYMMETRIC:
        require(value == 0 || value == 1, "FMM_OPT_NEAR_SYMMETRIC takes 0 or 1");
        tree->opt_near_sym = value;
        break;
      case FMM_OPT_M2L_BLOCKS_PER_SM:
        require(value >= 0 && value <= 32, "FMM_OPT_M2L_BLOCKS_PER_SM takes 0 .. 32");
        tree->opt_m2l_blocks_per_sm = value;
        break;
      default:
        require(false, "unknown option");
    }
  });
}

int fmm_tree_set_wait_limit(fmm_tree* tree, int64_t cycles) {
  if (!tree || cycles < 0) {
    set_error("invalid argument: %s", !tree ? "tree is NULL" : "cycles must be >= 0");
    return FMM_ERR_INVALID_ARG;
  }
  tree->wait_cycles = (long long)cycles;
  return FMM_OK;
}

int fmm_num_levels(int64_t n, int leaf_size, int splits) {
  if (n < 1 || splits < 1 || splits > 3 || leaf_size < (1 << splits)) return -1;
  int L = 0;
  for (;;) {
    const int64_t boxes = (int64_t)1 << (splits * L);
    if ((n + boxes - 1) / boxes <= leaf_size) return L;
    L++;
  }
}

int fmm_build_tree(const double* pos, int64_t n, const fmm_params* params, void* stream, fmm_tree** out) {
  if (out) *out = nullptr;
  fmm_tree* t = nullptr;
  int rc = guarded([&] {
    require(out != nullptr, "out is NULL");
    require(params != nullptr, "params is NULL");
    require(pos != nullptr, "pos is NULL");
    const fmm_params& p = *params;
    require(n >= 1 && n < (int64_t)1 << 31, "n must be in [1, 2^31)");
    require(p.p >= 1 && p.p <= FMM_MAX_P, "p must be in [1, FMM_MAX_P]");
    require(p.splits >= 1 && p.splits <= 3, "splits must be 1, 2 or 3");
    require(p.leaf_size >= (1 << p.splits) && p.leaf_size <= kMaxLeaf, "leaf_size must be in [2^splits, 256]");
    require(p.theta > 0.0 && p.theta < 1.0, "theta must be in (0, 1)");
    require(p.precision == FMM_FP64 || p.precision == FMM_FP32C || p.precision == FMM_FP64DF,
            "precision must be FMM_FP64, FMM_FP32C or FMM_FP64DF");
    require((p.flags & ~(FMM_TIE_TARGET | FMM_SAME_LEVEL | FMM_POS_SOA)) == 0, "unknown flags");
    auto t0 = std::chrono::steady_clock::now();
    TraceScope trace((cudaStream_t)stream);
    AllocScope scratch((cudaStream_t)stream);
    ensure_tables();
    t = new fmm_tree();
    t->prm = p;
    t->n = n;
    t->L = fmm_num_levels(n, p.leaf_size, p.splits);
    trace_mark("set-up");
    build_tree(t, pos, (cudaStream_t)stream);
    if (p.precision != FMM_FP32C) ensure_fp64(t, (cudaStream_t)stream);
    if (p.precision == FMM_FP64DF) prepare_df_far(t, (cudaStream_t)stream);
    t->build_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  });
  if (rc != FMM_OK) {
    free_tree(t);
    return rc;
  }
  *out = t;
  return FMM_OK;
}

int fmm_build_tree2(const double* src_pos, int64_t n_src, const double* trg_pos, int64_t n_trg,
                    const fmm_params* params, void* stream, fmm_tree** out) {
  if (out) *out = nullptr;
  fmm_tree* t = nullptr;
  int rc = guarded([&] {
    require(out != nullptr, "out is NULL");
    require(params != nullptr, "params is NULL");
    require(src_pos != nullptr && trg_pos != nullptr, "positions are NULL");
    const fmm_params& p = *params;
    require(n_src >= 1 && n_trg >= 1 && n_src + n_trg < (int64_t)1 << 31, "n_src, n_trg >= 1, n_src + n_trg < 2^31");
    require(p.p >= 1 && p.p <= FMM_MAX_P, "p must be in [1, FMM_MAX_P]");
    require(p.splits >= 1 && p.splits <= 3, "splits must be 1, 2 or 3");
    require(p.leaf_size >= (1 << p.splits) && p.leaf_size <= kMaxLeaf, "leaf_size must be in [2^splits, 256]");
    require(p.theta > 0.0 && p.theta < 1.0, "theta must be in (0, 1)");
    require(p.precision == FMM_FP64 || p.precision == FMM_FP32C || p.precision == FMM_FP64DF,
            "precision must be FMM_FP64, FMM_FP32C or FMM_FP64DF");
    require((p.flags & ~(FMM_TIE_TARGET | FMM_POS_SOA)) == 0,
            "flags must be 0 or FMM_TIE_TARGET (with or without FMM_POS_SOA) for two hierarchies");
    auto t0 = std::chrono::steady_clock::now();
    TraceScope trace((cudaStream_t)stream);
    AllocScope scratch((cudaStream_t)stream);
    ensure_tables();
    t = new fmm_tree();
    t->prm = p;
    build_tree2(t, src_pos, n_src, trg_pos, n_trg, (cudaStream_t)stream);
    if (p.precision != FMM_FP32C) ensure_fp64(t, (cudaStream_t)stream);
    t->build_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  });
  if (rc != FMM_OK) {
    free_tree(t);
    return rc;
  }
  *out = t;
  return FMM_OK;
}

void fmm_tree_free(fmm_tree* tree) { free_tree(tree); }

int fmm_tree_merge(fmm_tree* const* trees, int n_trees, void* stream, fmm_tree** out) {
  if (out) *out = nullptr;
  fmm_tree* m = nullptr;
  int rc = guarded([&] {
    require(out != nullptr && trees != nullptr, "NULL argument");
    require(n_trees >= 1, "n_trees must be >= 1");
    for (int k = 0; k < n_trees; k++)
      require(trees[k] == nullptr || !trees[k]->two_trees, "trees with separate source and target sets cannot be merged");
    auto t0 = std::chrono::steady_clock::now();
    AllocScope scratch((cudaStream_t)stream);
    m = new fmm_tree();
    merge_trees(trees, n_trees, (cudaStream_t)stream, m);
    if (m->prm.precision != FMM_FP32C) ensure_fp64(m, (cudaStream_t)stream);
    if (m->prm.precision == FMM_FP64DF) prepare_df_far(m, (cudaStream_t)stream);
    m->build_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  });
  if (rc != FMM_OK) {
    free_tree(m);
    return rc;
  }
  *out = m;
  return FMM_OK;
}

int fmm_tree_point_offsets(const fmm_tree* t, int64_t* offsets) {
  return guarded([&] {
    require(t != nullptr && offsets != nullptr, "NULL argument");
    if (t->tree_point_off_h) {
      for (int k = 0; k <= t->n_trees; k++) offsets[k] = t->tree_point_off_h[k];
    } else {
      offsets[0] = 0;
      offsets[1] = t->n;
    }
  });
}

int fmm_tree_set_precision(fmm_tree* tree, int precision) {
  return guarded([&] {
    require(tree != nullptr, "tree is NULL");
    require(precision == FMM_FP64 || precision == FMM_FP32C || precision == FMM_FP64DF,
            "precision must be FMM_FP64, FMM_FP32C or FMM_FP64DF");
    // FP64 rotation records, expansions and wide slots are made on the first
    // FP64 or FP64DF selection (on the legacy default stream, synchronously)
    if (precision != FMM_FP32C) ensure_fp64(tree, 0);
    if (precision == FMM_FP64DF) prepare_df_far(tree, 0);
    tree->prm.precision = precision;
  });
}

int fmm_tree_stats(const fmm_tree* t, fmm_stats* s) {
  return guarded([&] {
    require(t != nullptr && s != nullptr, "NULL argument");
    std::memset(s, 0, sizeof(*s));
    s->n = t->n;
    s->levels = t->L;
    s->p = t->prm.p;
    s->splits = t->prm.splits;
    s->leaf_size = t->prm.leaf_size;
    s->precision = t->prm.precision;
    s->theta = t->prm.theta;
    s->n_boxes = t->n_boxes;
    s->n_leaves = t->n_leaves;
    s->n_m2l = t->n_m2l;
    s->n_p2p = t->n_p2p;
    s->n_p2p_pairs = t->n_p2p_pairs;
    s->device_bytes = t->device_bytes;
    s->build_ms = t->build_ms;
    s->kernel_launches = t->launches;
    s->n_trees = t->n_trees;
    s->n_sources = t->n_charges;
    s->n_targets = t->two_trees ? t->n - t->n_charges : t->n;
    s->levels_src = t->two_trees ? t->L_src : t->L;
    s->n_src_leaves = t->n_src_leaves;
  });
}

int fmm_tree_profile(fmm_tree* t, int enable) {
  return guarded([&] {
    require(t != nullptr, "tree is NULL");
    if (enable && !t->prof_ev) {
      const int ne = fmm_tree::kProfCalls * fmm_tree::kProfSlots * 2;
      t->prof_ev = new cudaEvent_t[ne];
      for (int i = 0; i < ne; i++) FMM_CUDA_TRY(cudaEventCreate(&t->prof_ev[i]));
    }
    t->prof_on = enable ? 1 : 0;
    if (enable) t->prof_used = 0;
  });
}

int fmm_tree_stage_times(const fmm_tree* t, double* ms, int64_t* calls) {
  return guarded([&] {
    require(t != nullptr && ms != nullptr, "NULL argument");
    for (int s = 0; s < FMM_NUM_STAGES; s++) ms[s] = 0.0;
    if (calls) *calls = t->prof_ev ? t->prof_used : 0;
    if (!t->prof_ev) return;
    for (int c = 0; c < t->prof_used; c++) {
      cudaEvent_t* ev = t->prof_ev + c * fmm_tree::kProfSlots * 2;
      for (int s = 0; s < fmm_tree::kProfSlots; s++) {
        FMM_CUDA_TRY(cudaEventSynchronize(ev[2 * s + 1]));
        float x = 0.f;
        FMM_CUDA_TRY(cudaEventElapsedTime(&x, ev[2 * s], ev[2 * s + 1]));
        ms[s == fmm_tree::kStageP2P2 ? FMM_STAGE_P2P : s] += x;
      }
    }
  });
}

int fmm_tree_status(fmm_tree* t, void* stream) {
  int code = FMM_OK;
  int rc = guarded([&] {
    require(t != nullptr, "tree is NULL");
    cudaStream_t st = (cudaStream_t)stream;
    int h = 0;
    FMM_CUDA_TRY(cudaMemcpyAsync(&h, t->status, sizeof(int), cudaMemcpyDeviceToHost, st));
    FMM_CUDA_TRY(cudaStreamSynchronize(st));
    FMM_CUDA_TRY(cudaMemsetAsync(t->status, 0, sizeof(int), st));
    FMM_CUDA_TRY(cudaStreamSynchronize(st));
    if (h & ST_TIMEOUT) {
      set_error("a bounded device-side wait gave up (near-field tile copy)");
      code = FMM_ERR_TIMEOUT;
    }
  });
  return rc != FMM_OK ? rc : code;
}

int fmm_tree_export(const fmm_tree* t, int32_t* perm, int64_t* box_start, int64_t* box_count, double* center,
                    double* radius, double* level_avg_radius, int32_t* m2l_trg, int32_t* m2l_src,
                    int32_t* p2p_trg, int32_t* p2p_src) {
  return guarded([&] {
    require(t != nullptr, "tree is NULL");
    auto cp = [](void* dst, const void* src, size_t bytes) {
      if (dst && bytes) FMM_CUDA_TRY(cudaMemcpy(dst, src, bytes, cudaMemcpyDeviceToHost));
    };
    cp(perm, t->perm, sizeof(int32_t) * t->n);
    cp(box_start, t->box_start, sizeof(int64_t) * t->n_boxes);
    if (box_count) {
      std::vector<int32_t> c(t->n_boxes);
      cp(c.data(), t->box_count, sizeof(int32_t) * t->n_boxes);
      for (int64_t i = 0; i < t->n_boxes; i++) box_count[i] = c[i];
    }
    cp(center, t->center, sizeof(double) * 3 * t->n_boxes);
    cp(radius, t->radius, sizeof(double) * t->n_boxes);
    if (level_avg_radius)
      std::memcpy(level_avg_radius, t->level_avg_host,
                  sizeof(double) * (t->two_trees ? t->L_src + t->L + 2 : t->L + 1));
    cp(m2l_trg, t->m2l_trg, sizeof(int32_t) * t->n_m2l);
    cp(m2l_src, t->m2l_src, sizeof(int32_t) * t->n_m2l);
    cp(p2p_src, t->p2p_src, sizeof(int32_t) * t->n_p2p);
    if (p2p_trg) {
      std::vector<int64_t> off(t->n_leaves + 1);
      cp(off.data(), t->p2p_off, sizeof(int64_t) * (t->n_leaves + 1));
      for (int64_t l = 0; l < t->n_leaves; l++)
        for (int64_t e = off[l]; e < off[l + 1]; e++) p2p_trg[e] = (int32_t)l;
    }
  });
}

int fmm_eval_potential(const fmm_tree* t, const double* q, double* u, void* stream) {
  return guarded([&] {
    require(t != nullptr && q != nullptr && u != nullptr, "NULL argument");
    eval_any(t, q, u, nullptr, (cudaStream_t)stream);
  });
}

int fmm_eval_field(const fmm_tree* t, const double* q, double* u, double* field, void* stream) {
  return guarded([&] {
    require(t != nullptr && q != nullptr && field != nullptr, "NULL argument");
    if (t->prm.precision == FMM_FP32C && t->opt_near_sym) ensure_sym_vec(const_cast<fmm_tree*>(t), (cudaStream_t)stream);
    eval_any(t, q, u, field, (cudaStream_t)stream);
  });
}

int fmm_tree_workspace_bytes(const fmm_tree* t, size_t* bytes) {
  return guarded([&] {
    require(t != nullptr && bytes != nullptr, "NULL argument");
    *bytes = ws_bytes(ws_items(const_cast<fmm_tree*>(t)));
  });
}

int fmm_tree_set_workspace(fmm_tree* t, void* workspace, size_t ws_bytes_given) {
  return guarded([&] {
    require(t != nullptr, "tree is NULL");
    FMM_CUDA_TRY(cudaDeviceSynchronize());  // no evaluation may still use the old buffers
    std::vector<WsItem> items = ws_items(t);
    if (workspace == nullptr) {
      if (!t->ws_external) return;
      // the tree's own buffers again
      for (auto& w : items) {
        *w.ptr = tracked_malloc(w.bytes);
        t->device_bytes += w.bytes;
      }
      t->ws_external = 0;
      FMM_CUDA_TRY(cudaMemsetAsync(t->counters, 0, sizeof(int) * 8, 0));
      FMM_CUDA_TRY(cudaStreamSynchronize(0));
      return;
    }
    const size_t need = ws_bytes(items);
    if (ws_bytes_given < need) {
      set_error("workspace of %zu bytes is too small: this tree needs %zu (fmm_tree_workspace_bytes)",
                ws_bytes_given, need);
      throw Fail{FMM_ERR_CAPACITY};
    }
    require(((uintptr_t)workspace & 255) == 0, "workspace must be 256-byte aligned");
    unsigned char* base = static_cast<unsigned char*>(workspace);
    size_t off = 0;
    for (auto& w : items) {
      if (!t->ws_external) {
        dev_free(*w.ptr);
        t->device_bytes -= w.bytes;
      }
      *w.ptr = base + off;
      off += (w.bytes + 255) & ~(size_t)255;
    }
    t->ws_external = 1;
    FMM_CUDA_TRY(cudaMemsetAsync(t->counters, 0, sizeof(int) * 8, 0));
    FMM_CUDA_TRY(cudaStreamSynchronize(0));
  });
}

int fmm_eval_batched(const fmm_tree* t, int n_sets, const double* const* q_sets, double* const* u_sets,
                     void* stream) {
  return guarded([&] {
    require(t != nullptr && q_sets != nullptr && u_sets != nullptr, "NULL argument");
    require(!t->two_trees, "fmm_eval_batched takes batches of one-point-set trees");
    const int nt = t->n_trees;
    require(n_sets == nt, "n_sets must equal the number of trees of the batch");
    for (int k = 0; k < nt; k++) require(q_sets[k] != nullptr && u_sets[k] != nullptr, "NULL set pointer");
    cudaStream_t st = (cudaStream_t)stream;
    auto off = [&](int k) -> int64_t {
      return t->tree_point_off_h ? t->tree_point_off_h[k] : (k == 0 ? 0 : t->n);
    };
    for (int k0 = 0; k0 < nt; k0 += kBatchPtrs) {
      const int m = std::min(kBatchPtrs, nt - k0);
      SetPtrs sp;
      for (int k = 0; k < m; k++) sp.p[k] = q_sets[k0 + k];
      for (int k = 0; k <= m; k++) sp.off[k] = off(k0 + k);
      batch_gather_kernel<<<grid_for(sp.off[m] - sp.off[0], 256), 256, 0, st>>>(sp, m, t->q_stage);
      FMM_LAUNCH_CHECK();
    }
    eval_any(t, t->q_stage, t->u_stage, nullptr, st);
    for (int k0 = 0; k0 < nt; k0 += kBatchPtrs) {
      const int m = std::min(kBatchPtrs, nt - k0);
      SetPtrs sp;
      for (int k = 0; k < m; k++) sp.p[k] = u_sets[k0 + k];
      for (int k = 0; k <= m; k++) sp.off[k] = off(k0 + k);
      batch_scatter_kernel<<<grid_for(sp.off[m] - sp.off[0], 256), 256, 0, st>>>(sp, m, t->u_stage);
      FMM_LAUNCH_CHECK();
    }
    t->launches += 2 * ((nt + kBatchPtrs - 1) / kBatchPtrs);
  });
}

int fmm_eval_potential_host(const fmm_tree* t, const double* q_host, double* u_host, void* stream) {
  return guarded([&] {
    require(t != nullptr && q_host != nullptr && u_host != nullptr, "NULL argument");
    cudaStream_t st = (cudaStream_t)stream;
    const int64_t n_out = t->two_trees ? t->n - t->n_charges : t->n;
    FMM_CUDA_TRY(cudaMemcpyAsync(t->q_stage, q_host, sizeof(double) * t->n_charges, cudaMemcpyHostToDevice, st));
    eval_any(t, t->q_stage, t->u_stage, nullptr, st);
    FMM_CUDA_TRY(cudaMemcpyAsync(u_host, t->u_stage, sizeof(double) * n_out, cudaMemcpyDeviceToHost, st));
    FMM_CUDA_TRY(cudaStreamSynchronize(st));
  });
}

int fmm_backward(const fmm_tree* t, const double* q, const double* grad_u, double* grad_q, double* grad_pos,
                 void* stream) {
  return guarded([&] {
    require(t != nullptr && q != nullptr && grad_u != nullptr, "NULL argument");
    require(!t->two_trees,
            "fmm_backward needs one point set; for separate source and target trees evaluate the "
            "transposed problem (sources and targets swapped) instead");
    cudaStream_t st = (cudaStream_t)stream;
    const bool sym_vec = grad_pos && t->prm.precision == FMM_FP32C && t->src_dup2 && t->opt_near_sym &&
                         ensure_sym_vec(const_cast<fmm_tree*>(t), st);
    if (sym_vec) {
      // one symmetric near-field sweep for both charge vectors beside both far
      // fields, then a combine in tree order
      backward_sym_fp32(t, q, grad_u, grad_q, grad_pos, st);
    } else if (grad_pos && t->prm.precision == FMM_FP32C && t->src_dup2 && t->max_leaf <= 128) {
      // one near-field sweep for both charge vectors, then both far fields
      // (leaves of more than 128 points: two field evaluations below)
      backward_fp32(t, q, grad_u, grad_q, t->f_stage, t->g_stage, st);
      backward_combine_kernel<<<grid_for(t->n, 256), 256, 0, st>>>(t->n, q, grad_u, t->f_stage, t->g_stage,
                                                                   grad_pos);
      FMM_LAUNCH_CHECK();
    } else if (grad_pos) {
      eval_any(t, q, nullptr, t->f_stage, st);          // E of the charges
      eval_any(t, grad_u, grad_q, t->g_stage, st);      // v = K grad_u and E of grad_u
      backward_combine_kernel<<<grid_for(t->n, 256), 256, 0, st>>>(t->n, q, grad_u, t->f_stage, t->g_stage,
                                                                   grad_pos);
      FMM_LAUNCH_CHECK();
    } else if (grad_q) {
      eval_any(t, grad_u, grad_q, nullptr, st);
    }
  });
}

}  // extern "C"
