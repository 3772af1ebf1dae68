// Internal declarations shared by the CUDA translation units of the FMM
// library (C ABI in include/fmm.h).  Nothing here is part of the ABI.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <chrono>
#include <cstdio>
#include <cstdlib>
#include <string>

#include "../../include/fmm.h"

namespace fmm {

// ---- error handling -------------------------------------------------------
void set_error(const char* fmt, ...);
const char* last_error();

struct Fail {
  int code;
};

#define FMM_CUDA_TRY(expr)                                                      \
  do {                                                                          \
    cudaError_t e_ = (expr);                                                    \
    if (e_ != cudaSuccess) {                                                    \
      ::fmm::set_error("%s failed: %s (%s:%d)", #expr, cudaGetErrorString(e_),  \
                       __FILE__, __LINE__);                                     \
      throw ::fmm::Fail{e_ == cudaErrorMemoryAllocation ? FMM_ERR_OOM           \
                                                        : FMM_ERR_CUDA};        \
    }                                                                           \
  } while (0)

#define FMM_LAUNCH_CHECK() FMM_CUDA_TRY(cudaGetLastError())

inline void require(bool ok, const char* what) {
  if (!ok) {
    set_error("invalid argument: %s", what);
    throw Fail{FMM_ERR_INVALID_ARG};
  }
}

// Device status bits latched by kernels (read by fmm_tree_status).
enum : int { ST_TIMEOUT = 1 };

// Bounded waits: clock cycles a near-field warp waits for a staged source
// tile before it gives up and latches ST_TIMEOUT (about a second; settable
// per tree with fmm_tree_set_wait_limit), and the limit of the waits that let
// copies still in flight land before such a warp leaves.
constexpr long long kDefaultWaitCycles = 2000000000ll;
constexpr long long kDrainWaitCycles = 2000000000ll;

// ---- sizes -----------------------------------------------------------------
constexpr int kMaxP = FMM_MAX_P;
constexpr int kMaxLeaf = 256;     // largest leaf the leaf kernels accept
constexpr int kSmallCap = 2048;   // segments up to this size finish in one CTA

__host__ __device__ constexpr int ncoef(int p) { return (p + 1) * (p + 1); }
// Coefficient rows are padded to a multiple of 4 reals for vector loads.
__host__ __device__ constexpr int ncoef_pad(int p) { return (ncoef(p) + 3) & ~3; }

// Per-interaction geometry fields (structure of arrays, field-major):
//   M2L: [0] 1/r  [1] rho_S/r  [2] rho_T/r  [3] cos phi  [4] sin phi
//        [5] cos theta  [6] sin theta  (the M2L kernels make the multiples
//        m phi, m theta, m = 2..p, by angle addition in their own precision)
//   edges (per child box, M2M and L2L each): [0] r/rho_P  [1] rho_C/rho_P
//        then cos(m phi), sin(m phi), cos(m theta), sin(m theta) for m = 1..p
__host__ __device__ constexpr int m2l_fields(int /*p*/) { return 7; }
__host__ __device__ constexpr int edge_fields(int p) { return 2 + 4 * p; }

// Near-field entry for the FP32 path: source leaf (bit 31 set when the tree
// holds coincident points and the two leaves' bounding boxes touch, so that
// zero distances are possible outside the self pair) and the centre offset
// c_T - c_S rounded to FP32.
struct __align__(16) P2PEntry {
  int src;
  float dx, dy, dz;
};

// Tree-ordered FP64 point record (x, y, z, charge), 32-byte aligned for
// bulk copies.
struct __align__(32) dvec4 {
  double x, y, z, w;
};

// FP32 near-field source record with every component duplicated
// (x, x, y, y, z, z, q, q): 128-bit loads give packed f32x2 operands.
struct __align__(32) DupRec {
  float x0, x1, y0, y1, z0, z1, q0, q1;
};

// Double-float point record of the FP64DF near field: the position relative
// to its leaf's centre and the charge, each split as hi + lo.
struct __align__(32) DFRec {
  float xh, yh, zh, qh, xl, yl, zl, ql;
};

// Frame of a work entry's source leaf for the FP64DF near field: its centre
// (FP64).
struct __align__(32) SymFrame {
  double cx, cy, cz;
  float g, pad;
};

// One M2L work item: interactions b .. e - 1 of the list of target box g.
// Lists longer than kM2LItem are split into items of at most kM2LItem
// interactions whose sums go to rows prow, prow + 1, ... of a partial buffer
// and are added in item order afterwards (prow < 0: the item is the whole
// list and writes the target's local expansion itself).
struct __align__(8) M2LItem {
  int64_t b, e;
  int32_t g, prow;
};
constexpr int64_t kM2LItem = 8192;
// slots the symmetric near field's gather adds per chunk (one warp each)
constexpr int64_t kGatherChunk = 512;

// One work entry of the symmetric near field, read with one coalesced load:
// the source leaf's point range, the pair's slot (-1: one-sided), the FP32
// centre offset c_T - c_S and the coincidence threshold (< 0: no masking).
struct __align__(16) SymRec {
  int64_t start;
  int32_t count;
  int32_t slot;
  float dx, dy, dz, thr;
};

}  // namespace fmm

struct fmm_tree {
  fmm_params prm;
  int64_t n = 0;
  int L = 0;
  int s = 2;
  int64_t n_boxes = 0, n_leaves = 0;
  int64_t n_m2l = 0, n_p2p = 0, n_p2p_pairs = 0;
  int max_leaf = 0;          // largest leaf point count
  int min_leaf = 0;          // smallest target leaf point count
  int has_duplicates = 0;    // two distinct points share a position
  double build_ms = 0;
  size_t device_bytes = 0;
  double* level_avg_host = nullptr;  // L + 1

  // hierarchy (device)
  int32_t* perm = nullptr;       // n: tree position -> original index
  int64_t* box_start = nullptr;  // n_boxes
  int32_t* box_count = nullptr;  // n_boxes
  double* center = nullptr;      // 3 n_boxes
  double* radius = nullptr;      // n_boxes
  int64_t* m2l_off = nullptr;    // n_boxes + 1, CSR by target global box
  int32_t* m2l_src = nullptr;    // n_m2l
  int32_t* m2l_trg = nullptr;    // n_m2l
  int64_t n_m2l_items = 0;       // M2L work items (>= n_boxes)
  fmm::M2LItem* m2l_items = nullptr;  // longest first
  int64_t n_m2l_split = 0;       // targets whose list is split into several items
  int32_t* m2l_split_g = nullptr;     // those targets
  int64_t* m2l_split_row = nullptr;   // n_m2l_split + 1: their first partial row (CSR)
  double* m2l_partial = nullptr;      // partial rows (ncoef_pad doubles each; FP32 rows use the first half)
  int64_t m2l_partial_rows = 0;
  // symmetric near-field slot gather in chunks of at most kGatherChunk slots:
  // chunk c covers slots gch_r0[c] .. of leaf gch_leaf[c]; leaves with
  // several chunks (gmulti_leaf, their first chunk gch_off) add the chunks'
  // sums (gpart, stride rows of 8 bytes per point) in chunk order
  int64_t n_gchunks = 0;
  int32_t* gch_leaf = nullptr;
  int64_t* gch_r0 = nullptr;
  int64_t* gch_first = nullptr;       // n_leaves + 1: first chunk of each leaf
  int64_t n_gmulti = 0;
  int32_t* gmulti_leaf = nullptr;
  double* gpart = nullptr;            // n_gchunks x sym_stride
  int64_t* p2p_off = nullptr;    // n_leaves + 1, CSR by target leaf
  int32_t* p2p_src = nullptr;    // n_p2p
  fmm::P2PEntry* p2p32 = nullptr;  // n_p2p
  float* p2p_thr = nullptr;        // n_p2p: FP32 coincidence threshold on r^2
  // symmetric near field (one point set or a batch of them; symmetric.cu)
  int sym = 0;
  int64_t n_slots = 0;                // leaf pairs evaluated once for both sides
  int sym_stride = 0;                 // floats per slot (>= largest leaf)
  int32_t* sym_slot = nullptr;        // n_p2p: slot of a pair evaluated for both sides, else -1
  int64_t* sym_work_off = nullptr;    // n_leaves + 1
  int32_t* sym_work = nullptr;        // entries each leaf's warp evaluates, list order
  int64_t* sym_recv_off = nullptr;    // n_leaves + 1: the slots each leaf receives (contiguous)
  double* sym_partial = nullptr;      // n_slots x sym_stride floats (FP32C), doubles once
                                      // sym_partial_f64 is set (an FP64 precision was selected)
  int sym_partial_f64 = 0;
  // vector variants of the symmetric near field (FP32C field and backward):
  // (U, V) slot records, n_slots x sym_stride float4, and gather partials,
  // n_gchunks x sym_stride x 8 floats; made on the first such evaluation
  float* sym_partial4 = nullptr;
  float* gpart4 = nullptr;
  fmm::SymRec* sym_rec = nullptr;     // per work entry, in work-list order
  // FP64DF near field: per-point double-float records (coordinates set at
  // build, charges by every evaluation's gather) and the source frame of
  // every work entry
  fmm::DFRec* src_df = nullptr;       // n, tree order
  fmm::SymFrame* sym_frame = nullptr; // per work entry, in work-list order
  int32_t* leaf_order_sym = nullptr;  // n_leaves: heaviest symmetric work first
  int32_t* leaf_order = nullptr;   // n_leaves: target leaves, most work first
  int32_t* leaf_box = nullptr;     // n_leaves: global box id of each leaf
  int32_t* box_parent = nullptr;   // n_boxes: parent box id (-1 for a root)
  // M2M rounds (bottom-up): device lists of box ids with host offsets; the
  // children of a parent are consecutive
  int n_up = 0;
  int64_t* up_off_h = nullptr;     // n_up + 1
  int32_t* up_ids = nullptr;
  // L2L in direct form: per target leaf, its ancestors with a non-empty M2L
  // list (nearest first), CSR by leaf
  int64_t n_l2d = 0;
  int64_t* l2d_off = nullptr;      // n_leaves + 1
  int32_t* l2d_anc = nullptr;      // n_l2d ancestor boxes
  int n_trees = 1;                 // > 1 for a merged batch of trees
  int64_t* tree_point_off_h = nullptr;  // n_trees + 1 (merged batches)
  // Roles of points and leaves.  One point set: every point carries a charge
  // and is evaluated, every leaf is both a source and a target.  Separate
  // source and target hierarchies (two_trees): points 0 .. n_charges - 1 are
  // the charges, the rest the targets (output index perm[i] - out_base);
  // leaf_box / n_leaves are the target leaves, src_leaf_box / n_src_leaves
  // the source leaves; level_avg_host holds the source tree's L_src + 1
  // averages, then the target tree's L + 1.
  int two_trees = 0;
  int L_src = 0;
  int64_t n_charges = 0;
  int64_t out_base = 0;
  int64_t n_src_leaves = 0;
  int32_t* src_leaf_box = nullptr;  // == leaf_box unless two_trees

  // per-point and per-box constants
  float4* pos_local = nullptr;   // n: tree order, x - c_leaf (FP32), w = 0
  fmm::dvec4* pos64 = nullptr;   // n: tree order, x (FP64), w = 0
  float* inv_rho32 = nullptr;    // n_boxes: 1 / scaling radius (0 if radius 0)
  double* inv_rho64 = nullptr;

  // rotation / translation coefficients
  float* geo32 = nullptr;        // m2l_fields(p) x n_m2l
  float* geo_lo = nullptr;       // FP64DF: geo64 - geo32 rounded to FP32 (same layout), or null
  float2* m_df = nullptr;        // FP64DF: multipoles as double-float pairs, n_boxes x ncoef_pad(p)
  double* geo64 = nullptr;
  float* m2m32 = nullptr;        // edge_fields(p) x n_boxes (row = child id)
  double* m2m64 = nullptr;
  float* l2d32 = nullptr;         // edge_fields(p) x n_l2d (row = record)
  double* l2d64 = nullptr;

  // evaluation workspace
  float4* src32 = nullptr;       // n: (x_local, q) in tree order
  fmm::DupRec* src_dup = nullptr;  // n: duplicated FP32 near-field records
  fmm::dvec4* src64 = nullptr;   // n: (x, q) in tree order
  float* M32 = nullptr;          // n_boxes x ncoef_pad(p)
  float* Lam32 = nullptr;
  double* M64 = nullptr;
  double* Lam64 = nullptr;
  void* near_u = nullptr;        // n x 8 bytes: near-field potential sums
  void* near_f = nullptr;        // 3n x 8 bytes: near-field gradient sums
  // backward pass (one point set): records of the second charge vector and
  // its near-field potential (hi, lo) and field sums
  fmm::DupRec* src_dup2 = nullptr;
  float* near_u2 = nullptr;      // 2n
  float* near_f2 = nullptr;      // 3n
  double* q_stage = nullptr;     // n (host-buffer entry points, backward)
  double* u_stage = nullptr;     // n
  double* f_stage = nullptr;     // 3 n (backward)
  double* g_stage = nullptr;     // 3 n (backward)
  int* counters = nullptr;       // work counters, reset before each launch
  int* status = nullptr;         // latched kernel status bits
  int ws_external = 0;           // the evaluation workspace is the caller's (fmm_tree_set_workspace)
  int* m2m_ready = nullptr;      // n_boxes readiness flags of the one-launch M2M (NULL: one launch per round)
  // launch options (fmm_tree_set_option): stage order, M2M in one launch,
  // symmetric near field, cap on M2L blocks per SM (0: full occupancy)
  int opt_schedule = 1;
  int opt_m2m_one_launch = 1;
  int opt_near_sym = 1;
  int opt_m2l_blocks_per_sm = 0;
  long long wait_cycles = fmm::kDefaultWaitCycles;  // near-field tile wait limit

  // far-field stages run on a second, higher-priority stream forked from
  // and joined back into the caller's stream
  cudaStream_t far_stream = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;

  // per-stage timing (fmm_tree_profile) and launch accounting
  static constexpr int kProfCalls = 512;
  // per call and stage {begin, end}; one slot beyond the public stages holds
  // the second launch of a near field run in two parts (added to P2P)
  static constexpr int kProfSlots = FMM_NUM_STAGES + 1;
  static constexpr int kStageP2P2 = FMM_NUM_STAGES;
  cudaEvent_t* prof_ev = nullptr;      // kProfCalls x kProfSlots x {begin, end}
  mutable int prof_on = 0;
  mutable int prof_used = 0;
  mutable int prof_cur = -1;           // slot of the call being recorded
  mutable int64_t launches = 0;
};

namespace fmm {

// Begin (end = false) or end of stage s of the current evaluation call,
// recorded on the stream the stage runs on.
inline void stage_event(const fmm_tree* t, int s, bool end, cudaStream_t st) {
  if (!t->prof_on) return;
  if (s == FMM_STAGE_SORT && !end) {
    t->prof_cur = (t->prof_used < fmm_tree::kProfCalls) ? t->prof_used++ : -1;
  }
  if (t->prof_cur >= 0) cudaEventRecord(t->prof_ev[(t->prof_cur * fmm_tree::kProfSlots + s) * 2 + (end ? 1 : 0)], st);
}

// tree_build.cu
void build_tree(fmm_tree* t, const double* pos, cudaStream_t st);
// Separate source and target hierarchies (t->prm set on entry).
void build_tree2(fmm_tree* t, const double* src, int64_t n_src, const double* trg, int64_t n_trg, cudaStream_t st);
// symmetric.cu: symmetric near-field metadata of a one-point-set tree or batch
void build_symmetric(fmm_tree* t, cudaStream_t st);
// tree_build.cu: the direct L2L records of a tree with lists, geometry and
// parents in place
void build_l2l_direct(fmm_tree* t, cudaStream_t st);
// tree_build.cu: the FP64 data of a tree (FP64 rotation records, FP64
// expansions and point records, double-width near-field slots), made the
// first time a tree's precision is FMM_FP64 or FMM_FP64DF; synchronous
void ensure_fp64(fmm_tree* t, cudaStream_t st);
// tree_build.cu: the low parts of the rotation records and the double-float
// multipole buffer of the FP64DF far field, and (symmetric.cu,
// build_df_near) the double-float point records and per-entry source frames
// of its near field (once per tree)
void prepare_df_far(fmm_tree* t, cudaStream_t st);
void build_df_near(fmm_tree* t, cudaStream_t st);
// symmetric.cu: the slot buffers of the symmetric near field's vector
// variants (field and backward pass, FP32C; leaves of at most 128 points),
// made on the first evaluation that uses them unless the caller's workspace
// is attached; returns whether the tree has them.  Synchronous.
bool ensure_sym_vec(fmm_tree* t, cudaStream_t st);
// api.cu: releases every device array, stream and event of a tree
void free_tree(fmm_tree* t);
// merge.cu: a batch of trees as one tree-shaped object
void merge_trees(fmm_tree* const* in, int n, cudaStream_t st, fmm_tree* out);

// eval_f32.cu / eval_f64.cu: the evaluation pipelines.
//   q: device, original order; u / field: device outputs (nullable)
void eval_fp32(const fmm_tree* t, const double* q, double* u, double* field, cudaStream_t st);
void eval_fp64(const fmm_tree* t, const double* q, double* u, double* field, cudaStream_t st);
// FP32C backward of one point set: u of g (ug, nullable), fields of q and of
// g, caller's point order; one near-field sweep for both charge vectors.
void backward_fp32(const fmm_tree* t, const double* q, const double* g, double* ug, double* fq, double* fg,
                   cudaStream_t st);
// FP32C backward of one point set with the symmetric near field (vector slot
// buffers present, leaves of at most 128 points): dL/dq (grad_q) and dL/dx
// (grad_pos), both nullable, caller's point order.
void backward_sym_fp32(const fmm_tree* t, const double* q, const double* g, double* grad_q, double* grad_pos,
                       cudaStream_t st);
// Per-precision one-time set-up: constant tables for every order.
void init_tables_fp32();
void init_tables_fp64();

// Offset of degree n in the dense per-degree rotation tables.
__host__ __device__ constexpr int b_off(int n) {
  // sum_{j<n} (2j+1)^2 = n (4n^2 - 1) / 3
  return n * (4 * n * n - 1) / 3;
}

// sort.cu: perm = 0 .. n - 1 ordered by descending key (keys clamped to
// [0, 2^32)), equal keys in ascending index order; asynchronous on st.
void order_desc(const int64_t* key, int64_t n, int32_t* perm, cudaStream_t st);
// tree_build.cu: work orders of a tree whose lists are set (the M2L work
// items and leaf_order), on the device.
void build_work_orders(fmm_tree* t, cudaStream_t st);

// scan.cu: exclusive prefix sum of n int64 values (in place allowed), one
// launch; returns the total (synchronises the stream; FMM_ERR_TIMEOUT if a
// bounded wait of the look-back gave up).  The asynchronous form leaves the
// total in *total_dev and sets *err_dev (zeroed by the caller) on a timeout.
int64_t exclusive_scan(const int64_t* in, int64_t* out, int64_t n, cudaStream_t st);
void exclusive_scan_async(const int64_t* in, int64_t* out, int64_t n, int64_t* total_dev, int* err_dev,
                          cudaStream_t st);

// api.cu: every device allocation of the library goes through these two, so
// that the bytes it holds are known and can be capped
// (fmm_set_device_memory_limit): an allocation beyond the cap, or one that
// cudaMalloc refuses, throws Fail{FMM_ERR_OOM}.
void* tracked_malloc(size_t bytes);
void dev_free(void* p);

// Stream-ordered allocation for the duration of a build: while an AllocScope
// is alive on this thread, tracked_malloc takes memory from the library's
// pool on the scope's stream and dev_free returns it on that stream (no
// cudaMalloc, no implicit device synchronisation of cudaFree).  Pointers
// that outlive the scope (the tree's arrays) are freed later like any other.
inline thread_local cudaStream_t tl_alloc_stream = nullptr;
inline thread_local cudaMemPool_t tl_alloc_pool = nullptr;
// Returns the pool's unused memory to the device (outside a build).
void trim_pool();
struct AllocScope {
  cudaStream_t prev;
  cudaMemPool_t prev_pool;
  cudaMemPool_t pool;
  explicit AllocScope(cudaStream_t s);
  ~AllocScope();
};

template <class T>
T* dev_alloc(fmm_tree* t, size_t count) {
  if (count == 0) count = 1;
  T* p = static_cast<T*>(tracked_malloc(sizeof(T) * count));
  if (t) t->device_bytes += sizeof(T) * count;
  return p;
}

// Build-phase trace, on when the environment holds FMM_BUILD_TRACE=1: every
// trace_mark synchronises the build stream and prints the wall time since the
// previous mark to stderr (a diagnostic of where a build spends its time; the
// marks cost nothing when the trace is off).
struct BuildTrace {
  cudaStream_t st = nullptr;
  std::chrono::steady_clock::time_point t0;
  explicit BuildTrace(cudaStream_t s) : st(s), t0(std::chrono::steady_clock::now()) {}
  void mark(const char* what) {
    cudaStreamSynchronize(st);
    const auto t1 = std::chrono::steady_clock::now();
    fprintf(stderr, "fmm build: %-28s %8.3f ms\n", what, std::chrono::duration<double, std::milli>(t1 - t0).count());
    t0 = t1;
  }
};
inline thread_local BuildTrace* tl_trace = nullptr;
inline bool build_trace_enabled() {
  const char* e = std::getenv("FMM_BUILD_TRACE");
  return e && e[0] == '1';
}
inline void trace_mark(const char* what) {
  if (tl_trace) tl_trace->mark(what);
}
// Installs a trace for the current thread's build when the environment asks
// for one, and removes it when the build returns.
struct TraceScope {
  BuildTrace tr;
  explicit TraceScope(cudaStream_t s) : tr(s) {
    if (build_trace_enabled()) tl_trace = &tr;
  }
  ~TraceScope() { tl_trace = nullptr; }
};

template <class T>
T* scratch_alloc(size_t count) {
  return dev_alloc<T>(nullptr, count);
}

inline int grid_for(int64_t n, int block, int cap = 152 * 64) {
  int64_t g = (n + block - 1) / block;
  if (g < 1) g = 1;
  if (g > cap) g = cap;
  return (int)g;
}

}  // namespace fmm
