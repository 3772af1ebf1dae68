/*
 * fmm.h - C ABI of the GB300 (sm_103a) evaluator for the adaptive
 * point-charge Laplace Fast Multipole Method of Kraft, Bruckner, Suess and
 * Abert, "jaxFMM: An Adaptive, GPU-Parallel Implementation of the Fast
 * Multipole Method in JAX" (arXiv 2511.15269).
 *
 * What is computed (Sec. II, Eq. 1-3): for N point charges q_i at r_i,
 *     u_i = -1/(4 pi) * sum_{j != i} q_j / |r_i - r_j|          (potential)
 *     E_i = -grad u (r_i)                                       (field)
 * approximated by an FMM of expansion order p over a median-split 2^s-tree
 * (Sec. II.A) with level-marching cross-level interaction lists built from
 * the well-separation criterion R + theta r <= theta d (Eq. 4, Sec. II.B).
 * Pairs at zero distance (the self term and coincident points) contribute
 * nothing.
 *
 * Conventions shared by every entry point:
 *  - Data pointers are DEVICE pointers (cudaMalloc'd or equivalent) owned by
 *    the caller, contiguous, unless a function says "host".  Positions are
 *    N x 3 row-major doubles (x, y, z per point); charges, potentials and
 *    gradients with respect to charges are N doubles; fields and gradients
 *    with respect to positions are N x 3 doubles.  Outputs come back in the
 *    caller's point order.
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *    stream).  Evaluation calls only enqueue work on it and return; errors
 *    that kernels detect (a bounded wait that gave up) are latched in the
 *    tree and returned by fmm_tree_status().
 *  - Every call returns an fmm_status; on failure fmm_last_error() gives a
 *    thread-local message.  Nothing throws or aborts.
 *  - A tree owns the device workspace its evaluations use (allocated once
 *    by fmm_build_tree) and a second, higher-priority CUDA stream: an
 *    evaluation forks latency- or memory-bound stages onto it (P2M and M2M
 *    beside the near field, the near-field slot gather beside M2L) from the
 *    caller's stream and joins them back before the next dependent stage, so
 *    the caller sees ordinary stream-ordered semantics (stream capture
 *    included).  Evaluations of one tree must be ordered on one stream; two
 *    evaluations of the same tree in flight at once race.  Distinct trees are
 *    independent.
 */
#ifndef GB300_FMM_H
#define GB300_FMM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  FMM_OK = 0,
  FMM_ERR_INVALID_ARG = 1, /* bad size, parameter, null pointer, NaN/Inf position */
  FMM_ERR_CUDA = 2,        /* a CUDA runtime call failed (message has the CUDA error) */
  FMM_ERR_OOM = 3,         /* device allocation failed */
  FMM_ERR_CAPACITY = 4,    /* a fixed-capacity buffer overflowed (batched calls) */
  FMM_ERR_TIMEOUT = 5      /* a bounded device-side wait gave up */
} fmm_status;

enum {
  FMM_FP64 = 0,  /* every stage in FP64                                        */
  FMM_FP32C = 1, /* P2M/M2M/M2L/L2L/L2P/P2P in FP32 on box-radius-scaled
                    coefficients, compensated (two-sum) accumulation of leaf and
                    local sums; rotation coefficients generated in FP64; final
                    near + far combination in FP64                             */
  FMM_FP64DF = 2  /* FP64 accuracy: as FMM_FP64, except that the potential
                    near field and (for p <= 8) the M2L of a tree of one point
                    set (or a batch of them) run in double-float arithmetic (unevaluated
                    sums of two FP32 values, error-free transformations) on the
                    FP32 pipes, with results within a few 1e-14 of FP64;
                    fields, backward and two-hierarchy trees use FP64          */
};

enum {
  FMM_TIE_TARGET = 1, /* equal average radii advance the target level (the
                         same-vs-cross table of Sec. II.B) instead of the source
                         level (the text of Sec. II.B, the default)            */
  FMM_SAME_LEVEL = 2, /* same-level lists (Sec. II.B, steps 1-3): source and
                         target descend together and only boxes of one level
                         are compared; no cross-level M2L pairs.  Overrides
                         FMM_TIE_TARGET.  More M2L work than the default
                         level march (the same-vs-cross table of Sec. II.B);
                         kept for comparison                                   */
  FMM_POS_SOA = 4     /* positions passed to the build calls are three arrays
                         of n doubles (all x, then all y, then all z) instead
                         of n rows of (x, y, z); the hierarchy is the same    */
};

#define FMM_MAX_P 10 /* largest supported expansion order */

/* Parameters of the hierarchy and the expansion (Sec. II.A-II.D, Listing 1). */
typedef struct {
  int p;          /* expansion order, 1..FMM_MAX_P                              */
  int leaf_size;  /* N_max: levels are added until boxes hold <= N_max points;
                     must be >= 2^splits                                         */
  int splits;     /* s: bisections per level, 2^s children per box, 1..3        */
  double theta;   /* well-separation parameter of Eq. 4, 0 < theta < 1          */
  int precision;  /* FMM_FP64, FMM_FP32C or FMM_FP64DF, used by evaluations     */
  int flags;      /* 0 or a combination of FMM_TIE_TARGET, FMM_SAME_LEVEL,
                     FMM_POS_SOA                                                 */
} fmm_params;

typedef struct fmm_tree fmm_tree;

typedef struct {
  int64_t n;             /* points (sources + targets for two hierarchies)      */
  int levels;            /* L: the leaf level; the root is level 0 (the target
                            tree's for two hierarchies)                         */
  int p, splits, leaf_size, precision;
  double theta;
  int64_t n_boxes;       /* sum over levels of 2^(s l)                          */
  int64_t n_leaves;      /* 2^(s L) (target leaves for two hierarchies)         */
  int64_t n_m2l;         /* multipole-to-local interactions, all levels         */
  int64_t n_p2p;         /* near-field leaf pairs (self pairs included)         */
  int64_t n_p2p_pairs;   /* near-field point pairs: sum over leaf pairs |S||T|  */
  size_t device_bytes;   /* device memory owned by the tree                     */
  double build_ms;       /* wall time of fmm_build_tree                         */
  int64_t kernel_launches; /* kernels this library launched for evaluations of
                              this tree so far                                  */
  int n_trees;           /* 1, or the number of trees of a merged batch          */
  int levels_src;        /* source tree depth (== levels for one point set)      */
  int64_t n_sources;     /* charges (== n for one point set)                    */
  int64_t n_targets;     /* evaluated points (== n for one point set)           */
  int64_t n_src_leaves;  /* source leaves (== n_leaves for one point set)       */
} fmm_stats;

/* Evaluation stages in launch order, named after the stages of Sec. III.A:
 * sort (charges into tree order), evdir (P2P), mpls (P2M), M2M, M2L, L2L,
 * evloc (L2P, near + far combination and inverse sort). */
enum {
  FMM_STAGE_SORT = 0,
  FMM_STAGE_P2P = 1,
  FMM_STAGE_P2M = 2,
  FMM_STAGE_M2M = 3,
  FMM_STAGE_M2L = 4,
  FMM_STAGE_L2L = 5,
  FMM_STAGE_L2P = 6,
  FMM_NUM_STAGES = 7
};

/* Measured arithmetic throughput of the current device, the denominators of
 * the compute rooflines of the near field (FP32 FMA pipe and MUFU rsqrt) and
 * of the FP64 path: out[0] FP32 FMA TFLOP/s (fma.rn.f32), out[1] packed
 * FP32x2 FMA TFLOP/s (fma.rn.f32x2, 4 flops per lane), out[2] FP64 FMA
 * TFLOP/s, out[3] rsqrt.approx.f32 Gop/s.  out: host, 4 doubles.  Runs a
 * few short probe kernels on `stream` (tens of ms) and synchronises it; the
 * paper has no counterpart (it is a measurement aid). */
int fmm_device_peaks(double* out, void* stream);

/* Thread-local description of the last failure on this thread. */
const char* fmm_last_error(void);

/* Caps the device memory the library holds in total (every tree, batch and
 * build scratch of the process; 0 removes the cap, the default).  A device
 * allocation that would exceed the cap fails as if cudaMalloc had refused
 * it: the call returns FMM_ERR_OOM and leaves no tree behind.  Memory
 * already held is not released.  The paper has no counterpart (a budget for
 * processes that share a GPU with other allocators).  Always FMM_OK. */
int fmm_set_device_memory_limit(size_t bytes);

/* Device memory the library holds right now, in bytes (host pointer). */
int fmm_device_memory_in_use(size_t* bytes);

/* Device memory the library keeps reserved but unused after a build and
 * after a tree is freed (its stream-ordered pool), so that the next build
 * reuses it without mapping new memory; the rest goes back to the driver.
 * Default 2 GiB; 0 returns all of it at those points.  With a cap set
 * (fmm_set_device_memory_limit) at most the headroom under the cap is kept.
 * Kept memory is not counted by fmm_device_memory_in_use.  Trims the
 * current device's pool to the new size (after a device synchronisation).
 * The paper has no counterpart (an allocator setting).  Always FMM_OK. */
int fmm_set_pool_retention(size_t bytes);

/* Number of levels L for n points (Sec. II.A step 4): the smallest l with
 * ceil(n / 2^(splits l)) <= leaf_size.  Returns -1 on invalid arguments. */
int fmm_num_levels(int64_t n, int leaf_size, int splits);

/* Builds the hierarchy of Sec. II.A-II.B on the device: median-split tree
 * (Listing 2: longest-extent axis, ties to the lowest axis; ceil(n/2) points
 * to the lower child ordered by (coordinate, original index); leaf points in
 * ascending original index), box centres (bounding-box midpoints) and radii
 * (half diagonals) in FP64, level-march M2L lists and near-field lists, and
 * the rotation coefficients of every M2M and M2L translation and of the
 * L2L translations from each leaf's ancestors with M2L sums straight to the
 * leaf (the level-by-level L2L chain applied in one step; FP64, also stored
 * rounded to FP32).  -0.0 coordinates are treated as +0.0.
 *   pos     device, n x 3 doubles (x, y, z per point; with FMM_POS_SOA in
 *           params->flags: x[0..n), y[0..n), z[0..n)), read only during the
 *           call
 *   n       >= 1 points (< 2^31)
 *   params  host pointer, copied
 *   stream  work is enqueued on it; the call synchronises it before returning
 *   out     receives the new tree; free with fmm_tree_free
 * Errors: FMM_ERR_INVALID_ARG (n < 1, bad params, non-finite coordinate),
 * FMM_ERR_OOM, FMM_ERR_CUDA.  On error *out is set to NULL. */
int fmm_build_tree(const double* pos, int64_t n, const fmm_params* params, void* stream,
                   fmm_tree** out);

/* Separate source and target hierarchies (Sec. II.B, final part): the
 * potential of charges at n_src source positions evaluated at n_trg other
 * positions.  Two median-split trees are built with the same leaf_size,
 * splits and theta (their depths may differ) and compared by the level march
 * of Sec. II.B (ties as in fmm_params.flags; FMM_SAME_LEVEL is rejected
 * because same-level lists need equal depths).  src_pos, trg_pos: DEVICE,
 * 3 n_src / 3 n_trg doubles, x y z per point.  The resulting tree is used
 * with fmm_eval_potential / fmm_eval_field / fmm_eval_potential_host: q has
 * n_src entries (source order), u n_trg and field 3 n_trg (target order).  A
 * target at exactly the position of a source does not see that charge (zero
 * distances contribute nothing).  In fmm_tree_export the source boxes come
 * first (ids 0 .. NB_s - 1; box b of source level l at (2^(s l) - 1)/(2^s - 1)
 * + b), the target boxes follow (id NB_s + the same formula); perm maps
 * source tree positions 0 .. n_src - 1 to source indices and target tree
 * positions n_src .. to n_src + target index; level_avg_radius holds
 * levels_src + 1 source averages, then levels + 1 target averages;
 * near-field pairs are (target leaf, source leaf).  fmm_backward,
 * fmm_tree_merge and fmm_eval_potential_static reject such trees (the
 * transposed problem is a tree with the roles swapped).  Errors as for
 * fmm_build_tree. */
int fmm_build_tree2(const double* src_pos, int64_t n_src, const double* trg_pos,
                    int64_t n_trg, const fmm_params* params, void* stream, fmm_tree** out);

/* Releases a tree and its device memory (synchronises the device first).
 * NULL is accepted. */
void fmm_tree_free(fmm_tree* tree);

/* Batch of independent charge sets (many trees, uneven sizes) evaluated
 * together: builds one tree-shaped object holding copies of n_trees trees
 * (same p and splits; leaf sizes may differ), whose points are the
 * concatenation of the trees' points in the given order.  Every evaluation
 * entry point accepts it, with q, u, field, gradients of the concatenated
 * length; each stage then runs as one launch over the whole batch (M2M: one
 * per round; a whole
 * evaluation can be captured as one CUDA graph).  The input trees stay valid
 * and independent; free the batch with fmm_tree_free.  Synchronous.
 * Errors: FMM_ERR_INVALID_ARG (mismatched trees, nested batches), FMM_ERR_OOM,
 * FMM_ERR_CUDA. */
int fmm_tree_merge(fmm_tree* const* trees, int n_trees, void* stream, fmm_tree** out);

/* Point offsets of the trees of a batch: n_trees + 1 int64 (host); a plain
 * tree gives {0, n}. */
int fmm_tree_point_offsets(const fmm_tree* tree, int64_t* offsets);

/* Selects the precision of later evaluation calls (FMM_FP64, FMM_FP32C or
 * FMM_FP64DF).  A tree keeps only the data of the precisions selected so
 * far: the first selection of FMM_FP64 or FMM_FP64DF (at build or here)
 * computes the FP64 rotation records of every M2L, M2M and direct L2L
 * translation (4 m2l_fields(p) = 12 + 16 p more bytes per M2L interaction
 * than FP32C alone), FP64 expansion and point buffers and double-width
 * near-field slots; the first selection of FMM_FP64DF for a tree of one point
 * set (or a tree built or merged with it) also makes the low parts of the M2L
 * rotation records, a double-float multipole buffer and the double-float
 * near-field records.  These calls allocate and run synchronously on the
 * default stream.  Errors: FMM_ERR_INVALID_ARG, FMM_ERR_OOM, FMM_ERR_CUDA. */
int fmm_tree_set_precision(fmm_tree* tree, int precision);

/* Fills *stats (host pointer). */
int fmm_tree_stats(const fmm_tree* tree, fmm_stats* stats);

/* Synchronises `stream`, then returns and clears the status latched by the
 * kernels of earlier evaluations of this tree (FMM_OK or FMM_ERR_TIMEOUT). */
int fmm_tree_status(fmm_tree* tree, void* stream);

/* Launch options of later evaluations of a tree: the launch shapes the
 * autotuner searches (the paper tunes N_max by hand, Sec. III.A; these do
 * not change results beyond rounding, except FMM_OPT_NEAR_SYMMETRIC which
 * changes the summation order of the near field).
 *   FMM_OPT_SCHEDULE        0: every stage on the caller's stream in order;
 *                           1 (default): P2M and M2M on the tree's second
 *                           stream beside the near field, the near-field slot
 *                           gather beside M2L and L2L; 2: M2L and L2L beside
 *                           the near field; 3: the near field in two launches,
 *                           P2M and M2M beside the first, L2L beside the second
 *   FMM_OPT_M2M_ONE_LAUNCH  1 (default): every M2M round in one launch whose
 *                           warps wait (bounded) for their children's sums;
 *                           0: one launch per round
 *   FMM_OPT_NEAR_SYMMETRIC  1 (default): pairs listed both ways evaluated once
 *                           (potentials of one point set); 0: one-sided
 *   FMM_OPT_M2L_BLOCKS_PER_SM  cap on resident M2L blocks per SM (0: none)
 * Errors: FMM_ERR_INVALID_ARG (NULL tree, unknown option, value out of
 * range). */
enum {
  FMM_OPT_SCHEDULE = 1,
  FMM_OPT_M2M_ONE_LAUNCH = 2,
  FMM_OPT_NEAR_SYMMETRIC = 3,
  FMM_OPT_M2L_BLOCKS_PER_SM = 4
};
int fmm_tree_set_option(fmm_tree* tree, int option, int value);

/* Limit, in GPU clock cycles, of each bounded device-side wait: a near-field
 * warp's wait for a staged source tile (a bulk copy completing on a
 * shared-memory barrier; Sec. II.B near field) and the one-launch M2M's wait
 * for a child's sum.  A warp whose wait runs out latches FMM_ERR_TIMEOUT in the
 * tree (read by fmm_tree_status), lets its copies in flight land and stops;
 * that evaluation's results are then incomplete.  Default about 2e9 cycles
 * (about a second); 0 gives up before the first poll, which exercises the
 * timeout path without any fault.  Applies to later evaluations of this
 * tree.  Errors: FMM_ERR_INVALID_ARG (NULL tree, negative cycles). */
int fmm_tree_set_wait_limit(fmm_tree* tree, int64_t cycles);

/* Copies the hierarchy to HOST arrays for inspection; every pointer may be
 * NULL.  Sizes: perm n (tree position -> original index); box_start,
 * box_count, radius n_boxes; center 3 n_boxes; level_avg_radius levels+1;
 * m2l_trg, m2l_src n_m2l (global box ids, box b of level l has id
 * (2^(s l) - 1)/(2^s - 1) + b, sorted by (target, source)); p2p_trg, p2p_src
 * n_p2p (leaf indices, sorted by (target, source)).  Synchronous. */
int fmm_tree_export(const fmm_tree* tree, int32_t* perm, int64_t* box_start,
                    int64_t* box_count, double* center, double* radius,
                    double* level_avg_radius, int32_t* m2l_trg, int32_t* m2l_src,
                    int32_t* p2p_trg, int32_t* p2p_src);

/* Per-stage device timing.  enable = 1 clears the record and starts
 * recording CUDA events at the start and end of every stage of the next
 * evaluation calls of this tree (on the stream each stage runs on, up to 512
 * calls); enable = 0 stops.
 * fmm_tree_stage_times synchronises the recorded events and writes the summed
 * milliseconds per stage (FMM_NUM_STAGES doubles, host) and the number of
 * recorded calls. */
int fmm_tree_profile(fmm_tree* tree, int enable);
int fmm_tree_stage_times(const fmm_tree* tree, double* ms, int64_t* calls);

/* Potential u (n doubles) of charges q (n doubles) at the tree's points:
 * sort into tree order, P2M, M2M, M2L, L2L, L2P + P2P, inverse sort
 * (the stages of Sec. III.A). */
int fmm_eval_potential(const fmm_tree* tree, const double* q, double* u, void* stream);

/* Field E = -grad u (n x 3 doubles) and, if u != NULL, the potential;
 * L2P uses the gradient of the regular basis (App. A.3). */
int fmm_eval_field(const fmm_tree* tree, const double* q, double* u, double* field,
                   void* stream);

/* Batched charge sets (the batch form of the evaluation; the paper
 * evaluates one charge set per call, Sec. III.A): the potentials of n_sets
 * independent charge sets in one evaluation of a batch tree made by
 * fmm_tree_merge from n_sets trees.  q_sets and u_sets are HOST arrays of
 * n_sets DEVICE pointers; set k has offsets[k + 1] - offsets[k] points
 * (fmm_tree_point_offsets), in its own tree's point order.  The charges are
 * gathered into the batch's order and the potentials scattered back by
 * kernels that take the pointers as launch arguments (no host-to-device
 * copy, so the call can be captured in a CUDA graph).  n_sets must equal
 * the batch's tree count (1 for a plain tree).  Errors:
 * FMM_ERR_INVALID_ARG, FMM_ERR_CUDA. */
int fmm_eval_batched(const fmm_tree* batch, int n_sets, const double* const* q_sets, double* const* u_sets,
                     void* stream);

/* Evaluation workspace (Sec. III.A evaluations reuse one hierarchy; the
 * per-call scratch is separate from it): the buffers every evaluation of the
 * tree overwrites (tree-ordered point records, near-field sums and slots,
 * expansions, staging buffers, work counters) for the precisions selected so
 * far.  fmm_tree_workspace_bytes gives their size (host *bytes); a caller
 * that keeps device memory in its own allocator passes a buffer of at least
 * that size (device, 256-byte aligned) to fmm_tree_set_workspace, and the
 * tree releases its own buffers and uses the caller's for every later
 * evaluation; the caller keeps it valid until the tree is freed or another
 * workspace (or NULL: the tree's own again) is set.  Selecting a precision
 * that needs more workspace (FMM_FP64 or FMM_FP64DF for the first time)
 * requires the caller's workspace to be detached first.  The call
 * synchronises the device.  Errors: FMM_ERR_INVALID_ARG (NULL tree,
 * misaligned buffer), FMM_ERR_CAPACITY (buffer too small), FMM_ERR_OOM,
 * FMM_ERR_CUDA. */
int fmm_tree_workspace_bytes(const fmm_tree* tree, size_t* bytes);
int fmm_tree_set_workspace(fmm_tree* tree, void* workspace, size_t ws_bytes);

/* Same as fmm_eval_potential with HOST buffers: copies q to the device,
 * evaluates, copies u back and synchronises `stream`.  Pinned host memory
 * gives the fastest copies. */
int fmm_eval_potential_host(const fmm_tree* tree, const double* q_host, double* u_host,
                            void* stream);

/* Allocation-free variant of fmm_eval_potential (the paper has no
 * counterpart; it serves callers that may not allocate device memory at
 * evaluation time: code whose device memory budget belongs to another
 * allocator, latency-critical loops that cannot absorb cudaMalloc's implicit
 * synchronisation, plug-ins allowed to allocate only at start-up).
 * Same inputs and outputs as fmm_eval_potential; the per-call scratch (point
 * records, near-field sums, expansions, work counters) lives in one
 * file-scope device array of FMM_STATIC_SCRATCH_BYTES that every GPU loading
 * the library holds until the process exits.  It calls no
 * cudaMalloc/cudaFree and no allocating library routine.
 *   Results: the near field runs the one-sided kernel (every target leaf
 *   against its whole list; the symmetric kernel's per-pair slots are tree
 *   workspace), so FP32C results differ from fmm_eval_potential by rounding
 *   (within the FP32C tolerance), and a tree set to FMM_FP64DF is evaluated
 *   in plain FMM_FP64 (within about 1e-13 relative of the double-float
 *   results).  FMM_FP64 results equal fmm_eval_potential's up to the
 *   summation order of the near field.
 *   Limits: tree->n <= FMM_STATIC_MAX_POINTS and n_boxes <=
 *   FMM_STATIC_MAX_BOXES, else FMM_ERR_CAPACITY with a message.
 *   The first call on a device looks up the array's device address with
 *   that device current and keeps it for later calls; make that first call
 *   before any stream capture.  The kept address does not survive
 *   cudaDeviceReset (do not call this entry point after a reset).
 *   All calls share the array and it keeps the last call's contents (the
 *   work counters are cleared by each call before use): calls that overlap
 *   on the GPU, on any streams or trees, race and must be ordered. */
#define FMM_STATIC_MAX_POINTS 65536
#define FMM_STATIC_MAX_BOXES 5461
#define FMM_STATIC_SCRATCH_BYTES 16602368
int fmm_eval_potential_static(const fmm_tree* tree, const double* q, double* u, void* stream);

/* Vector-Jacobian product of u = K q at the tree's fixed geometry, for a loss
 * L(u) with grad_u = dL/du (n doubles):
 *     grad_q   = K grad_u                               (K is symmetric)
 *     grad_pos = grad_u_k * grad u(r_k) + q_k * grad v(r_k),  v = K grad_u
 * grad_q (n) and grad_pos (n x 3) may each be NULL.  The tree is held fixed
 * (gradients are taken with the hierarchy of the current positions).  With
 * FMM_FP32C and leaves of at most 128 points the near field of q and grad_u
 * is swept once (shared distances and 1/r), followed by the far field of
 * each; otherwise two field evaluations. */
int fmm_backward(const fmm_tree* tree, const double* q, const double* grad_u,
                 double* grad_q, double* grad_pos, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* GB300_FMM_H */
