/*
 * CPU FP64 oracle for the adaptive point-charge Laplace FMM of
 * Kraft, Bruckner, Suess, Abert, "jaxFMM: An Adaptive, GPU-Parallel
 * Implementation of the Fast Multipole Method in JAX" (arXiv 2511.15269).
 *
 * TEST INFRASTRUCTURE ONLY.  This library exists to check the CUDA path.
 * Only the test suite, the smoke check and the CPU-baseline leg of the
 * benchmark may load it; the product path never calls it and shares no
 * code, header, table or constant with it.
 *
 * Plain, slow, obviously correct: every routine follows the paper's
 * formula or step list, in FP64, with no blocking or fusion.  Floating
 * point expressions that decide integer results (tree, lists) are written
 * operation by operation and the library is compiled with
 * -ffp-contract=off so that no multiply-add is fused.
 *
 * Coefficient storage: real coefficient (n, m), 0 <= n <= p, -n <= m <= n,
 * lives at index n*n + n + m; an expansion of order p holds (p+1)^2 reals.
 */
#ifndef FMM_ORACLE_H
#define FMM_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- basis functions (App. A) ---- */
void orc_rhat(int p, double x, double y, double z, double* R);          /* App. A.1 */
void orc_shat(int p, double x, double y, double z, double* S);          /* App. A.2 */
void orc_grad_rhat(int p, double x, double y, double z, double* R, double* G); /* App. A.3, G[3*idx+c] */

/* ---- rotations and axial transforms (App. B) ---- */
void orc_wigner_d(int p, double beta, double* d);  /* d[(n*(2p+1)+(m+p))*(2p+1)+(k+p)] = d^n_{m,k}(beta) */
void orc_rotate_azimuthal(int p, int local, double dphi, const double* in, double* out); /* App. B.1 */
void orc_rotate_polar(int p, int local, double dtheta, const double* in, double* out);   /* App. B.2 */
void orc_axial_m2m(int p, double r, const double* in, double* out);   /* App. B.3 */
void orc_axial_m2l(int p, double r, const double* in, double* out);   /* App. B.3 */
void orc_axial_l2l(int p, double r, const double* in, double* out);   /* App. B.3 */

/* ---- complete operators between arbitrary centres; they ADD into out ---- */
void orc_p2m(int p, const double* pts, const double* q, int64_t n, const double c[3], double* out);
void orc_p2l(int p, const double* pts, const double* q, int64_t n, const double c[3], double* out);
void orc_m2m(int p, const double* C, const double c_old[3], const double c_new[3], double* out);
void orc_m2l(int p, const double* C, const double c_src[3], const double c_trg[3], double* out);
void orc_l2l(int p, const double* D, const double c_old[3], const double c_new[3], double* out);
/* potential sum without the -1/(4 pi) factor (the contraction of Sec. II.C) */
double orc_l2p(int p, const double* D, const double c[3], const double x[3], double* grad /*nullable, 3*/);
double orc_m2p(int p, const double* C, const double c[3], const double x[3]);

/* ---- hierarchy (Sec. II.A, II.B) ---- */
int orc_num_levels(int64_t n, int leaf_size, int s);
typedef struct orc_tree orc_tree;
/* flags bit 0 (tie target): equal average radii advance the target level
 * instead of the source level (text of Sec. II.B); bit 1 (same level): the
 * same-level lists of Sec. II.B steps 1-3 instead of level marching. */
orc_tree* orc_tree_build(const double* pos, int64_t n, int leaf_size, int s,
                         double theta, int flags);
void orc_tree_free(orc_tree* t);
/* info[0]=L, [1]=n_boxes, [2]=n_m2l, [3]=n_p2p, [4]=n_leaves */
void orc_tree_info(const orc_tree* t, int64_t* info);
void orc_tree_export(const orc_tree* t, int32_t* perm, int64_t* box_start,
                     int64_t* box_count, double* center, double* radius,
                     double* level_avg_radius);
void orc_tree_export_lists(const orc_tree* t, int32_t* m2l_trg, int32_t* m2l_src,
                           int32_t* p2p_trg, int32_t* p2p_src);

/* Separate source and target hierarchies (Sec. II.B, final part): two trees
 * with the same leaf_size, s and theta, lists by the level march between
 * them (flags bit 0: tie target; same-level lists are not offered).  M2L
 * pairs use combined ids (source boxes first, target box g at n_boxes_src +
 * g); near-field pairs are (target leaf, source leaf).  The two trees are
 * exported with orc_tree_export on orc_tree2_source / orc_tree2_target. */
typedef struct orc_tree2 orc_tree2;
orc_tree2* orc_tree2_build(const double* src_pos, int64_t n_src, const double* trg_pos,
                           int64_t n_trg, int leaf_size, int s, double theta, int flags);
void orc_tree2_free(orc_tree2* t2);
const orc_tree* orc_tree2_source(const orc_tree2* t2);
const orc_tree* orc_tree2_target(const orc_tree2* t2);
/* info[0]=n_m2l, [1]=n_p2p */
void orc_tree2_info(const orc_tree2* t2, int64_t* info);
void orc_tree2_export_lists(const orc_tree2* t2, int32_t* m2l_trg, int32_t* m2l_src,
                            int32_t* p2p_trg, int32_t* p2p_src);

/* ---- evaluation (Sec. II, Eq. 2-3, stages of Sec. III.A) ---- */
/* u[i] = -1/(4 pi) sum_{j != i} q_j / |r_i - r_j|, field = -grad u.
 * targets == NULL: all points; else only the listed original indices,
 * written to u[k], field[3k..3k+2] for k = 0..n_targets-1. */
void orc_fmm_eval(const orc_tree* t, int p, const double* q, const int64_t* targets,
                  int64_t n_targets, double* u, double* field);
/* As orc_fmm_eval, also reporting the stage wall times in seconds:
 * timing[0] sort and target bookkeeping, [1] P2M of every leaf, [2] M2M of
 * every box, [3] M2L into the boxes that feed the evaluated points, [4] L2L
 * into those boxes, [5] L2P + P2P at the evaluated points; and the work of
 * the restricted stages: [6] M2L interactions done, [7] L2L translations
 * done, [8] points evaluated.  (Measurement aid of the CPU baseline.) */
void orc_fmm_eval_timed(const orc_tree* t, int p, const double* q, const int64_t* targets,
                        int64_t n_targets, double* u, double* field, double* timing);
/* Sets the number of OpenMP threads of later calls (no effect without OpenMP). */
void orc_set_num_threads(int n);
void orc_direct(const double* pos, const double* q, int64_t n, const int64_t* targets,
                int64_t n_targets, double* u, double* field);
/* Potential and field of the charges q at src_pos evaluated at n_trg target
 * positions (target order); zero distances contribute nothing. */
void orc_fmm2_eval(const orc_tree2* t2, int p, const double* q, double* u, double* field);
void orc_direct2(const double* src_pos, const double* q, int64_t n_src, const double* trg_pos,
                 int64_t n_trg, double* u, double* field);
/* vector-Jacobian product of u = K q at a fixed geometry:
 * dq = K g,  dpos_k = g_k grad u(r_k) + q_k grad v(r_k) with v = K g. */
void orc_direct_vjp(const double* pos, const double* q, const double* g, int64_t n,
                    double* dq, double* dpos);
int orc_num_threads(void);

#ifdef __cplusplus
}
#endif
#endif
