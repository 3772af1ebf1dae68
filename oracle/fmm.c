/*
 * Oracle: FMM evaluation stages and the direct sum.  TEST INFRASTRUCTURE ONLY
 * (see fmm_oracle.h).
 *
 * The evaluation runs the stages in the paper's order (Sec. III.A stage
 * list): sort charges into tree order, leaf multipoles (P2M), upward M2M,
 * M2L over the whole interaction list, downward L2L, local evaluation (L2P)
 * and the direct near field (P2P), then the inverse sort.  The potential is
 * u_i = -1/(4 pi) sum_{j != i} q_j / |r_i - r_j| (Eq. 1-3); pairs at zero
 * distance contribute nothing (the self term, and coincident points).  The
 * field is -grad u.
 */
#define _POSIX_C_SOURCE 199309L
#include "fmm_oracle.h"
#include <math.h>
#include <stdlib.h>
#include <string.h>
#include <time.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* accessors defined in tree.c */
const int32_t* orc__perm(const orc_tree* t);
const double* orc__pos_tree(const orc_tree* t);
const int64_t* orc__box_start(const orc_tree* t);
const int64_t* orc__box_count(const orc_tree* t);
const double* orc__center(const orc_tree* t);
int orc__levels(const orc_tree* t);
int orc__splits(const orc_tree* t);
int64_t orc__n(const orc_tree* t);
int64_t orc__n_boxes(const orc_tree* t);
int64_t orc__n_m2l(const orc_tree* t);
const int32_t* orc__m2l_trg(const orc_tree* t);
const int32_t* orc__m2l_src(const orc_tree* t);
int64_t orc__n_p2p(const orc_tree* t);
const int32_t* orc__p2p_trg(const orc_tree* t);
const int32_t* orc__p2p_src(const orc_tree* t);
int64_t orc2__n_m2l(const orc_tree2* t2);
const int32_t* orc2__m2l_trg(const orc_tree2* t2);
const int32_t* orc2__m2l_src(const orc_tree2* t2);
int64_t orc2__n_p2p(const orc_tree2* t2);
const int32_t* orc2__p2p_trg(const orc_tree2* t2);
const int32_t* orc2__p2p_src(const orc_tree2* t2);

static const double FOUR_PI = 12.566370614359172953850573533118;

int orc_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

static int64_t level_off(int l, int s) {
  int64_t off = 0;
  for (int i = 0; i < l; i++) off += (int64_t)1 << (s * i);
  return off;
}

static int64_t first_ge(const int32_t* a, int64_t n, int32_t v) {
  int64_t lo = 0, hi = n;
  while (lo < hi) {
    int64_t mid = (lo + hi) / 2;
    if (a[mid] < v) lo = mid + 1;
    else hi = mid;
  }
  return lo;
}

/* Wall clock in seconds (stage timing of orc_fmm_eval_timed only). */
static double wall_s(void) {
#ifdef _OPENMP
  return omp_get_wtime();
#else
  struct timespec ts;
  clock_gettime(CLOCK_MONOTONIC, &ts);
  return (double)ts.tv_sec + 1e-9 * (double)ts.tv_nsec;
#endif
}

/* The evaluation of orc_fmm_eval; `timing` (nullable) receives the stage
 * wall times and the work done by the stages that are restricted to the
 * boxes feeding the evaluated points (see orc_fmm_eval_timed). */
static void fmm_eval_run(const orc_tree* t, int p, const double* q, const int64_t* targets,
                         int64_t n_targets, double* u, double* field, double* timing) {
  double tick = wall_s();
  int64_t done_m2l = 0, done_l2l = 0;
  const int64_t n = orc__n(t);
  const int L = orc__levels(t), s = orc__splits(t);
  const int64_t nch = (int64_t)1 << s;
  const int64_t nbox = orc__n_boxes(t);
  const int P = (p + 1) * (p + 1);
  const int32_t* perm = orc__perm(t);
  const double* X = orc__pos_tree(t);
  const int64_t* bs = orc__box_start(t);
  const int64_t* bc = orc__box_count(t);
  const double* cen = orc__center(t);
  const int64_t leaf_off = level_off(L, s);
  const int64_t n_leaves = (int64_t)1 << (s * L);

  /* sort: charges into tree order */
  double* qt = (double*)malloc(sizeof(double) * (size_t)n);
  for (int64_t i = 0; i < n; i++) qt[i] = q[perm[i]];

  /* which tree positions are evaluated, and which boxes feed them */
  int64_t* inv = (int64_t*)malloc(sizeof(int64_t) * (size_t)n);
  for (int64_t i = 0; i < n; i++) inv[perm[i]] = i;
  int64_t n_eval = targets ? n_targets : n;
  int64_t* tpos = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n_eval + 1));
  for (int64_t k = 0; k < n_eval; k++) tpos[k] = targets ? inv[targets[k]] : inv[k];
  char* need = (char*)calloc((size_t)nbox, 1);
  for (int64_t k = 0; k < n_eval; k++) {
    /* leaf holding tree position tpos[k] */
    int64_t lo = 0, hi = n_leaves - 1;
    while (lo < hi) {
      int64_t mid = (lo + hi + 1) / 2;
      if (bs[leaf_off + mid] <= tpos[k]) lo = mid;
      else hi = mid - 1;
    }
    int64_t b = lo;
    for (int l = L; l >= 0; l--) {
      need[level_off(l, s) + b] = 1;
      b /= nch;
    }
  }

  double* C = (double*)calloc((size_t)nbox * P, sizeof(double));
  double* D = (double*)calloc((size_t)nbox * P, sizeof(double));
  if (timing) {
    double now = wall_s();
    timing[0] = now - tick;
    tick = now;
  }

  /* mpls: P2M on every leaf */
#pragma omp parallel for schedule(dynamic, 16)
  for (int64_t b = 0; b < n_leaves; b++) {
    int64_t g = leaf_off + b;
    double* pts = (double*)malloc(sizeof(double) * 3 * (size_t)bc[g]);
    memcpy(pts, X + 3 * bs[g], sizeof(double) * 3 * (size_t)bc[g]);
    orc_p2m(p, pts, qt + bs[g], bc[g], cen + 3 * g, C + (size_t)g * P);
    free(pts);
  }
  if (timing) {
    double now = wall_s();
    timing[1] = now - tick;
    tick = now;
  }
  /* M2M: levels L-1 .. 0 */
  for (int l = L - 1; l >= 0; l--) {
    int64_t off = level_off(l, s), offc = level_off(l + 1, s);
    int64_t nb = (int64_t)1 << (s * l);
#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t b = 0; b < nb; b++) {
      int64_t g = off + b;
      for (int64_t c = 0; c < nch; c++) {
        int64_t gc = offc + nch * b + c;
        orc_m2m(p, C + (size_t)gc * P, cen + 3 * gc, cen + 3 * g, C + (size_t)g * P);
      }
    }
  }
  if (timing) {
    double now = wall_s();
    timing[2] = now - tick;
    tick = now;
  }
  /* M2L over the whole list, grouped by target */
  const int64_t nm = orc__n_m2l(t);
  const int32_t* mt = orc__m2l_trg(t);
  const int32_t* ms = orc__m2l_src(t);
#pragma omp parallel for schedule(dynamic, 8) reduction(+ : done_m2l)
  for (int64_t g = 0; g < nbox; g++) {
    if (!need[g]) continue;
    for (int64_t k = first_ge(mt, nm, (int32_t)g); k < nm && mt[k] == g; k++) {
      orc_m2l(p, C + (size_t)ms[k] * P, cen + 3 * (int64_t)ms[k], cen + 3 * g, D + (size_t)g * P);
      done_m2l++;
    }
  }
  if (timing) {
    double now = wall_s();
    timing[3] = now - tick;
    tick = now;
  }
  /* L2L: levels 1 .. L */
  for (int l = 1; l <= L; l++) {
    int64_t off = level_off(l, s), offp = level_off(l - 1, s);
    int64_t nb = (int64_t)1 << (s * l);
#pragma omp parallel for schedule(dynamic, 16) reduction(+ : done_l2l)
    for (int64_t b = 0; b < nb; b++) {
      int64_t g = off + b;
      if (!need[g]) continue;
      int64_t gp = offp + b / nch;
      orc_l2l(p, D + (size_t)gp * P, cen + 3 * gp, cen + 3 * g, D + (size_t)g * P);
      done_l2l++;
    }
  }
  if (timing) {
    double now = wall_s();
    timing[4] = now - tick;
    tick = now;
  }
  /* evloc (L2P) and evdir (P2P) for every evaluated point */
  const int64_t np = orc__n_p2p(t);
  const int32_t* pt = orc__p2p_trg(t);
  const int32_t* ps = orc__p2p_src(t);
#pragma omp parallel for schedule(dynamic, 64)
  for (int64_t k = 0; k < n_eval; k++) {
    int64_t i = tpos[k];
    int64_t lo = 0, hi = n_leaves - 1;
    while (lo < hi) {
      int64_t mid = (lo + hi + 1) / 2;
      if (bs[leaf_off + mid] <= i) lo = mid;
      else hi = mid - 1;
    }
    int64_t leaf = lo, g = leaf_off + leaf;
    double grad[3];
    double uf = orc_l2p(p, D + (size_t)g * P, cen + 3 * g, X + 3 * i, grad);
    double un = 0.0, gn[3] = {0.0, 0.0, 0.0};
    for (int64_t e = first_ge(pt, np, (int32_t)leaf); e < np && pt[e] == leaf; e++) {
      int64_t gs = leaf_off + ps[e];
      for (int64_t j = bs[gs]; j < bs[gs] + bc[gs]; j++) {
        double dx = X[3 * i] - X[3 * j], dy = X[3 * i + 1] - X[3 * j + 1], dz = X[3 * i + 2] - X[3 * j + 2];
        double r2 = dx * dx + dy * dy + dz * dz;
        if (r2 == 0.0) continue;
        double r = sqrt(r2);
        un += qt[j] / r;
        double w = qt[j] / (r2 * r);
        gn[0] -= w * dx;
        gn[1] -= w * dy;
        gn[2] -= w * dz;
      }
    }
    /* u = -1/(4 pi) (far + near); field = -grad u = +1/(4 pi) grad(far + near) */
    u[k] = -(uf + un) / FOUR_PI;
    if (field)
      for (int a = 0; a < 3; a++) field[3 * k + a] = (grad[a] + gn[a]) / FOUR_PI;
  }
  if (timing) {
    timing[5] = wall_s() - tick;
    timing[6] = (double)done_m2l;
    timing[7] = (double)done_l2l;
    timing[8] = (double)n_eval;
  }
  free(qt);
  free(inv);
  free(tpos);
  free(need);
  free(C);
  free(D);
}

void orc_fmm_eval(const orc_tree* t, int p, const double* q, const int64_t* targets,
                  int64_t n_targets, double* u, double* field) {
  fmm_eval_run(t, p, q, targets, n_targets, u, field, NULL);
}

void orc_fmm_eval_timed(const orc_tree* t, int p, const double* q, const int64_t* targets,
                        int64_t n_targets, double* u, double* field, double* timing) {
  fmm_eval_run(t, p, q, targets, n_targets, u, field, timing);
}

void orc_set_num_threads(int n) {
#ifdef _OPENMP
  if (n > 0) omp_set_num_threads(n);
#else
  (void)n;
#endif
}

/* Eq. 1-3 summed directly. */
void orc_direct(const double* pos, const double* q, int64_t n, const int64_t* targets,
                int64_t n_targets, double* u, double* field) {
  int64_t n_eval = targets ? n_targets : n;
#pragma omp parallel for schedule(static)
  for (int64_t k = 0; k < n_eval; k++) {
    int64_t i = targets ? targets[k] : k;
    double acc = 0.0, g0 = 0.0, g1 = 0.0, g2 = 0.0;
    for (int64_t j = 0; j < n; j++) {
      double dx = pos[3 * i] - pos[3 * j], dy = pos[3 * i + 1] - pos[3 * j + 1], dz = pos[3 * i + 2] - pos[3 * j + 2];
      double r2 = dx * dx + dy * dy + dz * dz;
      if (r2 == 0.0) continue;
      double r = sqrt(r2);
      acc += q[j] / r;
      double w = q[j] / (r2 * r);
      g0 += w * dx;
      g1 += w * dy;
      g2 += w * dz;
    }
    u[k] = -acc / FOUR_PI;
    /* grad(1/r) = -(r_i - r_j)/r^3, so field = -grad u = -(1/4pi) sum q (r_i - r_j)/r^3 */
    if (field) {
      field[3 * k] = -g0 / FOUR_PI;
      field[3 * k + 1] = -g1 / FOUR_PI;
      field[3 * k + 2] = -g2 / FOUR_PI;
    }
  }
}

/* Separate source and target trees (Sec. II.B, final part): multipoles on the
 * source tree (mpls, M2M), M2L from source boxes into target boxes, locals on
 * the target tree (L2L), evloc and evdir at every target point. */
void orc_fmm2_eval(const orc_tree2* t2, int p, const double* q, double* u, double* field) {
  const orc_tree* S = orc_tree2_source(t2);
  const orc_tree* T = orc_tree2_target(t2);
  const int s = orc__splits(S);
  const int64_t nch = (int64_t)1 << s;
  const int P = (p + 1) * (p + 1);
  const int Ls = orc__levels(S), Lt = orc__levels(T);
  const int64_t ns = orc__n(S), nt = orc__n(T);
  const int64_t nbs = orc__n_boxes(S), nbt = orc__n_boxes(T);
  const int32_t* perm_s = orc__perm(S);
  const int32_t* perm_t = orc__perm(T);
  const double* Xs = orc__pos_tree(S);
  const double* Xt = orc__pos_tree(T);
  const int64_t *bs_s = orc__box_start(S), *bc_s = orc__box_count(S);
  const int64_t *bs_t = orc__box_start(T), *bc_t = orc__box_count(T);
  const double* cen_s = orc__center(S);
  const double* cen_t = orc__center(T);
  const int64_t leaf_off_s = level_off(Ls, s), leaf_off_t = level_off(Lt, s);
  const int64_t nl_s = (int64_t)1 << (s * Ls), nl_t = (int64_t)1 << (s * Lt);

  /* sort: charges into source-tree order */
  double* qt = (double*)malloc(sizeof(double) * (size_t)ns);
  for (int64_t i = 0; i < ns; i++) qt[i] = q[perm_s[i]];
  double* C = (double*)calloc((size_t)nbs * P, sizeof(double));
  double* D = (double*)calloc((size_t)nbt * P, sizeof(double));

  /* mpls and M2M on the source tree */
#pragma omp parallel for schedule(dynamic, 16)
  for (int64_t b = 0; b < nl_s; b++) {
    int64_t g = leaf_off_s + b;
    orc_p2m(p, Xs + 3 * bs_s[g], qt + bs_s[g], bc_s[g], cen_s + 3 * g, C + (size_t)g * P);
  }
  for (int l = Ls - 1; l >= 0; l--) {
    int64_t off = level_off(l, s), offc = level_off(l + 1, s);
    int64_t nb = (int64_t)1 << (s * l);
#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t b = 0; b < nb; b++)
      for (int64_t c = 0; c < nch; c++) {
        int64_t gc = offc + nch * b + c;
        orc_m2m(p, C + (size_t)gc * P, cen_s + 3 * gc, cen_s + 3 * (off + b), C + (size_t)(off + b) * P);
      }
  }
  /* M2L: source box -> target box (combined target id = nbs + g) */
  const int64_t nm = orc2__n_m2l(t2);
  const int32_t* mt = orc2__m2l_trg(t2);
  const int32_t* ms = orc2__m2l_src(t2);
#pragma omp parallel for schedule(dynamic, 8)
  for (int64_t g = 0; g < nbt; g++)
    for (int64_t k = first_ge(mt, nm, (int32_t)(nbs + g)); k < nm && mt[k] == nbs + g; k++)
      orc_m2l(p, C + (size_t)ms[k] * P, cen_s + 3 * (int64_t)ms[k], cen_t + 3 * g, D + (size_t)g * P);
  /* L2L on the target tree */
  for (int l = 1; l <= Lt; l++) {
    int64_t off = level_off(l, s), offp = level_off(l - 1, s);
    int64_t nb = (int64_t)1 << (s * l);
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t b = 0; b < nb; b++) {
      int64_t gp = offp + b / nch;
      orc_l2l(p, D + (size_t)gp * P, cen_t + 3 * gp, cen_t + 3 * (off + b), D + (size_t)(off + b) * P);
    }
  }
  /* evloc and evdir at every target point, per target leaf */
  const int64_t np = orc2__n_p2p(t2);
  const int32_t* pt = orc2__p2p_trg(t2);
  const int32_t* ps = orc2__p2p_src(t2);
#pragma omp parallel for schedule(dynamic, 4)
  for (int64_t leaf = 0; leaf < nl_t; leaf++) {
    int64_t g = leaf_off_t + leaf;
    int64_t e0 = first_ge(pt, np, (int32_t)leaf);
    for (int64_t i = bs_t[g]; i < bs_t[g] + bc_t[g]; i++) {
      double grad[3];
      double uf = orc_l2p(p, D + (size_t)g * P, cen_t + 3 * g, Xt + 3 * i, grad);
      double un = 0.0, gn[3] = {0.0, 0.0, 0.0};
      for (int64_t e = e0; e < np && pt[e] == leaf; e++) {
        int64_t gs = leaf_off_s + ps[e];
        for (int64_t j = bs_s[gs]; j < bs_s[gs] + bc_s[gs]; j++) {
          double dx = Xt[3 * i] - Xs[3 * j], dy = Xt[3 * i + 1] - Xs[3 * j + 1], dz = Xt[3 * i + 2] - Xs[3 * j + 2];
          double r2 = dx * dx + dy * dy + dz * dz;
          if (r2 == 0.0) continue;
          double r = sqrt(r2);
          un += qt[j] / r;
          double w = qt[j] / (r2 * r);
          gn[0] -= w * dx;
          gn[1] -= w * dy;
          gn[2] -= w * dz;
        }
      }
      int64_t k = perm_t[i];
      u[k] = -(uf + un) / FOUR_PI;
      if (field)
        for (int a = 0; a < 3; a++) field[3 * k + a] = (grad[a] + gn[a]) / FOUR_PI;
    }
  }
  (void)nt;
  free(qt);
  free(C);
  free(D);
}

void orc_direct2(const double* src_pos, const double* q, int64_t n_src, const double* trg_pos,
                 int64_t n_trg, double* u, double* field) {
#pragma omp parallel for schedule(static)
  for (int64_t k = 0; k < n_trg; k++) {
    double acc = 0.0, g0 = 0.0, g1 = 0.0, g2 = 0.0;
    for (int64_t j = 0; j < n_src; j++) {
      double dx = trg_pos[3 * k] - src_pos[3 * j], dy = trg_pos[3 * k + 1] - src_pos[3 * j + 1],
             dz = trg_pos[3 * k + 2] - src_pos[3 * j + 2];
      double r2 = dx * dx + dy * dy + dz * dz;
      if (r2 == 0.0) continue;
      double r = sqrt(r2);
      acc += q[j] / r;
      double w = q[j] / (r2 * r);
      g0 += w * dx;
      g1 += w * dy;
      g2 += w * dz;
    }
    u[k] = -acc / FOUR_PI;
    if (field) {
      field[3 * k] = -g0 / FOUR_PI;
      field[3 * k + 1] = -g1 / FOUR_PI;
      field[3 * k + 2] = -g2 / FOUR_PI;
    }
  }
}

void orc_direct_vjp(const double* pos, const double* q, const double* g, int64_t n,
                    double* dq, double* dpos) {
  double* fu = (double*)malloc(sizeof(double) * 3 * (size_t)n);
  double* fv = (double*)malloc(sizeof(double) * 3 * (size_t)n);
  double* uq = (double*)malloc(sizeof(double) * (size_t)n);
  orc_direct(pos, q, n, NULL, 0, uq, fu);
  orc_direct(pos, g, n, NULL, 0, dq, fv);
  /* grad u = -field */
  for (int64_t k = 0; k < n; k++)
    for (int a = 0; a < 3; a++) dpos[3 * k + a] = -(g[k] * fu[3 * k + a] + q[k] * fv[3 * k + a]);
  free(fu);
  free(fv);
  free(uq);
}
