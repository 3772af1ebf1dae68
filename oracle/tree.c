/*
 * Oracle: median-split 2^s-tree, box geometry and level-marching interaction
 * lists (Sec. II.A, II.B, Listing 2).  TEST INFRASTRUCTURE ONLY (see
 * fmm_oracle.h).
 *
 * Readings taken where the paper is silent or ambiguous:
 *  - Coordinates equal to -0.0 are treated as +0.0.
 *  - Split (Sec. II.A steps 1-2, Listing 2): a box's axis is the one of largest
 *    extent of its points' bounding box, ties to the lowest axis index (as
 *    argmax does).  Its points are ordered by (coordinate on that axis,
 *    original index), with -0.0 equal to +0.0; the first ceil(n/2) form the
 *    lower child, the rest the upper child, lower child first.
 *  - Levels (step 4): L is the smallest l with ceil(N / 2^(l s)) <= N_max.
 *  - Leaf order (Listing 2, last line): ascending original index.
 *  - Box centre = midpoint of the tight bounding box of its points; radius =
 *    half the bounding-box diagonal (the paper does not define the radius).
 *  - Well separation (Eq. 4): R + theta r <= theta d evaluated in FP64 in that
 *    order, and additionally d > 0 (boxes with coincident centres never
 *    interact through expansions).
 *  - Average box radius of a level: pairwise sum of the radii over adjacent
 *    pairs, repeated until one value remains, divided by the box count.
 *  - Level march (Sec. II.B): equal average radii advance the source level
 *    (the text) unless tie_target is set (the reading of the same-vs-cross
 *    table, whose rows advance the target).  The march ends when no candidate
 *    is left or both sides are at the leaf level; the remaining leaf pairs,
 *    self pairs included, form the near field.  With same_level set, the
 *    lists are the same-level lists of Sec. II.B steps 1-3: both sides
 *    descend together and only boxes of one level are compared.
 *  - Canonical list order: M2L sorted by (target global box, source global
 *    box), near-field pairs by (target leaf, source leaf).  The global id of
 *    box b on level l is (2^(s l) - 1) / (2^s - 1) + b.
 */
#include "fmm_oracle.h"
#include <math.h>
#include <stdlib.h>
#include <string.h>

struct orc_tree {
  int64_t n;
  int L, s;
  double theta;
  int tie_target;
  int same_level;
  int64_t n_boxes, n_leaves;
  int32_t* perm;        /* tree position -> original index          */
  double* pos_tree;     /* positions in tree order, 3 per point     */
  int64_t* box_start;   /* per global box                           */
  int64_t* box_count;
  double* center;       /* 3 per global box                         */
  double* radius;
  double* level_avg;    /* L + 1                                    */
  int64_t n_m2l, n_p2p;
  int32_t *m2l_trg, *m2l_src; /* global box ids                     */
  int32_t *p2p_trg, *p2p_src; /* leaf indices                       */
};

int orc_num_levels(int64_t n, int leaf_size, int s) {
  int L = 0;
  for (;;) {
    int64_t boxes = (int64_t)1 << (s * L);
    int64_t largest = (n + boxes - 1) / boxes;
    if (largest <= leaf_size) return L;
    L++;
  }
}

static int64_t level_offset(int l, int s) {
  int64_t off = 0;
  for (int i = 0; i < l; i++) off += (int64_t)1 << (s * i);
  return off;
}

/* Sorting key for one bisection. */
static const double* g_sort_pos;
static int g_sort_axis;
static int cmp_axis_then_index(const void* a, const void* b) {
  int32_t ia = *(const int32_t*)a, ib = *(const int32_t*)b;
  double xa = g_sort_pos[3 * (int64_t)ia + g_sort_axis];
  double xb = g_sort_pos[3 * (int64_t)ib + g_sort_axis];
  if (xa < xb) return -1;
  if (xa > xb) return 1;
  return (ia < ib) ? -1 : (ia > ib) ? 1 : 0;
}
static int cmp_index(const void* a, const void* b) {
  int32_t ia = *(const int32_t*)a, ib = *(const int32_t*)b;
  return (ia < ib) ? -1 : (ia > ib) ? 1 : 0;
}

static void bbox(const double* pos, const int32_t* idx, int64_t cnt, double lo[3], double hi[3]) {
  for (int a = 0; a < 3; a++) {
    lo[a] = pos[3 * (int64_t)idx[0] + a];
    hi[a] = lo[a];
  }
  for (int64_t i = 1; i < cnt; i++)
    for (int a = 0; a < 3; a++) {
      double v = pos[3 * (int64_t)idx[i] + a];
      if (v < lo[a]) lo[a] = v;
      if (v > hi[a]) hi[a] = v;
    }
}

/* Well-separation criterion, Eq. 4, between a source box (centre cs, radius
 * rs) and a target box (centre ct, radius rt). */
static int well_separated(const double* cs, double rs, const double* ct, double rt, double theta) {
  double dx = cs[0] - ct[0];
  double dy = cs[1] - ct[1];
  double dz = cs[2] - ct[2];
  double dxx = dx * dx;
  double dyy = dy * dy;
  double dzz = dz * dz;
  double d2 = dxx + dyy;
  d2 = d2 + dzz;
  double d = sqrt(d2);
  double R = (rs > rt) ? rs : rt;
  double r = (rs > rt) ? rt : rs;
  double tr = theta * r;
  double lhs = R + tr;
  double rhs = theta * d;
  return (d > 0.0) && (lhs <= rhs);
}

typedef struct { int32_t t, s; } pair32;

static int cmp_pair(const void* a, const void* b) {
  const pair32* x = (const pair32*)a;
  const pair32* y = (const pair32*)b;
  if (x->t != y->t) return (x->t < y->t) ? -1 : 1;
  if (x->s != y->s) return (x->s < y->s) ? -1 : 1;
  return 0;
}

static void push(pair32** arr, int64_t* n, int64_t* cap, int32_t t, int32_t s) {
  if (*n == *cap) {
    *cap = (*cap == 0) ? 1024 : 2 * *cap;
    *arr = (pair32*)realloc(*arr, sizeof(pair32) * (size_t)*cap);
  }
  (*arr)[*n].t = t;
  (*arr)[*n].s = s;
  (*n)++;
}

typedef struct {
  int64_t n_m2l, n_p2p;
  int32_t *m2l_trg, *m2l_src;
  int32_t *p2p_trg, *p2p_src;
} lists;

/* Interaction lists between the boxes of a source tree S and a target tree T
 * (the same tree for the usual evaluation).  Level march of Sec. II.B: start
 * at both roots; well-separated candidate pairs go to the M2L list; the others
 * are replaced by the children of the side whose level has the larger average
 * radius (ties: the source, or the target with tie_target), the other side's
 * children once one side has no finer level; pairs left when both sides are
 * at their leaf levels form the near field.  same_level: both sides descend
 * together (Sec. II.B steps 1-3).  M2L target ids are offset by trg_base. */
static void march(const orc_tree* S, const orc_tree* T, double theta, int tie_target, int same_level,
                  int64_t trg_base, lists* out) {
  const int s = S->s;
  const int64_t nch = (int64_t)1 << s;
  pair32 *cand = NULL, *keep = NULL, *m2l = NULL;
  int64_t n_cand = 0, cap_cand = 0, n_keep = 0, cap_keep = 0, n_m2l = 0, cap_m2l = 0;
  push(&cand, &n_cand, &cap_cand, 0, 0);
  int ls = 0, lt = 0;
  out->n_p2p = 0;
  out->p2p_trg = out->p2p_src = NULL;
  for (;;) {
    int64_t offs = level_offset(ls, s), offt = level_offset(lt, s);
    n_keep = 0;
    for (int64_t i = 0; i < n_cand; i++) {
      int64_t gs = offs + cand[i].s, gt = offt + cand[i].t;
      if (well_separated(S->center + 3 * gs, S->radius[gs], T->center + 3 * gt, T->radius[gt], theta))
        push(&m2l, &n_m2l, &cap_m2l, (int32_t)(trg_base + gt), (int32_t)gs);
      else
        push(&keep, &n_keep, &cap_keep, cand[i].t, cand[i].s);
    }
    if (n_keep == 0) break;
    int can_s = ls < S->L, can_t = lt < T->L;
    if (!can_s && !can_t) {
      qsort(keep, (size_t)n_keep, sizeof(pair32), cmp_pair);
      out->n_p2p = n_keep;
      out->p2p_trg = (int32_t*)malloc(sizeof(int32_t) * (size_t)n_keep);
      out->p2p_src = (int32_t*)malloc(sizeof(int32_t) * (size_t)n_keep);
      for (int64_t i = 0; i < n_keep; i++) {
        out->p2p_trg[i] = keep[i].t;
        out->p2p_src[i] = keep[i].s;
      }
      break;
    }
    n_cand = 0;
    if (same_level) {
      /* same-level lists (Sec. II.B steps 1-3): both sides descend together */
      for (int64_t i = 0; i < n_keep; i++)
        for (int64_t ct = 0; ct < nch; ct++)
          for (int64_t cs = 0; cs < nch; cs++)
            push(&cand, &n_cand, &cap_cand, (int32_t)(nch * keep[i].t + ct), (int32_t)(nch * keep[i].s + cs));
      ls++;
      lt++;
      continue;
    }
    int adv_src;
    if (can_s && can_t) {
      double as = S->level_avg[ls], at = T->level_avg[lt];
      if (as > at) adv_src = 1;
      else if (as < at) adv_src = 0;
      else adv_src = !tie_target;
    } else {
      adv_src = can_s;
    }
    for (int64_t i = 0; i < n_keep; i++)
      for (int64_t c = 0; c < nch; c++) {
        if (adv_src) push(&cand, &n_cand, &cap_cand, keep[i].t, (int32_t)(nch * keep[i].s + c));
        else push(&cand, &n_cand, &cap_cand, (int32_t)(nch * keep[i].t + c), keep[i].s);
      }
    if (adv_src) ls++;
    else lt++;
  }
  qsort(m2l, (size_t)n_m2l, sizeof(pair32), cmp_pair);
  out->n_m2l = n_m2l;
  out->m2l_trg = (int32_t*)malloc(sizeof(int32_t) * (size_t)(n_m2l + 1));
  out->m2l_src = (int32_t*)malloc(sizeof(int32_t) * (size_t)(n_m2l + 1));
  for (int64_t i = 0; i < n_m2l; i++) {
    out->m2l_trg[i] = m2l[i].t;
    out->m2l_src[i] = m2l[i].s;
  }
  if (!out->p2p_trg) {
    out->p2p_trg = (int32_t*)malloc(sizeof(int32_t));
    out->p2p_src = (int32_t*)malloc(sizeof(int32_t));
  }
  free(cand);
  free(keep);
  free(m2l);
}

static void build_lists(orc_tree* t) {
  lists li;
  march(t, t, t->theta, t->tie_target, t->same_level, 0, &li);
  t->n_m2l = li.n_m2l;
  t->m2l_trg = li.m2l_trg;
  t->m2l_src = li.m2l_src;
  t->n_p2p = li.n_p2p;
  t->p2p_trg = li.p2p_trg;
  t->p2p_src = li.p2p_src;
}

orc_tree* orc_tree_build(const double* pos, int64_t n, int leaf_size, int s, double theta,
                         int flags) {
  if (n < 1 || s < 1 || leaf_size < (1 << s)) return NULL;
  orc_tree* t = (orc_tree*)calloc(1, sizeof(orc_tree));
  /* flags bit 2 (internal): hierarchy only, no lists */
  /* -0.0 is treated as +0.0 (x + 0.0 rounds -0.0 to +0.0) */
  double* canon = (double*)malloc(sizeof(double) * 3 * (size_t)n);
  for (int64_t i = 0; i < 3 * n; i++) canon[i] = pos[i] + 0.0;
  pos = canon;
  t->n = n;
  t->s = s;
  t->theta = theta;
  t->tie_target = (flags & 1) != 0;
  t->same_level = (flags & 2) != 0;
  t->L = orc_num_levels(n, leaf_size, s);
  int L = t->L;
  t->n_boxes = level_offset(L + 1, s);
  t->n_leaves = (int64_t)1 << (s * L);
  t->perm = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
  for (int64_t i = 0; i < n; i++) t->perm[i] = (int32_t)i;

  /* Bisection rounds (Listing 2): round j splits every segment in two. */
  int64_t nseg = 1;
  int64_t* seg_start = (int64_t*)malloc(sizeof(int64_t) * ((size_t)t->n_leaves + 1));
  int64_t* seg_next = (int64_t*)malloc(sizeof(int64_t) * ((size_t)t->n_leaves + 1));
  seg_start[0] = 0;
  seg_start[1] = n;
  for (int round = 0; round < L * s; round++) {
    for (int64_t j = 0; j < nseg; j++) {
      int64_t a = seg_start[j], b = seg_start[j + 1], cnt = b - a;
      double lo[3], hi[3];
      bbox(pos, t->perm + a, cnt, lo, hi);
      int axis = 0;
      double best = hi[0] - lo[0];
      for (int ax = 1; ax < 3; ax++)
        if (hi[ax] - lo[ax] > best) { best = hi[ax] - lo[ax]; axis = ax; }
      g_sort_pos = pos;
      g_sort_axis = axis;
      qsort(t->perm + a, (size_t)cnt, sizeof(int32_t), cmp_axis_then_index);
      seg_next[2 * j] = a;
      seg_next[2 * j + 1] = a + (cnt + 1) / 2;
    }
    seg_next[2 * nseg] = n;
    nseg *= 2;
    memcpy(seg_start, seg_next, sizeof(int64_t) * (size_t)(nseg + 1));
  }
  for (int64_t j = 0; j < nseg; j++)
    qsort(t->perm + seg_start[j], (size_t)(seg_start[j + 1] - seg_start[j]), sizeof(int32_t), cmp_index);
  free(seg_next);

  t->pos_tree = (double*)malloc(sizeof(double) * 3 * (size_t)n);
  for (int64_t i = 0; i < n; i++)
    for (int a = 0; a < 3; a++) t->pos_tree[3 * i + a] = pos[3 * (int64_t)t->perm[i] + a];

  /* Box ranges per level: leaf segment starts, coarsened by 2^s per level. */
  t->box_start = (int64_t*)malloc(sizeof(int64_t) * (size_t)t->n_boxes);
  t->box_count = (int64_t*)malloc(sizeof(int64_t) * (size_t)t->n_boxes);
  t->center = (double*)malloc(sizeof(double) * 3 * (size_t)t->n_boxes);
  t->radius = (double*)malloc(sizeof(double) * (size_t)t->n_boxes);
  t->level_avg = (double*)malloc(sizeof(double) * (size_t)(L + 1));
  for (int l = 0; l <= L; l++) {
    int64_t nb = (int64_t)1 << (s * l);
    int64_t stride = t->n_leaves / nb;
    int64_t off = level_offset(l, s);
    for (int64_t b = 0; b < nb; b++) {
      int64_t a = seg_start[b * stride], e = seg_start[(b + 1) * stride];
      int64_t g = off + b;
      t->box_start[g] = a;
      t->box_count[g] = e - a;
      double lo[3], hi[3];
      bbox(pos, t->perm + a, e - a, lo, hi);
      for (int ax = 0; ax < 3; ax++) {
        double sum = lo[ax] + hi[ax];
        t->center[3 * g + ax] = sum * 0.5;
      }
      double ex = hi[0] - lo[0], ey = hi[1] - lo[1], ez = hi[2] - lo[2];
      double exx = ex * ex;
      double eyy = ey * ey;
      double ezz = ez * ez;
      double d2 = exx + eyy;
      d2 = d2 + ezz;
      t->radius[g] = sqrt(d2) * 0.5;
    }
    /* average radius: adjacent-pair sums until one value remains */
    double* tmp = (double*)malloc(sizeof(double) * (size_t)nb);
    memcpy(tmp, t->radius + off, sizeof(double) * (size_t)nb);
    for (int64_t m = nb; m > 1; m /= 2)
      for (int64_t i = 0; i < m / 2; i++) tmp[i] = tmp[2 * i] + tmp[2 * i + 1];
    t->level_avg[l] = tmp[0] / (double)nb;
    free(tmp);
  }
  free(seg_start);
  free(canon);
  if (!(flags & 4)) build_lists(t);
  return t;
}

void orc_tree_free(orc_tree* t) {
  if (!t) return;
  free(t->perm);
  free(t->pos_tree);
  free(t->box_start);
  free(t->box_count);
  free(t->center);
  free(t->radius);
  free(t->level_avg);
  free(t->m2l_trg);
  free(t->m2l_src);
  free(t->p2p_trg);
  free(t->p2p_src);
  free(t);
}

void orc_tree_info(const orc_tree* t, int64_t* info) {
  info[0] = t->L;
  info[1] = t->n_boxes;
  info[2] = t->n_m2l;
  info[3] = t->n_p2p;
  info[4] = t->n_leaves;
}

void orc_tree_export(const orc_tree* t, int32_t* perm, int64_t* box_start, int64_t* box_count,
                     double* center, double* radius, double* level_avg_radius) {
  if (perm) memcpy(perm, t->perm, sizeof(int32_t) * (size_t)t->n);
  if (box_start) memcpy(box_start, t->box_start, sizeof(int64_t) * (size_t)t->n_boxes);
  if (box_count) memcpy(box_count, t->box_count, sizeof(int64_t) * (size_t)t->n_boxes);
  if (center) memcpy(center, t->center, sizeof(double) * 3 * (size_t)t->n_boxes);
  if (radius) memcpy(radius, t->radius, sizeof(double) * (size_t)t->n_boxes);
  if (level_avg_radius) memcpy(level_avg_radius, t->level_avg, sizeof(double) * (size_t)(t->L + 1));
}

void orc_tree_export_lists(const orc_tree* t, int32_t* m2l_trg, int32_t* m2l_src,
                           int32_t* p2p_trg, int32_t* p2p_src) {
  if (m2l_trg) memcpy(m2l_trg, t->m2l_trg, sizeof(int32_t) * (size_t)t->n_m2l);
  if (m2l_src) memcpy(m2l_src, t->m2l_src, sizeof(int32_t) * (size_t)t->n_m2l);
  if (p2p_trg) memcpy(p2p_trg, t->p2p_trg, sizeof(int32_t) * (size_t)t->n_p2p);
  if (p2p_src) memcpy(p2p_src, t->p2p_src, sizeof(int32_t) * (size_t)t->n_p2p);
}

/* ---- separate source and target hierarchies (Sec. II.B, final part) ----
 * Two trees built with the same N_max, s and theta; the lists compare source
 * boxes with target boxes by the level march (same-level lists are not
 * defined when the two trees have different depths).  Combined box ids:
 * source boxes 0 .. NB_s - 1, target box g at NB_s + g. */
struct orc_tree2 {
  orc_tree* src;
  orc_tree* trg;
  lists li;
};

orc_tree2* orc_tree2_build(const double* src_pos, int64_t n_src, const double* trg_pos, int64_t n_trg,
                           int leaf_size, int s, double theta, int flags) {
  if (flags & ~1) return NULL;
  orc_tree* S = orc_tree_build(src_pos, n_src, leaf_size, s, theta, 4);
  orc_tree* T = orc_tree_build(trg_pos, n_trg, leaf_size, s, theta, 4);
  if (!S || !T) {
    orc_tree_free(S);
    orc_tree_free(T);
    return NULL;
  }
  orc_tree2* t2 = (orc_tree2*)calloc(1, sizeof(orc_tree2));
  t2->src = S;
  t2->trg = T;
  march(S, T, theta, flags & 1, 0, S->n_boxes, &t2->li);
  return t2;
}

void orc_tree2_free(orc_tree2* t2) {
  if (!t2) return;
  orc_tree_free(t2->src);
  orc_tree_free(t2->trg);
  free(t2->li.m2l_trg);
  free(t2->li.m2l_src);
  free(t2->li.p2p_trg);
  free(t2->li.p2p_src);
  free(t2);
}

const orc_tree* orc_tree2_source(const orc_tree2* t2) { return t2->src; }
const orc_tree* orc_tree2_target(const orc_tree2* t2) { return t2->trg; }

void orc_tree2_info(const orc_tree2* t2, int64_t* info) {
  info[0] = t2->li.n_m2l;
  info[1] = t2->li.n_p2p;
}

void orc_tree2_export_lists(const orc_tree2* t2, int32_t* m2l_trg, int32_t* m2l_src, int32_t* p2p_trg,
                            int32_t* p2p_src) {
  const lists* li = &t2->li;
  if (m2l_trg) memcpy(m2l_trg, li->m2l_trg, sizeof(int32_t) * (size_t)li->n_m2l);
  if (m2l_src) memcpy(m2l_src, li->m2l_src, sizeof(int32_t) * (size_t)li->n_m2l);
  if (p2p_trg) memcpy(p2p_trg, li->p2p_trg, sizeof(int32_t) * (size_t)li->n_p2p);
  if (p2p_src) memcpy(p2p_src, li->p2p_src, sizeof(int32_t) * (size_t)li->n_p2p);
}

int64_t orc2__n_m2l(const orc_tree2* t2) { return t2->li.n_m2l; }
const int32_t* orc2__m2l_trg(const orc_tree2* t2) { return t2->li.m2l_trg; }
const int32_t* orc2__m2l_src(const orc_tree2* t2) { return t2->li.m2l_src; }
int64_t orc2__n_p2p(const orc_tree2* t2) { return t2->li.n_p2p; }
const int32_t* orc2__p2p_trg(const orc_tree2* t2) { return t2->li.p2p_trg; }
const int32_t* orc2__p2p_src(const orc_tree2* t2) { return t2->li.p2p_src; }

/* Internal accessors for the evaluation file. */
const int32_t* orc__perm(const orc_tree* t) { return t->perm; }
const double* orc__pos_tree(const orc_tree* t) { return t->pos_tree; }
const int64_t* orc__box_start(const orc_tree* t) { return t->box_start; }
const int64_t* orc__box_count(const orc_tree* t) { return t->box_count; }
const double* orc__center(const orc_tree* t) { return t->center; }
int orc__levels(const orc_tree* t) { return t->L; }
int orc__splits(const orc_tree* t) { return t->s; }
int64_t orc__n(const orc_tree* t) { return t->n; }
int64_t orc__n_boxes(const orc_tree* t) { return t->n_boxes; }
int64_t orc__n_m2l(const orc_tree* t) { return t->n_m2l; }
const int32_t* orc__m2l_trg(const orc_tree* t) { return t->m2l_trg; }
const int32_t* orc__m2l_src(const orc_tree* t) { return t->m2l_src; }
int64_t orc__n_p2p(const orc_tree* t) { return t->n_p2p; }
const int32_t* orc__p2p_trg(const orc_tree* t) { return t->p2p_trg; }
const int32_t* orc__p2p_src(const orc_tree* t) { return t->p2p_src; }
