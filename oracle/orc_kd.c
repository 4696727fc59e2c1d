/*
 * FP64 CPU oracle, ORB / k-d tree variant of the short-range FMM.
 *
 * TEST INFRASTRUCTURE ONLY, like orc.c (whose expansion operators it calls):
 * the test-suite, the smoke check and the benchmark's CPU-baseline leg are its
 * only users, and it shares nothing with the CUDA library.
 *
 * The tree of Sec. 2.1 (Fig. 1): an ORB tree with a leaf limiter, whose cells
 * hand their particles to two children of almost equal count down to the
 * leaves; Sec. 4 keeps such a k-d tree inside every domain.  The paper fixes no
 * more than that; the readings taken here:
 *   - positions are wrapped into the box as for the octree, x - L floor(x / L);
 *   - a node of n > leaf_max particles is split.  Its geometry is the tight
 *     bounding box [lo, hi] of its particles; the split axis is the axis of
 *     largest extent hi - lo (the lowest axis on a tie); its particles, ordered
 *     by (coordinate on that axis, input index), give their first floor(n / 2)
 *     to the first child and the others to the second.  The counts halve, so no
 *     depth cap is needed;
 *   - nodes are numbered breadth first, a level's children in the order of
 *     their parents, the first child before the second.  A node owns a
 *     contiguous range of the particle array: the first child the front part of
 *     its parent's range, the second the back part; inside a leaf the particles
 *     are ordered by (x, input index);
 *   - the expansion centre of a node is the centre of its box,
 *     c = (lo + hi) / 2, its half extents e = (hi - lo) / 2 and its side the
 *     largest extent;
 *   - the three rules of Sec. 2.3 on these boxes, in FP64 with the operations
 *     in the order written below (no contraction): S_c = |c_B + sL - c_A|,
 *     S_m and S_max from the per-axis gaps |dc| - (e_A + e_B) (at least 0) and
 *     spans |dc| + (e_A + e_B); skip if S_m > R_c, open in the transition region
 *     (S_c > R_c, or S_max > R_c with rule 1), accept if side^2 <= theta^2 S_c^2
 *     (side of the source, or of the larger cell with size rule 1) and
 *     theta^2 S_c^2 > 0: a box of one particle, or of coincident ones, has side
 *     0, and without the second condition it would be accepted against itself
 *     (R = 0) or at theta = 0;
 *   - the walk opens the cell of larger side (both on equal sides; the other
 *     one when a cell is a leaf), like the octree walk opens the cell of lower
 *     level.
 * The short-range kernel is the Gaussian one of Sec. 2.2, or (orc_kd_set_split) the
 * polynomial truncation that Sec. 5 allows in its place (the reading of orc.c).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* expansion operators and prefactors of orc.c (Eqs. p2m .. l2p, Sec. 2.2) */
int orc_ncoef(int p);
int orc_p2m(int64_t n, const double *x, const double *mu, const double *z, int p, double *M);
int orc_m2m(const double *Min, const double *x, int p, double *Mout);
int orc_m2l_split(const double *M, const double *R, double rs, double rc, int split, int p, double *L);
int orc_l2l(const double *Lin, const double *x, int p, double *Lout);
int orc_l2p(const double *L, const double *u, int p, double G, double *phi, double *acc);
int orc_prefactors(double r, double rs, int p, double *f);
int orc_prefactors_poly(double r, double rc, int p, double *f);

#define KD_PMAX 10
#define KD_NCMAX 286
#define KD_MAXLEV 64

typedef struct {
  double box, rs, rc, G, theta;
  int p, leaf_max, rule, size_rule;
  int split; /* short-range kernel: 0 Gaussian (Sec. 2.2), 1 polynomial (Sec. 5) */
  int64_t n;
  double *x;     /* [n][3] wrapped positions in tree order */
  double *m;     /* [n] */
  int64_t *idx;  /* [n] input index of each particle in tree order */
  int64_t nnodes, ncap;
  int nlevels;
  int64_t level_start[KD_MAXLEV + 1];
  int *lev, *axis;            /* axis = split axis, -1 for a leaf */
  int64_t *first, *count, *child;  /* child = first child, -1 for a leaf */
  double *lo, *hi;            /* [nnodes][3] */
  int64_t np2p, nm2l, cap_p2p, cap_m2l;
  int64_t *p2p, *m2l;         /* [len][3] sink, source, shift index */
  double *M, *L;
} orc_kd;

void orc_kd_destroy(orc_kd *c) {
  if (!c) return;
  free(c->x); free(c->m); free(c->idx);
  free(c->lev); free(c->axis); free(c->first); free(c->count); free(c->child); free(c->lo); free(c->hi);
  free(c->p2p); free(c->m2l); free(c->M); free(c->L);
  free(c);
}

orc_kd *orc_kd_create(double box, double rs, double rc, double G, double theta, int p, int leaf_max, int rule,
                      int size_rule) {
  if (!(box > 0) || !(rs > 0) || !(rc > 0) || !(rc < 0.5 * box) || p < 1 || p > KD_PMAX || leaf_max < 1 ||
      (rule != 0 && rule != 1) || (size_rule != 0 && size_rule != 1) || !(theta >= 0))
    return NULL;
  orc_kd *c = (orc_kd *)calloc(1, sizeof(orc_kd));
  c->box = box; c->rs = rs; c->rc = rc; c->G = G; c->theta = theta;
  c->p = p; c->leaf_max = leaf_max; c->rule = rule; c->size_rule = size_rule;
  return c;
}

/* Short-range kernel of the FMM and its pair force: 0 Gaussian, 1 polynomial (Sec. 5). */
int orc_kd_set_split(orc_kd *c, int split) {
  if (!c || split < 0 || split > 1) return -1;
  c->split = split;
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Tree                                                                      */
/* ------------------------------------------------------------------------ */

static double kd_wrap(double x, double box) {
  double q = floor(x / box);
  double t = box * q;
  return x - t;
}

typedef struct {
  double key;
  int64_t idx, slot;
} kd_item;

static int cmp_item(const void *a, const void *b) {
  const kd_item *x = (const kd_item *)a, *y = (const kd_item *)b;
  if (x->key != y->key) return x->key < y->key ? -1 : 1;
  return (x->idx > y->idx) - (x->idx < y->idx);
}

/* order the particles [f, f + n) by (coordinate on axis d, input index) */
static void sort_range(orc_kd *c, int64_t f, int64_t n, int d) {
  kd_item *it = (kd_item *)malloc(sizeof(kd_item) * (size_t)n);
  for (int64_t i = 0; i < n; ++i) {
    it[i].key = c->x[3 * (f + i) + d];
    it[i].idx = c->idx[f + i];
    it[i].slot = f + i;
  }
  qsort(it, (size_t)n, sizeof(kd_item), cmp_item);
  double *x = (double *)malloc(sizeof(double) * 3 * (size_t)n);
  double *m = (double *)malloc(sizeof(double) * (size_t)n);
  int64_t *ix = (int64_t *)malloc(sizeof(int64_t) * (size_t)n);
  for (int64_t i = 0; i < n; ++i) {
    int64_t s = it[i].slot;
    for (int k = 0; k < 3; ++k) x[3 * i + k] = c->x[3 * s + k];
    m[i] = c->m[s];
    ix[i] = c->idx[s];
  }
  memcpy(c->x + 3 * f, x, sizeof(double) * 3 * (size_t)n);
  memcpy(c->m + f, m, sizeof(double) * (size_t)n);
  memcpy(c->idx + f, ix, sizeof(int64_t) * (size_t)n);
  free(it); free(x); free(m); free(ix);
}

static void push_kd(orc_kd *c, int lev, int64_t first, int64_t count) {
  if (c->nnodes == c->ncap) {
    c->ncap = c->ncap ? 2 * c->ncap : 1024;
    c->lev = (int *)realloc(c->lev, sizeof(int) * c->ncap);
    c->axis = (int *)realloc(c->axis, sizeof(int) * c->ncap);
    c->first = (int64_t *)realloc(c->first, sizeof(int64_t) * c->ncap);
    c->count = (int64_t *)realloc(c->count, sizeof(int64_t) * c->ncap);
    c->child = (int64_t *)realloc(c->child, sizeof(int64_t) * c->ncap);
    c->lo = (double *)realloc(c->lo, sizeof(double) * 3 * c->ncap);
    c->hi = (double *)realloc(c->hi, sizeof(double) * 3 * c->ncap);
  }
  int64_t k = c->nnodes++;
  c->lev[k] = lev; c->axis[k] = -1;
  c->first[k] = first; c->count[k] = count; c->child[k] = -1;
}

/* Wrap the positions and build the tree (the readings in the header).  pos is SoA [3][n]. */
int orc_kd_build(orc_kd *c, int64_t n, const double *pos, const double *mass) {
  if (!c || n < 0) return -1;
  free(c->x); free(c->m); free(c->idx);
  c->x = NULL; c->m = NULL; c->idx = NULL;
  c->nnodes = 0; c->nlevels = 0; c->np2p = 0; c->nm2l = 0;
  c->n = n;
  if (n == 0) return 0;
  c->x = (double *)malloc(sizeof(double) * 3 * n);
  c->m = (double *)malloc(sizeof(double) * n);
  c->idx = (int64_t *)malloc(sizeof(int64_t) * n);
  for (int64_t i = 0; i < n; ++i) {
    for (int d = 0; d < 3; ++d) c->x[3 * i + d] = kd_wrap(pos[d * n + i], c->box);
    c->m[i] = mass[i];
    c->idx[i] = i;
  }
  push_kd(c, 0, 0, n);
  c->level_start[0] = 0;
  int lev = 0;
  for (;;) {
    if (lev >= KD_MAXLEV) return -2;
    int64_t lo = c->level_start[lev], hi = c->nnodes;
    c->level_start[lev + 1] = hi;
    for (int64_t k = lo; k < hi; ++k) {
      int64_t f = c->first[k], cnt = c->count[k];
      for (int d = 0; d < 3; ++d) {
        double a = c->x[3 * f + d], b = a;
        for (int64_t i = f + 1; i < f + cnt; ++i) {
          double v = c->x[3 * i + d];
          if (v < a) a = v;
          if (v > b) b = v;
        }
        c->lo[3 * k + d] = a;
        c->hi[3 * k + d] = b;
      }
      if (cnt <= c->leaf_max) continue;
      int ax = 0;
      double best = c->hi[3 * k] - c->lo[3 * k];
      for (int d = 1; d < 3; ++d) {
        double e = c->hi[3 * k + d] - c->lo[3 * k + d];
        if (e > best) { best = e; ax = d; }
      }
      c->axis[k] = ax;
      sort_range(c, f, cnt, ax);
      c->child[k] = c->nnodes;
      push_kd(c, lev + 1, f, cnt / 2);
      push_kd(c, lev + 1, f + cnt / 2, cnt - cnt / 2);
    }
    ++lev;
    if (c->nnodes == hi) break;
  }
  c->nlevels = lev;
  for (int64_t k = 0; k < c->nnodes; ++k)
    if (c->child[k] < 0) sort_range(c, c->first[k], c->count[k], 0);
  return 0;
}

static void kd_centre(const orc_kd *c, int64_t k, double *z) {
  for (int d = 0; d < 3; ++d) z[d] = 0.5 * (c->lo[3 * k + d] + c->hi[3 * k + d]);
}

static double kd_side(const orc_kd *c, int64_t k) {
  double s = c->hi[3 * k] - c->lo[3 * k];
  for (int d = 1; d < 3; ++d) {
    double e = c->hi[3 * k + d] - c->lo[3 * k + d];
    if (e > s) s = e;
  }
  return s;
}

/* ------------------------------------------------------------------------ */
/* Walk with the three rules of Sec. 2.3 on bounding boxes                   */
/* ------------------------------------------------------------------------ */

static void push3(int64_t **buf, int64_t *n, int64_t *cap, int64_t a, int64_t b, int64_t s) {
  if (*n == *cap) {
    *cap = *cap ? 2 * *cap : 4096;
    *buf = (int64_t *)realloc(*buf, sizeof(int64_t) * 3 * *cap);
  }
  (*buf)[3 * *n] = a; (*buf)[3 * *n + 1] = b; (*buf)[3 * *n + 2] = s;
  ++*n;
}

/* 0 skip, 1 M2L, 2 open: sink a, source b shifted by s (index (sx+1)*9+(sy+1)*3+(sz+1)).
 * conventional != 0: the opening-angle test alone (no skip, no transition region),
 * the acceptance of a conventional FMM (Sec. 3). */
static int kd_classify(const orc_kd *c, int64_t a, int64_t b, int s, int conventional) {
  const int sh[3] = {s / 9 - 1, (s / 3) % 3 - 1, s % 3 - 1};
  double sc2 = 0.0, sm2 = 0.0, sx2 = 0.0;
  for (int d = 0; d < 3; ++d) {
    double ca = 0.5 * (c->lo[3 * a + d] + c->hi[3 * a + d]);
    double cb = 0.5 * (c->lo[3 * b + d] + c->hi[3 * b + d]);
    double ea = 0.5 * (c->hi[3 * a + d] - c->lo[3 * a + d]);
    double eb = 0.5 * (c->hi[3 * b + d] - c->lo[3 * b + d]);
    double dc = (cb + (double)sh[d] * c->box) - ca;
    double ad = fabs(dc);
    double w = ea + eb;
    double gap = ad - w;
    if (gap < 0.0) gap = 0.0;
    double far = ad + w;
    sc2 = sc2 + dc * dc;
    sm2 = sm2 + gap * gap;
    sx2 = sx2 + far * far;
  }
  const double rc2 = c->rc * c->rc;
  if (!conventional && sm2 > rc2) return 0;
  int trans = conventional ? 0 : c->rule == 0 ? (sc2 > rc2) : (sx2 > rc2);
  double sa = kd_side(c, a), sb = kd_side(c, b);
  double wl = c->size_rule == 0 ? sb : (sa > sb ? sa : sb);
  const double lim = (c->theta * c->theta) * sc2; /* theta^2 S_c^2; a pair with theta S_c = 0 is never accepted */
  if (!trans && lim > 0.0 && wl * wl <= lim) return 1;
  return 2;
}

/* Dual walk from the root against its 27 nearest periodic images (R_c < L / 2);
 * conventional: the walk of a conventional FMM, from the single pair (root, root)
 * of the primary box (its periodic images go to an Ewald sum, Sec. 3). */
static int kd_walk(orc_kd *c, int conventional) {
  if (!c) return -1;
  c->np2p = 0; c->nm2l = 0;
  if (c->n == 0) return 0;
  int64_t *stk = NULL, nst = 0, cst = 0;
  if (conventional)
    push3(&stk, &nst, &cst, 0, 0, 13);
  else
    for (int s = 0; s < 27; ++s) push3(&stk, &nst, &cst, 0, 0, s);
  while (nst > 0) {
    --nst;
    int64_t a = stk[3 * nst], b = stk[3 * nst + 1];
    int s = (int)stk[3 * nst + 2];
    int cls = kd_classify(c, a, b, s, conventional);
    if (cls == 0) continue;
    if (cls == 1) {
      push3(&c->m2l, &c->nm2l, &c->cap_m2l, a, b, s);
      continue;
    }
    int leafa = c->child[a] < 0, leafb = c->child[b] < 0;
    if (leafa && leafb) {
      push3(&c->p2p, &c->np2p, &c->cap_p2p, a, b, s);
      continue;
    }
    int opena, openb;
    if (leafa) { opena = 0; openb = 1; }
    else if (leafb) { opena = 1; openb = 0; }
    else {
      double sa = kd_side(c, a), sb = kd_side(c, b);
      opena = sa >= sb;
      openb = sb >= sa;
    }
    int64_t a0 = opena ? c->child[a] : a, a1 = opena ? a0 + 2 : a + 1;
    int64_t b0 = openb ? c->child[b] : b, b1 = openb ? b0 + 2 : b + 1;
    for (int64_t x = a0; x < a1; ++x)
      for (int64_t y = b0; y < b1; ++y) push3(&stk, &nst, &cst, x, y, s);
  }
  free(stk);
  return 0;
}

int orc_kd_traverse(orc_kd *c) { return kd_walk(c, 0); }

/* The conventional walk: replaces the lists; for interaction counts only. */
int orc_kd_traverse_conventional(orc_kd *c) { return kd_walk(c, 1); }

/* ------------------------------------------------------------------------ */
/* FMM passes (Sec. 2.1 order), the same operators as the octree             */
/* ------------------------------------------------------------------------ */

static void kd_shift(int s, double box, double *v) {
  v[0] = (s / 9 - 1) * box;
  v[1] = ((s / 3) % 3 - 1) * box;
  v[2] = (s % 3 - 1) * box;
}

static int cmp_triple(const void *a, const void *b) {
  const int64_t *x = (const int64_t *)a, *y = (const int64_t *)b;
  for (int i = 0; i < 3; ++i)
    if (x[i] != y[i]) return x[i] < y[i] ? -1 : 1;
  return 0;
}

static int64_t *by_sink(int64_t *list, int64_t n, int64_t nnodes) {
  qsort(list, (size_t)n, 3 * sizeof(int64_t), cmp_triple);
  int64_t *off = (int64_t *)calloc((size_t)nnodes + 1, sizeof(int64_t));
  for (int64_t t = 0; t < n; ++t) off[list[3 * t] + 1]++;
  for (int64_t k = 0; k < nnodes; ++k) off[k + 1] += off[k];
  return off;
}

/* P2M at the leaves, M2M to the parents (Eqs. p2m, m2m), about the box centres. */
int orc_kd_upward(orc_kd *c) {
  if (!c) return -1;
  int nc = orc_ncoef(c->p);
  free(c->M);
  c->M = (double *)calloc((size_t)(c->nnodes ? c->nnodes : 1) * nc, sizeof(double));
  for (int l = c->nlevels - 1; l >= 0; --l) {
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t k = c->level_start[l]; k < c->level_start[l + 1]; ++k) {
      double z[3];
      kd_centre(c, k, z);
      if (c->child[k] < 0) {
        orc_p2m(c->count[k], c->x + 3 * c->first[k], c->m + c->first[k], z, c->p, c->M + k * nc);
      } else {
        double tmp[KD_NCMAX];
        for (int64_t ch = c->child[k]; ch < c->child[k] + 2; ++ch) {
          double zc[3], x[3];
          kd_centre(c, ch, zc);
          for (int d = 0; d < 3; ++d) x[d] = z[d] - zc[d];
          orc_m2m(c->M + ch * nc, x, c->p, tmp);
          for (int e = 0; e < nc; ++e) c->M[k * nc + e] += tmp[e];
        }
      }
    }
  }
  return 0;
}

/* M2L over the accepted pairs (Eq. m2l), R = c_A - (c_B + s L). */
int orc_kd_m2l_pass(orc_kd *c) {
  if (!c || !c->M) return -1;
  int nc = orc_ncoef(c->p);
  free(c->L);
  c->L = (double *)calloc((size_t)(c->nnodes ? c->nnodes : 1) * nc, sizeof(double));
  int64_t *off = by_sink(c->m2l, c->nm2l, c->nnodes);
#pragma omp parallel for schedule(dynamic, 16)
  for (int64_t a = 0; a < c->nnodes; ++a) {
    double za[3];
    kd_centre(c, a, za);
    for (int64_t t = off[a]; t < off[a + 1]; ++t) {
      int64_t b = c->m2l[3 * t + 1];
      double zb[3], sv[3], R[3];
      kd_centre(c, b, zb);
      kd_shift((int)c->m2l[3 * t + 2], c->box, sv);
      for (int d = 0; d < 3; ++d) R[d] = za[d] - (zb[d] + sv[d]);
      orc_m2l_split(c->M + b * nc, R, c->rs, c->rc, c->split, c->p, c->L + a * nc);
    }
  }
  free(off);
  return 0;
}

/* L2L to the children, L2P at the leaves (Eqs. l2l, l2p); acc_tree [n][3] is overwritten. */
int orc_kd_downward(orc_kd *c, double *acc_tree) {
  if (!c || !c->L) return -1;
  int nc = orc_ncoef(c->p);
  for (int l = 0; l < c->nlevels; ++l) {
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t k = c->level_start[l]; k < c->level_start[l + 1]; ++k) {
      double z[3];
      kd_centre(c, k, z);
      if (c->child[k] >= 0) {
        double tmp[KD_NCMAX];
        for (int64_t ch = c->child[k]; ch < c->child[k] + 2; ++ch) {
          double zc[3], x[3];
          kd_centre(c, ch, zc);
          for (int d = 0; d < 3; ++d) x[d] = zc[d] - z[d];
          orc_l2l(c->L + k * nc, x, c->p, tmp);
          for (int e = 0; e < nc; ++e) c->L[ch * nc + e] += tmp[e];
        }
      } else {
        for (int64_t i = c->first[k]; i < c->first[k] + c->count[k]; ++i) {
          double u[3];
          for (int d = 0; d < 3; ++d) u[d] = c->x[3 * i + d] - z[d];
          orc_l2p(c->L + k * nc, u, c->p, c->G, NULL, acc_tree + 3 * i);
        }
      }
    }
  }
  return 0;
}

/* P2P over the leaf pairs with the hard cut-off 0 < |r| < R_c (Sec. 2.2 force); adds into acc_tree. */
int orc_kd_p2p_pass(orc_kd *c, double *acc_tree) {
  if (!c) return -1;
  int64_t *off = by_sink(c->p2p, c->np2p, c->nnodes);
  const double rc2 = c->rc * c->rc;
#pragma omp parallel for schedule(dynamic, 16)
  for (int64_t a = 0; a < c->nnodes; ++a) {
    for (int64_t t = off[a]; t < off[a + 1]; ++t) {
      int64_t b = c->p2p[3 * t + 1];
      double sv[3];
      kd_shift((int)c->p2p[3 * t + 2], c->box, sv);
      for (int64_t i = c->first[a]; i < c->first[a] + c->count[a]; ++i) {
        double acc[3] = {0, 0, 0};
        for (int64_t j = c->first[b]; j < c->first[b] + c->count[b]; ++j) {
          double d[3];
          for (int k = 0; k < 3; ++k) d[k] = c->x[3 * i + k] - (c->x[3 * j + k] + sv[k]);
          double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
          if (!(r2 > 0.0) || !(r2 < rc2)) continue;
          double f[2];
          if (c->split == 1)
            orc_prefactors_poly(sqrt(r2), c->rc, 1, f);
          else
            orc_prefactors(sqrt(r2), c->rs, 1, f);
          for (int k = 0; k < 3; ++k) acc[k] += c->m[j] * f[1] * d[k];
        }
        for (int k = 0; k < 3; ++k) acc_tree[3 * i + k] += c->G * acc[k];
      }
    }
  }
  free(off);
  return 0;
}

/* Whole short-range FMM on the k-d tree; acc is SoA [3][n] in input order. */
int orc_kd_forces(orc_kd *c, double *acc) {
  if (!c) return -1;
  int64_t n = c->n;
  if (n == 0) return 0;
  double *as = (double *)calloc((size_t)3 * n, sizeof(double));
  int rc = orc_kd_traverse(c);
  if (!rc) rc = orc_kd_upward(c);
  if (!rc) rc = orc_kd_m2l_pass(c);
  if (!rc) rc = orc_kd_downward(c, as);
  if (!rc) rc = orc_kd_p2p_pass(c, as);
  if (!rc)
    for (int64_t s = 0; s < n; ++s)
      for (int d = 0; d < 3; ++d) acc[d * n + c->idx[s]] = as[3 * s + d];
  free(as);
  return rc;
}

/* ------------------------------------------------------------------------ */
/* Export                                                                    */
/* ------------------------------------------------------------------------ */

/* what: 0 n, 1 nodes, 2 levels, 3 P2P entries, 4 M2L entries */
int64_t orc_kd_size(const orc_kd *c, int what) {
  switch (what) {
    case 0: return c->n;
    case 1: return c->nnodes;
    case 2: return c->nlevels;
    case 3: return c->np2p;
    case 4: return c->nm2l;
  }
  return -1;
}

/* nodes [nnodes][5] i64: level, first, count, first child (-1 leaf), split axis (-1 leaf);
 * boxes [nnodes][6] f64: lo x y z, hi x y z; perm [n] i64: input index in tree order */
int orc_kd_export(const orc_kd *c, int64_t *nodes, double *boxes, int64_t *perm) {
  for (int64_t k = 0; k < c->nnodes; ++k) {
    if (nodes) {
      int64_t *o = nodes + 5 * k;
      o[0] = c->lev[k]; o[1] = c->first[k]; o[2] = c->count[k]; o[3] = c->child[k]; o[4] = c->axis[k];
    }
    if (boxes)
      for (int d = 0; d < 3; ++d) {
        boxes[6 * k + d] = c->lo[3 * k + d];
        boxes[6 * k + 3 + d] = c->hi[3 * k + d];
      }
  }
  if (perm) memcpy(perm, c->idx, sizeof(int64_t) * (size_t)c->n);
  return 0;
}

/* which = 0: P2P list, 1: M2L list; [len][3] i64 (sink, source, shift index) */
int orc_kd_export_list(const orc_kd *c, int which, int64_t *out) {
  int64_t n = which ? c->nm2l : c->np2p;
  memcpy(out, which ? c->m2l : c->p2p, sizeof(int64_t) * 3 * (size_t)n);
  return 0;
}

/* Replace the lists (the walk of another implementation), for forces on given lists. */
int orc_kd_set_lists(orc_kd *c, const int64_t *p2p, int64_t np2p, const int64_t *m2l, int64_t nm2l) {
  if (!c || np2p < 0 || nm2l < 0) return -1;
  for (int64_t t = 0; t < np2p; ++t)
    if (p2p[3 * t] < 0 || p2p[3 * t] >= c->nnodes || p2p[3 * t + 1] < 0 || p2p[3 * t + 1] >= c->nnodes ||
        p2p[3 * t + 2] < 0 || p2p[3 * t + 2] > 26)
      return -1;
  for (int64_t t = 0; t < nm2l; ++t)
    if (m2l[3 * t] < 0 || m2l[3 * t] >= c->nnodes || m2l[3 * t + 1] < 0 || m2l[3 * t + 1] >= c->nnodes ||
        m2l[3 * t + 2] < 0 || m2l[3 * t + 2] > 26)
      return -1;
  free(c->p2p); free(c->m2l);
  c->p2p = (int64_t *)malloc(sizeof(int64_t) * 3 * (size_t)(np2p ? np2p : 1));
  c->m2l = (int64_t *)malloc(sizeof(int64_t) * 3 * (size_t)(nm2l ? nm2l : 1));
  memcpy(c->p2p, p2p, sizeof(int64_t) * 3 * (size_t)np2p);
  memcpy(c->m2l, m2l, sizeof(int64_t) * 3 * (size_t)nm2l);
  c->np2p = c->cap_p2p = np2p;
  c->nm2l = c->cap_m2l = nm2l;
  if (c->cap_p2p == 0) c->cap_p2p = 1;
  if (c->cap_m2l == 0) c->cap_m2l = 1;
  return 0;
}

/* FMM forces on the current lists (no walk); acc SoA [3][n] in input order. */
int orc_kd_forces_given_lists(orc_kd *c, double *acc) {
  if (!c) return -1;
  int64_t n = c->n;
  if (n == 0) return 0;
  double *as = (double *)calloc((size_t)3 * n, sizeof(double));
  int rc = orc_kd_upward(c);
  if (!rc) rc = orc_kd_m2l_pass(c);
  if (!rc) rc = orc_kd_downward(c, as);
  if (!rc) rc = orc_kd_p2p_pass(c, as);
  if (!rc)
    for (int64_t s = 0; s < n; ++s)
      for (int d = 0; d < 3; ++d) acc[d * n + c->idx[s]] = as[3 * s + d];
  free(as);
  return rc;
}
