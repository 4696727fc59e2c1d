/*
 * FP64 CPU oracle for the Gaussian-truncated short-range FMM of
 * "A Hybrid Fast Multipole Method for Cosmological N-body Simulations" (Wang).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, plain, obviously-correct
 * statement of what the GPU library computes.  Only the test-suite, the smoke
 * check and the benchmark's CPU-baseline leg may load it.  It shares no code,
 * header, table or constant generator with the CUDA library.
 *
 * Contents, each with the passage it follows:
 *   - prefactors f_(k)(r) of the split kernel           Sec. 2.2, general-order equation
 *     (Newtonian f~_(k) as the r_s -> infinity limit)   Sec. 2.1, Eq. pref
 *   - derivative tensor D_n = grad^n psi_SR             Sec. 2.1 (after Eq. m2l), Sec. 2.2
 *   - P2M, M2M, M2L, L2L, L2P                           Eqs. p2m, m2m, m2l, l2l, l2p
 *   - direct truncated pair sum a = G sum m f_(1) r     Sec. 2.2, force equation g(r)
 *   - Morton-key octree with a leaf limit               Sec. 2.1 (leaf limiter)
 *   - dual-tree traversal with the three-rule MAC       Sec. 2.3, itemised criteria
 *   - the conventional-FMM walk the interaction counts  Sec. 3 (Figs. 5-6): the second
 *     are compared against                                criterion alone, from (root, root)
 *   - P2P with the hard cutoff                          Sec. 2.1 (P2P), Sec. 2.2
 *
 * Readings where the paper is silent or garbled:
 *   D_n uses erfc(r/2r_s) (the factor 2 of the potential equation), is NOT
 *   traceless, and is built from the radial derivatives f_(k) = ((1/r) d/dr)^k psi;
 *   expansion centres are geometric; total order |n|+|m| <= p; the MAC compares
 *   exact integer squared distances in units of L/2^22 against an FP64 threshold.
 *
 * Multi-index order (shared *format*, not code, with the GPU library): graded,
 * for k = 0..p, nx = k..0, ny = k-nx..0, nz = k-nx-ny.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_PMAX 10
#define ORC_NCMAX 286 /* C(ORC_PMAX+3,3) */
#define ORC_DEPTH 21
#define ORC_PI 3.14159265358979323846

static int g_mi[ORC_NCMAX][3];
static int g_idx[ORC_PMAX + 1][ORC_PMAX + 1][ORC_PMAX + 1];
static double g_fact[2 * ORC_PMAX + 2];

__attribute__((constructor)) static void orc_tables(void) {
  int c = 0;
  for (int k = 0; k <= ORC_PMAX; ++k)
    for (int nx = k; nx >= 0; --nx)
      for (int ny = k - nx; ny >= 0; --ny) {
        int nz = k - nx - ny;
        g_mi[c][0] = nx;
        g_mi[c][1] = ny;
        g_mi[c][2] = nz;
        g_idx[nx][ny][nz] = c;
        ++c;
      }
  g_fact[0] = 1.0;
  for (int i = 1; i < 2 * ORC_PMAX + 2; ++i) g_fact[i] = g_fact[i - 1] * i;
}

int orc_ncoef(int p) { return (p + 1) * (p + 2) * (p + 3) / 6; }

int orc_multi_index(int c, int *n3) {
  if (c < 0 || c >= ORC_NCMAX) return -1;
  n3[0] = g_mi[c][0];
  n3[1] = g_mi[c][1];
  n3[2] = g_mi[c][2];
  return 0;
}

static double dfact(int k) { /* k!! with (-1)!! = 0!! = 1 */
  double r = 1.0;
  for (int i = k; i > 1; i -= 2) r *= i;
  return r;
}

static double ipow(double x, int e) {
  double r = 1.0;
  for (int i = 0; i < e; ++i) r *= x;
  return r;
}

static double mpow(const double *x, const int *n) { /* x^n for a multi-index */
  return ipow(x[0], n[0]) * ipow(x[1], n[1]) * ipow(x[2], n[2]);
}

static double mfact(const int *n) { return g_fact[n[0]] * g_fact[n[1]] * g_fact[n[2]]; }

/* ------------------------------------------------------------------------ */
/* Prefactors.                                                               */
/* ------------------------------------------------------------------------ */

/*
 * f_(k)(r) for k = 0..p.  rs > 0: the closed form of Sec. 2.2 (general order),
 *   (-1)^k rs^(2k+1) f_(k) = (2k-1)!!/x^(2k+1) erfc(x/2)
 *                          + sum_{q=1..k} 2^(q-k) (2k-1)!!/(2k-2q+1)!! e^(-x^2/4)/(sqrt(pi) x^(2q)),
 *   x = r/rs.
 * rs <= 0: the Newtonian prefactors of Eq. pref, f~_(k) = (-1)^k (2k-1)!!/r^(2k+1).
 */
int orc_prefactors(double r, double rs, int p, double *f) {
  if (p < 0 || p > 2 * ORC_PMAX || !(r > 0.0)) return -1;
  if (rs <= 0.0) {
    for (int k = 0; k <= p; ++k) {
      double v = dfact(2 * k - 1) / ipow(r, 2 * k + 1);
      f[k] = (k & 1) ? -v : v;
    }
    return 0;
  }
  double x = r / rs;
  double g = exp(-x * x / 4.0) / sqrt(ORC_PI);
  double ec = erfc(x / 2.0);
  for (int k = 0; k <= p; ++k) {
    double df = dfact(2 * k - 1);
    double s = df / ipow(x, 2 * k + 1) * ec;
    for (int q = 1; q <= k; ++q) s += ldexp(1.0, q - k) * df / dfact(2 * k - 2 * q + 1) * g / ipow(x, 2 * q);
    double v = s / ipow(rs, 2 * k + 1);
    f[k] = (k & 1) ? -v : v;
  }
  return 0;
}

/*
 * The polynomial truncation of the split that Sec. 5 allows in place of the
 * Gaussian one (the paper names no polynomial; the reading taken is the even
 * quartic for which the kernel and its first two derivatives vanish at R_c):
 *   psi(r) = 1/r - P(r) for 0 < r < R_c,  P(r) = (15 - 10 w^2 + 3 w^4) / (8 R_c),  w = r / R_c.
 * Its prefactors f_(k) = ((1/r) d/dr)^k psi are the Newtonian ones minus those
 * of P, which vanish beyond k = 2:
 *   P_(0) = P,  P_(1) = (-5/2 + 3 w^2 / 2) / R_c^3,  P_(2) = 3 / R_c^5.
 */
int orc_prefactors_poly(double r, double rc, int p, double *f) {
  if (p < 0 || p > 2 * ORC_PMAX || !(r > 0.0) || !(rc > 0.0)) return -1;
  for (int k = 0; k <= p; ++k) {
    double v = dfact(2 * k - 1) / ipow(r, 2 * k + 1);
    f[k] = (k & 1) ? -v : v;
  }
  const double w2 = (r / rc) * (r / rc);
  f[0] -= (15.0 - 10.0 * w2 + 3.0 * w2 * w2) / (8.0 * rc);
  if (p >= 1) f[1] -= (-2.5 + 1.5 * w2) / ipow(rc, 3);
  if (p >= 2) f[2] -= 3.0 / ipow(rc, 5);
  return 0;
}

/* The short-range kernel in use: split 0 = erfc(r / 2 r_s) / r (Sec. 2.2; the
 * Newtonian 1/r when rs <= 0), split 1 = the polynomial truncation above. */
typedef struct {
  double rs, rc;
  int split;
} orc_kernel;

static int prefactors_k(double r, const orc_kernel *K, int p, double *f) {
  return K->split == 1 ? orc_prefactors_poly(r, K->rc, p, f) : orc_prefactors(r, K->rs, p, f);
}

/*
 * D_n(R) = d^n psi(R) for all |n| <= p (graded order), psi the kernel K.
 * Derivative of a radial function:
 *   d^n psi = sum_{k_d <= n_d/2} prod_d [ n_d! / (2^k_d k_d! (n_d-2k_d)!) R_d^(n_d-2k_d) ] f_(|n|-|k|)(r).
 */
static int deriv_tensor_k(const double *R, const orc_kernel *K, int p, double *D) {
  if (p < 0 || p > ORC_PMAX) return -1;
  double r = sqrt(R[0] * R[0] + R[1] * R[1] + R[2] * R[2]);
  double f[2 * ORC_PMAX + 1];
  if (prefactors_k(r, K, p, f)) return -1;
  int nc = orc_ncoef(p);
  for (int c = 0; c < nc; ++c) {
    const int *n = g_mi[c];
    int nn = n[0] + n[1] + n[2];
    double sum = 0.0;
    for (int kx = 0; 2 * kx <= n[0]; ++kx)
      for (int ky = 0; 2 * ky <= n[1]; ++ky)
        for (int kz = 0; 2 * kz <= n[2]; ++kz) {
          int k[3] = {kx, ky, kz};
          double coef = 1.0;
          for (int d = 0; d < 3; ++d)
            coef *= g_fact[n[d]] / (ldexp(1.0, k[d]) * g_fact[k[d]] * g_fact[n[d] - 2 * k[d]]) *
                    ipow(R[d], n[d] - 2 * k[d]);
          sum += coef * f[nn - kx - ky - kz];
        }
    D[c] = sum;
  }
  return 0;
}

/* D_n of psi = erfc(r/2rs)/r (Newtonian 1/r if rs <= 0). */
int orc_deriv_tensor(const double *R, double rs, int p, double *D) {
  const orc_kernel K = {rs, 0.0, 0};
  return deriv_tensor_k(R, &K, p, D);
}

/* D_n of the kernel of the given split (0 Gaussian with rs, 1 polynomial with rc). */
int orc_deriv_tensor_split(const double *R, double rs, double rc, int split, int p, double *D) {
  const orc_kernel K = {rs, rc, split};
  return deriv_tensor_k(R, &K, p, D);
}

/* ------------------------------------------------------------------------ */
/* Expansion operators on one cell (Sec. 2.1).                              */
/* ------------------------------------------------------------------------ */

/* Eq. p2m: M_m(z) = sum_a mu_a (-1)^|m| / m! (x_a - z)^m, |m| <= p.  x is [n][3]. */
int orc_p2m(int64_t n, const double *x, const double *mu, const double *z, int p, double *M) {
  int nc = orc_ncoef(p);
  for (int c = 0; c < nc; ++c) M[c] = 0.0;
  for (int64_t a = 0; a < n; ++a) {
    double d[3] = {x[3 * a] - z[0], x[3 * a + 1] - z[1], x[3 * a + 2] - z[2]};
    for (int c = 0; c < nc; ++c) {
      const int *m = g_mi[c];
      double sg = ((m[0] + m[1] + m[2]) & 1) ? -1.0 : 1.0;
      M[c] += mu[a] * sg / mfact(m) * mpow(d, m);
    }
  }
  return 0;
}

/* Eq. m2m: M_m(z + x) = sum_{n <= m} x^n / n! M_{m-n}(z).  Mout is overwritten. */
int orc_m2m(const double *Min, const double *x, int p, double *Mout) {
  int nc = orc_ncoef(p);
  for (int c = 0; c < nc; ++c) {
    const int *m = g_mi[c];
    double s = 0.0;
    for (int nx = 0; nx <= m[0]; ++nx)
      for (int ny = 0; ny <= m[1]; ++ny)
        for (int nz = 0; nz <= m[2]; ++nz) {
          int nn[3] = {nx, ny, nz};
          s += mpow(x, nn) / mfact(nn) * Min[g_idx[m[0] - nx][m[1] - ny][m[2] - nz]];
        }
    Mout[c] = s;
  }
  return 0;
}

/* Eq. m2l: L_n += sum_{|m| <= p-|n|} M_m D_{n+m}(R), R = z_sink - z_source. */
static int m2l_k(const double *M, const double *R, const orc_kernel *K, int p, double *L) {
  double D[ORC_NCMAX];
  if (deriv_tensor_k(R, K, p, D)) return -1;
  int nc = orc_ncoef(p);
  for (int c = 0; c < nc; ++c) {
    const int *n = g_mi[c];
    int rem = p - (n[0] + n[1] + n[2]);
    double s = 0.0;
    for (int e = 0; e < orc_ncoef(rem); ++e) {
      const int *m = g_mi[e];
      s += M[e] * D[g_idx[n[0] + m[0]][n[1] + m[1]][n[2] + m[2]]];
    }
    L[c] += s;
  }
  return 0;
}

int orc_m2l(const double *M, const double *R, double rs, int p, double *L) {
  const orc_kernel K = {rs, 0.0, 0};
  return m2l_k(M, R, &K, p, L);
}

/* The same for the kernel of a given split (0 Gaussian with rs, 1 polynomial with rc). */
int orc_m2l_split(const double *M, const double *R, double rs, double rc, int split, int p, double *L) {
  const orc_kernel K = {rs, rc, split};
  return m2l_k(M, R, &K, p, L);
}

/* Eq. l2l: L_n(z + x) = sum_{|m| <= p-|n|} x^m / m! L_{m+n}(z).  Lout is overwritten. */
int orc_l2l(const double *Lin, const double *x, int p, double *Lout) {
  int nc = orc_ncoef(p);
  for (int c = 0; c < nc; ++c) {
    const int *n = g_mi[c];
    int rem = p - (n[0] + n[1] + n[2]);
    double s = 0.0;
    for (int e = 0; e < orc_ncoef(rem); ++e) {
      const int *m = g_mi[e];
      s += mpow(x, m) / mfact(m) * Lin[g_idx[n[0] + m[0]][n[1] + m[1]][n[2] + m[2]]];
    }
    Lout[c] = s;
  }
  return 0;
}

/*
 * Eq. l2p: Psi(z + u) = sum_{|n| <= p} L_n u^n / n!, and its gradient
 * a_i = G dPsi/du_i = G sum_{|n| <= p-1} L_{n+e_i} u^n / n!.
 */
int orc_l2p(const double *L, const double *u, int p, double G, double *phi, double *acc) {
  double ph = 0.0, a[3] = {0, 0, 0};
  for (int c = 0; c < orc_ncoef(p); ++c) {
    const int *n = g_mi[c];
    double t = mpow(u, n) / mfact(n);
    ph += L[c] * t;
    if (n[0] + n[1] + n[2] <= p - 1) {
      a[0] += L[g_idx[n[0] + 1][n[1]][n[2]]] * t;
      a[1] += L[g_idx[n[0]][n[1] + 1][n[2]]] * t;
      a[2] += L[g_idx[n[0]][n[1]][n[2] + 1]] * t;
    }
  }
  if (phi) *phi = G * ph;
  for (int d = 0; d < 3; ++d) acc[d] = G * a[d];
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Periodic wrap and direct truncated sum.                                   */
/* ------------------------------------------------------------------------ */

/* x <- x - L floor(x / L): the particle's image inside the periodic box. */
static double wrap1(double x, double box) {
  double q = floor(x / box);
  double t = box * q;
  return x - t;
}

/* Pair force of Sec. 2.2: G m_j f_(1)(r) r, r = x_i - x_j, kept iff 0 < |r| < rc. */
static void pair_acc(const double *d, double mj, const orc_kernel *K, double rc2, double *acc) {
  double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
  if (!(r2 > 0.0) || !(r2 < rc2)) return;
  double f[2];
  prefactors_k(sqrt(r2), K, 1, f);
  for (int k = 0; k < 3; ++k) acc[k] += mj * f[1] * d[k];
}

/*
 * Direct truncated short-range sum (the quantity the FMM approximates):
 *   a_i = G sum_{j != i, 0 < |r_ij| < rc} m_j f_(1)(|r_ij|) r_ij,
 * r_ij the minimum-image separation x_i - x_j in the periodic box of side L
 * (rc < L/2, so that image is unique).  pos is SoA [3][n]; acc is SoA [3][nsink]
 * for the sinks listed (all particles when sinks == NULL).  A cell list with
 * cells of side >= rc restricts the candidates; it changes no result.
 */
int orc_direct_sr_split(int64_t n, const double *pos, const double *mass, double box, double rs, double rc,
                        int split, double G, int64_t nsink, const int64_t *sinks, double *acc) {
  if (n < 0 || nsink < 0 || !(rc > 0.0) || !(rc < 0.5 * box) || split < 0 || split > 1) return -1;
  const orc_kernel K = {rs, rc, split};
  if (n == 0 || nsink == 0) return 0;
  double *w = (double *)malloc(sizeof(double) * 3 * n);
  int nc = (int)floor(box / rc);
  if (nc < 1) nc = 1;
  if (nc > 256) nc = 256;
  int64_t ncell = (int64_t)nc * nc * nc;
  int64_t *head = (int64_t *)malloc(sizeof(int64_t) * (ncell + 1));
  int64_t *item = (int64_t *)malloc(sizeof(int64_t) * n);
  int64_t *cell = (int64_t *)malloc(sizeof(int64_t) * n);
  if (!w || !head || !item || !cell) {
    free(w); free(head); free(item); free(cell);
    return -2;
  }
  for (int64_t i = 0; i < n; ++i) {
    int64_t ci[3];
    for (int d = 0; d < 3; ++d) {
      w[3 * i + d] = wrap1(pos[d * n + i], box);
      int64_t k = (int64_t)floor(w[3 * i + d] / box * nc);
      if (k < 0) k = 0;
      if (k > nc - 1) k = nc - 1;
      ci[d] = k;
    }
    cell[i] = (ci[0] * nc + ci[1]) * nc + ci[2];
  }
  /* counting sort of particles by cell */
  memset(head, 0, sizeof(int64_t) * (ncell + 1));
  for (int64_t i = 0; i < n; ++i) head[cell[i] + 1]++;
  for (int64_t c = 0; c < ncell; ++c) head[c + 1] += head[c];
  {
    int64_t *fill = (int64_t *)malloc(sizeof(int64_t) * ncell);
    memcpy(fill, head, sizeof(int64_t) * ncell);
    for (int64_t i = 0; i < n; ++i) item[fill[cell[i]]++] = i;
    free(fill);
  }
  double rc2 = rc * rc;
#pragma omp parallel for schedule(dynamic, 16)
  for (int64_t s = 0; s < nsink; ++s) {
    int64_t i = sinks ? sinks[s] : s;
    double a[3] = {0, 0, 0};
    int64_t c0 = cell[i];
    int cz = (int)(c0 % nc), cy = (int)((c0 / nc) % nc), cx = (int)(c0 / ((int64_t)nc * nc));
    /* distinct neighbour cells (fewer than 27 when nc < 3) */
    int64_t nb[27];
    int nnb = 0;
    for (int dx = -1; dx <= 1; ++dx)
      for (int dy = -1; dy <= 1; ++dy)
        for (int dz = -1; dz <= 1; ++dz) {
          int64_t c = ((int64_t)((cx + dx + nc) % nc) * nc + (cy + dy + nc) % nc) * nc + (cz + dz + nc) % nc;
          int seen = 0;
          for (int t = 0; t < nnb; ++t) seen |= (nb[t] == c);
          if (!seen) nb[nnb++] = c;
        }
    for (int t = 0; t < nnb; ++t)
      for (int64_t q = head[nb[t]]; q < head[nb[t] + 1]; ++q) {
        int64_t j = item[q];
        double d[3];
        for (int k = 0; k < 3; ++k) {
          double dd = w[3 * i + k] - w[3 * j + k];
          d[k] = dd - box * nearbyint(dd / box);
        }
        pair_acc(d, mass[j], &K, rc2, a);
      }
    for (int k = 0; k < 3; ++k) acc[k * nsink + s] = G * a[k];
  }
  free(w); free(head); free(item); free(cell);
  return 0;
}

int orc_direct_sr(int64_t n, const double *pos, const double *mass, double box, double rs, double rc,
                  double G, int64_t nsink, const int64_t *sinks, double *acc) {
  return orc_direct_sr_split(n, pos, mass, box, rs, rc, 0, G, nsink, sinks, acc);
}

/* ------------------------------------------------------------------------ */
/* Octree (Sec. 2.1: tree with a leaf limiter; a Morton octree here).        */
/* ------------------------------------------------------------------------ */

typedef struct {
  uint64_t key;
  int64_t idx;
} keyidx;

static int cmp_keyidx(const void *a, const void *b) {
  const keyidx *x = (const keyidx *)a, *y = (const keyidx *)b;
  if (x->key != y->key) return x->key < y->key ? -1 : 1;
  return (x->idx > y->idx) - (x->idx < y->idx);
}

/* 63-bit Morton key: bit b of kx, ky, kz goes to bit 3b+2, 3b+1, 3b. */
static uint64_t morton(uint32_t kx, uint32_t ky, uint32_t kz) {
  uint64_t key = 0;
  for (int b = 0; b < ORC_DEPTH; ++b) {
    key |= (uint64_t)((kx >> b) & 1u) << (3 * b + 2);
    key |= (uint64_t)((ky >> b) & 1u) << (3 * b + 1);
    key |= (uint64_t)((kz >> b) & 1u) << (3 * b);
  }
  return key;
}

/* integer cell coordinate on the finest (2^21 per side) grid */
static uint32_t grid_coord(double w, double box) {
  double u = w / box;
  double t = floor(u * 2097152.0);
  if (t < 0.0) t = 0.0;
  if (t > 2097151.0) t = 2097151.0;
  return (uint32_t)t;
}

typedef struct {
  /* parameters */
  double box, rs, rc, G, theta;
  int p, leaf_max, rule, size_rule;
  int split; /* short-range kernel: 0 Gaussian (Sec. 2.2), 1 polynomial (Sec. 5) */
  /* particles, sorted by (key, input index) */
  int64_t n;
  double *x;      /* [n][3] wrapped positions */
  double *m;      /* [n] */
  uint64_t *key;  /* [n] */
  int64_t *perm;  /* [n] input index of sorted particle */
  /* nodes, breadth-first, key order within a level */
  int64_t nnodes, ncap;
  int nlevels;
  int64_t level_start[ORC_DEPTH + 2];
  int *lev;
  uint32_t *ic; /* [nnodes][3] cell coordinate at its level */
  int64_t *first, *count, *child_first;
  int *nchild;
  /* interaction lists: (sink, source, shift index 0..26) */
  int64_t np2p, nm2l, cap_p2p, cap_m2l;
  int64_t *p2p, *m2l;
  /* expansion order of each M2L entry (learned walk only; NULL: every entry has order p) */
  int64_t *m2l_ord, cap_ord;
  /* expansions [nnodes][ncoef(p)] */
  double *M, *L;
  /* MAC thresholds */
  double rc2h, theta2;
} orc_ctx;

void orc_destroy(orc_ctx *c) {
  if (!c) return;
  free(c->x); free(c->m); free(c->key); free(c->perm);
  free(c->lev); free(c->ic); free(c->first); free(c->count); free(c->child_first); free(c->nchild);
  free(c->p2p); free(c->m2l); free(c->m2l_ord); free(c->M); free(c->L);
  free(c);
}

/*
 * rule: 0 = transition region S_c > R_c > S_m (as printed), 1 = S_max > R_c > S_m.
 * size_rule: the length L in theta = L / S_c; 0 = side of the source cell (as
 * printed), 1 = the larger side of the two cells.
 */
orc_ctx *orc_create(double box, double rs, double rc, double G, double theta, int p, int leaf_max, int rule,
                    int size_rule) {
  if (!(box > 0) || !(rs > 0) || !(rc > 0) || !(rc < 0.5 * box) || p < 1 || p > ORC_PMAX || leaf_max < 1 ||
      (rule != 0 && rule != 1) || (size_rule != 0 && size_rule != 1) || !(theta >= 0))
    return NULL;
  orc_ctx *c = (orc_ctx *)calloc(1, sizeof(orc_ctx));
  c->box = box; c->rs = rs; c->rc = rc; c->G = G; c->theta = theta;
  c->p = p; c->leaf_max = leaf_max; c->rule = rule; c->size_rule = size_rule;
  double t = rc * 4194304.0;
  t = t / box;
  c->rc2h = t * t;
  c->theta2 = theta * theta;
  return c;
}

/* Short-range kernel of the FMM and its direct sums: 0 Gaussian, 1 polynomial (Sec. 5). */
int orc_set_split(orc_ctx *c, int split) {
  if (!c || split < 0 || split > 1) return -1;
  c->split = split;
  return 0;
}

static void push_node(orc_ctx *c, int lev, uint32_t ix, uint32_t iy, uint32_t iz, int64_t first, int64_t count) {
  if (c->nnodes == c->ncap) {
    c->ncap = c->ncap ? 2 * c->ncap : 1024;
    c->lev = (int *)realloc(c->lev, sizeof(int) * c->ncap);
    c->ic = (uint32_t *)realloc(c->ic, sizeof(uint32_t) * 3 * c->ncap);
    c->first = (int64_t *)realloc(c->first, sizeof(int64_t) * c->ncap);
    c->count = (int64_t *)realloc(c->count, sizeof(int64_t) * c->ncap);
    c->child_first = (int64_t *)realloc(c->child_first, sizeof(int64_t) * c->ncap);
    c->nchild = (int *)realloc(c->nchild, sizeof(int) * c->ncap);
  }
  int64_t k = c->nnodes++;
  c->lev[k] = lev;
  c->ic[3 * k] = ix; c->ic[3 * k + 1] = iy; c->ic[3 * k + 2] = iz;
  c->first[k] = first; c->count[k] = count;
  c->child_first[k] = -1; c->nchild[k] = 0;
}

/*
 * Wrap, key, sort and build the octree.  A cell is split into its non-empty
 * octants while it holds more than leaf_max particles and its level is below 21.
 * pos is SoA [3][n].
 */
int orc_build_tree(orc_ctx *c, int64_t n, const double *pos, const double *mass) {
  if (!c || n < 0) return -1;
  free(c->x); free(c->m); free(c->key); free(c->perm);
  c->x = NULL; c->m = NULL; c->key = NULL; c->perm = NULL;
  c->nnodes = 0; c->nlevels = 0; c->np2p = 0; c->nm2l = 0;
  c->n = n;
  if (n == 0) return 0;
  keyidx *ki = (keyidx *)malloc(sizeof(keyidx) * n);
  double *w = (double *)malloc(sizeof(double) * 3 * n);
  for (int64_t i = 0; i < n; ++i) {
    uint32_t k3[3];
    for (int d = 0; d < 3; ++d) {
      w[3 * i + d] = wrap1(pos[d * n + i], c->box);
      k3[d] = grid_coord(w[3 * i + d], c->box);
    }
    ki[i].key = morton(k3[0], k3[1], k3[2]);
    ki[i].idx = i;
  }
  qsort(ki, (size_t)n, sizeof(keyidx), cmp_keyidx);
  c->x = (double *)malloc(sizeof(double) * 3 * n);
  c->m = (double *)malloc(sizeof(double) * n);
  c->key = (uint64_t *)malloc(sizeof(uint64_t) * n);
  c->perm = (int64_t *)malloc(sizeof(int64_t) * n);
  for (int64_t s = 0; s < n; ++s) {
    int64_t i = ki[s].idx;
    for (int d = 0; d < 3; ++d) c->x[3 * s + d] = w[3 * i + d];
    c->m[s] = mass[i];
    c->key[s] = ki[s].key;
    c->perm[s] = i;
  }
  free(ki); free(w);

  push_node(c, 0, 0, 0, 0, 0, n);
  c->level_start[0] = 0;
  int lev = 0;
  for (;;) {
    int64_t lo = c->level_start[lev], hi = c->nnodes;
    c->level_start[lev + 1] = hi;
    int any = 0;
    for (int64_t k = lo; k < hi; ++k) {
      if (c->count[k] <= c->leaf_max || lev >= ORC_DEPTH) continue;
      int shift = 3 * (ORC_DEPTH - (lev + 1));
      int64_t f = c->first[k], e = f + c->count[k];
      c->child_first[k] = c->nnodes;
      for (uint32_t o = 0; o < 8; ++o) {
        int64_t a = f;
        while (a < e && (uint32_t)((c->key[a] >> shift) & 7u) < o) ++a;
        int64_t b = a;
        while (b < e && (uint32_t)((c->key[b] >> shift) & 7u) == o) ++b;
        if (b > a) {
          push_node(c, lev + 1, 2 * c->ic[3 * k] + ((o >> 2) & 1u), 2 * c->ic[3 * k + 1] + ((o >> 1) & 1u),
                    2 * c->ic[3 * k + 2] + (o & 1u), a, b - a);
          c->nchild[k]++;
          any = 1;
        }
      }
    }
    ++lev;
    if (!any) break;
  }
  c->nlevels = lev;
  c->level_start[lev] = c->nnodes;
  return 0;
}

/* geometric centre of node k (Sec. 2.1: expansion about the geometric centre) */
static void node_centre(const orc_ctx *c, int64_t k, double *z) {
  double h = c->box / (double)(1u << c->lev[k]);
  for (int d = 0; d < 3; ++d) z[d] = ((double)c->ic[3 * k + d] + 0.5) * h;
}

/* ------------------------------------------------------------------------ */
/* Dual-tree traversal with the hybrid MAC (Sec. 2.3).                       */
/* ------------------------------------------------------------------------ */

static void push3(int64_t **buf, int64_t *n, int64_t *cap, int64_t a, int64_t b, int64_t s) {
  if (*n == *cap) {
    *cap = *cap ? 2 * *cap : 4096;
    *buf = (int64_t *)realloc(*buf, sizeof(int64_t) * 3 * *cap);
  }
  (*buf)[3 * *n] = a; (*buf)[3 * *n + 1] = b; (*buf)[3 * *n + 2] = s;
  ++*n;
}

/*
 * Classify an ordered (sink a, source b shifted by s*L) cell pair.
 * Distances are exact integers in half units (L / 2^22):
 *   S_c  = |z_b + s L - z_a|, S_m = minimum box-box distance, S_max = maximum.
 * Returns 0 skip (S_m > R_c), 1 M2L, 2 open.
 *   transition (must open): S_c > R_c (rule 0) or S_max > R_c (rule 1);
 *   accept: L / S_c <= theta, i.e. (2 w)^2 <= theta^2 S_c^2, with w the half-unit
 *   side of the source (size_rule 0) or of the larger cell (size_rule 1).
 * conventional != 0: the acceptance test alone (no skip, no transition region),
 * the opening-angle criterion of a conventional FMM (Sec. 2.3, second item).
 */
static int mac_classify(const orc_ctx *c, int64_t a, int64_t b, int s, int conventional) {
  int64_t wa = (int64_t)1 << (ORC_DEPTH - c->lev[a]);
  int64_t wb = (int64_t)1 << (ORC_DEPTH - c->lev[b]);
  int sh[3] = {s / 9 - 1, (s / 3) % 3 - 1, s % 3 - 1};
  int64_t sc2 = 0, sm2 = 0, sx2 = 0;
  for (int d = 0; d < 3; ++d) {
    int64_t ca = 2 * ((int64_t)c->ic[3 * a + d] * wa) + wa;
    int64_t cb = 2 * ((int64_t)c->ic[3 * b + d] * wb) + wb + (int64_t)sh[d] * 4194304;
    int64_t dd = cb - ca;
    if (dd < 0) dd = -dd;
    int64_t gap = dd - (wa + wb);
    if (gap < 0) gap = 0;
    int64_t far = dd + (wa + wb);
    sc2 += dd * dd;
    sm2 += gap * gap;
    sx2 += far * far;
  }
  if (!conventional && (double)sm2 > c->rc2h) return 0;
  int trans = conventional ? 0 : c->rule == 0 ? ((double)sc2 > c->rc2h) : ((double)sx2 > c->rc2h);
  int64_t wl = (c->size_rule == 0) ? wb : (wa > wb ? wa : wb);
  if (!trans && (double)(4 * wl * wl) <= c->theta2 * (double)sc2) return 1;
  return 2;
}

/*
 * Dual-tree walk (Sec. 2.3): a stack of (sink, source, shift) cell pairs; an
 * accepted pair goes to the M2L list, two unaccepted leaves to the P2P list,
 * otherwise the larger cell is opened (both on a tie, the other one when the
 * larger is a leaf).  The hybrid walk starts from the root against the 27
 * nearest periodic images of itself (R_c < L / 2 reaches no further); the
 * conventional walk (Sec. 3) from the single pair (root, root): the walk of
 * the primary box, a conventional FMM treating the periodic images apart (by
 * Ewald summation, Sec. 3).
 */
static int walk(orc_ctx *c, int conventional) {
  if (!c) return -1;
  c->np2p = 0; c->nm2l = 0;
  free(c->m2l_ord); c->m2l_ord = NULL; c->cap_ord = 0;
  if (c->n == 0) return 0;
  int64_t *stk = NULL, nst = 0, cst = 0;
  if (conventional)
    push3(&stk, &nst, &cst, 0, 0, 13); /* shift index 13 = (0, 0, 0) */
  else
    for (int s = 0; s < 27; ++s) push3(&stk, &nst, &cst, 0, 0, s);
  while (nst > 0) {
    --nst;
    int64_t a = stk[3 * nst], b = stk[3 * nst + 1];
    int s = (int)stk[3 * nst + 2];
    int cls = mac_classify(c, a, b, s, conventional);
    if (cls == 0) continue;
    if (cls == 1) {
      push3(&c->m2l, &c->nm2l, &c->cap_m2l, a, b, s);
      continue;
    }
    int leafa = c->nchild[a] == 0, leafb = c->nchild[b] == 0;
    if (leafa && leafb) {
      push3(&c->p2p, &c->np2p, &c->cap_p2p, a, b, s);
      continue;
    }
    int opena, openb;
    if (leafa) { opena = 0; openb = 1; }
    else if (leafb) { opena = 1; openb = 0; }
    else if (c->lev[a] < c->lev[b]) { opena = 1; openb = 0; }
    else if (c->lev[b] < c->lev[a]) { opena = 0; openb = 1; }
    else { opena = 1; openb = 1; }
    int64_t a0 = opena ? c->child_first[a] : a, a1 = opena ? a0 + c->nchild[a] : a + 1;
    int64_t b0 = openb ? c->child_first[b] : b, b1 = openb ? b0 + c->nchild[b] : b + 1;
    for (int64_t x = a0; x < a1; ++x)
      for (int64_t y = b0; y < b1; ++y) push3(&stk, &nst, &cst, x, y, s);
  }
  free(stk);
  return 0;
}

int orc_traverse(orc_ctx *c) { return walk(c, 0); }

/* The conventional walk: replaces the lists; for interaction counts only. */
int orc_traverse_conventional(orc_ctx *c) { return walk(c, 1); }

/* ------------------------------------------------------------------------ */
/* FMM passes (Sec. 2.1 order: upward, M2L, downward, P2P).                  */
/* ------------------------------------------------------------------------ */

static void shift_vec(int s, double box, double *v) {
  v[0] = (s / 9 - 1) * box;
  v[1] = ((s / 3) % 3 - 1) * box;
  v[2] = (s % 3 - 1) * box;
}

int orc_upward(orc_ctx *c) {
  if (!c) return -1;
  int nc = orc_ncoef(c->p);
  free(c->M);
  c->M = (double *)calloc((size_t)(c->nnodes ? c->nnodes : 1) * nc, sizeof(double));
  for (int l = c->nlevels - 1; l >= 0; --l) {
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t k = c->level_start[l]; k < c->level_start[l + 1]; ++k) {
      double z[3];
      node_centre(c, k, z);
      if (c->nchild[k] == 0) {
        orc_p2m(c->count[k], c->x + 3 * c->first[k], c->m + c->first[k], z, c->p, c->M + k * nc);
      } else {
        double tmp[ORC_NCMAX];
        for (int64_t ch = c->child_first[k]; ch < c->child_first[k] + c->nchild[k]; ++ch) {
          double zc[3], x[3];
          node_centre(c, ch, zc);
          for (int d = 0; d < 3; ++d) x[d] = z[d] - zc[d];
          orc_m2m(c->M + ch * nc, x, c->p, tmp);
          for (int e = 0; e < nc; ++e) c->M[k * nc + e] += tmp[e];
        }
      }
    }
  }
  return 0;
}

static int cmp_triple(const void *a, const void *b) {
  const int64_t *x = (const int64_t *)a, *y = (const int64_t *)b;
  for (int i = 0; i < 3; ++i)
    if (x[i] != y[i]) return x[i] < y[i] ? -1 : 1;
  return 0;
}

/* sort a list by sink and return CSR offsets over nodes (caller frees) */
static int64_t *sink_offsets(int64_t *list, int64_t n, int64_t nnodes) {
  qsort(list, (size_t)n, 3 * sizeof(int64_t), cmp_triple);
  int64_t *off = (int64_t *)calloc((size_t)nnodes + 1, sizeof(int64_t));
  for (int64_t t = 0; t < n; ++t) off[list[3 * t] + 1]++;
  for (int64_t k = 0; k < nnodes; ++k) off[k + 1] += off[k];
  return off;
}

int orc_m2l_pass(orc_ctx *c) {
  if (!c || !c->M) return -1;
  int nc = orc_ncoef(c->p);
  free(c->L);
  c->L = (double *)calloc((size_t)(c->nnodes ? c->nnodes : 1) * nc, sizeof(double));
  int64_t *off = sink_offsets(c->m2l, c->nm2l, c->nnodes);
#pragma omp parallel for schedule(dynamic, 16)
  for (int64_t a = 0; a < c->nnodes; ++a) {
    double za[3];
    node_centre(c, a, za);
    for (int64_t t = off[a]; t < off[a + 1]; ++t) {
      int64_t b = c->m2l[3 * t + 1];
      int s = (int)c->m2l[3 * t + 2];
      double zb[3], sv[3], R[3];
      node_centre(c, b, zb);
      shift_vec(s, c->box, sv);
      for (int d = 0; d < 3; ++d) R[d] = za[d] - (zb[d] + sv[d]);
      const orc_kernel K = {c->rs, c->rc, c->split};
      m2l_k(c->M + b * nc, R, &K, c->p, c->L + a * nc);
    }
  }
  free(off);
  return 0;
}

/* L2L top-down (Eq. l2l) then L2P at the leaves (Eq. l2p); acc_sorted [n][3] is overwritten. */
int orc_downward(orc_ctx *c, double *acc_sorted) {
  if (!c || !c->L) return -1;
  int nc = orc_ncoef(c->p);
  for (int l = 0; l < c->nlevels; ++l) {
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t k = c->level_start[l]; k < c->level_start[l + 1]; ++k) {
      double z[3];
      node_centre(c, k, z);
      if (c->nchild[k] > 0) {
        double tmp[ORC_NCMAX];
        for (int64_t ch = c->child_first[k]; ch < c->child_first[k] + c->nchild[k]; ++ch) {
          double zc[3], x[3];
          node_centre(c, ch, zc);
          for (int d = 0; d < 3; ++d) x[d] = zc[d] - z[d];
          orc_l2l(c->L + k * nc, x, c->p, tmp);
          for (int e = 0; e < nc; ++e) c->L[ch * nc + e] += tmp[e];
        }
      } else {
        for (int64_t i = c->first[k]; i < c->first[k] + c->count[k]; ++i) {
          double u[3];
          for (int d = 0; d < 3; ++d) u[d] = c->x[3 * i + d] - z[d];
          orc_l2p(c->L + k * nc, u, c->p, c->G, NULL, acc_sorted + 3 * i);
        }
      }
    }
  }
  return 0;
}

/* P2P over the leaf-pair list with the hard cutoff 0 < |r| < R_c; adds into acc_sorted [n][3]. */
int orc_p2p_pass(orc_ctx *c, double *acc_sorted) {
  if (!c) return -1;
  const orc_kernel K = {c->rs, c->rc, c->split};
  int64_t *off = sink_offsets(c->p2p, c->np2p, c->nnodes);
  double rc2 = c->rc * c->rc;
#pragma omp parallel for schedule(dynamic, 16)
  for (int64_t a = 0; a < c->nnodes; ++a) {
    for (int64_t t = off[a]; t < off[a + 1]; ++t) {
      int64_t b = c->p2p[3 * t + 1];
      int s = (int)c->p2p[3 * t + 2];
      double sv[3];
      shift_vec(s, c->box, sv);
      for (int64_t i = c->first[a]; i < c->first[a] + c->count[a]; ++i) {
        double acc[3] = {0, 0, 0};
        for (int64_t j = c->first[b]; j < c->first[b] + c->count[b]; ++j) {
          double d[3];
          for (int k = 0; k < 3; ++k) d[k] = c->x[3 * i + k] - (c->x[3 * j + k] + sv[k]);
          pair_acc(d, c->m[j], &K, rc2, acc);
        }
        for (int k = 0; k < 3; ++k) acc_sorted[3 * i + k] += c->G * acc[k];
      }
    }
  }
  free(off);
  return 0;
}

/* Whole short-range FMM; acc is SoA [3][n] in input order. */
int orc_fmm_forces(orc_ctx *c, double *acc) {
  if (!c) return -1;
  int64_t n = c->n;
  if (n == 0) return 0;
  double *as = (double *)calloc((size_t)3 * n, sizeof(double));
  int rc = orc_traverse(c);
  if (!rc) rc = orc_upward(c);
  if (!rc) rc = orc_m2l_pass(c);
  if (!rc) rc = orc_downward(c, as);
  if (!rc) rc = orc_p2p_pass(c, as);
  if (!rc)
    for (int64_t s = 0; s < n; ++s)
      for (int d = 0; d < 3; ++d) acc[d * n + c->perm[s]] = as[3 * s + d];
  free(as);
  return rc;
}

/* ------------------------------------------------------------------------ */
/* Export for the tests.                                                     */
/* ------------------------------------------------------------------------ */

enum { ORC_N = 0, ORC_NNODES, ORC_NLEVELS, ORC_NP2P, ORC_NM2L };

int64_t orc_size(const orc_ctx *c, int what) {
  switch (what) {
    case ORC_N: return c->n;
    case ORC_NNODES: return c->nnodes;
    case ORC_NLEVELS: return c->nlevels;
    case ORC_NP2P: return c->np2p;
    case ORC_NM2L: return c->nm2l;
  }
  return -1;
}

/* keys [n] u64, perm [n] i64 */
int orc_export_particles(const orc_ctx *c, uint64_t *key, int64_t *perm, double *xs) {
  for (int64_t s = 0; s < c->n; ++s) {
    if (key) key[s] = c->key[s];
    if (perm) perm[s] = c->perm[s];
    if (xs)
      for (int d = 0; d < 3; ++d) xs[3 * s + d] = c->x[3 * s + d];
  }
  return 0;
}

/* nodes: [nnodes][8] i64 = level, ix, iy, iz, first, count, child_first(-1 for a leaf), nchild */
int orc_export_nodes(const orc_ctx *c, int64_t *out) {
  for (int64_t k = 0; k < c->nnodes; ++k) {
    int64_t *o = out + 8 * k;
    o[0] = c->lev[k];
    o[1] = c->ic[3 * k]; o[2] = c->ic[3 * k + 1]; o[3] = c->ic[3 * k + 2];
    o[4] = c->first[k]; o[5] = c->count[k];
    o[6] = c->nchild[k] ? c->child_first[k] : -1;
    o[7] = c->nchild[k];
  }
  return 0;
}

/* which = 0: P2P list, 1: M2L list; [len][3] i64 (sink, source, shift index) */
int orc_export_list(const orc_ctx *c, int which, int64_t *out) {
  int64_t n = which ? c->nm2l : c->np2p;
  const int64_t *src = which ? c->m2l : c->p2p;
  memcpy(out, src, sizeof(int64_t) * 3 * n);
  return 0;
}

/* expansions: which = 0 multipoles M, 1 locals L; [nnodes][ncoef] */
int orc_export_expansions(const orc_ctx *c, int which, double *out) {
  const double *src = which ? c->L : c->M;
  if (!src) return -1;
  memcpy(out, src, sizeof(double) * c->nnodes * orc_ncoef(c->p));
  return 0;
}

int orc_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

/* ------------------------------------------------------------------------ */
/* Learned acceptance: network reference and FMM on given lists.             */
/* ------------------------------------------------------------------------ */

/* FP32 value rounded to the nearest BF16 (ties to even), returned as double. */
double orc_bf16(double x) {
  float f = (float)x;
  uint32_t u;
  memcpy(&u, &f, 4);
  u += 0x7FFFu + ((u >> 16) & 1u);
  u &= 0xFFFF0000u;
  memcpy(&f, &u, 4);
  return (double)f;
}

#define MLP_IN 12
#define MLP_H 64
#define MLP_OUT 8
#define OFF_W1 0
#define OFF_B1 (OFF_W1 + MLP_H * MLP_IN)
#define OFF_W2 (OFF_B1 + MLP_H)
#define OFF_B2 (OFF_W2 + MLP_H * MLP_H)
#define OFF_W3 (OFF_B2 + MLP_H)
#define OFF_B3 (OFF_W3 + MLP_OUT * MLP_H)
#define MLP_W (OFF_B3 + MLP_OUT)

/* one sample: z1, h1, z2, h2 (hidden) and logits; rnd = 1 rounds inputs and hidden activations to BF16 */
static void mlp_fwd1(const double *w, const double *x, int rnd, double *z1, double *h1, double *z2, double *h2,
                     double *lo) {
  double xi[MLP_IN];
  for (int k = 0; k < MLP_IN; ++k) xi[k] = rnd ? orc_bf16(x[k]) : x[k];
  for (int u = 0; u < MLP_H; ++u) {
    double z = w[OFF_B1 + u];
    for (int k = 0; k < MLP_IN; ++k) z += w[OFF_W1 + u * MLP_IN + k] * xi[k];
    z1[u] = z;
    h1[u] = z > 0 ? (rnd ? orc_bf16(z) : z) : 0.0;
  }
  for (int u = 0; u < MLP_H; ++u) {
    double z = w[OFF_B2 + u];
    for (int k = 0; k < MLP_H; ++k) z += w[OFF_W2 + u * MLP_H + k] * h1[k];
    z2[u] = z;
    h2[u] = z > 0 ? (rnd ? orc_bf16(z) : z) : 0.0;
  }
  for (int o = 0; o < MLP_OUT; ++o) {
    double z = w[OFF_B3 + o];
    for (int k = 0; k < MLP_H; ++k) z += w[OFF_W3 + o * MLP_H + k] * h2[k];
    lo[o] = z;
  }
}

/* Network 12 -> 64 -> ReLU -> 64 -> ReLU -> 8 (the weight blob order of include/hfmm.h). */
int orc_mlp_forward(const double *w, const double *x, int64_t n, int rnd, double *logits) {
  for (int64_t i = 0; i < n; ++i) {
    double z1[MLP_H], h1[MLP_H], z2[MLP_H], h2[MLP_H];
    mlp_fwd1(w, x + i * MLP_IN, rnd, z1, h1, z2, h2, logits + i * MLP_OUT);
  }
  return 0;
}

/* Mean (class-weighted) softmax cross-entropy and its gradient; the BF16
 * rounding (rnd = 1) is treated as the identity in the backward pass. */
int orc_mlp_loss_grad(const double *w, const double *x, const int32_t *lab, const double *cw, int64_t n, int rnd,
                      double *grad, double *loss) {
  for (int i = 0; i < MLP_W; ++i) grad[i] = 0.0;
  double L = 0.0;
  for (int64_t s = 0; s < n; ++s) {
    double z1[MLP_H], h1[MLP_H], z2[MLP_H], h2[MLP_H], lo[MLP_OUT], xi[MLP_IN];
    const double *x0 = x + s * MLP_IN;
    for (int k = 0; k < MLP_IN; ++k) xi[k] = rnd ? orc_bf16(x0[k]) : x0[k];
    mlp_fwd1(w, x0, rnd, z1, h1, z2, h2, lo);
    double mx = lo[0];
    for (int o = 1; o < MLP_OUT; ++o) mx = lo[o] > mx ? lo[o] : mx;
    double se = 0.0, pr[MLP_OUT];
    for (int o = 0; o < MLP_OUT; ++o) se += exp(lo[o] - mx);
    for (int o = 0; o < MLP_OUT; ++o) pr[o] = exp(lo[o] - mx) / se;
    const int y = lab[s];
    const double wt = cw ? cw[y] : 1.0;
    L += -wt * log(pr[y]);
    double d3[MLP_OUT], d2[MLP_H], d1[MLP_H];
    for (int o = 0; o < MLP_OUT; ++o) d3[o] = wt * (pr[o] - (o == y ? 1.0 : 0.0));
    for (int o = 0; o < MLP_OUT; ++o) {
      grad[OFF_B3 + o] += d3[o];
      for (int k = 0; k < MLP_H; ++k) grad[OFF_W3 + o * MLP_H + k] += d3[o] * h2[k];
    }
    for (int k = 0; k < MLP_H; ++k) {
      double dh = 0.0;
      for (int o = 0; o < MLP_OUT; ++o) dh += w[OFF_W3 + o * MLP_H + k] * d3[o];
      d2[k] = z2[k] > 0 ? dh : 0.0;
    }
    for (int u = 0; u < MLP_H; ++u) {
      grad[OFF_B2 + u] += d2[u];
      for (int k = 0; k < MLP_H; ++k) grad[OFF_W2 + u * MLP_H + k] += d2[u] * h1[k];
    }
    for (int k = 0; k < MLP_H; ++k) {
      double dh = 0.0;
      for (int u = 0; u < MLP_H; ++u) dh += w[OFF_W2 + u * MLP_H + k] * d2[u];
      d1[k] = z1[k] > 0 ? dh : 0.0;
    }
    for (int u = 0; u < MLP_H; ++u) {
      grad[OFF_B1 + u] += d1[u];
      for (int k = 0; k < MLP_IN; ++k) grad[OFF_W1 + u * MLP_IN + k] += d1[u] * xi[k];
    }
  }
  for (int i = 0; i < MLP_W; ++i) grad[i] /= (double)n;
  if (loss) *loss = L / (double)n;
  return 0;
}

/*
 * Replace the context's lists (sink, source, shift index per row) and give
 * each M2L pair its own order q <= p (Eq. m2l truncated at |n| + |m| <= q).
 */
int orc_set_lists(orc_ctx *c, const int64_t *p2p, int64_t np2p, const int64_t *m2l, const int64_t *orders,
                  int64_t nm2l) {
  if (!c) return -1;
  free(c->p2p);
  free(c->m2l);
  free(c->m2l_ord); c->m2l_ord = NULL; c->cap_ord = 0;
  c->p2p = (int64_t *)malloc(sizeof(int64_t) * 3 * (np2p ? np2p : 1));
  c->m2l = (int64_t *)malloc(sizeof(int64_t) * 4 * (nm2l ? nm2l : 1));
  memcpy(c->p2p, p2p, sizeof(int64_t) * 3 * np2p);
  c->np2p = c->cap_p2p = np2p;
  /* the M2L rows keep (sink, source, shift) in the first three columns and the order in the fourth */
  for (int64_t t = 0; t < nm2l; ++t) {
    c->m2l[4 * t] = m2l[3 * t];
    c->m2l[4 * t + 1] = m2l[3 * t + 1];
    c->m2l[4 * t + 2] = m2l[3 * t + 2];
    c->m2l[4 * t + 3] = orders ? orders[t] : c->p;
  }
  c->nm2l = nm2l;
  c->cap_m2l = nm2l;
  return 0;
}

static int cmp_quad(const void *a, const void *b) {
  const int64_t *x = (const int64_t *)a, *y = (const int64_t *)b;
  for (int i = 0; i < 4; ++i)
    if (x[i] != y[i]) return x[i] < y[i] ? -1 : 1;
  return 0;
}

/* FMM forces on the lists given to orc_set_lists (order per M2L pair). */
int orc_fmm_forces_given_lists(orc_ctx *c, double *acc) {
  if (!c) return -1;
  int64_t n = c->n;
  if (n == 0) return 0;
  int nc = orc_ncoef(c->p);
  double *as = (double *)calloc((size_t)3 * n, sizeof(double));
  int rc = orc_upward(c);
  if (!rc) {
    free(c->L);
    c->L = (double *)calloc((size_t)(c->nnodes ? c->nnodes : 1) * nc, sizeof(double));
    qsort(c->m2l, (size_t)c->nm2l, 4 * sizeof(int64_t), cmp_quad);
    int64_t *off = (int64_t *)calloc((size_t)c->nnodes + 1, sizeof(int64_t));
    for (int64_t t = 0; t < c->nm2l; ++t) off[c->m2l[4 * t] + 1]++;
    for (int64_t k = 0; k < c->nnodes; ++k) off[k + 1] += off[k];
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t a = 0; a < c->nnodes; ++a) {
      double za[3];
      node_centre(c, a, za);
      for (int64_t t = off[a]; t < off[a + 1]; ++t) {
        int64_t b = c->m2l[4 * t + 1];
        int s = (int)c->m2l[4 * t + 2], q = (int)c->m2l[4 * t + 3];
        double zb[3], sv[3], R[3], Lq[ORC_NCMAX];
        node_centre(c, b, zb);
        shift_vec(s, c->box, sv);
        for (int d = 0; d < 3; ++d) R[d] = za[d] - (zb[d] + sv[d]);
        for (int e = 0; e < orc_ncoef(q); ++e) Lq[e] = 0.0;
        const orc_kernel K = {c->rs, c->rc, c->split};
        m2l_k(c->M + b * nc, R, &K, q, Lq);
        for (int e = 0; e < orc_ncoef(q); ++e) c->L[a * nc + e] += Lq[e];
      }
    }
    free(off);
    /* keep the list in the three-column layout the rest of the oracle uses */
    for (int64_t t = 0; t < c->nm2l; ++t)
      for (int j = 0; j < 3; ++j) c->m2l[3 * t + j] = c->m2l[4 * t + j];
  }
  if (!rc) rc = orc_downward(c, as);
  if (!rc) rc = orc_p2p_pass(c, as);
  if (!rc)
    for (int64_t s = 0; s < n; ++s)
      for (int d = 0; d < 3; ++d) acc[d * n + c->perm[s]] = as[3 * s + d];
  free(as);
  return rc;
}

/*
 * Error of accepting the pair (a, b, shift) with M2L at order q: up to 32
 * evenly strided particles of a, direct sum over b's particles vs
 * P2M(b, order q) -> M2L(order q) -> L2P (all FP64).  Returns
 * sqrt(sum |a_q - a|^2) / sqrt(sum |a|^2).
 */
double orc_pair_error(orc_ctx *c, int64_t a, int64_t b, int s, int q) {
  double za[3], zb[3], sv[3], R[3];
  node_centre(c, a, za);
  node_centre(c, b, zb);
  shift_vec(s, c->box, sv);
  for (int d = 0; d < 3; ++d) R[d] = za[d] - (zb[d] + sv[d]);
  double M[ORC_NCMAX], L[ORC_NCMAX];
  int64_t nb = c->count[b];
  double *xb = (double *)malloc(sizeof(double) * 3 * nb);
  for (int64_t j = 0; j < nb; ++j)
    for (int d = 0; d < 3; ++d) xb[3 * j + d] = c->x[3 * (c->first[b] + j) + d];
  orc_p2m(nb, xb, c->m + c->first[b], zb, q, M);
  for (int e = 0; e < orc_ncoef(q); ++e) L[e] = 0.0;
  const orc_kernel K = {c->rs, c->rc, c->split};
  m2l_k(M, R, &K, q, L);
  int64_t na = c->count[a];
  int ns = na < 32 ? (int)na : 32;
  double num = 0.0, den = 0.0;
  for (int k = 0; k < ns; ++k) {
    int64_t i = c->first[a] + (int64_t)(((uint64_t)k * (uint64_t)na) / (uint64_t)ns);
    double ex[3] = {0, 0, 0}, ap[3], u[3];
    for (int64_t j = 0; j < nb; ++j) {
      double d[3];
      for (int dd = 0; dd < 3; ++dd) d[dd] = c->x[3 * i + dd] - (xb[3 * j + dd] + sv[dd]);
      double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
      if (!(r2 > 0)) continue;
      double f[2];
      prefactors_k(sqrt(r2), &K, 1, f);
      for (int dd = 0; dd < 3; ++dd) ex[dd] += c->G * c->m[c->first[b] + j] * f[1] * d[dd];
    }
    for (int dd = 0; dd < 3; ++dd) u[dd] = c->x[3 * i + dd] - za[dd];
    orc_l2p(L, u, q, c->G, NULL, ap);
    for (int dd = 0; dd < 3; ++dd) {
      num += (ap[dd] - ex[dd]) * (ap[dd] - ex[dd]);
      den += ex[dd] * ex[dd];
    }
  }
  free(xb);
  return den > 0 ? sqrt(num / den) : 0.0;
}

/* index of the node with the given level and cell coordinates, or -1 */
int64_t orc_find_node(const orc_ctx *c, int lev, uint32_t ix, uint32_t iy, uint32_t iz) {
  if (lev < 0 || lev >= c->nlevels) return -1;
  for (int64_t k = c->level_start[lev]; k < c->level_start[lev + 1]; ++k)
    if (c->ic[3 * k] == ix && c->ic[3 * k + 1] == iy && c->ic[3 * k + 2] == iz) return k;
  return -1;
}

/* ------------------------------------------------------------------------ */
/* Learned acceptance: the pair features, the network with a bound on any   */
/* FP32 evaluation of it, and the walk that applies it.                      */
/* ------------------------------------------------------------------------ */

/*
 * The 12 features of an ordered cell pair (sink a, source b displaced by
 * shift s), all dimensionless (the feature list of the learned acceptance):
 *   0 S_c / r_s       1 S_m / r_s        2 S_max / R_c
 *   3 h_a / S_c       4 h_b / S_c        5 max(h_a, h_b) / S_c
 *   6 (level_a - level_b) / 8            7 log2(1 + n_a) / 16   8 log2(1 + n_b) / 16
 *   9 |(M~_100, M~_010, M~_001)| / |M~_000|    10 |(M~_m, |m| = 2)| / |M~_000|
 *  11 S_c / R_c
 * with S_c the centre distance, S_m and S_max the least and greatest distance
 * between the two cubes (Sec. 2.3), h the cell sides, n the particle counts
 * and M~_m = M_m / h_b^|m| the source's multipoles of Eq. p2m about its
 * geometric centre in units of its side.  A massless source (M_000 = 0) has
 * |M~_000| read as 1e-30, so its moment features are 0 or huge, never NaN.
 * Needs the multipoles (orc_upward).  Plain FP64 from the exact integer cell
 * geometry.
 */
int orc_pair_features(const orc_ctx *c, int64_t a, int64_t b, int s, double *f) {
  if (!c || !c->M || a < 0 || b < 0 || a >= c->nnodes || b >= c->nnodes || s < 0 || s > 26) return -1;
  int64_t wa = (int64_t)1 << (ORC_DEPTH - c->lev[a]);
  int64_t wb = (int64_t)1 << (ORC_DEPTH - c->lev[b]);
  int sh[3] = {s / 9 - 1, (s / 3) % 3 - 1, s % 3 - 1};
  double sc2 = 0, sm2 = 0, sx2 = 0;
  for (int d = 0; d < 3; ++d) {
    int64_t ca = 2 * ((int64_t)c->ic[3 * a + d] * wa) + wa;
    int64_t cb = 2 * ((int64_t)c->ic[3 * b + d] * wb) + wb + (int64_t)sh[d] * 4194304;
    int64_t dd = cb - ca;
    if (dd < 0) dd = -dd;
    int64_t gap = dd - (wa + wb);
    if (gap < 0) gap = 0;
    int64_t far = dd + (wa + wb);
    sc2 += (double)dd * (double)dd;
    sm2 += (double)gap * (double)gap;
    sx2 += (double)far * (double)far;
  }
  const double unit = c->box / 4194304.0; /* one half unit */
  const double Sc = sqrt(sc2) * unit, Sm = sqrt(sm2) * unit, Sx = sqrt(sx2) * unit;
  const double ha = 2.0 * (double)wa * unit, hb = 2.0 * (double)wb * unit;
  f[0] = Sc / c->rs;
  f[1] = Sm / c->rs;
  f[2] = Sx / c->rc;
  f[3] = ha / Sc;
  f[4] = hb / Sc;
  f[5] = (ha > hb ? ha : hb) / Sc;
  f[6] = (double)(c->lev[a] - c->lev[b]) / 8.0;
  f[7] = log2(1.0 + (double)c->count[a]) / 16.0;
  f[8] = log2(1.0 + (double)c->count[b]) / 16.0;
  const int nc = orc_ncoef(c->p);
  const double *M = c->M + b * nc;
  const double m0 = fabs(M[0]) + 1e-30;
  double d2 = 0.0, q2 = 0.0;
  for (int e = 1; e < 10 && e < nc; ++e) {
    const int *m = g_mi[e];
    const int deg = m[0] + m[1] + m[2];
    const double v = M[e] / pow(hb, deg);
    if (deg == 1) d2 += v * v; else q2 += v * v;
  }
  f[9] = sqrt(d2) / m0;
  f[10] = sqrt(q2) / m0;
  f[11] = Sc / c->rc;
  return 0;
}

/* t > 0 rounded to FP32 and then to BF16, else 0: the activation of a hidden
 * unit (rounding to FP32 first, as the network's FP32 accumulator does). */
static double act_bf16(double t) { return t > 0 ? orc_bf16(t) : 0.0; }

/*
 * One layer, out = act(b + W in), with a bound on how far any FP32 evaluation
 * can be from `out`.  Its inputs may differ from `in` by up to `ein`; the sum
 * of the K products and the bias, accumulated in FP32 in any order (rounded
 * or truncated at each step), differs from the exact sum by at most
 * (K + 2) 2^-23 times the sum of the magnitudes.  A hidden unit's activation
 * (FP32 -> BF16 after the ReLU) is monotone in the pre-activation, so the
 * evaluation lies between the activations of the interval's two ends.
 */
static void layer_bound(const double *W, const double *bias, int nout, int nin, const double *in,
                        const double *ein, int hidden, double *out, double *eout) {
  const double gam = (double)(nin + 2) * ldexp(1.0, -23);
  for (int u = 0; u < nout; ++u) {
    double z = bias[u], mag = fabs(bias[u]), e = 0.0;
    for (int k = 0; k < nin; ++k) {
      const double wk = W[u * nin + k];
      z += wk * in[k];
      mag += fabs(wk) * (fabs(in[k]) + ein[k]);
      e += fabs(wk) * ein[k];
    }
    e += gam * mag;
    if (hidden) {
      out[u] = act_bf16(z);
      const double hi = act_bf16(z + e) - out[u], lo = out[u] - act_bf16(z - e);
      eout[u] = hi > lo ? hi : lo;
    } else {
      out[u] = z;
      eout[u] = e;
    }
  }
}

/*
 * The network on one feature row, at its rounding points (inputs and hidden
 * activations rounded to BF16, FP32 sums), and bounds elo[8] on the deviation
 * of any FP32 evaluation's logits.  xtol (may be NULL): the evaluated
 * features may differ from x by up to xtol[k] before their BF16 rounding.
 * Returns the bit mask of the classes that can be the evaluation's argmax
 * (ties to the lower class): classes whose upper bound reaches the largest
 * lower bound.
 */
static uint32_t mlp_bound1(const double *w, const double *x, const double *xtol, double *lo, double *elo) {
  double xi[MLP_IN], ex[MLP_IN], h1[MLP_H], e1[MLP_H], h2[MLP_H], e2[MLP_H];
  for (int k = 0; k < MLP_IN; ++k) {
    xi[k] = orc_bf16(x[k]);
    ex[k] = 0.0;
    if (xtol && xtol[k] > 0) {
      const double up = orc_bf16(x[k] + xtol[k]) - xi[k], dn = xi[k] - orc_bf16(x[k] - xtol[k]);
      ex[k] = up > dn ? up : dn;
    }
  }
  layer_bound(w + OFF_W1, w + OFF_B1, MLP_H, MLP_IN, xi, ex, 1, h1, e1);
  layer_bound(w + OFF_W2, w + OFF_B2, MLP_H, MLP_H, h1, e1, 1, h2, e2);
  layer_bound(w + OFF_W3, w + OFF_B3, MLP_OUT, MLP_H, h2, e2, 0, lo, elo);
  double lmax = -HUGE_VAL;
  for (int o = 0; o < MLP_OUT; ++o)
    if (lo[o] - elo[o] > lmax) lmax = lo[o] - elo[o];
  uint32_t mask = 0;
  for (int o = 0; o < MLP_OUT; ++o)
    if (lo[o] + elo[o] >= lmax) mask |= 1u << o;
  return mask;
}

/* Batch form: logits and bounds [n][8], class [n] (argmax of the nominal
 * logits, ties to the lower class), plausible-class mask [n]. */
int orc_mlp_forward_bound(const double *w, const double *x, const double *xtol, int64_t n, double *logits,
                          double *bound, int32_t *cls, uint32_t *mask) {
  for (int64_t i = 0; i < n; ++i) {
    double *lo = logits + i * MLP_OUT, *el = bound + i * MLP_OUT;
    const uint32_t m = mlp_bound1(w, x + i * MLP_IN, xtol ? xtol + i * MLP_IN : NULL, lo, el);
    int best = 0;
    for (int o = 1; o < MLP_OUT; ++o)
      if (lo[o] > lo[best]) best = o;
    if (cls) cls[i] = best;
    if (mask) mask[i] = m;
  }
  return 0;
}

static void push1(int64_t **buf, int64_t *cap, int64_t n, int64_t v) {
  if (n >= *cap) {
    *cap = *cap ? 2 * *cap : 4096;
    while (*cap <= n) *cap *= 2;
    *buf = (int64_t *)realloc(*buf, sizeof(int64_t) * *cap);
  }
  (*buf)[n] = v;
}

static int cmp_ref4(const void *key, const void *row) {
  const int64_t *x = (const int64_t *)key, *y = (const int64_t *)row;
  for (int i = 0; i < 3; ++i)
    if (x[i] != y[i]) return x[i] < y[i] ? -1 : 1;
  return 0;
}

/*
 * Dual-tree walk with the learned acceptance (the network in place of the
 * opening-angle rule; the feature list above): rules 1 and 3 of Sec. 2.3 and
 * the opening rules unchanged; a pair that the geometric rule would accept at
 * the context's theta (the safety bound) is a candidate, and the network's
 * class decides: 0 = open the pair as the geometric walk would, k >= 1 = M2L
 * at order min(k + 1, p).  The decision is the argmax of the nominal logits
 * (mlp_bound1, with the features within ftol_rel |f| + ftol_abs of these FP64
 * values).  Where the bound admits more than one class, an FP32 evaluation
 * may take any of them; with `ref` (an M2L list [nref][4] = sink, source,
 * shift, order, sorted by the first three columns) the walk then takes the
 * decision that list records (M2L at its order when the pair is in it, else
 * open) and checks that it is one of the admitted classes.
 * stats[6]: candidates, candidates with more than one admitted class, those
 * resolved from ref, ref decisions outside the admitted classes, the largest
 * logit bound seen, (reserved, 0).  The lists (with their orders,
 * orc_export_m2l_orders) replace the context's.  Computes the multipoles
 * (orc_upward) when they are missing.
 */
int orc_traverse_learned(orc_ctx *c, const double *w, const double *ftol_rel, const double *ftol_abs,
                         const int64_t *ref, int64_t nref, double *stats) {
  if (!c || !w) return -1;
  c->np2p = 0; c->nm2l = 0;
  free(c->m2l_ord); c->m2l_ord = NULL; c->cap_ord = 0;
  double st[6] = {0, 0, 0, 0, 0, 0};
  if (c->n == 0) {
    if (stats) memcpy(stats, st, sizeof st);
    return 0;
  }
  if (!c->M && orc_upward(c)) return -1;
  int64_t *stk = NULL, nst = 0, cst = 0;
  for (int s = 0; s < 27; ++s) push3(&stk, &nst, &cst, 0, 0, s);
  while (nst > 0) {
    --nst;
    int64_t a = stk[3 * nst], b = stk[3 * nst + 1];
    int s = (int)stk[3 * nst + 2];
    int cls = mac_classify(c, a, b, s, 0);
    if (cls == 0) continue;
    if (cls == 1) { /* candidate: the network decides */
      double f[MLP_IN], tol[MLP_IN], lo[MLP_OUT], el[MLP_OUT];
      orc_pair_features(c, a, b, s, f);
      for (int k = 0; k < MLP_IN; ++k) tol[k] = ftol_rel[k] * fabs(f[k]) + ftol_abs[k];
      const uint32_t mask = mlp_bound1(w, f, tol, lo, el);
      int k = 0;
      for (int o = 1; o < MLP_OUT; ++o)
        if (lo[o] > lo[k]) k = o;
      st[0] += 1;
      for (int o = 0; o < MLP_OUT; ++o)
        if (el[o] > st[4]) st[4] = el[o];
      if (mask != (1u << k)) {
        st[1] += 1;
        if (ref) {
          const int64_t key[3] = {a, b, s};
          const int64_t *hit = (const int64_t *)bsearch(key, ref, (size_t)nref, 4 * sizeof(int64_t), cmp_ref4);
          int kr = 0;
          if (hit) kr = (int)hit[3] - 1; /* order q = k + 1 (orders above p were capped at p) */
          /* with the cap, class k >= p - 1 all give order p: admitted if any such class is */
          int ok = 0;
          if (kr <= 0) ok = (mask & 1u) != 0, kr = 0;
          else if (kr >= c->p - 1) {
            for (int o = c->p - 1; o < MLP_OUT; ++o) ok |= (mask >> o) & 1u;
          } else ok = (mask >> kr) & 1u;
          st[2] += 1;
          if (!ok) st[3] += 1;
          k = kr;
        }
      }
      if (k > 0) {
        const int q = k + 1 < c->p ? k + 1 : c->p;
        push1(&c->m2l_ord, &c->cap_ord, c->nm2l, q);
        push3(&c->m2l, &c->nm2l, &c->cap_m2l, a, b, s);
        continue;
      }
      cls = 2; /* open */
    }
    int leafa = c->nchild[a] == 0, leafb = c->nchild[b] == 0;
    if (leafa && leafb) {
      push3(&c->p2p, &c->np2p, &c->cap_p2p, a, b, s);
      continue;
    }
    int opena, openb;
    if (leafa) { opena = 0; openb = 1; }
    else if (leafb) { opena = 1; openb = 0; }
    else if (c->lev[a] < c->lev[b]) { opena = 1; openb = 0; }
    else if (c->lev[b] < c->lev[a]) { opena = 0; openb = 1; }
    else { opena = 1; openb = 1; }
    int64_t a0 = opena ? c->child_first[a] : a, a1 = opena ? a0 + c->nchild[a] : a + 1;
    int64_t b0 = openb ? c->child_first[b] : b, b1 = openb ? b0 + c->nchild[b] : b + 1;
    for (int64_t x = a0; x < a1; ++x)
      for (int64_t y = b0; y < b1; ++y) push3(&stk, &nst, &cst, x, y, s);
  }
  free(stk);
  if (stats) memcpy(stats, st, sizeof st);
  return 0;
}

/* Order of each M2L entry of the current list (p for every entry after a geometric walk). */
int orc_export_m2l_orders(const orc_ctx *c, int64_t *out) {
  for (int64_t t = 0; t < c->nm2l; ++t) out[t] = c->m2l_ord ? c->m2l_ord[t] : c->p;
  return 0;
}
