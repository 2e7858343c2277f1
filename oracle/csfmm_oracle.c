/*
 * csfmm_oracle.c -- plain FP64 CPU oracle for the cubed-sphere fast multipole
 * method (CSFMM) evaluation pass of Chen & Krasny, "A cubed sphere fast
 * multipole method" (arXiv 2508.13550).
 *
 * TEST INFRASTRUCTURE.  Only the tests, the smoke check and the benchmark's
 * CPU-baseline leg may load this library.  It shares no code, header or table
 * generator with the CUDA library; both sides only agree on the conventions
 * listed below, which each side implements on its own.
 *
 * It provides
 *   - the direct sum phi_i = sum_{j != i} K(x_i, x_j) w_j  (Sec. 1, Eq. nbodysum)
 *     with Neumaier-compensated summation, and
 *   - the CSFMM: quadtree on the equiangular gnomonic cubed sphere (Sec. 3),
 *     barycentric Lagrange interpolation at Chebyshev points (Sec. 4,
 *     Eq. barycentric), the PP/PC/CP/CC interactions (Sec. 5, Eqs. PP, PC,
 *     CP, CC), the upward pass (Sec. 6, Eq. upwardpass2), the dual tree
 *     traversal (Sec. 8, Algorithm "CSFMM") and the downward pass (Sec. 8.1,
 *     Eq. downward_2),
 *   - the cubed sphere tree code (CSTC, Sec. 7, Algorithm "CSTC") on the
 *     same tree, proxies and upward pass,
 *   - cells shrunk to bound their points (Sec. 3, optional),
 *   - the Laplace, Biot-Savart, Newtonian, biharmonic (Eq. G_B) and SAL
 *     (Eq. G_SAL_approx) kernels,
 * all in double precision, written for clarity rather than speed (OpenMP over
 * independent targets only).  Numbered planted mistakes (oracle_set_mutation)
 * let the tests show that their pins catch each one.
 *
 * Readings of points the paper leaves open (each listed in the design notes):
 *   - 1 - x.y is evaluated as |x - y|^2 / 2 for unit vectors, and x cross y
 *     as x cross (y - x), so that neither cancels for nearby points.
 *   - A cell splits iff it holds more than N0 points; "big" (|C| > N0) means
 *     "has children", "small" means "leaf".  Empty children are dropped.
 *   - Children split their parent's (xi, eta) square at its midpoint; a
 *     coordinate on the midpoint goes to the upper child.
 *   - A cell's box is its dyadic square, or, when the plan shrinks cells
 *     (Sec. 3: cells shrunk to bound their particles), the smallest box of
 *     fine cells holding its points, each edge moved out to an even fine
 *     coordinate so that the midpoint is a table entry.  The Chebyshev grid
 *     spans the box (separate half-widths along xi and eta); a child's nodes
 *     are placed in its parent's coordinates from the boxes' integer edges.
 *   - Centre = sphere image of the box midpoint; radius = largest chord from
 *     the centre to the four corners; R = chord between centres.
 *   - Well separated iff (r_t + r_s) < MAC * R.  In Algorithm "CSFMM" the
 *     PC / CP / CC choice is read as exclusive; when not well separated and
 *     at least one cluster is big, the shallower cluster is split (equal
 *     levels: the target), and if that one is a leaf the other one is split.
 *   - If the evaluation point equals a Chebyshev node exactly, L_k = delta.
 *   - CSTC: x_i and C_s are well separated iff r_s < MAC * R, R the chord from
 *     x_i to the centre of C_s; "|C_s| > N0" means C_s has children; a leaf
 *     that is not well separated interacts directly (it has no children to
 *     pass x_i to).
 *
 * Conventions (agreed with the CUDA library, implemented independently):
 *   - face f = 2*axis + (component < 0), axis = argmax |x_axis| (ties: lowest
 *     axis); face-plane coordinates a = x_u/|x_axis|, b = x_v/|x_axis| with
 *     u = (axis+1) mod 3, v = (axis+2) mod 3; inverse map
 *     q = sqrt((1 + a*a) + b*b), x_axis = +-1/q, x_u = a/q, x_v = b/q.
 *   - tangent table T[k] = tan(k * ((pi/2)/2^D) - pi/4), k = 0..2^D, D = 18,
 *     evaluated on the host with the C library's tan;  a point's integer
 *     coordinate is the largest k < 2^D with k == 0 or T[k] <= a.
 *   - cells live on levels 0..17; the (xi, eta) midpoint and corners of a
 *     cell (f, l, ia, ib) are table entries.
 *   - proxy index k = k1*(n+1) + k2, k1 along xi (a), k2 along eta (b).
 *   - geometry used in decisions is evaluated without fused multiply-add
 *     (this file must be compiled with -ffp-contract=off).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_KERNEL_LAPLACE 0
#define OR_KERNEL_BIOT_SAVART 1
#define OR_KERNEL_NEWTON 2
#define OR_KERNEL_BIHARMONIC 3
#define OR_KERNEL_SAL 4
#define OR_KERNEL_ONE 100

/* Load Love number fit of Sec. 2.4: k'_n ~ a1/n, h'_n ~ b0 + b1/n. */
#define OR_SAL_A1 (-2.7)
#define OR_SAL_B0 (-6.21196)
#define OR_SAL_B1 (6.1)

#define OR_D 18            /* tangent table resolution: 2^D intervals per face */
#define OR_LMAX 17         /* deepest cell level */

#define OR_PP 0
#define OR_PC 1
#define OR_CP 2
#define OR_CC 3

static const double OR_PI = 3.14159265358979323846;
static const double OR_HALF_PI = 1.57079632679489661923;
static const double OR_QUARTER_PI = 0.78539816339744830962;

/* Planted mistakes, used only by the tests that show each pin catches them.
 * 0 = the oracle as written. */
static int g_mutation = 0;
void oracle_set_mutation(int m) { g_mutation = m; }
int oracle_get_mutation(void) { return g_mutation; }

int oracle_kernel_dim(int kid) { return kid == OR_KERNEL_BIOT_SAVART ? 3 : 1; }

/* Dilogarithm dilog(x) = -int_0^x log(1 - t)/t dt = Li2(x), 0 <= x <= 1, by the
 * Bernoulli-number series Li2(x) = sum_{n>=0} B_n u^(n+1)/(n+1)!, u = -log(1 - x)
 * (convergent for |u| < 2 pi), used for x <= 1/2 (u <= log 2), and Euler's
 * reflection Li2(x) = pi^2/6 - log(x) log(1 - x) - Li2(1 - x) for x > 1/2. */
static double li2_series(double u) {
  /* B_{2k} / (2k+1)!, k = 1..10 */
  static const double c[10] = {
      1.0 / 36.0, -1.0 / 3600.0, 1.0 / 211680.0, -1.0 / 10886400.0, 1.0 / 526901760.0,
      -691.0 / 16999766784000.0, 7.0 / 6.0 / 1307674368000.0, -3617.0 / 510.0 / 355687428096000.0,
      43867.0 / 798.0 / 121645100408832000.0, -174611.0 / 330.0 / 51090942171709440000.0};
  double u2 = u * u, p = u * u2, s = 0.0;
  for (int k = 0; k < 10; ++k) { s += c[k] * p; p *= u2; }
  return u - 0.25 * u2 + s;
}
double oracle_dilog(double x) {
  if (x <= 0.5) return li2_series(-log1p(-x));
  if (x >= 1.0) return OR_PI * OR_PI / 6.0;
  return OR_PI * OR_PI / 6.0 - ((g_mutation == 14) ? 0.0 : log(x) * log1p(-x)) -
         li2_series(-log(x));
}

static int kernel_valid(int kid) {
  return kid == OR_KERNEL_LAPLACE || kid == OR_KERNEL_BIOT_SAVART ||
         kid == OR_KERNEL_NEWTON || kid == OR_KERNEL_BIHARMONIC || kid == OR_KERNEL_SAL ||
         kid == OR_KERNEL_ONE;
}

/* ------------------------------------------------------------------------ */
/* Kernels (Sec. 2): Laplace G_L = -(1/4pi) ln(1 - x.y)  (Eq. G_L);          */
/* biharmonic G_B = (1/4pi) dilog((1 + x.y)/2)  (Eq. G_B);                    */
/* Biot-Savart K_BS = -(1/4pi) (x cross y)/(1 - x.y)  (Eq. K_BS);            */
/* Newtonian 1/sqrt(2(1 - x.y)), the leading term 1/gamma of Eq.             */
/* G_SAL_approx;  SAL: the bracket of Eq. G_SAL_approx,                       */
/* (1 - b0)/gamma - (a1 - b1) ln(gamma/2 + gamma^2/4), gamma = |x - y|,       */
/* without the factor 3 rho_w / (4 pi rho_e);  K = 1 (test kernel).           */
/* ------------------------------------------------------------------------ */
static void kernel_eval(int kid, const double *x, const double *y, double *k) {
  double dx = x[0] - y[0], dy = x[1] - y[1], dz = x[2] - y[2];
  double d2 = dx * dx + dy * dy + dz * dz;
  double omc = 0.5 * d2; /* 1 - x.y */
  switch (kid) {
  case OR_KERNEL_LAPLACE: {
    double g = -log(omc) / (4.0 * OR_PI);
    k[0] = (g_mutation == 2) ? -g : g;
    break;
  }
  case OR_KERNEL_BIOT_SAVART: {
    /* x cross y = x cross (y - x): the same vector, without the cancellation
     * of x cross y for nearby unit vectors (as 1 - x.y is |x - y|^2 / 2) */
    double cx = -(x[1] * dz - x[2] * dy);
    double cy = -(x[2] * dx - x[0] * dz);
    double cz = -(x[0] * dy - x[1] * dx);
    double s = -1.0 / (4.0 * OR_PI * omc);
    k[0] = s * cx;
    k[1] = s * cy;
    k[2] = s * cz;
    break;
  }
  case OR_KERNEL_NEWTON:
    k[0] = 1.0 / sqrt(d2);
    break;
  case OR_KERNEL_SAL: {
    double g = sqrt(d2);
    k[0] = (1.0 - OR_SAL_B0) / g - (OR_SAL_A1 - OR_SAL_B1) * log(0.5 * g + 0.25 * d2);
    break;
  }
  case OR_KERNEL_BIHARMONIC: /* Eq. G_B: dilog((1 + x.y)/2) / (4 pi), (1 + x.y)/2 = 1 - d2/4 */
    k[0] = oracle_dilog(1.0 - 0.25 * d2) / (4.0 * OR_PI);
    break;
  default:
    k[0] = 1.0;
    break;
  }
}

/* Neumaier's compensated summation. */
typedef struct { double s, c; } ksum;
static inline void ksum_add(ksum *a, double v) {
  double t = a->s + v;
  if (fabs(a->s) >= fabs(v))
    a->c += (a->s - t) + v;
  else
    a->c += (v - t) + a->s;
  a->s = t;
}

/* ------------------------------------------------------------------------ */
/* Direct sum (Eq. nbodysum), i = j omitted.  out[r][t][d] for the targets   */
/* listed in tgt (all N points if tgt == NULL).                              */
/* ------------------------------------------------------------------------ */
int oracle_direct(const double *pts, int64_t N, int kid, const double *w,
                  int nrhs, const int64_t *tgt, int64_t ntgt, double *out) {
  if (!pts || N < 0 || !kernel_valid(kid) || nrhs < 1 || !w || !out) return 1;
  int dim = oracle_kernel_dim(kid);
  int64_t nt = tgt ? ntgt : N;
#pragma omp parallel for schedule(dynamic, 16)
  for (int64_t t = 0; t < nt; ++t) {
    int64_t i = tgt ? tgt[t] : t;
    for (int r = 0; r < nrhs; ++r) {
      ksum acc[3] = {{0, 0}, {0, 0}, {0, 0}};
      const double *wr = w + (int64_t)r * N;
      for (int64_t j = 0; j < N; ++j) {
        if (j == i) continue;
        double k[3];
        kernel_eval(kid, pts + 3 * i, pts + 3 * j, k);
        for (int d = 0; d < dim; ++d) ksum_add(&acc[d], k[d] * wr[j]);
      }
      for (int d = 0; d < dim; ++d)
        out[((int64_t)r * nt + t) * dim + d] = acc[d].s + acc[d].c;
    }
  }
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Barycentric Lagrange interpolation at Chebyshev points (Sec. 4).          */
/* ------------------------------------------------------------------------ */
void oracle_cheb_nodes(int n, double *s) {
  for (int k = 0; k <= n; ++k) {
    double den = (g_mutation == 4) ? (double)(n + 1) : (double)n;
    s[k] = cos((double)k * OR_PI / den);
  }
}

static double bary_weight(int k, int n) {
  double w = (k % 2 == 0) ? 1.0 : -1.0;
  if ((k == 0 || k == n) && g_mutation != 8) w *= 0.5;
  return w;
}

/* L_k(u), k = 0..n, Eq. (barycentric). */
void oracle_lagrange(int n, const double *s, double u, double *L) {
  for (int k = 0; k <= n; ++k) {
    if (u == s[k]) {
      for (int j = 0; j <= n; ++j) L[j] = (j == k) ? 1.0 : 0.0;
      return;
    }
  }
  double den = 0.0;
  for (int k = 0; k <= n; ++k) {
    L[k] = bary_weight(k, n) / (u - s[k]);
    den += L[k];
  }
  for (int k = 0; k <= n; ++k) L[k] /= den;
}

/* ------------------------------------------------------------------------ */
/* Cubed-sphere geometry (Sec. 3).                                           */
/* ------------------------------------------------------------------------ */
static double *g_tan = NULL; /* T[k], k = 0..2^D */

static const double *tan_table(void) {
  if (g_tan) return g_tan;
#pragma omp critical(oracle_tan_table)
  {
    if (!g_tan) {
      int64_t M = (int64_t)1 << OR_D;
      double H = ldexp(OR_HALF_PI, -OR_D);
      double *t = (double *)malloc(sizeof(double) * (size_t)(M + 1));
      for (int64_t k = 0; k <= M; ++k) t[k] = tan((double)k * H - OR_QUARTER_PI);
      g_tan = t;
    }
  }
  return g_tan;
}

/* Face of a point and its face-plane coordinates. */
static void face_coords(const double *x, int *face, double *a, double *b) {
  int ax = 0;
  double m = fabs(x[0]);
  if (fabs(x[1]) > m) { ax = 1; m = fabs(x[1]); }
  if (fabs(x[2]) > m) { ax = 2; m = fabs(x[2]); }
  int u = (ax + 1) % 3, v = (ax + 2) % 3;
  *face = 2 * ax + (x[ax] < 0.0 ? 1 : 0);
  *a = x[u] / m;
  *b = x[v] / m;
}

/* Sphere point of face-plane coordinates (a, b) on face f. */
static void face_point(int f, double a, double b, double *x) {
  int ax = f / 2;
  double sg = (f % 2) ? -1.0 : 1.0;
  int u = (ax + 1) % 3, v = (ax + 2) % 3;
  double q = sqrt((1.0 + a * a) + b * b);
  x[ax] = sg / q;
  x[u] = a / q;
  x[v] = b / q;
}

static double chord(const double *x, const double *y) {
  double dx = x[0] - y[0], dy = x[1] - y[1], dz = x[2] - y[2];
  return sqrt((dx * dx + dy * dy) + dz * dz);
}

/* Largest k < 2^D with k == 0 or T[k] <= a. */
static int64_t fine_coord(const double *T, double a) {
  int64_t lo = 0, hi = ((int64_t)1 << OR_D) - 1;
  while (lo < hi) {
    int64_t mid = (lo + hi + 1) / 2;
    if (T[mid] <= a) lo = mid; else hi = mid - 1;
  }
  return lo;
}

static uint64_t interleave(uint64_t qa, uint64_t qb) {
  uint64_t key = 0;
  for (int i = 0; i < OR_D; ++i) {
    key |= ((qa >> i) & 1u) << (2 * i);
    key |= ((qb >> i) & 1u) << (2 * i + 1);
  }
  return key;
}

/* ------------------------------------------------------------------------ */
/* Tree and plan.                                                             */
/* ------------------------------------------------------------------------ */
typedef struct {
  int face, level;
  int64_t ia, ib;
  int64_t begin, end; /* range in sorted order */
  int parent;
  int child[4];       /* by quadrant c = 2*bit_b + bit_a; -1 if empty */
  int nchild;
  double c[3], r;
  /* the cell's box in fine face coordinates (even edges): a in [alo, ahi],
   * b in [blo, bhi]; the dyadic square of the cell, or with shrinking the
   * smallest such box around its points */
  int64_t alo, ahi, blo, bhi;
  double xi_mid, eta_mid, hx, hy; /* box midpoint and half-widths in angle */
} ocell;

typedef struct { int t, s; } opair;

typedef struct {
  int64_t N;
  int n, p, P, N0;
  int shrink;       /* boxes shrunk to bound their points */
  double theta;
  double *x;        /* points in sorted order [N][3] */
  int64_t *order;   /* sorted position -> input index */
  double *u, *v;    /* local coordinates of each point in its leaf */
  int *leaf_of;     /* sorted position -> leaf cell */
  ocell *cells;
  int ncells, nlevels;
  int *level_begin; /* cells of level l are [level_begin[l], level_begin[l+1]) */
  opair *list[4];
  int64_t nlist[4], caplist[4];
  double *s;        /* Chebyshev nodes */
  double *proxy;    /* [ncells][P][3] */
  double margin;    /* min |(r_t+r_s) - MAC R| / (MAC R) over MAC tests, R > 0 */
  int64_t n_mac_tests;
} oplan;

static void list_push(oplan *pl, int type, int t, int s) {
  if (pl->nlist[type] == pl->caplist[type]) {
    pl->caplist[type] = pl->caplist[type] ? 2 * pl->caplist[type] : 1024;
    pl->list[type] = (opair *)realloc(pl->list[type],
                                      sizeof(opair) * (size_t)pl->caplist[type]);
  }
  pl->list[type][pl->nlist[type]].t = t;
  pl->list[type][pl->nlist[type]].s = s;
  pl->nlist[type]++;
}

typedef struct { uint64_t key; int64_t idx; } okey;
static int okey_cmp(const void *A, const void *B) {
  const okey *a = (const okey *)A, *b = (const okey *)B;
  if (a->key != b->key) return a->key < b->key ? -1 : 1;
  return a->idx < b->idx ? -1 : (a->idx > b->idx);
}

/* Geometry of a cell from its box: centre at the box midpoint (an integer
 * fine coordinate: the edges are even), radius the largest chord to the four
 * corners, midpoint angles and half-widths for the Chebyshev grid. */
static void cell_geometry(oplan *pl, ocell *C) {
  const double *T = tan_table();
  int64_t amid = (C->alo + C->ahi) / 2, bmid = (C->blo + C->bhi) / 2;
  face_point(C->face, T[amid], T[bmid], C->c);
  double corner[3];
  double r = 0.0, d;
  face_point(C->face, T[C->alo], T[C->blo], corner); d = chord(corner, C->c); if (d > r) r = d;
  face_point(C->face, T[C->ahi], T[C->blo], corner); d = chord(corner, C->c); if (d > r) r = d;
  face_point(C->face, T[C->alo], T[C->bhi], corner); d = chord(corner, C->c); if (d > r) r = d;
  face_point(C->face, T[C->ahi], T[C->bhi], corner); d = chord(corner, C->c); if (d > r) r = d;
  C->r = r;
  double H = ldexp(OR_HALF_PI, -OR_D);      /* angle of one fine step */
  double H2 = ldexp(OR_HALF_PI, -(OR_D + 1));
  C->hx = (double)(C->ahi - C->alo) * H2;
  C->hy = (double)(C->bhi - C->blo) * H2;
  C->xi_mid = (double)amid * H - OR_QUARTER_PI;
  C->eta_mid = (double)bmid * H - OR_QUARTER_PI;
  (void)pl;
}

/* Position of child node s in the parent's interpolation coordinate along
 * one axis, from the boxes in fine units: (2 (mid_c - mid_p) + w_c s) / w_p. */
static double child_node(int64_t clo, int64_t chi, int64_t plo, int64_t phi, double s) {
  double dm = (double)((clo + chi) - (plo + phi));
  return (dm + (double)(chi - clo) * s) / (double)(phi - plo);
}

/* Dual tree traversal, Algorithm "CSFMM" (Sec. 8). */
static void traverse(oplan *pl, int t, int s) {
  const ocell *T = &pl->cells[t], *S = &pl->cells[s];
  double R = chord(T->c, S->c);
  double lhs = T->r + S->r, rhs = pl->theta * R;
  int sep = (g_mutation == 7) ? (lhs > rhs) : (lhs < rhs);
  if (R > 0.0) {
    double m = fabs(lhs - rhs) / rhs;
    if (m < pl->margin) pl->margin = m;
    pl->n_mac_tests++;
  }
  int bigT = T->nchild > 0, bigS = S->nchild > 0;
  if (sep && (bigT || bigS)) {
    if (!bigT && bigS) list_push(pl, OR_PC, t, s);
    else if (bigT && !bigS) list_push(pl, OR_CP, t, s);
    else list_push(pl, OR_CC, t, s);
  } else if (bigT || bigS) {
    int split_t;
    if (bigT && bigS) split_t = (T->level <= S->level);
    else split_t = bigT;
    if (split_t) {
      for (int c = 0; c < 4; ++c)
        if (T->child[c] >= 0) traverse(pl, T->child[c], s);
    } else {
      for (int c = 0; c < 4; ++c)
        if (S->child[c] >= 0) traverse(pl, t, S->child[c]);
    }
  } else {
    list_push(pl, OR_PP, t, s);
  }
}

void oracle_fmm_destroy(void *h);

/* Builds the tree (Sec. 3), the cell geometry and proxies (Sec. 4) and the
 * interaction lists (Sec. 8).  Returns NULL on invalid input. */
void *oracle_fmm_create(const double *pts, int64_t N, int n, double theta, int N0, int shrink) {
  if (!pts || N < 1 || n < 1 || n > 64 || !(theta > 0.0) || N0 < 1) return NULL;
  const double *T = tan_table();
  oplan *pl = (oplan *)calloc(1, sizeof(oplan));
  pl->N = N; pl->n = n; pl->p = n + 1; pl->P = (n + 1) * (n + 1); pl->N0 = N0;
  pl->shrink = shrink != 0;
  pl->theta = theta;
  pl->margin = INFINITY;

  /* keys: face, then Morton interleave of the fine (a, b) coordinates */
  okey *keys = (okey *)malloc(sizeof(okey) * (size_t)N);
  int64_t *qa = (int64_t *)malloc(sizeof(int64_t) * (size_t)N);
  int64_t *qb = (int64_t *)malloc(sizeof(int64_t) * (size_t)N);
  int *fc = (int *)malloc(sizeof(int) * (size_t)N);
#pragma omp parallel for
  for (int64_t i = 0; i < N; ++i) {
    int f; double a, b;
    face_coords(pts + 3 * i, &f, &a, &b);
    qa[i] = fine_coord(T, a);
    qb[i] = fine_coord(T, b);
    fc[i] = f;
    keys[i].key = ((uint64_t)f << (2 * OR_D)) | interleave((uint64_t)qa[i], (uint64_t)qb[i]);
    keys[i].idx = i;
  }
  qsort(keys, (size_t)N, sizeof(okey), okey_cmp);
  pl->order = (int64_t *)malloc(sizeof(int64_t) * (size_t)N);
  pl->x = (double *)malloc(sizeof(double) * 3 * (size_t)N);
  uint64_t *skey = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)N);
  int64_t *sqa = (int64_t *)malloc(sizeof(int64_t) * (size_t)N);
  int64_t *sqb = (int64_t *)malloc(sizeof(int64_t) * (size_t)N);
  for (int64_t i = 0; i < N; ++i) {
    pl->order[i] = keys[i].idx;
    skey[i] = keys[i].key;
    sqa[i] = qa[keys[i].idx];
    sqb[i] = qb[keys[i].idx];
    memcpy(pl->x + 3 * i, pts + 3 * keys[i].idx, 3 * sizeof(double));
  }
  free(keys);

  /* cells, level by level; a cell is the key range sharing its prefix */
  int cap = 1024;
  pl->cells = (ocell *)malloc(sizeof(ocell) * (size_t)cap);
  pl->level_begin = (int *)malloc(sizeof(int) * (OR_LMAX + 2));
  int nc = 0;
  pl->level_begin[0] = 0;
  {
    int64_t pos = 0;
    for (int f = 0; f < 6; ++f) {
      int64_t b = pos;
      while (pos < N && (int)(skey[pos] >> (2 * OR_D)) == f) ++pos;
      if (pos > b) {
        ocell C; memset(&C, 0, sizeof C);
        C.face = f; C.level = 0; C.ia = 0; C.ib = 0; C.begin = b; C.end = pos;
        C.parent = -1; for (int c = 0; c < 4; ++c) C.child[c] = -1;
        pl->cells[nc++] = C;
      }
    }
  }
  int nlev = 1;
  for (int l = 0; l < OR_LMAX; ++l) {
    int lb = pl->level_begin[l], le = nc;
    pl->level_begin[l + 1] = le;
    int any = 0;
    for (int ci = lb; ci < le; ++ci) {
      if (pl->cells[ci].end - pl->cells[ci].begin <= N0) continue;
      int sh = 2 * (OR_D - l - 1);
      int64_t pos = pl->cells[ci].begin;
      for (int q = 0; q < 4; ++q) {
        int64_t b = pos;
        while (pos < pl->cells[ci].end && (int)((skey[pos] >> sh) & 3u) == q) ++pos;
        if (pos == b) continue;
        if (nc == cap) { cap *= 2; pl->cells = (ocell *)realloc(pl->cells, sizeof(ocell) * (size_t)cap); }
        ocell C; memset(&C, 0, sizeof C);
        C.face = pl->cells[ci].face; C.level = l + 1;
        C.ia = 2 * pl->cells[ci].ia + (q & 1);
        C.ib = 2 * pl->cells[ci].ib + (q >> 1);
        C.begin = b; C.end = pos; C.parent = ci;
        for (int c = 0; c < 4; ++c) C.child[c] = -1;
        pl->cells[ci].child[q] = nc;
        pl->cells[ci].nchild++;
        pl->cells[nc++] = C;
        any = 1;
      }
    }
    if (!any) break;
    nlev = l + 2;
  }
  pl->level_begin[nlev] = nc;
  pl->ncells = nc;
  pl->nlevels = nlev;
  /* boxes: the dyadic square, or (shrinking) the fine cells of the points
   * widened to even edges */
  for (int ci = 0; ci < nc; ++ci) {
    ocell *C = &pl->cells[ci];
    int sh = OR_D - C->level;
    C->alo = C->ia << sh; C->ahi = (C->ia + 1) << sh;
    C->blo = C->ib << sh; C->bhi = (C->ib + 1) << sh;
    if (pl->shrink) {
      int64_t amin = INT64_MAX, amax = -1, bmin = INT64_MAX, bmax = -1;
      for (int64_t i = C->begin; i < C->end; ++i) {
        if (sqa[i] < amin) amin = sqa[i];
        if (sqa[i] > amax) amax = sqa[i];
        if (sqb[i] < bmin) bmin = sqb[i];
        if (sqb[i] > bmax) bmax = sqb[i];
      }
      C->alo = amin & ~(int64_t)1;
      C->ahi = (amax + (g_mutation == 15 ? 0 : 2)) & ~(int64_t)1;
      C->blo = bmin & ~(int64_t)1; C->bhi = (bmax + 2) & ~(int64_t)1;
    }
  }
  free(skey); free(qa); free(qb); free(fc); free(sqa); free(sqb);

  /* geometry, proxies, leaf membership and local coordinates */
  pl->s = (double *)malloc(sizeof(double) * (size_t)pl->p);
  oracle_cheb_nodes(n, pl->s);
  pl->proxy = (double *)malloc(sizeof(double) * 3 * (size_t)nc * (size_t)pl->P);
  pl->leaf_of = (int *)malloc(sizeof(int) * (size_t)N);
  pl->u = (double *)malloc(sizeof(double) * (size_t)N);
  pl->v = (double *)malloc(sizeof(double) * (size_t)N);
#pragma omp parallel for schedule(dynamic, 8)
  for (int ci = 0; ci < nc; ++ci) {
    ocell *C = &pl->cells[ci];
    cell_geometry(pl, C);
    for (int k1 = 0; k1 <= n; ++k1)
      for (int k2 = 0; k2 <= n; ++k2) {
        double a = tan(C->xi_mid + C->hx * pl->s[k1]);
        double b = tan(C->eta_mid + C->hy * pl->s[k2]);
        face_point(C->face, a, b, pl->proxy + 3 * ((int64_t)ci * pl->P + k1 * pl->p + k2));
      }
    if (C->nchild == 0) {
      for (int64_t i = C->begin; i < C->end; ++i) {
        int f; double a, b;
        face_coords(pl->x + 3 * i, &f, &a, &b);
        pl->leaf_of[i] = ci;
        pl->u[i] = (atan(a) - C->xi_mid) / C->hx;
        pl->v[i] = (atan(b) - C->eta_mid) / C->hy;
      }
    }
  }

  /* dual tree traversal over all ordered pairs of root clusters */
  int nroots = pl->level_begin[1];
  for (int t = 0; t < nroots; ++t)
    for (int s = 0; s < nroots; ++s) traverse(pl, t, s);
  return pl;
}

void oracle_fmm_destroy(void *h) {
  oplan *pl = (oplan *)h;
  if (!pl) return;
  free(pl->x); free(pl->order); free(pl->u); free(pl->v); free(pl->leaf_of);
  free(pl->cells); free(pl->level_begin); free(pl->s); free(pl->proxy);
  for (int t = 0; t < 4; ++t) free(pl->list[t]);
  free(pl);
}

/* info[0..] = ncells, nleaves, nlevels, nPP, nPC, nCP, nCC, n_mac_tests,
 *             kernel evaluations (PP excl. self, PC, CP, CC), pairs covered */
int oracle_fmm_info(void *h, int64_t *info, double *margin) {
  oplan *pl = (oplan *)h;
  if (!pl) return 1;
  int64_t nleaves = 0;
  for (int c = 0; c < pl->ncells; ++c) nleaves += pl->cells[c].nchild == 0;
  int64_t evals = 0, covered = 0;
  for (int ty = 0; ty < 4; ++ty)
    for (int64_t e = 0; e < pl->nlist[ty]; ++e) {
      const ocell *T = &pl->cells[pl->list[ty][e].t], *S = &pl->cells[pl->list[ty][e].s];
      int64_t nt = T->end - T->begin, ns = S->end - S->begin;
      covered += nt * ns;
      if (ty == OR_PP) evals += nt * ns - (pl->list[ty][e].t == pl->list[ty][e].s ? nt : 0);
      else if (ty == OR_PC) evals += nt * pl->P;
      else if (ty == OR_CP) evals += (int64_t)pl->P * ns;
      else evals += (int64_t)pl->P * pl->P;
    }
  info[0] = pl->ncells; info[1] = nleaves; info[2] = pl->nlevels;
  info[3] = pl->nlist[OR_PP]; info[4] = pl->nlist[OR_PC];
  info[5] = pl->nlist[OR_CP]; info[6] = pl->nlist[OR_CC];
  info[7] = pl->n_mac_tests; info[8] = evals; info[9] = covered;
  if (margin) *margin = pl->margin;
  return 0;
}

/* Cells in the oracle's order: face, level, ia, ib, begin, end, parent,
 * child[4]; centre [3] and radius. */
int oracle_fmm_cells(void *h, int32_t *face, int32_t *level, int64_t *ia, int64_t *ib,
                     int64_t *begin, int64_t *end, int32_t *parent, int32_t *child,
                     double *centre, double *radius) {
  oplan *pl = (oplan *)h;
  if (!pl) return 1;
  for (int c = 0; c < pl->ncells; ++c) {
    const ocell *C = &pl->cells[c];
    face[c] = C->face; level[c] = C->level; ia[c] = C->ia; ib[c] = C->ib;
    begin[c] = C->begin; end[c] = C->end; parent[c] = C->parent;
    for (int q = 0; q < 4; ++q) child[4 * c + q] = C->child[q];
    memcpy(centre + 3 * c, C->c, 3 * sizeof(double));
    radius[c] = C->r;
  }
  return 0;
}

int oracle_fmm_list(void *h, int type, int32_t *t, int32_t *s) {
  oplan *pl = (oplan *)h;
  if (!pl || type < 0 || type > 3) return 1;
  for (int64_t e = 0; e < pl->nlist[type]; ++e) {
    t[e] = pl->list[type][e].t;
    s[e] = pl->list[type][e].s;
  }
  return 0;
}

int oracle_fmm_order(void *h, int64_t *order) {
  oplan *pl = (oplan *)h;
  if (!pl) return 1;
  memcpy(order, pl->order, sizeof(int64_t) * (size_t)pl->N);
  return 0;
}

int oracle_fmm_proxies(void *h, double *proxy) {
  oplan *pl = (oplan *)h;
  if (!pl) return 1;
  memcpy(proxy, pl->proxy, sizeof(double) * 3 * (size_t)pl->ncells * (size_t)pl->P);
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Evaluation.                                                                */
/* ------------------------------------------------------------------------ */

/* CSR of a list grouped by target cell (stable in list order). */
static void group_by_target(const oplan *pl, int type, int64_t **off, int **src) {
  int nc = pl->ncells;
  int64_t *o = (int64_t *)calloc((size_t)nc + 1, sizeof(int64_t));
  for (int64_t e = 0; e < pl->nlist[type]; ++e) o[pl->list[type][e].t + 1]++;
  for (int c = 0; c < nc; ++c) o[c + 1] += o[c];
  int64_t *fill = (int64_t *)malloc(sizeof(int64_t) * (size_t)nc);
  memcpy(fill, o, sizeof(int64_t) * (size_t)nc);
  int *sv = (int *)malloc(sizeof(int) * (size_t)(pl->nlist[type] + 1));
  for (int64_t e = 0; e < pl->nlist[type]; ++e) sv[fill[pl->list[type][e].t]++] = pl->list[type][e].s;
  free(fill);
  *off = o; *src = sv;
}

/* Proxy weights wbar[c][r][k] for every cell: leaves directly by Eq. (PC),
 * parents from their children by Eq. (upwardpass2), bottom-up (Sec. 6). */
static void upward_pass(const oplan *pl, const double *ws, int nrhs, double *wbar) {
  int n = pl->n, p = pl->p, P = pl->P;
  int64_t N = pl->N;
  /* P2M at the leaves */
#pragma omp parallel for schedule(dynamic, 4)
  for (int c = 0; c < pl->ncells; ++c) {
    const ocell *C = &pl->cells[c];
    if (C->nchild) continue;
    double La[65], Lb[65];
    for (int r = 0; r < nrhs; ++r)
      for (int k = 0; k < P; ++k) wbar[((int64_t)c * nrhs + r) * P + k] = 0.0;
    for (int64_t j = C->begin; j < C->end; ++j) {
      oracle_lagrange(n, pl->s, pl->u[j], La);
      oracle_lagrange(n, pl->s, pl->v[j], Lb);
      for (int r = 0; r < nrhs; ++r) {
        double wj = ws[(int64_t)r * N + ((g_mutation == 10) ? pl->order[j] % N : j)];
        for (int k1 = 0; k1 <= n; ++k1)
          for (int k2 = 0; k2 <= n; ++k2)
            wbar[((int64_t)c * nrhs + r) * P + k1 * p + k2] += La[k1] * Lb[k2] * wj;
      }
    }
  }
  /* M2M: parent proxy weights from child proxy weights, deepest level first */
  for (int l = pl->nlevels - 2; l >= 0; --l) {
#pragma omp parallel for schedule(dynamic, 4)
    for (int c = pl->level_begin[l]; c < pl->level_begin[l + 1]; ++c) {
      const ocell *C = &pl->cells[c];
      if (!C->nchild) continue;
      double *wp = wbar + (int64_t)c * nrhs * P;
      for (int k = 0; k < nrhs * P; ++k) wp[k] = 0.0;
      for (int q = 0; q < 4; ++q) {
        int ch = C->child[q];
        if (ch < 0) continue;
        const ocell *K = &pl->cells[ch];
        double La[65 * 65], Lb[65 * 65]; /* [m][k]: parent L_k at child node m */
        for (int m = 0; m <= n; ++m) {
          double ta = child_node(K->alo, K->ahi, C->alo, C->ahi, pl->s[m]);
          if (g_mutation == 3)  /* the child's box mirrored inside the parent */
            ta = child_node(C->alo + C->ahi - K->ahi, C->alo + C->ahi - K->alo, C->alo, C->ahi,
                            pl->s[m]);
          oracle_lagrange(n, pl->s, ta, La + m * p);
          oracle_lagrange(n, pl->s, child_node(K->blo, K->bhi, C->blo, C->bhi, pl->s[m]), Lb + m * p);
        }
        const double *wc = wbar + (int64_t)ch * nrhs * P;
        for (int r = 0; r < nrhs; ++r)
          for (int k1 = 0; k1 <= n; ++k1)
            for (int k2 = 0; k2 <= n; ++k2) {
              double acc = 0.0;
              for (int m1 = 0; m1 <= n; ++m1)
                for (int m2 = 0; m2 <= n; ++m2)
                  acc += La[m1 * p + k1] * Lb[m2 * p + k2] * wc[r * P + m1 * p + m2];
              wp[r * P + k1 * p + k2] += acc;
            }
      }
    }
  }
}

/* CSFMM evaluation (Algorithm "CSFMM").  w[r][N] in input order.  If tgt is
 * NULL, out[r][N][dim] receives every potential in input order; otherwise
 * out[r][t][dim] receives the potentials of the ntgt input indices tgt[t],
 * and only the cells on the paths from the root to their leaves are
 * visited in the interaction and downward phases (same arithmetic). */
static int fmm_evaluate(oplan *pl, int kid, const double *w, int nrhs,
                        const int64_t *tgt, int64_t ntgt, double *out) {
  int n = pl->n, p = pl->p, P = pl->P, nc = pl->ncells;
  int dim = oracle_kernel_dim(kid);
  int64_t N = pl->N;

  /* which sorted positions and cells are needed */
  char *need_pt = (char *)malloc((size_t)N);
  char *need_cell = (char *)malloc((size_t)nc);
  int64_t *pos_of = NULL;
  if (tgt) {
    memset(need_pt, 0, (size_t)N);
    memset(need_cell, 0, (size_t)nc);
    int64_t *inv = (int64_t *)malloc(sizeof(int64_t) * (size_t)N);
    for (int64_t i = 0; i < N; ++i) inv[pl->order[i]] = i;
    pos_of = (int64_t *)malloc(sizeof(int64_t) * (size_t)ntgt);
    for (int64_t t = 0; t < ntgt; ++t) {
      if (tgt[t] < 0 || tgt[t] >= N) { free(inv); free(pos_of); free(need_pt); free(need_cell); return 1; }
      int64_t i = inv[tgt[t]];
      pos_of[t] = i;
      need_pt[i] = 1;
      for (int c = pl->leaf_of[i]; c >= 0; c = pl->cells[c].parent) need_cell[c] = 1;
    }
    free(inv);
  } else {
    memset(need_pt, 1, (size_t)N);
    memset(need_cell, 1, (size_t)nc);
  }

  /* weights in sorted order */
  double *ws = (double *)malloc(sizeof(double) * (size_t)N * (size_t)nrhs);
  for (int r = 0; r < nrhs; ++r)
    for (int64_t i = 0; i < N; ++i) ws[(int64_t)r * N + i] = w[(int64_t)r * N + pl->order[i]];

  /* Algorithm "CSFMM": upward pass */
  double *wbar = (double *)malloc(sizeof(double) * (size_t)nc * (size_t)nrhs * (size_t)P);
  upward_pass(pl, ws, nrhs, wbar);

  int64_t *off[4]; int *src[4];
  for (int ty = 0; ty < 4; ++ty) group_by_target(pl, ty, &off[ty], &src[ty]);

  /* CP and CC proxy potentials, accumulated per target cell
   * (Eq. CP_CC_accumulated).  psi[c][r][m][d]. */
  size_t psz = (size_t)nc * (size_t)nrhs * (size_t)P * (size_t)dim;
  double *psi = (double *)calloc(psz, sizeof(double));
#pragma omp parallel for schedule(dynamic, 1)
  for (int t = 0; t < nc; ++t) {
    if (!need_cell[t]) continue;
    const double *tp = pl->proxy + 3 * (int64_t)t * P;
    double *pt = psi + (int64_t)t * nrhs * P * dim;
    /* CP: sources are the particles of a small cluster (Eq. CP) */
    for (int64_t e = off[OR_CP][t]; e < off[OR_CP][t + 1]; ++e) {
      const ocell *S = &pl->cells[src[OR_CP][e]];
      for (int m = 0; m < P; ++m)
        for (int64_t j = S->begin; j < S->end; ++j) {
          double k[3];
          kernel_eval(kid, tp + 3 * m, pl->x + 3 * j, k);
          for (int r = 0; r < nrhs; ++r)
            for (int d = 0; d < dim; ++d)
              pt[(r * P + m) * dim + d] += k[d] * ws[(int64_t)r * N + j];
        }
    }
    /* CC: sources are the proxies of a big cluster (Eq. CC) */
    for (int64_t e = off[OR_CC][t]; e < off[OR_CC][t + 1]; ++e) {
      int s = src[OR_CC][e];
      const double *sp = pl->proxy + 3 * (int64_t)s * P;
      for (int m = 0; m < P; ++m)
        for (int kk = 0; kk < P; ++kk) {
          double k[3];
          kernel_eval(kid, tp + 3 * m, sp + 3 * kk, k);
          for (int r = 0; r < nrhs; ++r)
            for (int d = 0; d < dim; ++d)
              pt[(r * P + m) * dim + d] += k[d] * wbar[((int64_t)s * nrhs + r) * P + kk];
        }
    }
  }

  /* PC and PP potentials at the target particles. */
  double *phi = (double *)calloc((size_t)N * (size_t)nrhs * (size_t)dim, sizeof(double));
#pragma omp parallel for schedule(dynamic, 1)
  for (int t = 0; t < nc; ++t) {
    const ocell *T = &pl->cells[t];
    if (!need_cell[t] || (off[OR_PP][t] == off[OR_PP][t + 1] && off[OR_PC][t] == off[OR_PC][t + 1]))
      continue;
    double *a = (double *)malloc(sizeof(double) * (size_t)(nrhs * dim));
    for (int64_t i = T->begin; i < T->end; ++i) {
      if (!need_pt[i]) continue;
      for (int q = 0; q < nrhs * dim; ++q) a[q] = 0.0;
      /* PP (Eq. PP), the i = j term omitted */
      for (int64_t e = off[OR_PP][t]; e < off[OR_PP][t + 1]; ++e) {
        const ocell *S = &pl->cells[src[OR_PP][e]];
        for (int64_t j = S->begin; j < S->end; ++j) {
          if (j == i && g_mutation != 5) continue;
          double k[3];
          kernel_eval(kid, pl->x + 3 * i, pl->x + 3 * j, k);
          for (int r = 0; r < nrhs; ++r)
            for (int d = 0; d < dim; ++d) a[r * dim + d] += k[d] * ws[(int64_t)r * N + j];
        }
      }
      /* PC (Eq. PC) */
      if (g_mutation != 1) {
        for (int64_t e = off[OR_PC][t]; e < off[OR_PC][t + 1]; ++e) {
          int s = src[OR_PC][e];
          const double *sp = pl->proxy + 3 * (int64_t)s * P;
          for (int kk = 0; kk < P; ++kk) {
            double k[3];
            kernel_eval(kid, pl->x + 3 * i, sp + 3 * kk, k);
            for (int r = 0; r < nrhs; ++r)
              for (int d = 0; d < dim; ++d)
                a[r * dim + d] += k[d] * wbar[((int64_t)s * nrhs + r) * P + kk];
          }
        }
      }
      for (int r = 0; r < nrhs; ++r)
        for (int d = 0; d < dim; ++d) phi[((int64_t)r * N + i) * dim + d] = a[r * dim + d];
    }
    free(a);
  }

  /* Downward pass.  L2L through all levels (Eq. downward_2) ... */
  for (int l = 0; l + 1 < pl->nlevels; ++l) {
    if (g_mutation == 9 && l == pl->nlevels - 2) continue;
#pragma omp parallel for schedule(dynamic, 4)
    for (int c = pl->level_begin[l]; c < pl->level_begin[l + 1]; ++c) {
      const ocell *C = &pl->cells[c];
      if (!need_cell[c]) continue;
      const double *pp = psi + (int64_t)c * nrhs * P * dim;
      for (int q = 0; q < 4; ++q) {
        int ch = C->child[q];
        if (ch < 0 || !need_cell[ch]) continue;
        const ocell *K = &pl->cells[ch];
        double La[65 * 65], Lb[65 * 65]; /* [nn][m]: parent L_m at child node nn */
        for (int nn = 0; nn <= n; ++nn) {
          oracle_lagrange(n, pl->s, child_node(K->alo, K->ahi, C->alo, C->ahi, pl->s[nn]),
                          La + nn * p);
          oracle_lagrange(n, pl->s, child_node(K->blo, K->bhi, C->blo, C->bhi, pl->s[nn]),
                          Lb + nn * p);
        }
        double *pc = psi + (int64_t)ch * nrhs * P * dim;
        for (int r = 0; r < nrhs; ++r)
          for (int n1 = 0; n1 <= n; ++n1)
            for (int n2 = 0; n2 <= n; ++n2)
              for (int d = 0; d < dim; ++d) {
                double acc = 0.0;
                for (int m1 = 0; m1 <= n; ++m1)
                  for (int m2 = 0; m2 <= n; ++m2)
                    acc += pp[(r * P + m1 * p + m2) * dim + d] * La[n1 * p + m1] * Lb[n2 * p + m2];
                pc[(r * P + n1 * p + n2) * dim + d] += acc;
              }
      }
    }
  }
  /* ... then from the leaf proxies to the particles. */
#pragma omp parallel for schedule(dynamic, 4)
  for (int c = 0; c < nc; ++c) {
    const ocell *C = &pl->cells[c];
    if (C->nchild || !need_cell[c]) continue;
    const double *pc = psi + (int64_t)c * nrhs * P * dim;
    double La[65], Lb[65];
    for (int64_t i = C->begin; i < C->end; ++i) {
      if (!need_pt[i]) continue;
      oracle_lagrange(n, pl->s, pl->u[i], La);
      oracle_lagrange(n, pl->s, (g_mutation == 6) ? pl->u[i] : pl->v[i], Lb);
      for (int r = 0; r < nrhs; ++r)
        for (int d = 0; d < dim; ++d) {
          double acc = 0.0;
          for (int m1 = 0; m1 <= n; ++m1)
            for (int m2 = 0; m2 <= n; ++m2)
              acc += pc[(r * P + m1 * p + m2) * dim + d] * La[m1] * Lb[m2];
          phi[((int64_t)r * N + i) * dim + d] += acc;
        }
    }
  }

  /* Output */
  if (tgt) {
    for (int r = 0; r < nrhs; ++r)
      for (int64_t t = 0; t < ntgt; ++t)
        for (int d = 0; d < dim; ++d)
          out[((int64_t)r * ntgt + t) * dim + d] = phi[((int64_t)r * N + pos_of[t]) * dim + d];
  } else {
    for (int r = 0; r < nrhs; ++r)
      for (int64_t i = 0; i < N; ++i)
        for (int d = 0; d < dim; ++d)
          out[((int64_t)r * N + pl->order[i]) * dim + d] = phi[((int64_t)r * N + i) * dim + d];
  }

  free(ws); free(wbar); free(psi); free(phi); free(need_pt); free(need_cell); free(pos_of);
  for (int ty = 0; ty < 4; ++ty) { free(off[ty]); free(src[ty]); }
  return 0;
}

int oracle_fmm_evaluate(void *h, int kid, const double *w, int nrhs, double *out) {
  oplan *pl = (oplan *)h;
  if (!pl || !kernel_valid(kid) || nrhs < 1 || !w || !out) return 1;
  return fmm_evaluate(pl, kid, w, nrhs, NULL, 0, out);
}

int oracle_fmm_evaluate_targets(void *h, int kid, const double *w, int nrhs,
                                const int64_t *tgt, int64_t ntgt, double *out) {
  oplan *pl = (oplan *)h;
  if (!pl || !kernel_valid(kid) || nrhs < 1 || !w || !out || !tgt || ntgt < 0) return 1;
  return fmm_evaluate(pl, kid, w, nrhs, tgt, ntgt, out);
}

/* ------------------------------------------------------------------------ */
/* Cubed sphere tree code (Sec. 7, Algorithm "CSTC").  Each target particle  */
/* x_i walks the source tree from the six root cells.  A cluster C_s that is */
/* well separated from x_i (r_s < MAC R, R = |x_i - c_s|) contributes through */
/* its proxies by Eq. (PC) if it has more than N0 particles (it has           */
/* children) and directly by Eq. (PP) otherwise; a cluster that is not well  */
/* separated passes x_i on to its children, and a leaf that is not well      */
/* separated contributes directly.  The proxy weights come from the same     */
/* upward pass as the CSFMM (Sec. 6).                                        */
/* ------------------------------------------------------------------------ */
typedef struct {
  const oplan *pl;
  int kid, nrhs, dim;
  const double *ws, *wbar;
  int64_t i;          /* target, sorted position */
  ksum *acc;          /* [nrhs][dim] */
  int64_t npc, npp, evals;
  double margin;
} cstc_walk;

static void cstc_visit(cstc_walk *X, int c) {
  const oplan *pl = X->pl;
  const ocell *C = &pl->cells[c];
  const double *x = pl->x + 3 * X->i;
  const int P = pl->P, nrhs = X->nrhs, dim = X->dim;
  const int64_t N = pl->N;
  double R = chord(x, C->c);
  double rhs = pl->theta * R;
  int sep = (g_mutation == 11) ? (C->r > rhs) : (C->r < rhs);
  if (R > 0.0) {
    double m = fabs(C->r - rhs) / rhs;
    if (m < X->margin) X->margin = m;
  }
  double k[3];
  if (sep && C->nchild > 0) {
    /* PC: x_i against the proxies of C_s with their proxy weights */
    for (int q = 0; q < P; ++q) {
      kernel_eval(X->kid, x, pl->proxy + 3 * ((int64_t)c * P + q), k);
      for (int r = 0; r < nrhs; ++r) {
        double wq = X->wbar[((int64_t)c * nrhs + r) * P + q];
        for (int d = 0; d < dim; ++d) ksum_add(&X->acc[r * dim + d], k[d] * wq);
      }
    }
    X->npc++;
    X->evals += P;
  } else if (sep || C->nchild == 0) {
    if (!sep && g_mutation == 12) return;
    /* PP: x_i against the particles of C_s, j = i omitted */
    for (int64_t j = C->begin; j < C->end; ++j) {
      if (j == X->i) continue;
      kernel_eval(X->kid, x, pl->x + 3 * j, k);
      for (int r = 0; r < nrhs; ++r) {
        double wj = X->ws[(int64_t)r * N + j];
        for (int d = 0; d < dim; ++d) ksum_add(&X->acc[r * dim + d], k[d] * wj);
      }
      X->evals++;
    }
    X->npp++;
  } else {
    for (int q = 0; q < 4; ++q)
      if (C->child[q] >= 0) cstc_visit(X, (g_mutation == 13 && q == 3) ? C->child[0] : C->child[q]);
  }
}

/* CSTC potentials out[r][t][dim] of the input indices tgt[t] (every point if
 * tgt == NULL); stats (optional) = {PC interactions, PP interactions, kernel
 * evaluations} summed over the targets, and *margin the smallest
 * |r_s - MAC R| / (MAC R) over all separation tests. */
int oracle_cstc_evaluate(void *h, int kid, const double *w, int nrhs, const int64_t *tgt,
                         int64_t ntgt, double *out, int64_t *stats, double *margin) {
  oplan *pl = (oplan *)h;
  if (!pl || !kernel_valid(kid) || nrhs < 1 || nrhs > 64 || !w || !out || (tgt && ntgt < 0))
    return 1;
  const int64_t N = pl->N;
  const int dim = oracle_kernel_dim(kid), P = pl->P;
  if (!tgt) ntgt = N;
  int64_t *inv = (int64_t *)malloc(sizeof(int64_t) * (size_t)N);
  for (int64_t i = 0; i < N; ++i) inv[pl->order[i]] = i;
  for (int64_t t = 0; tgt && t < ntgt; ++t)
    if (tgt[t] < 0 || tgt[t] >= N) { free(inv); return 1; }
  double *ws = (double *)malloc(sizeof(double) * (size_t)N * (size_t)nrhs);
  for (int r = 0; r < nrhs; ++r)
    for (int64_t i = 0; i < N; ++i) ws[(int64_t)r * N + i] = w[(int64_t)r * N + pl->order[i]];
  double *wbar = (double *)malloc(sizeof(double) * (size_t)pl->ncells * (size_t)nrhs * (size_t)P);
  upward_pass(pl, ws, nrhs, wbar);
  int64_t tot_pc = 0, tot_pp = 0, tot_ev = 0;
  double mg = INFINITY;
#pragma omp parallel for schedule(dynamic, 64) reduction(+ : tot_pc, tot_pp, tot_ev) reduction(min : mg)
  for (int64_t t = 0; t < ntgt; ++t) {
    ksum acc[64 * 3];
    for (int u = 0; u < nrhs * dim; ++u) { acc[u].s = 0.0; acc[u].c = 0.0; }
    const int64_t in = tgt ? tgt[t] : t;
    cstc_walk X = {pl, kid, nrhs, dim, ws, wbar, inv[in], acc, 0, 0, 0, INFINITY};
    for (int c = pl->level_begin[0]; c < pl->level_begin[1]; ++c) cstc_visit(&X, c);
    for (int r = 0; r < nrhs; ++r)
      for (int d = 0; d < dim; ++d)
        out[((int64_t)r * ntgt + t) * dim + d] = acc[r * dim + d].s + acc[r * dim + d].c;
    tot_pc += X.npc;
    tot_pp += X.npp;
    tot_ev += X.evals;
    if (X.margin < mg) mg = X.margin;
  }
  if (stats) { stats[0] = tot_pc; stats[1] = tot_pp; stats[2] = tot_ev; }
  if (margin) *margin = mg;
  free(ws); free(wbar); free(inv);
  return 0;
}

/* Proxy weights of every cell after the upward pass, [ncells][nrhs][P],
 * for the moment-identity pins. */
int oracle_fmm_upward(void *h, const double *w, int nrhs, double *wbar) {
  oplan *pl = (oplan *)h;
  if (!pl || nrhs < 1 || !w || !wbar) return 1;
  int64_t N = pl->N;
  double *ws = (double *)malloc(sizeof(double) * (size_t)N * (size_t)nrhs);
  for (int r = 0; r < nrhs; ++r)
    for (int64_t i = 0; i < N; ++i) ws[(int64_t)r * N + i] = w[(int64_t)r * N + pl->order[i]];
  upward_pass(pl, ws, nrhs, wbar);
  free(ws);
  return 0;
}

/* Local (u, v) coordinates of each sorted point in its leaf, and its leaf. */
int oracle_fmm_local(void *h, double *u, double *v, int32_t *leaf) {
  oplan *pl = (oplan *)h;
  if (!pl) return 1;
  for (int64_t i = 0; i < pl->N; ++i) { u[i] = pl->u[i]; v[i] = pl->v[i]; leaf[i] = pl->leaf_of[i]; }
  return 0;
}

int oracle_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

/* Number of OpenMP threads of later calls (n >= 1). */
void oracle_set_num_threads(int n) {
#ifdef _OPENMP
  if (n >= 1) omp_set_num_threads(n);
#else
  (void)n;
#endif
}
