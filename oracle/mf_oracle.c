/*
 * mf_oracle.c -- plain FP64 CPU oracle for manifold tracing over the Coxeter
 * triangulation and for the capsule/obstacle certification of the traced points.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test-suite, the package smoke check and
 * the benchmark's CPU-baseline leg load this library.  The CUDA library shares
 * no code, header, table or constant with it, and neither calls the other.
 *
 * Every routine restates one passage of arXiv 2406.04795 ("Scaling Motion
 * Planning Infeasibility Proofs", Li & Dantam) in the most literal form:
 * general simplices as (vertex, ordered partition) records, the paper's query
 * types written out one by one, sums in index order, no blocking and no
 * fusion.  The file is compiled with -ffp-contract=off so that each product
 * and each sum is rounded on its own.
 *
 * Readings where the paper is silent or garbled (each one is also listed in
 * the repository design notes):
 *   R1  Ã_d realisation (Sec. II-B only names "root systems"): x = lam*L*y + o
 *       with L = I - c*1*1^T, c = (1 - 1/sqrt(d+1))/d.
 *   R2  Canonical permutahedral code: the part that holds d is last
 *       (Fig. 2 codes; the vertex is then the lexicographically smallest).
 *   R3  Locate: floor of the inverse map, fractional parts sorted descending,
 *       ties broken towards the lower index.
 *   R4  Sign: s(v) = [f(v) >= 0]; an edge crosses iff s(v1) != s(v2)
 *       (Sec. IV-A uses the strict product f(v1)f(v2) < 0, which loses exact zeros).
 *   R5  Domain: a simplex is inside iff all its vertices lie in the closed box.
 *   R6  Root: bisection on [0,1] to 2^-50 under the sign rule R4 (the paper
 *       only says "an iterative algorithm", Sec. VI).
 *   R7  Cells: the crossing n-simplices (n-cofaces of traced edges, Sec. IV-B).
 *   R8  Robot links are capsules (segment + radius); a sphere is a zero-length
 *       capsule.  Collision iff distance <= radius (App. A: "no collision"
 *       needs a strict ">").
 *
 * Parity status: every exported function is pinned by the tests under
 * tests/ (worked examples of Fig. 2 and Fig. 5, closed forms, brute force).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_MAXD 8

/* ------------------------------------------------------------------------ */
/* A generic insertion-ordered hash set of fixed-size records (plain C).     */
/* The first key_size bytes of a record are its key.                         */
/* ------------------------------------------------------------------------ */
typedef struct {
  size_t rec_size, key_size;
  size_t n, cap;          /* records stored / allocated */
  unsigned char *recs;
  size_t tcap;            /* table slots, power of two */
  long *table;            /* record index or -1 */
} or_set;

static uint64_t bytes_hash(const unsigned char *p, size_t n) {
  uint64_t h = 1469598103934665603ULL; /* FNV-1a */
  for (size_t i = 0; i < n; i++) { h ^= p[i]; h *= 1099511628211ULL; }
  h ^= h >> 29;
  return h;
}

static int set_init(or_set *s, size_t rec_size, size_t key_size) {
  s->rec_size = rec_size; s->key_size = key_size;
  s->n = 0; s->cap = 1024;
  s->recs = (unsigned char *)malloc(s->cap * rec_size);
  s->tcap = 2048;
  s->table = (long *)malloc(s->tcap * sizeof(long));
  if (!s->recs || !s->table) return -1;
  for (size_t i = 0; i < s->tcap; i++) s->table[i] = -1;
  return 0;
}

static void set_free(or_set *s) { free(s->recs); free(s->table); s->recs = NULL; s->table = NULL; }

static long set_find(const or_set *s, const void *key) {
  size_t h = (size_t)bytes_hash((const unsigned char *)key, s->key_size) & (s->tcap - 1);
  for (;;) {
    long idx = s->table[h];
    if (idx < 0) return -1;
    if (memcmp(s->recs + (size_t)idx * s->rec_size, key, s->key_size) == 0) return idx;
    h = (h + 1) & (s->tcap - 1);
  }
}

static int set_grow(or_set *s) {
  size_t ntcap = s->tcap * 2;
  long *nt = (long *)malloc(ntcap * sizeof(long));
  if (!nt) return -1;
  for (size_t i = 0; i < ntcap; i++) nt[i] = -1;
  for (size_t r = 0; r < s->n; r++) {
    size_t h = (size_t)bytes_hash(s->recs + r * s->rec_size, s->key_size) & (ntcap - 1);
    while (nt[h] >= 0) h = (h + 1) & (ntcap - 1);
    nt[h] = (long)r;
  }
  free(s->table); s->table = nt; s->tcap = ntcap;
  return 0;
}

/* Returns the record index; *inserted = 1 if the record is new. -1 on OOM. */
static long set_insert(or_set *s, const void *rec, int *inserted) {
  long f = set_find(s, rec);
  if (f >= 0) { *inserted = 0; return f; }
  if ((s->n + 1) * 2 > s->tcap && set_grow(s)) return -1;
  if (s->n == s->cap) {
    size_t ncap = s->cap * 2;
    unsigned char *nr = (unsigned char *)realloc(s->recs, ncap * s->rec_size);
    if (!nr) return -1;
    s->recs = nr; s->cap = ncap;
  }
  memcpy(s->recs + s->n * s->rec_size, rec, s->rec_size);
  size_t h = (size_t)bytes_hash((const unsigned char *)rec, s->key_size) & (s->tcap - 1);
  while (s->table[h] >= 0) h = (h + 1) & (s->tcap - 1);
  s->table[h] = (long)s->n;
  *inserted = 1;
  return (long)s->n++;
}

/* ------------------------------------------------------------------------ */
/* Permutahedral representation (Sec. II-B, Fig. 2).                          */
/* A k-simplex is a vertex y in Z^d and an ordered partition of {0..d} into  */
/* k+1 parts (bitmasks over {0..d}).  The j-th vertex is y plus the steps of */
/* parts 0..j-1, where step e_i is the unit vector for i < d and e_d is      */
/* -(1,...,1), so the d+1 steps sum to zero and the walk closes (Sec. II-B). */
/* ------------------------------------------------------------------------ */
typedef struct {
  int32_t y[OR_MAXD];
  int32_t k;
  uint32_t part[OR_MAXD + 1];
} or_simplex;

static void or_simplex_zero(or_simplex *s) { memset(s, 0, sizeof(*s)); }

static void step_add(int d, int32_t *v, uint32_t part) {
  for (int i = 0; i < d; i++)
    if ((part >> i) & 1u) v[i] += 1;
  if ((part >> d) & 1u)
    for (int i = 0; i < d; i++) v[i] -= 1;
}

/* Query type 5 (Sec. IV-A): the k+1 vertices, in walk order. */
void or_simplex_vertices(int d, const or_simplex *s, int32_t *verts) {
  int32_t v[OR_MAXD];
  for (int i = 0; i < d; i++) v[i] = s->y[i];
  for (int j = 0; j <= s->k; j++) {
    for (int i = 0; i < d; i++) verts[j * d + i] = v[i];
    if (j < s->k) step_add(d, v, s->part[j]);
  }
}

/* Reading R2: rotate the cyclic walk so that the part holding d is last. */
void or_canonicalize(int d, or_simplex *s) {
  int j = 0;
  while (j <= s->k && !((s->part[j] >> d) & 1u)) j++;
  if (j >= s->k) return; /* already last (or malformed) */
  /* new start vertex = vertex j+1 of the walk */
  int32_t v[OR_MAXD];
  for (int i = 0; i < d; i++) v[i] = s->y[i];
  for (int t = 0; t <= j; t++) step_add(d, v, s->part[t]);
  uint32_t np[OR_MAXD + 1];
  int n = 0;
  for (int t = j + 1; t <= s->k; t++) np[n++] = s->part[t];
  for (int t = 0; t <= j; t++) np[n++] = s->part[t];
  or_simplex r;
  or_simplex_zero(&r);
  for (int i = 0; i < d; i++) r.y[i] = v[i];
  r.k = s->k;
  for (int t = 0; t <= s->k; t++) r.part[t] = np[t];
  *s = r;
}

/* The edge between walk vertices i < j of a k-simplex: first part is the
 * union of parts i..j-1 (query type 2 for k = n, type 4 for k = 2). */
static void simplex_edge(int d, const or_simplex *s, int i, int j, or_simplex *e) {
  int32_t v[OR_MAXD];
  for (int t = 0; t < d; t++) v[t] = s->y[t];
  for (int t = 0; t < i; t++) step_add(d, v, s->part[t]);
  uint32_t p1 = 0, all = (2u << d) - 1u;
  for (int t = i; t < j; t++) p1 |= s->part[t];
  or_simplex_zero(e);
  for (int t = 0; t < d; t++) e->y[t] = v[t];
  e->k = 1;
  e->part[0] = p1;
  e->part[1] = all & ~p1;
  or_canonicalize(d, e);
}

/* Query type 4 (Sec. IV-A): the three edges of a 2-simplex. */
int or_triangle_edges(int d, const or_simplex *tri, or_simplex *edges) {
  simplex_edge(d, tri, 0, 1, &edges[0]);
  simplex_edge(d, tri, 0, 2, &edges[1]);
  simplex_edge(d, tri, 1, 2, &edges[2]);
  return 3;
}

/* Query type 2 (Sec. IV-A): the (n+1)n/2 edges of an n-simplex, pairs i<j. */
int or_nsimplex_edges(int d, const or_simplex *s, or_simplex *edges) {
  int n = 0;
  for (int i = 0; i <= s->k; i++)
    for (int j = i + 1; j <= s->k; j++) simplex_edge(d, s, i, j, &edges[n++]);
  return n;
}

/* Query type 3 (Sec. IV-A): the 2-simplex cofaces of an edge (y,(p1,p2)).
 * Every ordered two-set partition (A,B) of p1 gives (y,(A,B,p2)); every one
 * of p2 gives (y,(p1,A,B)); each is then put in canonical form.  The count is
 * |osp(p1)| + |osp(p2)| = (2^|p1|-2) + (2^|p2|-2). */
int or_edge_cofaces(int d, const or_simplex *e, or_simplex *tris) {
  int n = 0;
  for (int side = 0; side < 2; side++) {
    uint32_t P = e->part[side];
    /* all sub-masks A of P, A != 0, A != P */
    for (uint32_t A = (P - 1) & P; A; A = (A - 1) & P) {
      uint32_t B = P & ~A;
      or_simplex t;
      or_simplex_zero(&t);
      for (int i = 0; i < d; i++) t.y[i] = e->y[i];
      t.k = 2;
      if (side == 0) { t.part[0] = A; t.part[1] = B; t.part[2] = e->part[1]; }
      else { t.part[0] = e->part[0]; t.part[1] = A; t.part[2] = B; }
      or_canonicalize(d, &t);
      tris[n++] = t;
    }
  }
  return n;
}

static int next_perm(int *a, int n) {
  int i = n - 2;
  while (i >= 0 && a[i] >= a[i + 1]) i--;
  if (i < 0) return 0;
  int j = n - 1;
  while (a[j] <= a[i]) j--;
  int t = a[i]; a[i] = a[j]; a[j] = t;
  for (int l = i + 1, r = n - 1; l < r; l++, r--) { t = a[l]; a[l] = a[r]; a[r] = t; }
  return 1;
}

/* The n-simplex cofaces of an edge (y,(p1,p2)) (Sec. IV-C): every total order
 * of p1 followed by every total order of p2, as singleton parts; |p1|!|p2|! of
 * them. */
int or_edge_ncofaces(int d, const or_simplex *e, or_simplex *cells) {
  int e1[OR_MAXD + 1], e2[OR_MAXD + 1], n1 = 0, n2 = 0, n = 0;
  for (int i = 0; i <= d; i++) {
    if ((e->part[0] >> i) & 1u) e1[n1++] = i;
    if ((e->part[1] >> i) & 1u) e2[n2++] = i;
  }
  int a[OR_MAXD + 1], b[OR_MAXD + 1];
  for (int i = 0; i < n1; i++) a[i] = e1[i];
  do {
    for (int i = 0; i < n2; i++) b[i] = e2[i];
    do {
      or_simplex c;
      or_simplex_zero(&c);
      for (int i = 0; i < d; i++) c.y[i] = e->y[i];
      c.k = d;
      for (int i = 0; i < n1; i++) c.part[i] = 1u << a[i];
      for (int i = 0; i < n2; i++) c.part[n1 + i] = 1u << b[i];
      or_canonicalize(d, &c);
      cells[n++] = c;
    } while (next_perm(b, n2));
  } while (next_perm(a, n1));
  return n;
}

/* ------------------------------------------------------------------------ */
/* Ã_d realisation (reading R1) and the locate query (type 1, reading R3).    */
/* ------------------------------------------------------------------------ */
double or_lattice_c(int d) { return (1.0 - 1.0 / sqrt((double)(d + 1))) / (double)d; }
double or_lattice_cinv(int d) { return or_lattice_c(d) * sqrt((double)(d + 1)); }

void or_vertex_x(int d, double lam, const double *o, const int32_t *y, double *x) {
  long s = 0;
  for (int i = 0; i < d; i++) s += y[i];
  double c = or_lattice_c(d);
  double cs = c * (double)s;
  for (int i = 0; i < d; i++) {
    double u = (double)y[i] - cs;
    double w = lam * u;
    x[i] = w + o[i];
  }
}

void or_locate(int d, double lam, const double *o, const double *x, or_simplex *out) {
  double cp = or_lattice_cinv(d);
  double s = 0.0;
  for (int j = 0; j < d; j++) s += (x[j] - o[j]);
  double yp[OR_MAXD], fr[OR_MAXD];
  int perm[OR_MAXD];
  or_simplex_zero(out);
  for (int i = 0; i < d; i++) {
    double u = (x[i] - o[i]) + cp * s;
    yp[i] = u / lam;
    double fl = floor(yp[i]);
    out->y[i] = (int32_t)fl;
    fr[i] = yp[i] - fl;
    perm[i] = i;
  }
  /* insertion sort: fractional parts descending, ties -> lower index first */
  for (int i = 1; i < d; i++) {
    int p = perm[i], j = i - 1;
    while (j >= 0 && fr[perm[j]] < fr[p]) { perm[j + 1] = perm[j]; j--; }
    perm[j + 1] = p;
  }
  out->k = d;
  for (int i = 0; i < d; i++) out->part[i] = 1u << perm[i];
  out->part[d] = 1u << d;
}

/* ------------------------------------------------------------------------ */
/* The learned manifold: RBF-SVM decision function (Sec. IV-A, ThunderSVM).  */
/* f(q) = sum_i alpha_i exp(-gamma |q - s_i|^2) + b, summed in index order.   */
/* ------------------------------------------------------------------------ */
typedef struct {
  int32_t d;
  int64_t n_sv;
  const double *sv;    /* [n_sv][d] */
  const double *alpha; /* [n_sv] */
  double gamma, b;
} or_rbf;

double or_f(const or_rbf *r, const double *q) {
  double acc = 0.0;
  for (int64_t i = 0; i < r->n_sv; i++) {
    double d2 = 0.0;
    for (int k = 0; k < r->d; k++) {
      double t = q[k] - r->sv[i * r->d + k];
      d2 += t * t;
    }
    acc += r->alpha[i] * exp(-r->gamma * d2);
  }
  return acc + r->b;
}

void or_f_batch(const or_rbf *r, const double *q, int64_t n, double *out) {
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n; i++) out[i] = or_f(r, q + i * r->d);
}

static int in_box(int d, const double *x, const double *lo, const double *hi) {
  for (int i = 0; i < d; i++)
    if (!(x[i] >= lo[i] && x[i] <= hi[i])) return 0;
  return 1;
}

/* ------------------------------------------------------------------------ */
/* Manifold tracing (Sec. IV-A, Figs. 3 and 4) and cells (Sec. IV-C).        */
/* ------------------------------------------------------------------------ */
typedef struct { int32_t y[OR_MAXD]; double f; } vrec;

typedef struct {
  int d;
  double lam;
  const double *o, *lo, *hi;
  const or_rbf *rbf;
  or_set vmap;
  int64_t n_near_zero;
} tctx;

/* f at a lattice vertex, evaluated once per distinct vertex. */
static int vertex_f(tctx *c, const int32_t *y, double *f) {
  vrec r;
  memset(&r, 0, sizeof(r));
  for (int i = 0; i < c->d; i++) r.y[i] = y[i];
  long idx = set_find(&c->vmap, &r);
  if (idx >= 0) { *f = ((vrec *)c->vmap.recs)[idx].f; return 0; }
  double x[OR_MAXD];
  or_vertex_x(c->d, c->lam, c->o, y, x);
  r.f = or_f(c->rbf, x);
  if (fabs(r.f) < 1e-12) c->n_near_zero++;
  int ins;
  if (set_insert(&c->vmap, &r, &ins) < 0) return -1;
  *f = r.f;
  return 0;
}

static int vertex_in(tctx *c, const int32_t *y) {
  double x[OR_MAXD];
  or_vertex_x(c->d, c->lam, c->o, y, x);
  return in_box(c->d, x, c->lo, c->hi);
}

/* An edge is traced iff both endpoints are in the domain (R5) and the signs
 * differ (R4).  Returns 1/0, or -1 on error; f0/f1 receive the values. */
static int edge_crosses(tctx *c, const or_simplex *e, double *f0, double *f1) {
  int32_t v[2 * OR_MAXD];
  or_simplex_vertices(c->d, e, v);
  if (!vertex_in(c, v) || !vertex_in(c, v + c->d)) return 0;
  if (vertex_f(c, v, f0) || vertex_f(c, v + c->d, f1)) return -1;
  return ((*f0 >= 0.0) != (*f1 >= 0.0)) ? 1 : 0;
}

typedef struct {
  int32_t d;
  int64_t n_edges;
  int32_t *edge_y;       /* [E][d] first vertex */
  uint32_t *edge_mask;   /* [E] first part as a mask over {0..d-1} */
  int32_t *edge_level;   /* [E] BFS level */
  double *edge_f;        /* [E][2] f at both endpoints */
  double *edge_t;        /* [E] root parameter */
  double *edge_pt;       /* [E][d] intersection point */
  uint8_t *edge_multiroot; /* [E] more than one sign change in 17 samples */
  int64_t n_cells;
  int32_t *cell_y;       /* [C][d] */
  uint8_t *cell_perm;    /* [C][d] the order of the singleton parts before {d} */
  int64_t *cell_off;     /* [C+1] */
  int64_t *cell_idx;     /* [cell_off[C]] indices into the edge list */
  int64_t n_vertices, n_near_zero, n_boundary, n_dead_seeds, levels;
  int64_t n_crossing_triangles;
} or_trace_result;

void or_trace_free(or_trace_result *r) {
  free(r->edge_y); free(r->edge_mask); free(r->edge_level); free(r->edge_f);
  free(r->edge_t); free(r->edge_pt); free(r->edge_multiroot);
  free(r->cell_y); free(r->cell_perm); free(r->cell_off); free(r->cell_idx);
  memset(r, 0, sizeof(*r));
}

/* Root of g(t) = f(v1 + t (v2 - v1)) on [0,1] by bisection (reading R6). */
static double seg_point(double a, double b, double t) { double w = b - a; double u = t * w; return a + u; }

static double root_bisect(const or_rbf *rbf, int d, const double *x1, const double *x2, double f1) {
  int s1 = f1 >= 0.0;
  double lo = 0.0, hi = 1.0, q[OR_MAXD];
  for (int it = 0; it < 50; it++) {
    double mid = 0.5 * (lo + hi);
    for (int i = 0; i < d; i++) q[i] = seg_point(x1[i], x2[i], mid);
    if ((or_f(rbf, q) >= 0.0) == s1) lo = mid; else hi = mid;
  }
  return 0.5 * (lo + hi);
}

static int multiroot(const or_rbf *rbf, int d, const double *x1, const double *x2) {
  double q[OR_MAXD];
  int changes = 0, prev = -1;
  for (int k = 0; k <= 16; k++) {
    double t = (double)k / 16.0;
    for (int i = 0; i < d; i++) q[i] = seg_point(x1[i], x2[i], t);
    int s = or_f(rbf, q) >= 0.0;
    if (prev >= 0 && s != prev) changes++;
    prev = s;
  }
  return changes > 1;
}

/* For given edges (y, p1): f at both vertices, the bisection root t, the
 * intersection point and the multi-root flag (used to check sampled edges of
 * a traced set too large to trace here). */
void or_edge_roots(const or_rbf *rbf, double lam, const double *o, const int32_t *ey,
                   const uint32_t *emask, int64_t n, double *f2, double *t, double *pt,
                   uint8_t *mr) {
  int d = rbf->d;
#pragma omp parallel for schedule(dynamic, 16)
  for (int64_t i = 0; i < n; i++) {
    or_simplex e;
    or_simplex_zero(&e);
    for (int k = 0; k < d; k++) e.y[k] = ey[i * d + k];
    e.k = 1;
    e.part[0] = emask[i];
    e.part[1] = ((2u << d) - 1u) & ~emask[i];
    int32_t v[2 * OR_MAXD];
    double x1[OR_MAXD], x2[OR_MAXD];
    or_simplex_vertices(d, &e, v);
    or_vertex_x(d, lam, o, v, x1);
    or_vertex_x(d, lam, o, v + d, x2);
    f2[2 * i] = or_f(rbf, x1);
    f2[2 * i + 1] = or_f(rbf, x2);
    t[i] = root_bisect(rbf, d, x1, x2, f2[2 * i]);
    for (int k = 0; k < d; k++) pt[i * d + k] = seg_point(x1[k], x2[k], t[i]);
    mr[i] = (uint8_t)multiroot(rbf, d, x1, x2);
  }
}

/* Trace the zero set of f from the seeds.  Returns 0, or -1 on allocation
 * failure / bad arguments.  want_cells: also build cells and their CSR;
 * want_roots: also solve the roots. */
int or_trace(const or_rbf *rbf, double lam, const double *o, const double *lo, const double *hi,
             const double *seeds, int64_t n_seeds, int want_roots, int want_cells,
             int64_t max_edges, or_trace_result *res) {
  int d = rbf->d;
  memset(res, 0, sizeof(*res));
  if (d < 2 || d > OR_MAXD || !(lam > 0.0)) return -1;
  res->d = d;
  tctx c;
  c.d = d; c.lam = lam; c.o = o; c.lo = lo; c.hi = hi; c.rbf = rbf; c.n_near_zero = 0;
  if (set_init(&c.vmap, sizeof(vrec), sizeof(int32_t) * OR_MAXD)) return -1;
  or_set eset;
  if (set_init(&eset, sizeof(or_simplex), sizeof(or_simplex))) return -1;
  /* per-edge side data in insertion order */
  size_t side_cap = 1024;
  int32_t *level = (int32_t *)malloc(side_cap * sizeof(int32_t));
  double *ef = (double *)malloc(side_cap * 2 * sizeof(double));
  int rc = -1;
  if (!level || !ef) goto out;

  /* Locate edges (Fig. 3): seed -> n-simplex -> its crossing edges -> set. */
  for (int64_t si = 0; si < n_seeds; si++) {
    or_simplex ns;
    or_locate(d, lam, o, seeds + si * d, &ns);
    or_simplex edges[(OR_MAXD + 1) * OR_MAXD / 2];
    int ne = or_nsimplex_edges(d, &ns, edges), any = 0;
    for (int k = 0; k < ne; k++) {
      double f0, f1;
      int x = edge_crosses(&c, &edges[k], &f0, &f1);
      if (x < 0) goto out;
      if (!x) continue;
      any = 1;
      int ins;
      long idx = set_insert(&eset, &edges[k], &ins);
      if (idx < 0) goto out;
      if (ins) {
        if ((size_t)idx >= side_cap) {
          side_cap *= 2;
          level = (int32_t *)realloc(level, side_cap * sizeof(int32_t));
          ef = (double *)realloc(ef, side_cap * 2 * sizeof(double));
          if (!level || !ef) goto out;
        }
        level[idx] = 0; ef[2 * idx] = f0; ef[2 * idx + 1] = f1;
      }
    }
    if (!any) res->n_dead_seeds++;
  }

  /* Search edges (Fig. 4): breadth-first over 2-simplex cofaces. */
  {
    size_t head = 0;
    or_simplex tris[2 * (1 << OR_MAXD)];
    /* max_edges > 0 bounds the sample: expansion stops once that many edges exist */
    while (head < eset.n && !(max_edges > 0 && (int64_t)eset.n >= max_edges)) {
      or_simplex e = ((or_simplex *)eset.recs)[head];
      int lev = level[head];
      head++;
      int nt = or_edge_cofaces(d, &e, tris);
      for (int ti = 0; ti < nt; ti++) {
        int32_t tv[3 * OR_MAXD];
        or_simplex_vertices(d, &tris[ti], tv);
        if (!vertex_in(&c, tv) || !vertex_in(&c, tv + d) || !vertex_in(&c, tv + 2 * d)) {
          res->n_boundary++;
          continue;
        }
        or_simplex fe[3];
        or_triangle_edges(d, &tris[ti], fe);
        for (int k = 0; k < 3; k++) {
          double f0, f1;
          int x = edge_crosses(&c, &fe[k], &f0, &f1);
          if (x < 0) goto out;
          if (!x) continue;
          int ins;
          long idx = set_insert(&eset, &fe[k], &ins);
          if (idx < 0) goto out;
          if (ins) {
            if ((size_t)idx >= side_cap) {
              side_cap *= 2;
              level = (int32_t *)realloc(level, side_cap * sizeof(int32_t));
              ef = (double *)realloc(ef, side_cap * 2 * sizeof(double));
              if (!level || !ef) goto out;
            }
            level[idx] = lev + 1; ef[2 * idx] = f0; ef[2 * idx + 1] = f1;
          }
        }
      }
    }
  }

  int64_t E = (int64_t)eset.n;
  res->n_edges = E;
  res->edge_y = (int32_t *)malloc((size_t)(E ? E : 1) * d * sizeof(int32_t));
  res->edge_mask = (uint32_t *)malloc((size_t)(E ? E : 1) * sizeof(uint32_t));
  res->edge_level = (int32_t *)malloc((size_t)(E ? E : 1) * sizeof(int32_t));
  res->edge_f = (double *)malloc((size_t)(E ? E : 1) * 2 * sizeof(double));
  res->edge_t = (double *)malloc((size_t)(E ? E : 1) * sizeof(double));
  res->edge_pt = (double *)malloc((size_t)(E ? E : 1) * d * sizeof(double));
  res->edge_multiroot = (uint8_t *)malloc((size_t)(E ? E : 1));
  if (!res->edge_y || !res->edge_mask || !res->edge_level || !res->edge_f || !res->edge_t ||
      !res->edge_pt || !res->edge_multiroot)
    goto out;
  res->levels = 0;
  for (int64_t i = 0; i < E; i++) {
    const or_simplex *e = &((or_simplex *)eset.recs)[i];
    for (int k = 0; k < d; k++) res->edge_y[i * d + k] = e->y[k];
    res->edge_mask[i] = e->part[0];
    res->edge_level[i] = level[i];
    if (level[i] + 1 > res->levels) res->levels = level[i] + 1;
    res->edge_f[2 * i] = ef[2 * i];
    res->edge_f[2 * i + 1] = ef[2 * i + 1];
    res->edge_t[i] = 0.0;
    res->edge_multiroot[i] = 0;
  }
  /* The roots are independent per edge: the loop runs on all host threads
   * (OpenMP), each edge with the same arithmetic as a serial loop. */
  if (want_roots) {
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t i = 0; i < E; i++) {
      const or_simplex *e = &((or_simplex *)eset.recs)[i];
      int32_t v[2 * OR_MAXD];
      double x1[OR_MAXD], x2[OR_MAXD];
      or_simplex_vertices(d, e, v);
      or_vertex_x(d, lam, o, v, x1);
      or_vertex_x(d, lam, o, v + d, x2);
      double t = root_bisect(rbf, d, x1, x2, ef[2 * i]);
      res->edge_t[i] = t;
      for (int k = 0; k < d; k++) res->edge_pt[i * d + k] = seg_point(x1[k], x2[k], t);
      res->edge_multiroot[i] = (uint8_t)multiroot(rbf, d, x1, x2);
    }
  }

  if (want_cells) {
    /* crossing 2-simplices: cofaces (inside the domain) of traced edges */
    or_set tset;
    if (set_init(&tset, sizeof(or_simplex), sizeof(or_simplex))) goto out;
    or_simplex tris[2 * (1 << OR_MAXD)];
    for (int64_t i = 0; i < E; i++) {
      const or_simplex *e = &((or_simplex *)eset.recs)[i];
      int nt = or_edge_cofaces(d, e, tris);
      for (int ti = 0; ti < nt; ti++) {
        int32_t tv[3 * OR_MAXD];
        or_simplex_vertices(d, &tris[ti], tv);
        if (!vertex_in(&c, tv) || !vertex_in(&c, tv + d) || !vertex_in(&c, tv + 2 * d)) continue;
        int ins;
        if (set_insert(&tset, &tris[ti], &ins) < 0) { set_free(&tset); goto out; }
      }
    }
    res->n_crossing_triangles = (int64_t)tset.n;
    set_free(&tset);

    /* cells: n-simplex cofaces of traced edges, de-duplicated */
    or_set cset;
    if (set_init(&cset, sizeof(or_simplex), sizeof(or_simplex))) goto out;
    long maxnc = 1;
    for (int i = 2; i <= d; i++) maxnc *= i; /* d! >= |p1|!|p2|! */
    maxnc *= (d + 1);
    or_simplex *nc = (or_simplex *)malloc((size_t)maxnc * sizeof(or_simplex));
    if (!nc) { set_free(&cset); goto out; }
    for (int64_t i = 0; i < E; i++) {
      const or_simplex *e = &((or_simplex *)eset.recs)[i];
      int n = or_edge_ncofaces(d, e, nc);
      for (int k = 0; k < n; k++) {
        int ins;
        if (set_insert(&cset, &nc[k], &ins) < 0) { free(nc); set_free(&cset); goto out; }
      }
    }
    free(nc);
    int64_t C = (int64_t)cset.n;
    res->n_cells = C;
    res->cell_y = (int32_t *)malloc((size_t)(C ? C : 1) * d * sizeof(int32_t));
    res->cell_perm = (uint8_t *)malloc((size_t)(C ? C : 1) * d);
    res->cell_off = (int64_t *)malloc((size_t)(C + 1) * sizeof(int64_t));
    int nedg = (d + 1) * d / 2;
    res->cell_idx = (int64_t *)malloc((size_t)(C ? C : 1) * nedg * sizeof(int64_t));
    if (!res->cell_y || !res->cell_perm || !res->cell_off || !res->cell_idx) { set_free(&cset); goto out; }
    int64_t pos = 0;
    or_simplex ce[(OR_MAXD + 1) * OR_MAXD / 2];
    for (int64_t ci = 0; ci < C; ci++) {
      const or_simplex *cs = &((or_simplex *)cset.recs)[ci];
      for (int k = 0; k < d; k++) res->cell_y[ci * d + k] = cs->y[k];
      for (int k = 0; k < d; k++) {
        int el = 0;
        while (!((cs->part[k] >> el) & 1u)) el++;
        res->cell_perm[ci * d + k] = (uint8_t)el;
      }
      res->cell_off[ci] = pos;
      int n = or_nsimplex_edges(d, cs, ce);
      for (int k = 0; k < n; k++) {
        long idx = set_find(&eset, &ce[k]);
        if (idx >= 0) res->cell_idx[pos++] = idx;
      }
    }
    res->cell_off[C] = pos;
    set_free(&cset);
  }
  res->n_vertices = (int64_t)c.vmap.n;
  res->n_near_zero = c.n_near_zero;
  rc = 0;
out:
  free(level);
  free(ef);
  set_free(&eset);
  set_free(&c.vmap);
  if (rc) or_trace_free(res);
  return rc;
}

/* ------------------------------------------------------------------------ */
/* Batch triangulation (Sec. V-B, Figs. 5-6, Eqs. bc and local).             */
/* ------------------------------------------------------------------------ */
/* Inside test of a local vertex v' of the subdivided n-simplex (Eq. local,
 * read with "no less than 0": the closed simplex, so that the local edges on
 * its faces, such as the first edge of Fig. 5, are kept):
 *   k - v'_0 >= 0,  v'_{i-1} - v'_i >= 0,  v'_{n-1} >= 0. */
static int local_inside(int d, int k, const int32_t *m) {
  if (k - m[0] < 0) return 0;
  for (int i = 1; i < d; i++)
    if (m[i - 1] - m[i] < 0) return 0;
  return m[d - 1] >= 0;
}

/* The local triangulation of the subdivided reference n-simplex (computed
 * once and shared by all n-simplices, Sec. V-B): its vertices (all v' that
 * pass the inside test) and its edges (v', v' + e(M') for a non-empty local
 * mask M', both inside).  verts [nv][d], edges [ne][2] = (vertex index, M');
 * NULL arrays only count.  Returns 0. */
int or_subdiv_template(int d, int k, int32_t *verts, int64_t *nv, int32_t *edges, int64_t *ne) {
  int64_t cv = 0, ce = 0;
  int32_t m[OR_MAXD], m2[OR_MAXD];
  /* every v' in [0, k]^d in lexicographic order, kept if inside */
  int64_t total = 1;
  for (int i = 0; i < d; i++) total *= (k + 1);
  for (int64_t code = 0; code < total; code++) {
    int64_t c = code;
    for (int i = d - 1; i >= 0; i--) { m[i] = (int32_t)(c % (k + 1)); c /= (k + 1); }
    if (!local_inside(d, k, m)) continue;
    for (uint32_t M = 1; M < (1u << d); M++) {
      for (int i = 0; i < d; i++) m2[i] = m[i] + (int32_t)((M >> i) & 1u);
      if (!local_inside(d, k, m2)) continue;
      if (edges) { edges[2 * ce] = (int32_t)cv; edges[2 * ce + 1] = (int32_t)M; }
      ce++;
    }
    if (verts) for (int i = 0; i < d; i++) verts[cv * d + i] = m[i];
    cv++;
  }
  *nv = cv;
  *ne = ce;
  return 0;
}

/* Batch triangulation: trace at the coarse scale k * lam (same offset o),
 * take its crossing n-simplices, and in each the local triangulation of
 * scale lam: local vertex v' maps to the lattice vertex
 *   y = k z + sum_j v'_j e(pi_j)                    (Eq. bc, lattice units)
 * of the n-simplex (z, pi), local edge (v', M') to the edge (y, pi(M')).
 * The result is every such edge with both vertices in the box and a sign
 * change, de-duplicated (edges on shared faces come from several
 * n-simplices), with roots as in or_trace.  res->levels = the coarse trace's
 * BFS levels; *n_coarse receives its crossing n-simplices. */
int or_subdiv(const or_rbf *rbf, double lam, int k, const double *o, const double *lo,
              const double *hi, const double *seeds, int64_t n_seeds, int want_roots,
              or_trace_result *res, int64_t *n_coarse) {
  int d = rbf->d;
  memset(res, 0, sizeof(*res));
  if (d < 2 || d > OR_MAXD || !(lam > 0.0) || k < 1 || k > 64) return -1;
  or_trace_result coarse;
  if (or_trace(rbf, k * lam, o, lo, hi, seeds, n_seeds, 0, 1, 0, &coarse)) return -1;
  *n_coarse = coarse.n_cells;
  int64_t nv, ne;
  or_subdiv_template(d, k, NULL, &nv, NULL, &ne);
  int32_t *tv = (int32_t *)malloc((size_t)(nv ? nv : 1) * d * sizeof(int32_t));
  int32_t *te = (int32_t *)malloc((size_t)(ne ? ne : 1) * 2 * sizeof(int32_t));
  tctx c;
  c.d = d; c.lam = lam; c.o = o; c.lo = lo; c.hi = hi; c.rbf = rbf; c.n_near_zero = 0;
  or_set eset;
  int rc = -1, have_v = 0, have_e = 0;
  size_t cap = 1024;
  double *ef = (double *)malloc(cap * 2 * sizeof(double));
  if (!tv || !te || !ef) goto out0;
  or_subdiv_template(d, k, tv, &nv, te, &ne);
  if (set_init(&c.vmap, sizeof(vrec), sizeof(int32_t) * OR_MAXD)) goto out0;
  have_v = 1;
  if (set_init(&eset, sizeof(or_simplex), sizeof(or_simplex))) goto out0;
  have_e = 1;
  for (int64_t ci = 0; ci < coarse.n_cells; ci++) {
    const int32_t *z = coarse.cell_y + ci * d;
    const uint8_t *pi = coarse.cell_perm + ci * d;
    for (int64_t ei = 0; ei < ne; ei++) {
      const int32_t *m = tv + (int64_t)te[2 * ei] * d;
      uint32_t Ml = (uint32_t)te[2 * ei + 1];
      or_simplex e;
      or_simplex_zero(&e);
      for (int i = 0; i < d; i++) e.y[i] = k * z[i];
      uint32_t M = 0;
      for (int j = 0; j < d; j++) {
        e.y[pi[j]] += m[j];
        if ((Ml >> j) & 1u) M |= 1u << pi[j];
      }
      e.k = 1;
      e.part[0] = M;
      e.part[1] = ((2u << d) - 1u) & ~M;
      double f0, f1;
      int x = edge_crosses(&c, &e, &f0, &f1);
      if (x < 0) goto out0;
      if (!x) continue;
      int ins;
      long idx = set_insert(&eset, &e, &ins);
      if (idx < 0) goto out0;
      if (ins) {
        if ((size_t)idx >= cap) {
          cap *= 2;
          ef = (double *)realloc(ef, cap * 2 * sizeof(double));
          if (!ef) goto out0;
        }
        ef[2 * idx] = f0;
        ef[2 * idx + 1] = f1;
      }
    }
  }
  {
    int64_t E = (int64_t)eset.n;
    res->d = d;
    res->n_edges = E;
    res->edge_y = (int32_t *)malloc((size_t)(E ? E : 1) * d * sizeof(int32_t));
    res->edge_mask = (uint32_t *)malloc((size_t)(E ? E : 1) * sizeof(uint32_t));
    res->edge_level = (int32_t *)calloc((size_t)(E ? E : 1), sizeof(int32_t));
    res->edge_f = (double *)malloc((size_t)(E ? E : 1) * 2 * sizeof(double));
    res->edge_t = (double *)calloc((size_t)(E ? E : 1), sizeof(double));
    res->edge_pt = (double *)calloc((size_t)(E ? E : 1) * d, sizeof(double));
    res->edge_multiroot = (uint8_t *)calloc((size_t)(E ? E : 1), 1);
    if (!res->edge_y || !res->edge_mask || !res->edge_level || !res->edge_f || !res->edge_t ||
        !res->edge_pt || !res->edge_multiroot)
      goto out0;
    for (int64_t i = 0; i < E; i++) {
      const or_simplex *e = &((or_simplex *)eset.recs)[i];
      for (int q = 0; q < d; q++) res->edge_y[i * d + q] = e->y[q];
      res->edge_mask[i] = e->part[0];
      res->edge_f[2 * i] = ef[2 * i];
      res->edge_f[2 * i + 1] = ef[2 * i + 1];
    }
    if (want_roots) {
#pragma omp parallel for schedule(dynamic, 16)
      for (int64_t i = 0; i < E; i++) {
        const or_simplex *e = &((or_simplex *)eset.recs)[i];
        int32_t v[2 * OR_MAXD];
        double x1[OR_MAXD], x2[OR_MAXD];
        or_simplex_vertices(d, e, v);
        or_vertex_x(d, lam, o, v, x1);
        or_vertex_x(d, lam, o, v + d, x2);
        double t = root_bisect(rbf, d, x1, x2, ef[2 * i]);
        res->edge_t[i] = t;
        for (int q = 0; q < d; q++) res->edge_pt[i * d + q] = seg_point(x1[q], x2[q], t);
        res->edge_multiroot[i] = (uint8_t)multiroot(rbf, d, x1, x2);
      }
    }
    res->levels = coarse.levels;
    res->n_vertices = (int64_t)c.vmap.n;
    res->n_near_zero = c.n_near_zero;
    res->n_dead_seeds = coarse.n_dead_seeds;
  }
  rc = 0;
out0:
  free(tv);
  free(te);
  free(ef);
  if (have_e) set_free(&eset);
  if (have_v) set_free(&c.vmap);
  or_trace_free(&coarse);
  if (rc) or_trace_free(res);
  return rc;
}

/* ------------------------------------------------------------------------ */
/* Certification (Sec. V-C, App. A): forward kinematics of a serial DH arm   */
/* and the exact capsule/obstacle distance.                                   */
/* ------------------------------------------------------------------------ */
typedef struct {
  int32_t n_links;
  const double *dh;     /* [n][4]: theta0, d, a, alpha */
  const double *radius; /* [n] capsule radius of link i; NULL: no capsules */
  /* Spheres fixed to the links (the paper's robot model, Sec. VI): sphere s
   * rides on link sphere_link[s], its centre sphere_center[s] given in the
   * frame T_{link+1} of the body that joint `link` turns. */
  int32_t n_spheres;
  const int32_t *sphere_link;
  const double *sphere_center; /* [n_spheres][3] */
  const double *sphere_radius; /* [n_spheres] */
} or_robot;

typedef struct {
  int32_t n;
  const int32_t *type;  /* 0 = box, 1 = sphere, 2 = cylinder */
  const double *pose;   /* [n][12]: R (row-major, obstacle frame -> world), then t */
  const double *dims;   /* [n][3]: box side lengths l_x,l_y,l_z; sphere radius in [0];
                           cylinder radius r_c in [0] and height h in [1] (axis = local z) */
} or_scene;

static void mat4_mul(const double *A, const double *B, double *C) {
  for (int i = 0; i < 4; i++)
    for (int j = 0; j < 4; j++) {
      double s = 0.0;
      for (int k = 0; k < 4; k++) s += A[i * 4 + k] * B[k * 4 + j];
      C[i * 4 + j] = s;
    }
}

/* Frame origins of the chain T_{i+1} = T_i Rz(q_i+theta_i) Tz(d_i) Tx(a_i) Rx(alpha_i),
 * T_0 = identity; origins[(n+1)][3]. */
void or_fk(const or_robot *r, const double *q, double *origins) {
  double T[16] = {1, 0, 0, 0, 0, 1, 0, 0, 0, 0, 1, 0, 0, 0, 0, 1};
  origins[0] = 0; origins[1] = 0; origins[2] = 0;
  for (int i = 0; i < r->n_links; i++) {
    double th = q[i] + r->dh[4 * i + 0], dd = r->dh[4 * i + 1], aa = r->dh[4 * i + 2], al = r->dh[4 * i + 3];
    double ct = cos(th), st = sin(th), ca = cos(al), sa = sin(al);
    double Rz[16] = {ct, -st, 0, 0, st, ct, 0, 0, 0, 0, 1, 0, 0, 0, 0, 1};
    double Tz[16] = {1, 0, 0, 0, 0, 1, 0, 0, 0, 0, 1, dd, 0, 0, 0, 1};
    double Tx[16] = {1, 0, 0, aa, 0, 1, 0, 0, 0, 0, 1, 0, 0, 0, 0, 1};
    double Rx[16] = {1, 0, 0, 0, 0, ca, -sa, 0, 0, sa, ca, 0, 0, 0, 0, 1};
    double A[16], B[16], C[16];
    mat4_mul(T, Rz, A);
    mat4_mul(A, Tz, B);
    mat4_mul(B, Tx, C);
    mat4_mul(C, Rx, T);
    origins[3 * (i + 1) + 0] = T[3];
    origins[3 * (i + 1) + 1] = T[7];
    origins[3 * (i + 1) + 2] = T[11];
  }
}

/* All frames T_0 .. T_n of the chain as 3x4 row-major [R | t]. */
void or_fk_frames(const or_robot *r, const double *q, double *frames) {
  double T[16] = {1, 0, 0, 0, 0, 1, 0, 0, 0, 0, 1, 0, 0, 0, 0, 1};
  for (int k = 0; k < 12; k++) frames[k] = T[k];
  for (int i = 0; i < r->n_links; i++) {
    double th = q[i] + r->dh[4 * i + 0], dd = r->dh[4 * i + 1], aa = r->dh[4 * i + 2], al = r->dh[4 * i + 3];
    double ct = cos(th), st = sin(th), ca = cos(al), sa = sin(al);
    double Rz[16] = {ct, -st, 0, 0, st, ct, 0, 0, 0, 0, 1, 0, 0, 0, 0, 1};
    double Tz[16] = {1, 0, 0, 0, 0, 1, 0, 0, 0, 0, 1, dd, 0, 0, 0, 1};
    double Tx[16] = {1, 0, 0, aa, 0, 1, 0, 0, 0, 0, 1, 0, 0, 0, 0, 1};
    double Rx[16] = {1, 0, 0, 0, 0, ca, -sa, 0, 0, sa, ca, 0, 0, 0, 0, 1};
    double A[16], B[16], C[16];
    mat4_mul(T, Rz, A);
    mat4_mul(A, Tz, B);
    mat4_mul(B, Tx, C);
    mat4_mul(C, Rx, T);
    for (int k = 0; k < 12; k++) frames[12 * (i + 1) + k] = T[k];
  }
}

static double dot3(const double *a, const double *b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }
static double clamp01(double x) { return x < 0.0 ? 0.0 : (x > 1.0 ? 1.0 : x); }

/* Distance between segments [p1,q1] and [p2,q2]: minimise the convex quadratic
 * |p1 + s d1 - p2 - t d2|^2 over the unit square by the clamped closed form. */
double or_segseg_dist(const double *p1, const double *q1, const double *p2, const double *q2) {
  double d1[3], d2[3], r[3];
  for (int i = 0; i < 3; i++) { d1[i] = q1[i] - p1[i]; d2[i] = q2[i] - p2[i]; r[i] = p1[i] - p2[i]; }
  double a = dot3(d1, d1), e = dot3(d2, d2), f = dot3(d2, r), s, t;
  if (a <= 1e-300 && e <= 1e-300) { s = 0.0; t = 0.0; }
  else if (a <= 1e-300) { s = 0.0; t = clamp01(f / e); }
  else {
    double cc = dot3(d1, r);
    if (e <= 1e-300) { t = 0.0; s = clamp01(-cc / a); }
    else {
      double b = dot3(d1, d2), den = a * e - b * b;
      s = den > 0.0 ? clamp01((b * f - cc * e) / den) : 0.0;
      t = (b * s + f) / e;
      if (t < 0.0) { t = 0.0; s = clamp01(-cc / a); }
      else if (t > 1.0) { t = 1.0; s = clamp01((b - cc) / a); }
    }
  }
  double w[3];
  for (int i = 0; i < 3; i++) w[i] = (p1[i] + s * d1[i]) - (p2[i] + t * d2[i]);
  return sqrt(dot3(w, w));
}

/* Distance from a point to an origin-centred box of half extents h. */
static double point_box(const double *p, const double *h) {
  double s = 0.0;
  for (int i = 0; i < 3; i++) {
    double u = fabs(p[i]) - h[i];
    if (u > 0.0) s += u * u;
  }
  return sqrt(s);
}

/* Distance from segment [a,b] (box frame) to an origin-centred box: zero if
 * the segment meets the box (slab clipping); otherwise the smallest of the
 * two end-point distances and the twelve segment/box-edge distances. */
static double segment_box_local(const double *a, const double *b, const double *h) {
  double t0 = 0.0, t1 = 1.0;
  int meets = 1;
  for (int i = 0; i < 3 && meets; i++) {
    double dir = b[i] - a[i];
    if (dir == 0.0) {
      if (a[i] < -h[i] || a[i] > h[i]) meets = 0;
    } else {
      double ta = (-h[i] - a[i]) / dir, tb = (h[i] - a[i]) / dir;
      if (ta > tb) { double tt = ta; ta = tb; tb = tt; }
      if (ta > t0) t0 = ta;
      if (tb < t1) t1 = tb;
      if (t0 > t1) meets = 0;
    }
  }
  if (meets) return 0.0;
  double best = point_box(a, h), pb = point_box(b, h);
  if (pb < best) best = pb;
  for (int ax = 0; ax < 3; ax++) {
    int u = (ax + 1) % 3, v = (ax + 2) % 3;
    for (int su = -1; su <= 1; su += 2)
      for (int sv = -1; sv <= 1; sv += 2) {
        double e0[3], e1[3];
        e0[ax] = -h[ax]; e1[ax] = h[ax];
        e0[u] = e1[u] = su * h[u];
        e0[v] = e1[v] = sv * h[v];
        double dd = or_segseg_dist(a, b, e0, e1);
        if (dd < best) best = dd;
      }
  }
  return best;
}

static void to_local(const double *pose, const double *p, double *out) {
  /* pose: R row-major (local -> world), t; local = R^T (p - t) */
  double w[3] = {p[0] - pose[9], p[1] - pose[10], p[2] - pose[11]};
  for (int i = 0; i < 3; i++) out[i] = pose[0 + i] * w[0] + pose[3 + i] * w[1] + pose[6 + i] * w[2];
}

/* Distance from a point to the origin-centred solid cylinder of radius rc
 * and height h with axis z (App. A, sphere vs cylinder): the radial excess
 * sqrt(x^2 + y^2) - rc and the axial excess |z| - h/2, each counted when
 * positive; inside both it is 0. */
static double point_cylinder(const double *p, double rc, double h) {
  double rho = sqrt(p[0] * p[0] + p[1] * p[1]);
  double u = rho - rc, v = fabs(p[2]) - 0.5 * h;
  if (u < 0.0) u = 0.0;
  if (v < 0.0) v = 0.0;
  return sqrt(u * u + v * v);
}

/* Distance from segment [a,b] (cylinder frame) to the cylinder: the distance
 * to a convex set is convex along the segment, so golden-section search on
 * [0,1] finds its minimum (100 steps shrink the bracket below 1e-20; the end
 * points are checked too). */
static double segment_cylinder_local(const double *a, const double *b, double rc, double h) {
  const double g = 0.6180339887498949;
  double p[3];
#define OR_CYL_AT(t) (p[0] = a[0] + (t) * (b[0] - a[0]), p[1] = a[1] + (t) * (b[1] - a[1]), \
                      p[2] = a[2] + (t) * (b[2] - a[2]), point_cylinder(p, rc, h))
  double lo = 0.0, hi = 1.0;
  double x1 = hi - g * (hi - lo), x2 = lo + g * (hi - lo);
  double f1 = OR_CYL_AT(x1), f2 = OR_CYL_AT(x2);
  for (int it = 0; it < 100; it++) {
    if (f1 <= f2) {
      hi = x2; x2 = x1; f2 = f1;
      x1 = hi - g * (hi - lo); f1 = OR_CYL_AT(x1);
    } else {
      lo = x1; x1 = x2; f1 = f2;
      x2 = lo + g * (hi - lo); f2 = OR_CYL_AT(x2);
    }
  }
  double best = f1 < f2 ? f1 : f2;
  double e0 = OR_CYL_AT(0.0), e1 = OR_CYL_AT(1.0);
  double em = OR_CYL_AT(0.5 * (lo + hi));
#undef OR_CYL_AT
  if (e0 < best) best = e0;
  if (e1 < best) best = e1;
  if (em < best) best = em;
  return best;
}

double or_segment_obstacle_dist(const double *a, const double *b, int32_t type, const double *pose,
                                const double *dims) {
  double la[3], lb[3];
  to_local(pose, a, la);
  to_local(pose, b, lb);
  if (type == 0) {
    double h[3] = {0.5 * dims[0], 0.5 * dims[1], 0.5 * dims[2]};
    return segment_box_local(la, lb, h);
  }
  if (type == 2) return segment_cylinder_local(la, lb, dims[0], dims[1]);
  /* sphere at the frame origin: distance from the centre to the segment */
  double d[3] = {lb[0] - la[0], lb[1] - la[1], lb[2] - la[2]};
  double m[3] = {-la[0], -la[1], -la[2]};
  double dd = dot3(d, d);
  double t = dd > 0.0 ? clamp01(dot3(m, d) / dd) : 0.0;
  double w[3] = {la[0] + t * d[0], la[1] + t * d[1], la[2] + t * d[2]};
  double cd = sqrt(dot3(w, w)) - dims[0];
  return cd > 0.0 ? cd : 0.0;
}

#define OR_ELEM_TIE 1e-9

/* Robot elements: the link capsules (when radius is given), then the spheres.
 * Element e's end points at a configuration, from the frames of or_fk_frames. */
static int n_elements(const or_robot *r) { return (r->radius ? r->n_links : 0) + r->n_spheres; }

static void element_at(const or_robot *r, const double *frames, int e, double *pa, double *pb,
                       double *rad, int *link) {
  int nc = r->radius ? r->n_links : 0;
  if (e < nc) {
    for (int k = 0; k < 3; k++) {
      pa[k] = frames[12 * e + 4 * k + 3];
      pb[k] = frames[12 * (e + 1) + 4 * k + 3];
    }
    *rad = r->radius[e];
    *link = e;
    return;
  }
  int s = e - nc, l = r->sphere_link[s];
  const double *F = frames + 12 * (l + 1), *c = r->sphere_center + 3 * s;
  for (int k = 0; k < 3; k++) pa[k] = pb[k] = F[4 * k] * c[0] + F[4 * k + 1] * c[1] + F[4 * k + 2] * c[2] + F[4 * k + 3];
  *rad = r->sphere_radius[s];
  *link = l;
}

/* Lipschitz constants of the robot elements (the whole-cell certificate):
 * turning joint k by dq moves a point x of the body by at most |dq| times
 * its distance to the joint axis, which is at most |x - o_k|.  For a point of
 * element e on link l >= k that is at most sum_{m=k..l} |o_{m+1} - o_m| (+ |c|
 * for a sphere centre c in frame T_{l+1}), with |o_{m+1} - o_m| =
 * sqrt(d_m^2 + a_m^2) whatever the configuration; joints after l do not move
 * it.  L[e * n_links + k]. */
void or_lipschitz(const or_robot *r, double *L) {
  int ne = n_elements(r), nc = r->radius ? r->n_links : 0;
  for (int e = 0; e < ne; e++) {
    int l = e < nc ? e : r->sphere_link[e - nc];
    double extra = 0.0;
    if (e >= nc) {
      const double *c = r->sphere_center + 3 * (e - nc);
      extra = sqrt(c[0] * c[0] + c[1] * c[1] + c[2] * c[2]);
    }
    for (int k = 0; k < r->n_links; k++) {
      double s = 0.0;
      if (k <= l) {
        for (int m = k; m <= l; m++)
          s += sqrt(r->dh[4 * m + 1] * r->dh[4 * m + 1] + r->dh[4 * m + 2] * r->dh[4 * m + 2]);
        s += extra;
      }
      L[e * r->n_links + k] = s;
    }
  }
}

/* Per point: margin = max over robot elements and obstacles of
 * (radius - distance); verdict = 1 (in collision, i.e. in C_obs) iff
 * margin >= 0; element = the lowest-index element whose own margin is within
 * 1e-9 of that maximum.  Per cell
 * (cell_off/cell_idx index the points): the AND of its points' verdicts, and
 * the whole-cell certificate: the cell's piece of the traced manifold is the
 * convex hull of its points, every q in it has |q_k - p_jk| <= span_jk =
 * max_l |p_lk - p_jk|, and element e's margin is at least its margin at p_j
 * minus sum_k L[e][k] |q_k - p_jk| (distances are 1-Lipschitz in the
 * element's points); so slack = max_j (margin_j - 1e-9 - sum_k L[e_j][k]
 * span_jk) >= 0 certifies every point of the piece (whole = 1). */
void or_certify_ex(const or_robot *r, const or_scene *sc, const double *points, int64_t P,
                   int32_t d, const int64_t *cell_off, const int64_t *cell_idx, int64_t n_cells,
                   uint8_t *verdict, double *margin, int32_t *element, uint8_t *cell_verdict,
                   uint8_t *cell_whole, double *cell_slack) {
  int ne = n_elements(r);
#pragma omp parallel for schedule(dynamic, 64)
  for (int64_t p = 0; p < P; p++) {
    double frames[12 * (OR_MAXD + 1)];
    or_fk_frames(r, points + p * d, frames);
    double best = -INFINITY, em[OR_MAXD + 256]; /* up to 256 spheres */
    for (int e = 0; e < ne; e++) {
      double pa[3], pb[3], rad;
      int link;
      element_at(r, frames, e, pa, pb, &rad, &link);
      em[e] = -INFINITY;
      for (int k = 0; k < sc->n; k++) {
        double dist = or_segment_obstacle_dist(pa, pb, sc->type[k], sc->pose + 12 * k, sc->dims + 3 * k);
        double m = rad - dist;
        if (m > em[e]) em[e] = m;
      }
      if (em[e] > best) best = em[e];
    }
    /* the deciding element: the lowest index whose margin is within
     * OR_ELEM_TIE of the maximum (elements inside obstacles all reach their
     * radius; the certificate below subtracts the same OR_ELEM_TIE) */
    int be = -1;
    for (int e = 0; e < ne && be < 0; e++)
      if (em[e] >= best - OR_ELEM_TIE) be = e;
    margin[p] = best;
    verdict[p] = best >= 0.0 ? 1 : 0;
    if (element) element[p] = be;
  }
  double *L = NULL;
  if (cell_whole || cell_slack) {
    L = (double *)malloc(sizeof(double) * (size_t)(ne > 0 ? ne : 1) * (size_t)r->n_links);
    if (L) or_lipschitz(r, L);
  }
  for (int64_t c = 0; c < n_cells; c++) {
    uint8_t v = 1;
    for (int64_t j = cell_off[c]; j < cell_off[c + 1]; j++) v = (uint8_t)(v & verdict[cell_idx[j]]);
    if (cell_verdict) cell_verdict[c] = v;
    if (!L) continue;
    double slack = -INFINITY;
    for (int64_t j = cell_off[c]; j < cell_off[c + 1]; j++) {
      int64_t pj = cell_idx[j];
      int e = element ? element[pj] : -1;
      if (e < 0) continue;
      double drop = 0.0;
      for (int k = 0; k < d; k++) {
        double span = 0.0;
        for (int64_t l = cell_off[c]; l < cell_off[c + 1]; l++) {
          double u = fabs(points[cell_idx[l] * d + k] - points[pj * d + k]);
          if (u > span) span = u;
        }
        drop += L[e * r->n_links + k] * span;
      }
      double s = (margin[pj] - OR_ELEM_TIE) - drop;
      if (s > slack) slack = s;
    }
    if (cell_slack) cell_slack[c] = slack;
    if (cell_whole) cell_whole[c] = slack >= 0.0 ? 1 : 0;
  }
  free(L);
}

void or_certify(const or_robot *r, const or_scene *sc, const double *points, int64_t P, int32_t d,
                const int64_t *cell_off, const int64_t *cell_idx, int64_t n_cells,
                uint8_t *verdict, double *margin, uint8_t *cell_verdict) {
  or_certify_ex(r, sc, points, P, d, cell_off, cell_idx, n_cells, verdict, margin, NULL,
                cell_verdict, NULL, NULL);
}

/* Host threads of the parallel loops (roots, f batches, certification);
 * n <= 0 restores all cores.  Returns the count now in use. */
#ifdef _OPENMP
#include <omp.h>
#endif
int or_set_threads(int n) {
#ifdef _OPENMP
  if (n <= 0) n = omp_get_num_procs();
  omp_set_num_threads(n);
  return omp_get_max_threads();
#else
  (void)n;
  return 1;
#endif
}
