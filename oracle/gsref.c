/*
 * gsref.c -- plain FP64 CPU oracle for point-set geodesic shooting with the
 * Barnes-Hut approximation (arXiv 1907.04834).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the reference that the CUDA path is
 * checked against.  It shares no code, header, table or constant with the CUDA
 * library; only the test suite, the smoke check and the benchmark's CPU
 * baseline leg load it.  Nothing here is tuned: every sum is a plain loop in
 * the order the definition states (OpenMP only splits the independent target
 * points across threads; each target's sum keeps its sequential order).
 *
 * Notation (Sec. 2.1): q_i, p_i in R^3, i = 0..N-1; d_ij = q_i - q_j;
 * g_ij = G(|d_ij|) = exp(-|d_ij|^2 / (2 sigma^2)) (the paper names a Gaussian
 * kernel without a formula: taken unnormalised, G(0) = 1); c_ij = p_i . p_j.
 * Hamiltonian (Sec. 2.1, with a factor 1/2 so that Eq. 1 gives dq/dt = K p):
 *     H(q,p) = 1/2 sum_i sum_j g_ij c_ij.
 * Hamilton's equations (Eq. 1):
 *     dq_i/dt =  dH/dp_i = F_i   = sum_j g_ij p_j                (j = i included)
 *     dp_i/dt = -dH/dq_i = Phi_i = sigma^-2 sum_j c_ij g_ij d_ij
 * Time discretisation (Sec. 2.1 says only "discretized in time"; taken as):
 *     explicit Euler, h = 1/T, q^{k+1} = q^k + h F^k, p^{k+1} = p^k + h Phi^k.
 * Objective (Eq. 2, p0* = argmin E):  E(p0) = H(q0,p0) + lambda sum_i |q_i^T - X_i|^2.
 * Backward stage (Sec. 2.2; taken as the discrete adjoint of the Euler map),
 *     alpha = dE/dq, beta = dE/dp; alpha^T = 2 lambda (q^T - X), beta^T = 0,
 *     alpha^k = alpha^{k+1} + h [ (dF/dq)^T alpha^{k+1} + (dPhi/dq)^T beta^{k+1} ]
 *     beta^k  = beta^{k+1}  + h [ (dF/dp)^T alpha^{k+1} + (dPhi/dp)^T beta^{k+1} ]
 *     dE/dp0  = beta^0 + F(q0, p0).
 *   Written out per pair (a = alpha^{k+1}, b = beta^{k+1}, w_ij = b_i - b_j):
 *     (dF/dq)^T a   |_i = -sigma^-2 sum_j g_ij ((a_i.p_j) + (a_j.p_i)) d_ij
 *     (dPhi/dq)^T b |_i =  sigma^-2 sum_j c_ij g_ij (w_ij - (w_ij.d_ij) d_ij / sigma^2)
 *     (dF/dp)^T a   |_i =  sum_j g_ij a_j
 *     (dPhi/dp)^T b |_i =  sigma^-2 sum_j g_ij (w_ij.d_ij) p_j
 *
 * Barnes-Hut (Sec. 2.2), rebuilt at every forward and backward step:
 *   - root cell = FP32 bounding box of the FP32-rounded positions; cells are
 *     per-axis bisections; a point's child octant at depth d is bit (9-d) of its
 *     10-bit quantised coordinates (quantisation taken as: ext = hi-lo; inv = 1024/ext;
 *     u = (x-lo)*inv; k = min((uint32)u, 1023); k = 0 when ext == 0; all FP32,
 *     round to nearest, no contraction); octant = (kx_b << 2) | (ky_b << 1) | kz_b.
 *   - points are inserted one by one in index order with the three-case rule
 *     (internal -> descend; empty leaf -> store; occupied leaf -> split into
 *     eight and pass both points down); depth 10 cannot split and keeps a list.
 *   - node statistics updated as each point is passed to a node: n, total
 *     momentum P = sum p, position sum (centroid = sum q / n, the plain mean), the
 *     FP32 "actual range" [lo, hi]; the backward stage adds A = sum alpha and
 *     B = sum beta.
 *   - traversal for a target point m (three cases of Sec. 2.2): a node with
 *     n >= 2 whose actual range lies farther than the threshold from q_m is one
 *     interaction with its summary; a leaf is computed exactly point by point;
 *     any other node is opened.  "Farther than the threshold" is taken as
 *     dist^2(q32_m, [lo,hi]) > r*r in FP32, with r = (float)(thresh * sigma),
 *     dx = max(lo - x, 0, x - hi) per axis, d2 = (dx*dx + dy*dy) + dz*dz.
 *   - summary interaction (Eq. 4 and the replacement rules after it, with the
 *     n_k members each counted, so the node acts as one source point
 *     at the centroid with momentum P, position derivative A and momentum
 *     derivative B/n.
 */
#include <float.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#if !defined(FLT_EVAL_METHOD) || FLT_EVAL_METHOD != 0
#error "the FP32 decision rule needs FLT_EVAL_METHOD == 0 (no excess precision)"
#endif

#define GSREF_EXACT 0
#define GSREF_BH 1
#define GSREF_TRUNC 2 /* pure truncation: only pairs within the threshold */
#define MAX_DEPTH 10

/* ------------------------------------------------------------------------ */
/* Pair interactions.  A "source" s is either a point or a node summary.      */
/* ------------------------------------------------------------------------ */

/* Forward contribution of source (qs, ps) to target (qm, pm): Eq. 1 / Eq. 3. */
static void fwd_pair(const double *qm, const double *pm, const double *qs,
                     const double *ps, double sigma, double *f, double *phi) {
  double d0 = qm[0] - qs[0], d1 = qm[1] - qs[1], d2 = qm[2] - qs[2];
  double r2 = d0 * d0 + d1 * d1 + d2 * d2;
  double g = exp(-r2 / (2.0 * sigma * sigma));
  double c = pm[0] * ps[0] + pm[1] * ps[1] + pm[2] * ps[2];
  f[0] += g * ps[0];
  f[1] += g * ps[1];
  f[2] += g * ps[2];
  phi[0] += c * g * d0;
  phi[1] += c * g * d1;
  phi[2] += c * g * d2;
}

/* Adjoint contribution of source (qs, ps, as, bs) to target m (formulas in the
 * header).  da and db receive the bracketed sums without the factor h; the
 * sigma^-2 factors are applied per term so the code reads like the formula. */
static void adj_pair(const double *qm, const double *pm, const double *am,
                     const double *bm, const double *qs, const double *ps,
                     const double *as, const double *bs, double sigma,
                     double *da, double *db) {
  double s2 = sigma * sigma;
  double d[3] = {qm[0] - qs[0], qm[1] - qs[1], qm[2] - qs[2]};
  double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
  double g = exp(-r2 / (2.0 * s2));
  double c = pm[0] * ps[0] + pm[1] * ps[1] + pm[2] * ps[2];
  double am_ps = am[0] * ps[0] + am[1] * ps[1] + am[2] * ps[2];
  double as_pm = as[0] * pm[0] + as[1] * pm[1] + as[2] * pm[2];
  double w[3] = {bm[0] - bs[0], bm[1] - bs[1], bm[2] - bs[2]};
  double wd = w[0] * d[0] + w[1] * d[1] + w[2] * d[2];
  for (int a = 0; a < 3; a++) {
    da[a] += -(g * (am_ps + as_pm) * d[a]) / s2;
    da[a] += (c * g * (w[a] - wd * d[a] / s2)) / s2;
    db[a] += g * as[a];
    db[a] += (g * wd * ps[a]) / s2;
  }
}

/* ------------------------------------------------------------------------ */
/* Exact all-pairs right-hand sides.                                         */
/* ------------------------------------------------------------------------ */

static void rhs_exact_row(int64_t N, const double *q, const double *p,
                          double sigma, int64_t i, double *F, double *Phi) {
  double f[3] = {0, 0, 0}, ph[3] = {0, 0, 0};
  for (int64_t j = 0; j < N; j++)
    fwd_pair(q + 3 * i, p + 3 * i, q + 3 * j, p + 3 * j, sigma, f, ph);
  for (int a = 0; a < 3; a++) {
    F[a] = f[a];
    Phi[a] = ph[a] / (sigma * sigma);
  }
}

/* Pure 3-sigma truncation (a variant of the method, not the paper's
 * approximation): the sums of Eq. 1 and of the adjoint over the pairs whose
 * FP32-rounded positions lie within the threshold r = (float)(thresh *
 * sigma): dx = x32_m - x32_j per axis, d2 = (dx*dx + dy*dy) + dz*dz in FP32
 * (each operation rounded, no contraction), pair taken iff d2 <= r*r.  The
 * relation is symmetric, and a point is always within its own threshold. */
static int within_cut(const float *a, const float *b, float thr) {
  float dx = a[0] - b[0];
  float dy = a[1] - b[1];
  float dz = a[2] - b[2];
  float d2 = dx * dx;
  d2 = d2 + dy * dy;
  d2 = d2 + dz * dz;
  return d2 <= thr;
}

static int64_t rhs_trunc_row(int64_t N, const double *q, const double *p,
                             const float *q32, float thr, double sigma,
                             int64_t i, double *F, double *Phi) {
  double f[3] = {0, 0, 0}, ph[3] = {0, 0, 0};
  int64_t n = 0;
  for (int64_t j = 0; j < N; j++)
    if (within_cut(q32 + 3 * i, q32 + 3 * j, thr)) {
      fwd_pair(q + 3 * i, p + 3 * i, q + 3 * j, p + 3 * j, sigma, f, ph);
      n++;
    }
  for (int a = 0; a < 3; a++) {
    F[a] = f[a];
    Phi[a] = ph[a] / (sigma * sigma);
  }
  return n;
}

static void adj_exact_row(int64_t N, const double *q, const double *p,
                          const double *al, const double *be, double sigma,
                          int64_t i, double *dA, double *dB) {
  double da[3] = {0, 0, 0}, db[3] = {0, 0, 0};
  for (int64_t j = 0; j < N; j++)
    adj_pair(q + 3 * i, p + 3 * i, al + 3 * i, be + 3 * i, q + 3 * j,
             p + 3 * j, al + 3 * j, be + 3 * j, sigma, da, db);
  for (int a = 0; a < 3; a++) {
    dA[a] = da[a];
    dB[a] = db[a];
  }
}

static int64_t adj_trunc_row(int64_t N, const double *q, const double *p,
                             const double *al, const double *be,
                             const float *q32, float thr, double sigma,
                             int64_t i, double *dA, double *dB) {
  double da[3] = {0, 0, 0}, db[3] = {0, 0, 0};
  int64_t n = 0;
  for (int64_t j = 0; j < N; j++)
    if (within_cut(q32 + 3 * i, q32 + 3 * j, thr)) {
      adj_pair(q + 3 * i, p + 3 * i, al + 3 * i, be + 3 * i, q + 3 * j,
               p + 3 * j, al + 3 * j, be + 3 * j, sigma, da, db);
      n++;
    }
  for (int a = 0; a < 3; a++) {
    dA[a] = da[a];
    dB[a] = db[a];
  }
  return n;
}

static float *round_positions(int64_t N, const double *q) {
  float *q32 = (float *)malloc((size_t)(N > 0 ? N : 1) * 3 * sizeof(float));
  for (int64_t i = 0; i < 3 * N; i++) q32[i] = (float)q[i];
  return q32;
}

/* ------------------------------------------------------------------------ */
/* Pointer octree built by the paper's insertion rule.                        */
/* ------------------------------------------------------------------------ */

typedef struct {
  int depth;
  int leaf;          /* 1 = leaf (holds points), 0 = internal */
  int64_t child[8];  /* internal: child node ids, -1 = empty cell */
  int64_t head, tail;/* leaf: member list (in insertion order) */
  int64_t n;         /* statistics: number of points passed to this node */
  double sq[3], sp[3], sa[3], sb[3];
  float lo[3], hi[3];
} onode;

typedef struct {
  onode *nodes;
  int64_t count, cap;
  int64_t *next;     /* member list links, one per point */
  uint32_t *kq;      /* quantised coordinates, 3 per point */
  float *q32;        /* FP32-rounded positions, 3 per point */
  const double *q, *p, *al, *be;
} otree;

static int64_t new_node(otree *t, int depth) {
  if (t->count == t->cap) {
    t->cap = t->cap ? 2 * t->cap : 64;
    t->nodes = (onode *)realloc(t->nodes, (size_t)t->cap * sizeof(onode));
  }
  onode *nd = &t->nodes[t->count];
  memset(nd, 0, sizeof(*nd));
  nd->depth = depth;
  nd->leaf = 1;
  nd->head = nd->tail = -1;
  for (int c = 0; c < 8; c++) nd->child[c] = -1;
  for (int a = 0; a < 3; a++) {
    nd->lo[a] = INFINITY;
    nd->hi[a] = -INFINITY;
  }
  return t->count++;
}

/* Statistics update when point i is passed to node k (Sec. 2.2). */
static void add_stats(otree *t, int64_t k, int64_t i) {
  onode *nd = &t->nodes[k];
  nd->n += 1;
  for (int a = 0; a < 3; a++) {
    nd->sq[a] += t->q[3 * i + a];
    nd->sp[a] += t->p[3 * i + a];
    if (t->al) nd->sa[a] += t->al[3 * i + a];
    if (t->be) nd->sb[a] += t->be[3 * i + a];
    float x = t->q32[3 * i + a];
    if (x < nd->lo[a]) nd->lo[a] = x;
    if (x > nd->hi[a]) nd->hi[a] = x;
  }
}

static int octant(const otree *t, int64_t i, int depth) {
  int b = 9 - depth;
  return (int)((((t->kq[3 * i + 0] >> b) & 1u) << 2) |
               (((t->kq[3 * i + 1] >> b) & 1u) << 1) |
               ((t->kq[3 * i + 2] >> b) & 1u));
}

static void leaf_append(otree *t, int64_t k, int64_t i) {
  onode *nd = &t->nodes[k];
  t->next[i] = -1;
  if (nd->tail < 0) nd->head = i;
  else t->next[nd->tail] = i;
  nd->tail = i;
}

/* Pass point i to node k: the three-case recursion of Sec. 2.2. */
static void insert(otree *t, int64_t k, int64_t i) {
  for (;;) {
    add_stats(t, k, i);
    onode *nd = &t->nodes[k];
    if (!nd->leaf) { /* case 1: internal node, descend */
      int o = octant(t, i, nd->depth);
      if (nd->child[o] < 0) {
        int64_t c = new_node(t, nd->depth + 1);
        t->nodes[k].child[o] = c;
      }
      k = t->nodes[k].child[o];
      continue;
    }
    if (nd->head < 0) { /* case 2: empty leaf, store and stop */
      leaf_append(t, k, i);
      return;
    }
    if (nd->depth == MAX_DEPTH) { /* finest cell: keep a list */
      leaf_append(t, k, i);
      return;
    }
    /* case 3: occupied leaf -> subdivide, pass the resident point down, then
     * continue passing point i down from this (now internal) node.  The
     * resident point's statistics are already counted in this node. */
    int64_t e = nd->head;
    nd->leaf = 0;
    nd->head = nd->tail = -1;
    int oe = octant(t, e, nd->depth);
    int64_t ce = new_node(t, t->nodes[k].depth + 1);
    t->nodes[k].child[oe] = ce;
    add_stats(t, ce, e);
    leaf_append(t, ce, e);
    /* point i: descend from the new internal node without re-counting it */
    int oi = octant(t, i, t->nodes[k].depth);
    if (t->nodes[k].child[oi] < 0) {
      int64_t ci = new_node(t, t->nodes[k].depth + 1);
      t->nodes[k].child[oi] = ci;
    }
    k = t->nodes[k].child[oi];
  }
}

/* Quantised coordinates (rule in the header) from the FP32 positions. */
static void quantise(int64_t N, const float *q32, float lo[3], float hi[3],
                     uint32_t *kq) {
  for (int a = 0; a < 3; a++) {
    lo[a] = INFINITY;
    hi[a] = -INFINITY;
  }
  for (int64_t i = 0; i < N; i++)
    for (int a = 0; a < 3; a++) {
      if (q32[3 * i + a] < lo[a]) lo[a] = q32[3 * i + a];
      if (q32[3 * i + a] > hi[a]) hi[a] = q32[3 * i + a];
    }
  for (int a = 0; a < 3; a++) {
    float ext = hi[a] - lo[a];
    float inv = ext > 0.0f ? 1024.0f / ext : 0.0f;
    for (int64_t i = 0; i < N; i++) {
      uint32_t k = 0;
      if (ext > 0.0f) {
        float u = (q32[3 * i + a] - lo[a]) * inv;
        k = (uint32_t)u;
        if (k > 1023u) k = 1023u;
      }
      kq[3 * i + a] = k;
    }
  }
}

static void tree_build(otree *t, int64_t N, const double *q, const double *p,
                       const double *al, const double *be) {
  memset(t, 0, sizeof(*t));
  t->q = q;
  t->p = p;
  t->al = al;
  t->be = be;
  t->next = (int64_t *)malloc((size_t)N * sizeof(int64_t));
  t->kq = (uint32_t *)malloc((size_t)N * 3 * sizeof(uint32_t));
  t->q32 = (float *)malloc((size_t)N * 3 * sizeof(float));
  for (int64_t i = 0; i < 3 * N; i++) t->q32[i] = (float)q[i];
  float lo[3], hi[3];
  quantise(N, t->q32, lo, hi, t->kq);
  new_node(t, 0); /* root */
  for (int64_t i = 0; i < N; i++) insert(t, 0, i);
}

static void tree_free(otree *t) {
  free(t->nodes);
  free(t->next);
  free(t->kq);
  free(t->q32);
}

/* Threshold r*r of the far test, in FP32. */
static float far_threshold(double thresh, double sigma) {
  float r = (float)(thresh * sigma);
  return r * r;
}

/* Is the node's actual range farther than the threshold (rule in the header)? */
static int is_far(const float *x, const onode *nd, float thr) {
  float dd[3];
  for (int a = 0; a < 3; a++) {
    float t = 0.0f;
    float u = nd->lo[a] - x[a];
    float v = x[a] - nd->hi[a];
    if (u > t) t = u;
    if (v > t) t = v;
    dd[a] = t;
  }
  float d2 = dd[0] * dd[0];
  d2 = d2 + dd[1] * dd[1];
  d2 = d2 + dd[2] * dd[2];
  return d2 > thr;
}

/* Opening-angle variant (classic Barnes-Hut form, not the paper's rule): with
 * s the largest side of the node's FP32 actual range and c its centre,
 * c = (lo + hi) * 0.5, the node is summarised iff s*s < theta^2 * d2, where
 * d2 = (dx*dx + dy*dy) + dz*dz, dx = x - c per axis, and thr = theta32 *
 * theta32 (theta32 = (float)theta); all FP32, each operation rounded. */
static int is_far_angle(const float *x, const onode *nd, float thr) {
  float s = nd->hi[0] - nd->lo[0];
  float sy = nd->hi[1] - nd->lo[1];
  float sz = nd->hi[2] - nd->lo[2];
  if (sy > s) s = sy;
  if (sz > s) s = sz;
  float d[3];
  for (int a = 0; a < 3; a++) {
    float c = (nd->lo[a] + nd->hi[a]) * 0.5f;
    d[a] = x[a] - c;
  }
  float d2 = d[0] * d[0];
  d2 = d2 + d[1] * d[1];
  d2 = d2 + d[2] * d[2];
  float ss = s * s;
  float td = thr * d2;
  return ss < td;
}

static float angle_threshold(double theta) {
  float t = (float)theta;
  return t * t;
}

static float rule_threshold(int crit, double thresh, double sigma) {
  return crit ? angle_threshold(thresh) : far_threshold(thresh, sigma);
}

/* Interaction lists are produced by the same traversal, so tests can check
 * which sources each target took (kind 0 = point, 1 = node summary). */
typedef struct {
  int64_t *kind, *id;
  int64_t len, cap;
} ilist;

typedef struct {
  const otree *t;
  double sigma;
  float thr;
  int adjoint;
  int64_t leaf; /* leaf-size variant: near nodes of <= leaf points taken exactly */
  int crit;     /* 0: the paper's distance rule; 1: opening-angle variant */
  int64_t m;
  /* the target: point m of the tree, or an outside point (tracer) */
  const double *tq, *tp, *ta, *tb;
  const float *tq32;
  double acc0[3], acc1[3];
  int64_t n_point, n_node;
  ilist *list;
  /* decision fingerprint (gsref_bh_tally): DFS position of each point, DFS
   * first position of each node's members; NULL when not wanted */
  const int64_t *tpos, *tfirst;
  uint64_t h_point, h_node;
  int64_t n_reached; /* nodes of >= 2 points reached, a chain of single-child cells once */
} visit_ctx;

/* splitmix64 (Steele, Lea and Flood, "Fast splittable pseudorandom number
 * generators", OOPSLA 2014): the output of the generator whose state is
 * `key`, used as a 64-bit mix of an interaction's identity. */
static uint64_t mix64(uint64_t key) {
  uint64_t z = key + 0x9e3779b97f4a7c15ull;
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
  return z ^ (z >> 31);
}

/* Identity of a source as the set of points it stands for: the DFS position
 * of its first member (the DFS order is the stable Morton order) and its
 * member count; a point is the set of itself. */
static uint64_t source_key(int64_t first, int64_t n) {
  return ((uint64_t)first << 32) | (uint64_t)n;
}

static void record(visit_ctx *v, int64_t kind, int64_t id) {
  if (v->tpos) {
    if (kind == 0)
      v->h_point += mix64(source_key(v->tpos[id], 1));
    else
      v->h_node += mix64(source_key(v->tfirst[id], v->t->nodes[id].n));
  }
  if (!v->list) return;
  if (v->list->len < v->list->cap) {
    v->list->kind[v->list->len] = kind;
    v->list->id[v->list->len] = id;
  }
  v->list->len++;
}

static void point_source(visit_ctx *v, int64_t s) {
  const otree *t = v->t;
  if (!v->adjoint)
    fwd_pair(v->tq, v->tp, t->q + 3 * s, t->p + 3 * s, v->sigma, v->acc0, v->acc1);
  else
    adj_pair(v->tq, v->tp, v->ta, v->tb,
             t->q + 3 * s, t->p + 3 * s, t->al + 3 * s, t->be + 3 * s,
             v->sigma, v->acc0, v->acc1);
  v->n_point++;
  record(v, 0, s);
}

static void node_source(visit_ctx *v, int64_t k) {
  const otree *t = v->t;
  const onode *nd = &t->nodes[k];
  double n = (double)nd->n;
  double qc[3] = {nd->sq[0] / n, nd->sq[1] / n, nd->sq[2] / n};
  if (!v->adjoint) {
    fwd_pair(v->tq, v->tp, qc, nd->sp, v->sigma, v->acc0, v->acc1);
  } else {
    double bavg[3] = {nd->sb[0] / n, nd->sb[1] / n, nd->sb[2] / n};
    adj_pair(v->tq, v->tp, v->ta, v->tb, qc,
             nd->sp, nd->sa, bavg, v->sigma, v->acc0, v->acc1);
  }
  v->n_node++;
  record(v, 1, k);
}

/* Every point of node k, exactly (children in octant order). */
static void all_points(visit_ctx *v, int64_t k) {
  const otree *t = v->t;
  const onode *nd = &t->nodes[k];
  if (nd->n == 0) return;
  if (nd->leaf) {
    for (int64_t s = nd->head; s >= 0; s = t->next[s]) point_source(v, s);
    return;
  }
  for (int c = 0; c < 8; c++)
    if (nd->child[c] >= 0) all_points(v, nd->child[c]);
}

/* top: k is the root or its parent has >= 2 non-empty children, i.e. k is
 * the first of a chain of cells with the same members (and the same range,
 * so the same decision); only that one is counted as reached. */
static void visit(visit_ctx *v, int64_t k, int top) {
  const otree *t = v->t;
  const onode *nd = &t->nodes[k];
  if (nd->n == 0) return;
  int nc = 0;
  if (!nd->leaf)
    for (int c = 0; c < 8; c++) nc += nd->child[c] >= 0;
  if (nd->n >= 2 && top) v->n_reached++;
  const float *x = v->tq32;
  if (nd->n >= 2 && (v->crit ? is_far_angle(x, nd, v->thr) : is_far(x, nd, v->thr))) {
    node_source(v, k); /* case 2: summarised far node */
    return;
  }
  if (nd->leaf) { /* case 1 (and a finest-cell list): exact */
    for (int64_t s = nd->head; s >= 0; s = t->next[s]) point_source(v, s);
    return;
  }
  if (nd->n <= v->leaf) { /* leaf-size variant: a near node of <= leaf points, exactly */
    all_points(v, k);
    return;
  }
  for (int c = 0; c < 8; c++) /* case 3: open the node */
    if (nd->child[c] >= 0) visit(v, nd->child[c], nc >= 2);
}

static void bh_target(const otree *t, double sigma, float thr, int64_t leaf,
                      int crit, int adjoint, int64_t m, double *o0, double *o1,
                      int64_t *np, int64_t *nn, ilist *list) {
  visit_ctx v;
  memset(&v, 0, sizeof(v));
  v.t = t;
  v.sigma = sigma;
  v.thr = thr;
  v.leaf = leaf;
  v.crit = crit;
  v.tq = t->q + 3 * m;
  v.tp = t->p + 3 * m;
  v.ta = adjoint ? t->al + 3 * m : NULL;
  v.tb = adjoint ? t->be + 3 * m : NULL;
  v.tq32 = t->q32 + 3 * m;
  v.adjoint = adjoint;
  v.m = m;
  v.list = list;
  visit(&v, 0, 1);
  for (int a = 0; a < 3; a++) {
    o0[a] = v.acc0[a];
    o1[a] = v.acc1[a];
  }
  *np = v.n_point;
  *nn = v.n_node;
}

/* ------------------------------------------------------------------------ */
/* Public right-hand sides.                                                   */
/* ------------------------------------------------------------------------ */

/* Forward right-hand side (F, Phi) of Eq. 1 for every point.  mode 0 = exact
 * all pairs (Sec. 2.1); mode 1 = Barnes-Hut (Sec. 2.2); mode 2 = pure
 * truncation (pairs within the threshold only; counts[0] = those pairs).  counts (optional,
 * 2 entries) receives the number of point-point and point-node interactions. */
void gsref_rhs(int64_t N, const double *q, const double *p, double sigma,
               int mode, double thresh, int leaf, int crit, double *F,
               double *Phi, int64_t *counts) {
  int64_t np_tot = 0, nn_tot = 0;
  if (mode == GSREF_EXACT) {
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < N; i++)
      rhs_exact_row(N, q, p, sigma, i, F + 3 * i, Phi + 3 * i);
    np_tot = N * N;
  } else if (mode == GSREF_TRUNC) {
    float *q32 = round_positions(N, q);
    float thr = far_threshold(thresh, sigma);
#pragma omp parallel for schedule(static) reduction(+ : np_tot)
    for (int64_t i = 0; i < N; i++)
      np_tot += rhs_trunc_row(N, q, p, q32, thr, sigma, i, F + 3 * i, Phi + 3 * i);
    free(q32);
  } else {
    otree t;
    tree_build(&t, N, q, p, NULL, NULL);
    float thr = rule_threshold(crit, thresh, sigma);
#pragma omp parallel for schedule(dynamic, 64) reduction(+ : np_tot, nn_tot)
    for (int64_t i = 0; i < N; i++) {
      int64_t a, b;
      bh_target(&t, sigma, thr, leaf, crit, 0, i, F + 3 * i, Phi + 3 * i, &a, &b, NULL);
      for (int c = 0; c < 3; c++) Phi[3 * i + c] /= sigma * sigma;
      np_tot += a;
      nn_tot += b;
    }
    tree_free(&t);
  }
  if (counts) {
    counts[0] = np_tot;
    counts[1] = nn_tot;
  }
}

/* Exact forward right-hand side for selected rows only (sampled parity). */
void gsref_rhs_rows(int64_t N, const double *q, const double *p, double sigma,
                    int64_t nrows, const int64_t *rows, double *F,
                    double *Phi) {
#pragma omp parallel for schedule(static)
  for (int64_t r = 0; r < nrows; r++)
    rhs_exact_row(N, q, p, sigma, rows[r], F + 3 * r, Phi + 3 * r);
}

/* Adjoint right-hand side: dA, dB such that alpha^k = a + h dA and
 * beta^k = b + h dB (a = alpha^{k+1}, b = beta^{k+1}). */
void gsref_adj_rhs(int64_t N, const double *q, const double *p,
                   const double *al, const double *be, double sigma, int mode,
                   double thresh, int leaf, int crit, double *dA, double *dB,
                   int64_t *counts) {
  int64_t np_tot = 0, nn_tot = 0;
  if (mode == GSREF_EXACT) {
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < N; i++)
      adj_exact_row(N, q, p, al, be, sigma, i, dA + 3 * i, dB + 3 * i);
    np_tot = N * N;
  } else if (mode == GSREF_TRUNC) {
    float *q32 = round_positions(N, q);
    float thr = far_threshold(thresh, sigma);
#pragma omp parallel for schedule(static) reduction(+ : np_tot)
    for (int64_t i = 0; i < N; i++)
      np_tot += adj_trunc_row(N, q, p, al, be, q32, thr, sigma, i, dA + 3 * i, dB + 3 * i);
    free(q32);
  } else {
    otree t;
    tree_build(&t, N, q, p, al, be);
    float thr = rule_threshold(crit, thresh, sigma);
#pragma omp parallel for schedule(dynamic, 64) reduction(+ : np_tot, nn_tot)
    for (int64_t i = 0; i < N; i++) {
      int64_t a, b;
      bh_target(&t, sigma, thr, leaf, crit, 1, i, dA + 3 * i, dB + 3 * i, &a, &b, NULL);
      np_tot += a;
      nn_tot += b;
    }
    tree_free(&t);
  }
  if (counts) {
    counts[0] = np_tot;
    counts[1] = nn_tot;
  }
}

void gsref_adj_rhs_rows(int64_t N, const double *q, const double *p,
                        const double *al, const double *be, double sigma,
                        int64_t nrows, const int64_t *rows, double *dA,
                        double *dB) {
#pragma omp parallel for schedule(static)
  for (int64_t r = 0; r < nrows; r++)
    adj_exact_row(N, q, p, al, be, sigma, rows[r], dA + 3 * r, dB + 3 * r);
}

/* ------------------------------------------------------------------------ */
/* Shooting and its gradient.                                                 */
/* ------------------------------------------------------------------------ */

static double half_p_dot_F(int64_t N, const double *p, const double *F) {
  double s = 0.0;
  for (int64_t i = 0; i < 3 * N; i++) s += p[i] * F[i];
  return 0.5 * s;
}

/* Geodesic shooting (Eq. 1, Euler, h = 1/T).  H (optional, 2 entries) gets
 * H(q^0,p^0) and H(q^T,p^T) = 1/2 sum_i p_i . F_i in the same mode. */
void gsref_shoot(int64_t N, const double *q0, const double *p0, double sigma,
                 int T, int mode, double thresh, int leaf, int crit,
                 double *q1, double *p1, double *H) {
  double *F = (double *)malloc((size_t)N * 3 * sizeof(double));
  double *Phi = (double *)malloc((size_t)N * 3 * sizeof(double));
  double h = 1.0 / (double)T;
  memcpy(q1, q0, (size_t)N * 3 * sizeof(double));
  memcpy(p1, p0, (size_t)N * 3 * sizeof(double));
  for (int k = 0; k < T; k++) {
    gsref_rhs(N, q1, p1, sigma, mode, thresh, leaf, crit, F, Phi, NULL);
    if (k == 0 && H) H[0] = half_p_dot_F(N, p1, F);
    for (int64_t i = 0; i < 3 * N; i++) {
      q1[i] += h * F[i];
      p1[i] += h * Phi[i];
    }
  }
  if (H) {
    gsref_rhs(N, q1, p1, sigma, mode, thresh, leaf, crit, F, Phi, NULL);
    H[1] = half_p_dot_F(N, p1, F);
  }
  free(F);
  free(Phi);
}

/* Classical fourth-order Runge-Kutta shooting (test infrastructure for the
 * right-hand side: its trajectories converge at fourth order to the exact
 * flow, so an error in F or Phi shows as a lost order; not a scheme of the
 * method).  h = 1/T; k1 = f(y), k2 = f(y + h/2 k1), k3 = f(y + h/2 k2),
 * k4 = f(y + h k3), y += h/6 (k1 + 2 k2 + 2 k3 + k4), f = (F, Phi). */
void gsref_shoot_rk4(int64_t N, const double *q0, const double *p0, double sigma, int T,
                     double *q1, double *p1) {
  size_t sz = (size_t)N * 3;
  double *kq = (double *)malloc(4 * sz * sizeof(double));
  double *kp = (double *)malloc(4 * sz * sizeof(double));
  double *yq = (double *)malloc(sz * sizeof(double));
  double *yp = (double *)malloc(sz * sizeof(double));
  double h = 1.0 / (double)T;
  const double c[4] = {0.0, 0.5, 0.5, 1.0};
  memcpy(q1, q0, sz * sizeof(double));
  memcpy(p1, p0, sz * sizeof(double));
  for (int k = 0; k < T; k++) {
    for (int s = 0; s < 4; s++) {
      for (size_t i = 0; i < sz; i++) {
        yq[i] = s ? q1[i] + c[s] * h * kq[(size_t)(s - 1) * sz + i] : q1[i];
        yp[i] = s ? p1[i] + c[s] * h * kp[(size_t)(s - 1) * sz + i] : p1[i];
      }
      gsref_rhs(N, yq, yp, sigma, 0, 0.0, 1, 0, kq + (size_t)s * sz, kp + (size_t)s * sz, NULL);
    }
    for (size_t i = 0; i < sz; i++) {
      q1[i] += h / 6.0 * (kq[i] + 2.0 * kq[sz + i] + 2.0 * kq[2 * sz + i] + kq[3 * sz + i]);
      p1[i] += h / 6.0 * (kp[i] + 2.0 * kp[sz + i] + 2.0 * kp[2 * sz + i] + kp[3 * sz + i]);
    }
  }
  free(kq);
  free(kp);
  free(yq);
  free(yp);
}

/* Semi-implicit symplectic Euler (a variant of the time discretisation, not
 * the paper's scheme; its Sec. 2.1 only says the flow is discretised in
 * time).  H is not separable (K depends on q), so the symplectic Euler step
 *     p^{k+1} = p^k + h Phi(q^k, p^{k+1}),   q^{k+1} = q^k + h F(q^k, p^{k+1})
 * is implicit in p.  It is solved approximately by `iters` fixed-point passes
 * with q held at q^k:  r^0 = p^k,  r^{m+1} = p^k + h Phi(q^k, r^m), followed
 * by the update  q^{k+1} = q^k + h F(q^k, r^iters),  p^{k+1} = p^k + h Phi(q^k,
 * r^iters).  iters = 0 is the explicit Euler step of gsref_shoot; as iters
 * grows the step tends to the symplectic Euler step.  H as in gsref_shoot. */
void gsref_shoot_sympl(int64_t N, const double *q0, const double *p0, double sigma,
                       int T, int mode, double thresh, int leaf, int crit, int iters,
                       double *q1, double *p1, double *H) {
  size_t sz = (size_t)N * 3;
  double *F = (double *)malloc(sz * sizeof(double));
  double *Phi = (double *)malloc(sz * sizeof(double));
  double *r = (double *)malloc(sz * sizeof(double));
  double h = 1.0 / (double)T;
  memcpy(q1, q0, sz * sizeof(double));
  memcpy(p1, p0, sz * sizeof(double));
  for (int k = 0; k < T; k++) {
    memcpy(r, p1, sz * sizeof(double));
    for (int m = 0; m <= iters; m++) {
      gsref_rhs(N, q1, r, sigma, mode, thresh, leaf, crit, F, Phi, NULL);
      if (k == 0 && m == 0 && H) H[0] = half_p_dot_F(N, p1, F);
      if (m < iters)
        for (size_t i = 0; i < sz; i++) r[i] = p1[i] + h * Phi[i];
    }
    for (size_t i = 0; i < sz; i++) {
      q1[i] += h * F[i];
      p1[i] += h * Phi[i];
    }
  }
  if (H) {
    gsref_rhs(N, q1, p1, sigma, mode, thresh, leaf, crit, F, Phi, NULL);
    H[1] = half_p_dot_F(N, p1, F);
  }
  free(F);
  free(Phi);
  free(r);
}

/* Objective (Eq. 2) and its gradient with respect to p0 by the discrete
 * adjoint.  E gets {total, H(q0,p0), lambda * sum |q^T - X|^2}; q1 (optional)
 * gets q^T.  The whole trajectory is stored (plain, no checkpointing). */
void gsref_shoot_grad(int64_t N, const double *q0, const double *p0,
                      const double *X, double sigma, int T, double lambda,
                      int mode, double thresh, int leaf, int crit, double *E,
                      double *grad, double *q1) {
  size_t sz = (size_t)N * 3;
  double *qs = (double *)malloc((size_t)(T + 1) * sz * sizeof(double));
  double *ps = (double *)malloc((size_t)(T + 1) * sz * sizeof(double));
  double *F = (double *)malloc(sz * sizeof(double));
  double *F0 = (double *)malloc(sz * sizeof(double));
  double *Phi = (double *)malloc(sz * sizeof(double));
  double *al = (double *)malloc(sz * sizeof(double));
  double *be = (double *)malloc(sz * sizeof(double));
  double *dA = (double *)malloc(sz * sizeof(double));
  double *dB = (double *)malloc(sz * sizeof(double));
  double h = 1.0 / (double)T;
  memcpy(qs, q0, sz * sizeof(double));
  memcpy(ps, p0, sz * sizeof(double));
  for (int k = 0; k < T; k++) {
    double *qk = qs + (size_t)k * sz, *pk = ps + (size_t)k * sz;
    gsref_rhs(N, qk, pk, sigma, mode, thresh, leaf, crit, F, Phi, NULL);
    if (k == 0) memcpy(F0, F, sz * sizeof(double));
    for (size_t i = 0; i < sz; i++) {
      qk[sz + i] = qk[i] + h * F[i];
      pk[sz + i] = pk[i] + h * Phi[i];
    }
  }
  const double *qT = qs + (size_t)T * sz;
  double data = 0.0;
  for (size_t i = 0; i < sz; i++) {
    double r = qT[i] - X[i];
    data += r * r;
  }
  double H0 = half_p_dot_F(N, p0, F0);
  E[0] = H0 + lambda * data;
  E[1] = H0;
  E[2] = lambda * data;
  for (size_t i = 0; i < sz; i++) {
    al[i] = 2.0 * lambda * (qT[i] - X[i]);
    be[i] = 0.0;
  }
  for (int k = T - 1; k >= 0; k--) {
    gsref_adj_rhs(N, qs + (size_t)k * sz, ps + (size_t)k * sz, al, be, sigma,
                  mode, thresh, leaf, crit, dA, dB, NULL);
    for (size_t i = 0; i < sz; i++) {
      al[i] += h * dA[i];
      be[i] += h * dB[i];
    }
  }
  for (size_t i = 0; i < sz; i++) grad[i] = be[i] + F0[i];
  if (q1) memcpy(q1, qT, sz * sizeof(double));
  free(qs);
  free(ps);
  free(F);
  free(F0);
  free(Phi);
  free(al);
  free(be);
  free(dA);
  free(dB);
}

/* Objective (Eq. 2) and its gradient with respect to p0 for the
 * semi-implicit scheme of gsref_shoot_sympl (M = iters fixed-point passes
 * per step): the discrete adjoint of that step, in the same spirit as the
 * backward stage of gsref_shoot_grad.  With r_0 = p^k and r_m = p^k + h
 * Phi(q^k, r_{m-1}), a = dE/dq^{k+1}, b = dE/dp^{k+1}, and [x, y](r) the
 * adjoint right-hand side of gsref_adj_rhs at (q^k, r) with alpha = x,
 * beta = y (its two parts dA, dB):
 *   rho_M     = h dB[a, b](r_M)
 *   rho_{m-1} = h dB[0, rho_m](r_{m-1}),                m = M .. 1
 *   dE/dq^k   = a + h dA[a, b](r_M) + sum_{m=1..M} h dA[0, rho_m](r_{m-1})
 *   dE/dp^k   = b + sum_{m=0..M} rho_m
 * (r_M enters the update q^{k+1} = q^k + h F(q^k, r_M), p^{k+1} = p^k + h
 * Phi(q^k, r_M); each r_m depends on p^k directly and through r_{m-1}, and
 * on q^k).  dE/dp0 = beta^0 + F(q0, p0).  The passes are recomputed from
 * (q^k, p^k) in the backward sweep.  M = 0 is gsref_shoot_grad. */
void gsref_shoot_grad_sympl(int64_t N, const double *q0, const double *p0,
                            const double *X, double sigma, int T, double lambda,
                            int mode, double thresh, int leaf, int crit, int iters,
                            double *E, double *grad, double *q1) {
  size_t sz = (size_t)N * 3;
  int M = iters;
  double *qs = (double *)malloc((size_t)(T + 1) * sz * sizeof(double));
  double *ps = (double *)malloc((size_t)(T + 1) * sz * sizeof(double));
  double *rs = (double *)malloc((size_t)(M + 1) * sz * sizeof(double));
  double *F = (double *)malloc(sz * sizeof(double));
  double *F0 = (double *)malloc(sz * sizeof(double));
  double *Phi = (double *)malloc(sz * sizeof(double));
  double *al = (double *)malloc(sz * sizeof(double));
  double *be = (double *)malloc(sz * sizeof(double));
  double *dA = (double *)malloc(sz * sizeof(double));
  double *dB = (double *)malloc(sz * sizeof(double));
  double *rho = (double *)malloc(sz * sizeof(double));
  double *zero = (double *)calloc(sz, sizeof(double));
  double h = 1.0 / (double)T;
  memcpy(qs, q0, sz * sizeof(double));
  memcpy(ps, p0, sz * sizeof(double));
  for (int k = 0; k < T; k++) {
    double *qk = qs + (size_t)k * sz, *pk = ps + (size_t)k * sz;
    memcpy(rs, pk, sz * sizeof(double));
    for (int m = 0; m <= M; m++) {
      gsref_rhs(N, qk, rs, sigma, mode, thresh, leaf, crit, F, Phi, NULL);
      if (k == 0 && m == 0) memcpy(F0, F, sz * sizeof(double));
      if (m < M)
        for (size_t i = 0; i < sz; i++) rs[i] = pk[i] + h * Phi[i];
    }
    for (size_t i = 0; i < sz; i++) {
      qk[sz + i] = qk[i] + h * F[i];
      pk[sz + i] = pk[i] + h * Phi[i];
    }
  }
  const double *qT = qs + (size_t)T * sz;
  double data = 0.0;
  for (size_t i = 0; i < sz; i++) {
    double r = qT[i] - X[i];
    data += r * r;
  }
  double H0 = half_p_dot_F(N, p0, F0);
  E[0] = H0 + lambda * data;
  E[1] = H0;
  E[2] = lambda * data;
  for (size_t i = 0; i < sz; i++) {
    al[i] = 2.0 * lambda * (qT[i] - X[i]);
    be[i] = 0.0;
  }
  for (int k = T - 1; k >= 0; k--) {
    const double *qk = qs + (size_t)k * sz, *pk = ps + (size_t)k * sz;
    /* the passes of step k: rs[m] = r_m */
    memcpy(rs, pk, sz * sizeof(double));
    for (int m = 1; m <= M; m++) {
      gsref_rhs(N, qk, rs + (size_t)(m - 1) * sz, sigma, mode, thresh, leaf, crit, F, Phi,
                NULL);
      for (size_t i = 0; i < sz; i++) rs[(size_t)m * sz + i] = pk[i] + h * Phi[i];
    }
    /* the update's terms at r_M, then the passes' terms back to r_0; al and
     * be accumulate dE/dq^k and dE/dp^k */
    gsref_adj_rhs(N, qk, rs + (size_t)M * sz, al, be, sigma, mode, thresh, leaf, crit, dA,
                  dB, NULL);
    for (size_t i = 0; i < sz; i++) {
      al[i] += h * dA[i];
      rho[i] = h * dB[i];
      be[i] += rho[i];
    }
    for (int m = M; m >= 1; m--) {
      gsref_adj_rhs(N, qk, rs + (size_t)(m - 1) * sz, zero, rho, sigma, mode, thresh, leaf,
                    crit, dA, dB, NULL);
      for (size_t i = 0; i < sz; i++) {
        al[i] += h * dA[i];
        rho[i] = h * dB[i];
        be[i] += rho[i];
      }
    }
  }
  for (size_t i = 0; i < sz; i++) grad[i] = be[i] + F0[i];
  if (q1) memcpy(q1, qT, sz * sizeof(double));
  free(qs);
  free(ps);
  free(rs);
  free(F);
  free(F0);
  free(Phi);
  free(al);
  free(be);
  free(dA);
  free(dB);
  free(rho);
  free(zero);
}

/* ------------------------------------------------------------------------ */
/* Dense velocity field (Eq. 3) and points carried by it.                     */
/* ------------------------------------------------------------------------ */

/* Velocity of Eq. 3 at M points x of the domain (mesh vertices, grid nodes):
 * v(x) = sum_i G(|x - q_i|) p_i, all N particles, exact sums. */
void gsref_velocity(int64_t N, const double *q, const double *p, int64_t M,
                    const double *x, double sigma, double *v) {
  double inv2s2 = 1.0 / (2.0 * sigma * sigma);
#pragma omp parallel for schedule(static)
  for (int64_t m = 0; m < M; m++) {
    double acc[3] = {0.0, 0.0, 0.0};
    for (int64_t i = 0; i < N; i++) {
      double e0 = x[3 * m] - q[3 * i];
      double e1 = x[3 * m + 1] - q[3 * i + 1];
      double e2 = x[3 * m + 2] - q[3 * i + 2];
      double G = exp(-(e0 * e0 + e1 * e1 + e2 * e2) * inv2s2);
      for (int a = 0; a < 3; a++) acc[a] += G * p[3 * i + a];
    }
    for (int a = 0; a < 3; a++) v[3 * m + a] = acc[a];
  }
}

/* Velocity of Eq. 3 at M outside points with the Barnes-Hut approximation
 * of Sec. 2.2 over the particles' tree: each point is a target of the
 * three-case traversal (its FP32 position decides), with no momentum of its
 * own, so only the velocity sums are formed.  leaf, crit as in gsref_rhs. */
void gsref_velocity_bh(int64_t N, const double *q, const double *p, int64_t M,
                       const double *x, double sigma, double thresh, int leaf,
                       int crit, double *v) {
  otree t;
  tree_build(&t, N, q, p, NULL, NULL);
  float thr = rule_threshold(crit, thresh, sigma);
  float *x32 = round_positions(M, x);
  static const double zero[3] = {0.0, 0.0, 0.0};
#pragma omp parallel for schedule(dynamic, 64)
  for (int64_t m = 0; m < M; m++) {
    visit_ctx vc;
    memset(&vc, 0, sizeof(vc));
    vc.t = &t;
    vc.sigma = sigma;
    vc.thr = thr;
    vc.leaf = leaf;
    vc.crit = crit;
    vc.tq = x + 3 * m;
    vc.tp = zero;
    vc.tq32 = x32 + 3 * m;
    visit(&vc, 0, 1);
    for (int a = 0; a < 3; a++) v[3 * m + a] = vc.acc0[a];
  }
  free(x32);
  tree_free(&t);
}

/* Shooting (Eq. 1; mode 0 exact, 1 Barnes-Hut) with M tracer points x
 * carried by the velocity field of Eq. 3 (same mode).  The tracers do not
 * act on the particles; they take the same explicit Euler steps, from the
 * particles' state at the start of each step:
 * x^{k+1} = x^k + h v(x^k; q^k, p^k). */
void gsref_flow(int64_t N, const double *q0, const double *p0, int64_t M,
                const double *x0, double sigma, int T, int mode, double thresh,
                int leaf, int crit, double *q1, double *p1, double *x1) {
  double *F = (double *)malloc((size_t)N * 3 * sizeof(double));
  double *Phi = (double *)malloc((size_t)N * 3 * sizeof(double));
  double *v = (double *)malloc((size_t)(M > 0 ? M : 1) * 3 * sizeof(double));
  double h = 1.0 / (double)T;
  memcpy(q1, q0, (size_t)N * 3 * sizeof(double));
  memcpy(p1, p0, (size_t)N * 3 * sizeof(double));
  memcpy(x1, x0, (size_t)M * 3 * sizeof(double));
  for (int k = 0; k < T; k++) {
    if (mode == GSREF_BH)
      gsref_velocity_bh(N, q1, p1, M, x1, sigma, thresh, leaf, crit, v);
    else
      gsref_velocity(N, q1, p1, M, x1, sigma, v);
    gsref_rhs(N, q1, p1, sigma, mode == GSREF_BH ? GSREF_BH : GSREF_EXACT, thresh, leaf,
              crit, F, Phi, NULL);
    for (int64_t i = 0; i < 3 * M; i++) x1[i] += h * v[i];
    for (int64_t i = 0; i < 3 * N; i++) {
      q1[i] += h * F[i];
      p1[i] += h * Phi[i];
    }
  }
  free(F);
  free(Phi);
  free(v);
}

/* ------------------------------------------------------------------------ */
/* Tree inspection for tests.                                                 */
/* ------------------------------------------------------------------------ */

/* Per-point quantised coordinates and the 30-bit Morton code of the rule in the header
 * (bit 3b+2 = x bit b, 3b+1 = y bit b, 3b = z bit b). */
void gsref_morton(int64_t N, const double *q, uint32_t *kq, uint32_t *code) {
  float *q32 = (float *)malloc((size_t)N * 3 * sizeof(float));
  for (int64_t i = 0; i < 3 * N; i++) q32[i] = (float)q[i];
  float lo[3], hi[3];
  quantise(N, q32, lo, hi, kq);
  for (int64_t i = 0; i < N; i++) {
    uint32_t c = 0;
    for (int b = 0; b < 10; b++) {
      c |= ((kq[3 * i + 0] >> b) & 1u) << (3 * b + 2);
      c |= ((kq[3 * i + 1] >> b) & 1u) << (3 * b + 1);
      c |= ((kq[3 * i + 2] >> b) & 1u) << (3 * b);
    }
    code[i] = c;
  }
  free(q32);
}

typedef struct {
  const otree *t;
  int64_t *order;   /* DFS point order */
  int64_t npos;
  int64_t *remap;   /* pool id -> preorder id */
  int64_t nid;
} dfs_ctx;

static void dfs(dfs_ctx *c, int64_t k) {
  const onode *nd = &c->t->nodes[k];
  c->remap[k] = c->nid++;
  if (nd->leaf) {
    for (int64_t s = nd->head; s >= 0; s = c->t->next[s]) c->order[c->npos++] = s;
    return;
  }
  for (int o = 0; o < 8; o++)
    if (nd->child[o] >= 0) dfs(c, nd->child[o]);
}

/* Builds the tree on (q, p, alpha, beta) (alpha/beta may be NULL) and exports
 * it in DFS preorder (children in octant order).  order[N] gets the DFS point
 * order.  For each node (up to cap): info[6*k..] = {depth, leaf, n, first
 * DFS position of its points, number of non-empty children, parent preorder
 * id (-1 for the root)}; stat[12*k..] = {sum q (3), sum p (3), sum alpha (3),
 * sum beta (3)} in FP64 (12 per node) and range[6*k..] = {lo (3), hi (3)} in FP32.
 * Returns the number of nodes. */
int64_t gsref_tree(int64_t N, const double *q, const double *p,
                   const double *al, const double *be, int64_t *order,
                   int64_t cap, int64_t *info, double *stat, float *range) {
  otree t;
  tree_build(&t, N, q, p, al, be);
  dfs_ctx c;
  c.t = &t;
  c.order = order;
  c.npos = 0;
  c.remap = (int64_t *)malloc((size_t)t.count * sizeof(int64_t));
  c.nid = 0;
  dfs(&c, 0);
  /* first DFS position of each node: smallest position among its members,
   * found by a second walk that tracks the running position */
  int64_t *first = (int64_t *)malloc((size_t)t.count * sizeof(int64_t));
  int64_t *parent = (int64_t *)malloc((size_t)t.count * sizeof(int64_t));
  for (int64_t k = 0; k < t.count; k++) parent[k] = -1;
  for (int64_t k = 0; k < t.count; k++)
    if (!t.nodes[k].leaf)
      for (int o = 0; o < 8; o++)
        if (t.nodes[k].child[o] >= 0) parent[t.nodes[k].child[o]] = k;
  {
    /* explicit-stack walk in the same order as dfs() */
    int64_t *stack = (int64_t *)malloc((size_t)(t.count + 1) * sizeof(int64_t));
    int64_t sp = 0, pos = 0;
    stack[sp++] = 0;
    while (sp) {
      int64_t k = stack[--sp];
      first[k] = pos;
      if (t.nodes[k].leaf) {
        for (int64_t s = t.nodes[k].head; s >= 0; s = t.next[s]) pos++;
      } else {
        for (int o = 7; o >= 0; o--)
          if (t.nodes[k].child[o] >= 0) stack[sp++] = t.nodes[k].child[o];
      }
    }
    free(stack);
  }
  for (int64_t k = 0; k < t.count; k++) {
    int64_t id = c.remap[k];
    if (id >= cap) continue;
    const onode *nd = &t.nodes[k];
    int nc = 0;
    if (!nd->leaf)
      for (int o = 0; o < 8; o++)
        if (nd->child[o] >= 0) nc++;
    info[6 * id + 0] = nd->depth;
    info[6 * id + 1] = nd->leaf;
    info[6 * id + 2] = nd->n;
    info[6 * id + 3] = first[k];
    info[6 * id + 4] = nc;
    info[6 * id + 5] = parent[k] >= 0 ? c.remap[parent[k]] : -1;
    for (int a = 0; a < 3; a++) {
      stat[12 * id + a] = nd->sq[a];
      stat[12 * id + 3 + a] = nd->sp[a];
      stat[12 * id + 6 + a] = nd->sa[a];
      stat[12 * id + 9 + a] = nd->sb[a];
      range[6 * id + a] = nd->lo[a];
      range[6 * id + 3 + a] = nd->hi[a];
    }
  }
  int64_t count = t.count;
  free(first);
  free(parent);
  free(c.remap);
  tree_free(&t);
  return count;
}

/* Interaction list of target m under Barnes-Hut: kind[r] = 0 (point, id =
 * point index) or 1 (node summary, id = preorder node id as exported by
 * gsref_tree).  Returns the list length (entries beyond cap are dropped). */
int64_t gsref_bh_list(int64_t N, const double *q, const double *p,
                      double sigma, double thresh, int leaf, int crit,
                      int64_t m, int64_t cap, int64_t *kind, int64_t *id) {
  otree t;
  tree_build(&t, N, q, p, NULL, NULL);
  dfs_ctx c;
  int64_t *order = (int64_t *)malloc((size_t)N * sizeof(int64_t));
  c.t = &t;
  c.order = order;
  c.npos = 0;
  c.remap = (int64_t *)malloc((size_t)t.count * sizeof(int64_t));
  c.nid = 0;
  dfs(&c, 0);
  ilist L;
  L.kind = kind;
  L.id = id;
  L.len = 0;
  L.cap = cap;
  double o0[3], o1[3];
  int64_t a, b;
  bh_target(&t, sigma, rule_threshold(crit, thresh, sigma), leaf, crit, 0, m, o0, o1,
            &a, &b, &L);
  for (int64_t r = 0; r < L.len && r < cap; r++)
    if (kind[r] == 1) id[r] = c.remap[id[r]];
  free(order);
  free(c.remap);
  tree_free(&t);
  return L.len;
}

/* DFS positions (children in octant order, a leaf's points in insertion
 * order): pos[i] of every point i, first[k] of every node k (the position
 * of its first member). */
static void dfs_positions(const otree *t, int64_t N, int64_t *pos, int64_t *first) {
  int64_t *stack = (int64_t *)malloc((size_t)(t->count + 1) * sizeof(int64_t));
  int64_t sp = 0, at = 0;
  stack[sp++] = 0;
  while (sp) {
    int64_t k = stack[--sp];
    first[k] = at;
    if (t->nodes[k].leaf) {
      for (int64_t s = t->nodes[k].head; s >= 0; s = t->next[s]) pos[s] = at++;
    } else {
      for (int o = 7; o >= 0; o--)
        if (t->nodes[k].child[o] >= 0) stack[sp++] = t->nodes[k].child[o];
    }
  }
  (void)N;
  free(stack);
}

/* Per-target record of the Barnes-Hut decisions (Sec. 2.2, three cases) on
 * the tree of positions q: tally[5 m .. 5 m + 4] = {point interactions,
 * node interactions, sum over the point interactions of mix64(key), the same
 * sum over the node interactions, nodes of >= 2 points reached} for every
 * target m, sums modulo 2^64.  A source's key is (DFS first position << 32) |
 * member count, so two targets' records agree exactly when they took the
 * same sources, whatever the order.  Reached nodes are those the recursion
 * tests (summarised, opened, or taken whole), a chain of cells with a single
 * non-empty child counted once (its cells have the same members and range,
 * so the first one decides); with the points taken they are the
 * traversal's node visits. */
void gsref_bh_tally(int64_t N, const double *q, double sigma, double thresh, int leaf,
                    int crit, int64_t *tally) {
  otree t;
  tree_build(&t, N, q, q, NULL, NULL); /* decisions depend on positions only */
  int64_t *pos = (int64_t *)malloc((size_t)N * sizeof(int64_t));
  int64_t *first = (int64_t *)malloc((size_t)t.count * sizeof(int64_t));
  dfs_positions(&t, N, pos, first);
  float thr = rule_threshold(crit, thresh, sigma);
#pragma omp parallel for schedule(dynamic, 64)
  for (int64_t m = 0; m < N; m++) {
    visit_ctx v;
    memset(&v, 0, sizeof(v));
    v.t = &t;
    v.sigma = sigma;
    v.thr = thr;
    v.leaf = leaf;
    v.crit = crit;
    v.tq = t.q + 3 * m;
    v.tp = t.p + 3 * m;
    v.tq32 = t.q32 + 3 * m;
    v.m = m;
    v.tpos = pos;
    v.tfirst = first;
    visit(&v, 0, 1);
    tally[5 * m + 0] = v.n_point;
    tally[5 * m + 1] = v.n_node;
    tally[5 * m + 2] = (int64_t)v.h_point;
    tally[5 * m + 3] = (int64_t)v.h_node;
    tally[5 * m + 4] = v.n_reached;
  }
  free(pos);
  free(first);
  tree_free(&t);
}

int gsref_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}
