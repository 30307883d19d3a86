/*
 * vd_oracle.c -- plain, slow FP64 CPU oracle for clipped / restricted Voronoi
 * diagrams.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the package smoke check and
 * the bench's CPU-baseline leg load this library; the product path never does.
 * It shares no code with the CUDA path.
 *
 * What it computes (paper Sec. 2.1, Eq. 1 and Sec. 2.2):
 *   for a site v_i and a domain simplex T_a (triangle in 2D or on a surface,
 *   tetrahedron in 3D) the piece
 *       P_{a,i} = T_a  intersected with  H_ij for all j != i,
 *       H_ij = { x : |x - v_i| <= |x - v_j| }                      (Eq. 1)
 *   together with its measure (area or volume), its first moment and the flags
 *   of its faces (Sec. 2.2): a face on the bisector of v_i and v_j carries +j,
 *   a face shared with simplex T_b carries -(b+1) (the paper writes -b with
 *   1-based indices), a face on the mesh boundary carries ORC_FLAG_BOUNDARY.
 *
 * How (not the paper's search -- the textbook security-radius criterion):
 *   the piece starts as T_a and is clipped by the half-spaces H_ij taken in
 *   increasing |v_j - v_i| order; clipping stops once |v_j - v_i| exceeds twice
 *   the largest distance from v_i to a corner of the piece (no later bisector
 *   can then cut it).  In brute-force mode every j != i is used, in index
 *   order, with no pruning.
 *
 * Sign decisions.  All arithmetic runs in the frame centred on v_i.  A corner
 * of a piece is the intersection of three planes (simplex faces, triangle
 * edges and the triangle's own plane, bisectors).  Whether corner q lies in a
 * half-space n.x <= c is the sign of s = c - n.q; with q defined by planes
 * 1..3, s = det M / det N where N stacks n_1..n_3 and M stacks the rows
 * (n_r, c_r), r = 1..4.  The sign is taken from a running error bound
 * (Wilkinson's running error analysis) in float64, then in binary128 when the
 * float64 value is within its bound; a binary128 value of exactly zero is a
 * tie and counts as inside (Eq. 1 uses <=).  Decisions left uncertain are
 * counted in the stats.
 *
 * The measure and moment are integrated in float64 from corner coordinates:
 * a fan of tetrahedra from v_i (3D) or a triangle fan (2D, surface).
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#define ORC_MODE_2D 2
#define ORC_MODE_SURFACE 3
#define ORC_MODE_3D 4
#define ORC_FLAG_BOUNDARY INT32_MIN

enum { ST_FAST = 0, ST_EXACT64, ST_EXACT128, ST_TIE, ST_UNCERTAIN, ST_CLIPS, ST_PIECES, ST_ERROR, ST_N };

/* ------------------------------------------------------------------------- */
/* error-tracked arithmetic: value + bound on its absolute error             */
/* ------------------------------------------------------------------------- */
typedef __float128 q128;
typedef struct { double v, e; } ed;
typedef struct { q128 v, e; } eq;

static inline double dabs(double x) { return x < 0 ? -x : x; }
static inline q128 qabs(q128 x) { return x < 0 ? -x : x; }
#define U64 (1.1102230246251565e-16)              /* 2^-53 */
#define U128 ((q128)9.62964972193617926527988971292463659e-35Q) /* 2^-113 */

#define DEF_EARITH(T, S, R, U, ABS)                                                    \
  static inline T S##_c(double x) { T r; r.v = (R)x; r.e = 0; return r; }              \
  static inline T S##_add(T a, T b) {                                                  \
    T r; r.v = a.v + b.v; r.e = a.e + b.e + U * ABS(r.v); return r; }                 \
  static inline T S##_sub(T a, T b) {                                                  \
    T r; r.v = a.v - b.v; r.e = a.e + b.e + U * ABS(r.v); return r; }                 \
  static inline T S##_mul(T a, T b) {                                                  \
    T r; r.v = a.v * b.v;                                                              \
    r.e = ABS(a.v) * b.e + ABS(b.v) * a.e + a.e * b.e + U * ABS(r.v); return r; }      \
  static inline T S##_scale(T a, double k) { /* k = +-1 or +-0.5: exact */             \
    T r; r.v = a.v * (R)k; r.e = a.e * (R)dabs(k); return r; }                         \
  static inline T S##_dot3(const T* a, const T* b) {                                   \
    return S##_add(S##_add(S##_mul(a[0], b[0]), S##_mul(a[1], b[1])), S##_mul(a[2], b[2])); } \
  static inline void S##_cross(const T* a, const T* b, T* r) {                         \
    r[0] = S##_sub(S##_mul(a[1], b[2]), S##_mul(a[2], b[1]));                          \
    r[1] = S##_sub(S##_mul(a[2], b[0]), S##_mul(a[0], b[2]));                          \
    r[2] = S##_sub(S##_mul(a[0], b[1]), S##_mul(a[1], b[0])); }                        \
  static inline T S##_det3(const T* a, const T* b, const T* c) {                       \
    T bc[3]; S##_cross(b, c, bc); return S##_dot3(a, bc); }

DEF_EARITH(ed, e64, double, U64, dabs)
DEF_EARITH(eq, e128, q128, U128, qabs)

/* a sign is certified when |value| exceeds its bound (inflated for the rounding
 * of the bound computation itself) */
static inline int e64_sign(ed a) {
  double b = a.e * (1.0 + 1e-12) + 1e-300;
  return a.v > b ? 1 : (a.v < -b ? -1 : 0);
}
static inline int e128_sign(eq a) {
  q128 b = a.e * (q128)(1.0 + 1e-12) + (q128)1e-300;
  return a.v > b ? 1 : (a.v < -b ? -1 : 0);
}

/* ------------------------------------------------------------------------- */
/* input context                                                              */
/* ------------------------------------------------------------------------- */
typedef struct {
  int64_t n; double* p; int64_t* idx; int64_t nnodes;
} kdtree;

typedef struct {
  int mode;          /* ORC_MODE_* */
  int k;             /* vertices per simplex: 3 or 4 */
  int brute;         /* 1: clip by every other site, in index order */
  int nthreads;
  int64_t n, nv, m;
  double* sites;     /* n*3 */
  double* verts;     /* nv*3 */
  int32_t* simp;     /* m*k */
  int32_t* adj;      /* m*k: neighbour across the face/edge opposite local vertex f, or -1 */
  kdtree kd_sites;
  kdtree kd_cent;    /* simplex centroids */
  double* cent;      /* m*3 */
  double* w;         /* n power weights (power diagram), or NULL (Voronoi diagram) */
  double wmax;       /* largest weight */
} orc_ctx;

/* ------------------------------------------------------------------------- */
/* kd-tree (implicit, balanced; node = median of its index range)             */
/* ------------------------------------------------------------------------- */
static void kd_select(const double* p, int64_t* idx, int64_t lo, int64_t hi, int64_t kth, int ax) {
  /* quickselect so that idx[kth] holds the kth smallest p[.,ax] in [lo,hi) */
  while (hi - lo > 1) {
    double pv = p[3 * idx[(lo + hi) / 2] + ax];
    int64_t i = lo, j = hi - 1;
    while (i <= j) {
      while (p[3 * idx[i] + ax] < pv) ++i;
      while (p[3 * idx[j] + ax] > pv) --j;
      if (i <= j) { int64_t t = idx[i]; idx[i] = idx[j]; idx[j] = t; ++i; --j; }
    }
    if (kth <= j) hi = j + 1;
    else if (kth >= i) lo = i;
    else return;
  }
}

static void kd_build_rec(kdtree* t, int64_t lo, int64_t hi, int depth) {
  if (hi - lo <= 1) return;
  int64_t mid = (lo + hi) / 2;
  kd_select(t->p, t->idx, lo, hi, mid, depth % 3);
  kd_build_rec(t, lo, mid, depth + 1);
  kd_build_rec(t, mid + 1, hi, depth + 1);
}

static void kd_build(kdtree* t, const double* pts, int64_t n) {
  t->n = n;
  t->p = (double*)malloc(sizeof(double) * 3 * (n ? n : 1));
  memcpy(t->p, pts, sizeof(double) * 3 * n);
  t->idx = (int64_t*)malloc(sizeof(int64_t) * (n ? n : 1));
  for (int64_t i = 0; i < n; ++i) t->idx[i] = i;
  kd_build_rec(t, 0, n, 0);
}

static void kd_free(kdtree* t) { free(t->p); free(t->idx); }

static inline double d2(const double* a, const double* b) {
  double x = a[0] - b[0], y = a[1] - b[1], z = a[2] - b[2];
  return x * x + y * y + z * z;
}

/* (distance^2, index) ordering, smaller index first on ties */
static inline int kless(double da, int64_t ia, double db, int64_t ib) {
  return da < db || (da == db && ia < ib);
}

typedef struct { int64_t k, cnt; double* d; int64_t* id; } kheap; /* max-heap */

static void kh_push(kheap* h, double d, int64_t id) {
  if (h->cnt < h->k) {
    int64_t c = h->cnt++;
    h->d[c] = d; h->id[c] = id;
    while (c > 0) {
      int64_t par = (c - 1) / 2;
      if (kless(h->d[par], h->id[par], h->d[c], h->id[c])) {
        double td = h->d[par]; h->d[par] = h->d[c]; h->d[c] = td;
        int64_t ti = h->id[par]; h->id[par] = h->id[c]; h->id[c] = ti;
        c = par;
      } else break;
    }
  } else if (kless(d, id, h->d[0], h->id[0])) {
    h->d[0] = d; h->id[0] = id;
    int64_t c = 0;
    for (;;) {
      int64_t l = 2 * c + 1, r = l + 1, big = c;
      if (l < h->cnt && kless(h->d[big], h->id[big], h->d[l], h->id[l])) big = l;
      if (r < h->cnt && kless(h->d[big], h->id[big], h->d[r], h->id[r])) big = r;
      if (big == c) break;
      double td = h->d[big]; h->d[big] = h->d[c]; h->d[c] = td;
      int64_t ti = h->id[big]; h->id[big] = h->id[c]; h->id[c] = ti;
      c = big;
    }
  }
}

static void kd_knn_rec(const kdtree* t, const double* q, int64_t lo, int64_t hi, int depth,
                       int64_t skip, kheap* h) {
  while (hi > lo) {
    int64_t mid = (lo + hi) / 2;
    int64_t id = t->idx[mid];
    int ax = depth % 3;
    if (id != skip) kh_push(h, d2(q, t->p + 3 * id), id);
    double diff = q[ax] - t->p[3 * id + ax];
    int64_t nlo, nhi, flo, fhi;
    if (diff < 0) { nlo = lo; nhi = mid; flo = mid + 1; fhi = hi; }
    else { nlo = mid + 1; nhi = hi; flo = lo; fhi = mid; }
    kd_knn_rec(t, q, nlo, nhi, depth + 1, skip, h);
    if (h->cnt == h->k && diff * diff > h->d[0]) return;
    lo = flo; hi = fhi; ++depth;
  }
}

static int cmp_pair(const void* a, const void* b) {
  const double* x = (const double*)a; const double* y = (const double*)b;
  if (x[0] < y[0]) return -1;
  if (x[0] > y[0]) return 1;
  int64_t ix, iy; memcpy(&ix, x + 1, 8); memcpy(&iy, y + 1, 8);
  return ix < iy ? -1 : (ix > iy ? 1 : 0);
}

/* k nearest (excluding index skip), sorted by (distance, index); returns count */
static int64_t kd_knn(const kdtree* t, const double* q, int64_t k, int64_t skip, int64_t* out_id,
                      double* out_d) {
  kheap h; h.k = k; h.cnt = 0;
  h.d = (double*)malloc(sizeof(double) * k); h.id = (int64_t*)malloc(sizeof(int64_t) * k);
  kd_knn_rec(t, q, 0, t->n, 0, skip, &h);
  double* tmp = (double*)malloc(sizeof(double) * 2 * (h.cnt ? h.cnt : 1));
  for (int64_t j = 0; j < h.cnt; ++j) { tmp[2 * j] = h.d[j]; memcpy(tmp + 2 * j + 1, &h.id[j], 8); }
  qsort(tmp, h.cnt, 2 * sizeof(double), cmp_pair);
  for (int64_t j = 0; j < h.cnt; ++j) { out_d[j] = tmp[2 * j]; memcpy(&out_id[j], tmp + 2 * j + 1, 8); }
  int64_t c = h.cnt;
  free(tmp); free(h.d); free(h.id);
  return c;
}

typedef struct { int64_t n, cap; int64_t* v; } ivec;
static void iv_push(ivec* a, int64_t x) {
  if (a->n == a->cap) { a->cap = a->cap ? 2 * a->cap : 64; a->v = (int64_t*)realloc(a->v, 8 * a->cap); }
  a->v[a->n++] = x;
}

static void kd_range_rec(const kdtree* t, const double* q, double r2, int64_t lo, int64_t hi, int depth,
                         ivec* out) {
  while (hi > lo) {
    int64_t mid = (lo + hi) / 2;
    int64_t id = t->idx[mid];
    int ax = depth % 3;
    if (d2(q, t->p + 3 * id) <= r2) iv_push(out, id);
    double diff = q[ax] - t->p[3 * id + ax];
    if (diff <= 0 || diff * diff <= r2) kd_range_rec(t, q, r2, lo, mid, depth + 1, out);
    if (diff >= 0 || diff * diff <= r2) { lo = mid + 1; ++depth; continue; }
    return;
  }
}

/* ------------------------------------------------------------------------- */
/* planes, defined exactly from input coordinates                             */
/* ------------------------------------------------------------------------- */
enum { PL_BIS = 1, PL_FACE, PL_EDGE };

typedef struct {
  int kind;
  int32_t a, b, c;   /* PL_BIS: a = site j.  PL_FACE: plane through verts a,b,c.
                        PL_EDGE: plane through edge (a,b) of triangle (a,b,c), normal
                        to the triangle's plane */
  double sgn;        /* +-1: orientation so that the piece lies on n.x <= c */
  int32_t flag;      /* face flag written to the output */
} oplane;

#define DEF_PLANE(T, S)                                                               \
  static void S##_plane(const orc_ctx* C, int64_t site, const oplane* p, T* n, T* c) { \
    const double* vi = C->sites + 3 * site;                                          \
    if (p->kind == PL_BIS) {                                                          \
      const double* vj = C->sites + 3 * (int64_t)p->a;                               \
      for (int d = 0; d < 3; ++d) n[d] = S##_sub(S##_c(vj[d]), S##_c(vi[d]));         \
      if (C->w)  /* power bisector: |x-v_i|^2 - w_i <= |x-v_j|^2 - w_j */              \
        *c = S##_scale(S##_sub(S##_dot3(n, n), S##_sub(S##_c(C->w[p->a]), S##_c(C->w[site]))), 0.5); \
      else                                                                            \
        *c = S##_scale(S##_dot3(n, n), 0.5);                                          \
      return;                                                                         \
    }                                                                                 \
    const double* A = C->verts + 3 * (int64_t)p->a;                                  \
    const double* B = C->verts + 3 * (int64_t)p->b;                                  \
    const double* Cc = C->verts + 3 * (int64_t)p->c;                                 \
    T e1[3], e2[3], a[3], cr[3];                                                      \
    for (int d = 0; d < 3; ++d) {                                                     \
      e1[d] = S##_sub(S##_c(B[d]), S##_c(A[d]));                                      \
      e2[d] = S##_sub(S##_c(Cc[d]), S##_c(A[d]));                                     \
      a[d] = S##_sub(S##_c(A[d]), S##_c(vi[d]));                                      \
    }                                                                                 \
    S##_cross(e1, e2, cr);                                                            \
    if (p->kind == PL_FACE) {                                                         \
      for (int d = 0; d < 3; ++d) n[d] = S##_scale(cr[d], p->sgn);                    \
    } else {                                                                          \
      T ed_[3]; S##_cross(e1, cr, ed_);                                               \
      for (int d = 0; d < 3; ++d) n[d] = S##_scale(ed_[d], p->sgn);                   \
    }                                                                                 \
    *c = S##_dot3(n, a);                                                              \
  }

DEF_PLANE(ed, e64)
DEF_PLANE(eq, e128)

/* ------------------------------------------------------------------------- */
/* corners and the exact side test                                            */
/* ------------------------------------------------------------------------- */
typedef struct {
  double q[3];     /* coordinates in the frame of v_i */
  double qe;       /* bound on the absolute error of each coordinate (INFINITY: unknown) */
  int pl[3];       /* the three defining planes (indices into the piece's plane table) */
} overt;

enum { CL_OUT = -1, CL_ON = 0, CL_IN = 1 };

typedef struct {
  const orc_ctx* C;
  int64_t site;
  int np, npcap;
  oplane* pl;
  int64_t* st;     /* stats */
} pctx;

static int add_plane(pctx* P, oplane p) {
  if (P->np == P->npcap) {
    P->npcap = P->npcap ? 2 * P->npcap : 64;
    P->pl = (oplane*)realloc(P->pl, sizeof(oplane) * P->npcap);
  }
  P->pl[P->np] = p;
  return P->np++;
}

/* sign of c4 - n4.q for the corner q defined by planes pl[0..2]: +1 in, 0 tie, -1 out */
static int side_exact(pctx* P, const int* pl, int p4) {
  const orc_ctx* C = P->C;
  {
    ed n[4][3], c[4];
    for (int r = 0; r < 3; ++r) e64_plane(C, P->site, &P->pl[pl[r]], n[r], &c[r]);
    e64_plane(C, P->site, &P->pl[p4], n[3], &c[3]);
    ed dN = e64_det3(n[0], n[1], n[2]);
    /* det M = -c1 det(n2,n3,n4) + c2 det(n1,n3,n4) - c3 det(n1,n2,n4) + c4 det(n1,n2,n3) */
    ed dM = e64_add(e64_add(e64_scale(e64_mul(c[0], e64_det3(n[1], n[2], n[3])), -1.0),
                            e64_mul(c[1], e64_det3(n[0], n[2], n[3]))),
                    e64_add(e64_scale(e64_mul(c[2], e64_det3(n[0], n[1], n[3])), -1.0),
                            e64_mul(c[3], dN)));
    int sN = e64_sign(dN), sM = e64_sign(dM);
    if (sN != 0 && sM != 0) { P->st[ST_EXACT64]++; return sN * sM; }
  }
  {
    eq n[4][3], c[4];
    for (int r = 0; r < 3; ++r) e128_plane(C, P->site, &P->pl[pl[r]], n[r], &c[r]);
    e128_plane(C, P->site, &P->pl[p4], n[3], &c[3]);
    eq dN = e128_det3(n[0], n[1], n[2]);
    eq dM = e128_add(e128_add(e128_scale(e128_mul(c[0], e128_det3(n[1], n[2], n[3])), -1.0),
                              e128_mul(c[1], e128_det3(n[0], n[2], n[3]))),
                     e128_add(e128_scale(e128_mul(c[2], e128_det3(n[0], n[1], n[3])), -1.0),
                              e128_mul(c[3], dN)));
    int sN = e128_sign(dN), sM = e128_sign(dM);
    if (sN != 0 && sM != 0) { P->st[ST_EXACT128]++; return sN * sM; }
    if (sN != 0 && dM.v == 0) { P->st[ST_TIE]++; return CL_ON; }
    P->st[ST_UNCERTAIN]++;
    if (dM.v == 0 || dN.v == 0) return CL_ON;
    return ((dM.v > 0) == (dN.v > 0)) ? CL_IN : CL_OUT;
  }
}

static int classify(pctx* P, const overt* v, int p4) {
  ed n[3], c;
  e64_plane(P->C, P->site, &P->pl[p4], n, &c);
  if (v->qe < INFINITY) {
    ed s = c;
    for (int d = 0; d < 3; ++d) {
      ed q; q.v = v->q[d]; q.e = v->qe;
      s = e64_sub(s, e64_mul(n[d], q));
    }
    int sg = e64_sign(s);
    if (sg != 0) { P->st[ST_FAST]++; return sg; }
  }
  return side_exact(P, v->pl, p4);
}

/* corner at the intersection of three planes (Cramer's rule, with error bound) */
static overt make_corner(pctx* P, int p0, int p1, int p2) {
  overt v; v.pl[0] = p0; v.pl[1] = p1; v.pl[2] = p2;
  ed n[3][3], c[3];
  for (int r = 0; r < 3; ++r) e64_plane(P->C, P->site, &P->pl[v.pl[r]], n[r], &c[r]);
  ed D = e64_det3(n[0], n[1], n[2]);
  ed x12[3], x20[3], x01[3];
  e64_cross(n[1], n[2], x12); e64_cross(n[2], n[0], x20); e64_cross(n[0], n[1], x01);
  double emax = 0;
  double den = dabs(D.v) - D.e;
  for (int d = 0; d < 3; ++d) {
    ed A = e64_add(e64_add(e64_mul(c[0], x12[d]), e64_mul(c[1], x20[d])), e64_mul(c[2], x01[d]));
    v.q[d] = A.v / D.v;
    double e = den > 0 ? (A.e + dabs(v.q[d]) * D.e) / den + 2 * U64 * dabs(v.q[d]) : INFINITY;
    if (e > emax) emax = e;
  }
  v.qe = emax * (1 + 1e-9);
  return v;
}

/* ------------------------------------------------------------------------- */
/* convex polyhedron as a face list (3D pieces)                               */
/* ------------------------------------------------------------------------- */
#define PV_MAX 2048
#define PF_MAX 256
#define PFV_MAX 96

typedef struct {
  int nv; overt v[PV_MAX];
  int nf; int fpl[PF_MAX]; int fn[PF_MAX]; int fv[PF_MAX][PFV_MAX];
  /* scratch */
  int cls[PV_MAX]; int remap[PV_MAX]; int succ[PV_MAX];
  int nf2; int fpl2[PF_MAX]; int fn2[PF_MAX]; int fv2[PF_MAX][PFV_MAX];
  int ekn; int eka[PV_MAX], ekb[PV_MAX], ekv[PV_MAX];
} opoly;

static int poly_other_face(const opoly* G, int f, int a, int b) {
  for (int g = 0; g < G->nf; ++g) {
    if (g == f) continue;
    int n = G->fn[g];
    for (int k = 0; k < n; ++k) {
      int u = G->fv[g][k], w = G->fv[g][(k + 1) % n];
      if ((u == a && w == b) || (u == b && w == a)) return g;
    }
  }
  return -1;
}

/* corner on the edge a-b (a kept, b cut away) of face f, shared with the other face */
static int poly_edge_vertex(pctx* P, opoly* G, int f, int a, int b, int pidx, int* err) {
  int lo = a < b ? a : b, hi = a < b ? b : a;
  for (int k = 0; k < G->ekn; ++k)
    if (G->eka[k] == lo && G->ekb[k] == hi) return G->ekv[k];
  int g = poly_other_face(G, f, a, b);
  if (g < 0 || G->nv >= PV_MAX) { *err = 1; return a; }
  int id = G->nv++;
  G->v[id] = make_corner(P, G->fpl[f], G->fpl[g], pidx);
  G->cls[id] = CL_IN;
  G->eka[G->ekn] = lo; G->ekb[G->ekn] = hi; G->ekv[G->ekn] = id; G->ekn++;
  return id;
}

/* P <- P intersected with {plane pidx}.  returns 0 ok, 1 empty, -1 inconsistent */
static int poly_clip(pctx* P, opoly* G, int pidx) {
  int nin = 0, nout = 0;
  for (int v = 0; v < G->nv; ++v) {
    G->cls[v] = classify(P, &G->v[v], pidx);
    if (G->cls[v] == CL_IN) ++nin;
    if (G->cls[v] == CL_OUT) ++nout;
  }
  if (nout == 0) return 0;
  P->st[ST_CLIPS]++;
  if (nin == 0) { G->nv = 0; G->nf = 0; return 1; }
  int nv0 = G->nv;
  for (int v = 0; v < PV_MAX; ++v) G->succ[v] = -1;
  G->ekn = 0; G->nf2 = 0;
  int err = 0, nseg = 0, first_y = -1;
  for (int f = 0; f < G->nf; ++f) {
    int n = G->fn[f], m = 0, nx = 0, X = -1, Y = -1;
    int* out = G->fv2[G->nf2];
    for (int k = 0; k < n; ++k) {
      int u = G->fv[f][k], w = G->fv[f][(k + 1) % n];
      int cu = G->cls[u], cw = G->cls[w];
      if (cu != CL_OUT) {
        if (m < PFV_MAX) out[m++] = u; else err = 1;
        if (cw == CL_OUT) {
          X = (cu == CL_ON) ? u : poly_edge_vertex(P, G, f, u, w, pidx, &err);
          if (X != u) { if (m < PFV_MAX) out[m++] = X; else err = 1; }
          ++nx;
        }
      } else if (cw != CL_OUT) {
        Y = (cw == CL_ON) ? w : poly_edge_vertex(P, G, f, w, u, pidx, &err);
        if (Y != w) { if (m < PFV_MAX) out[m++] = Y; else err = 1; }
      }
    }
    if (nx > 1) err = 1;
    if (X >= 0 && Y >= 0 && X != Y) {
      if (G->succ[Y] != -1) err = 1;
      G->succ[Y] = X; ++nseg; first_y = Y;
    }
    if (m >= 3) { G->fpl2[G->nf2] = G->fpl[f]; G->fn2[G->nf2] = m; G->nf2++; }
  }
  (void)nv0;
  if (err) { P->st[ST_ERROR]++; return -1; }
  /* the new face on plane pidx: follow succ from one entry point */
  if (nseg >= 3) {
    int* out = G->fv2[G->nf2];
    int m = 0, v = first_y;
    do {
      if (m >= PFV_MAX) { P->st[ST_ERROR]++; return -1; }
      out[m++] = v;
      v = G->succ[v];
    } while (v >= 0 && v != first_y && m <= nseg);
    if (v != first_y || m != nseg) { P->st[ST_ERROR]++; return -1; }
    G->fpl2[G->nf2] = pidx; G->fn2[G->nf2] = m; G->nf2++;
  }
  /* compact: drop cut-away corners */
  int nk = 0;
  for (int v = 0; v < G->nv; ++v) {
    if (G->cls[v] != CL_OUT) { G->remap[v] = nk; G->v[nk++] = G->v[v]; }
    else G->remap[v] = -1;
  }
  G->nv = nk;
  G->nf = G->nf2;
  for (int f = 0; f < G->nf; ++f) {
    G->fpl[f] = G->fpl2[f]; G->fn[f] = G->fn2[f];
    for (int k = 0; k < G->fn[f]; ++k) G->fv[f][k] = G->remap[G->fv2[f][k]];
  }
  if (G->nf < 4) { G->nv = 0; G->nf = 0; return 1; }
  return 0;
}

/* ------------------------------------------------------------------------- */
/* convex polygon in the plane of a triangle (2D and surface pieces)          */
/* ------------------------------------------------------------------------- */
#define PG_MAX 256
typedef struct {
  int n; overt v[PG_MAX]; int e[PG_MAX];  /* e[k]: plane of the edge v[k] -> v[k+1] */
  int sp;                                   /* the triangle's own plane */
  int n2; overt v2[PG_MAX]; int e2[PG_MAX]; int cls[PG_MAX];
} opgon;

static int pgon_clip(pctx* P, opgon* G, int pidx) {
  int nin = 0, nout = 0;
  for (int k = 0; k < G->n; ++k) {
    G->cls[k] = classify(P, &G->v[k], pidx);
    if (G->cls[k] == CL_IN) ++nin;
    if (G->cls[k] == CL_OUT) ++nout;
  }
  if (nout == 0) return 0;
  P->st[ST_CLIPS]++;
  if (nin == 0) { G->n = 0; return 1; }
  int m = 0, nx = 0;
  for (int k = 0; k < G->n; ++k) {
    int k1 = (k + 1) % G->n;
    int cu = G->cls[k], cw = G->cls[k1];
    if (m + 2 >= PG_MAX) { P->st[ST_ERROR]++; return -1; }
    if (cu != CL_OUT) {
      if (cw == CL_OUT) {
        ++nx;
        if (cu == CL_ON) { G->v2[m] = G->v[k]; G->e2[m++] = pidx; }
        else {
          G->v2[m] = G->v[k]; G->e2[m++] = G->e[k];
          G->v2[m] = make_corner(P, G->sp, G->e[k], pidx); G->e2[m++] = pidx;
        }
      } else { G->v2[m] = G->v[k]; G->e2[m++] = G->e[k]; }
    } else if (cw == CL_IN) {
      G->v2[m] = make_corner(P, G->sp, pidx, G->e[k]); G->e2[m++] = G->e[k];
    }
  }
  if (nx != 1) { P->st[ST_ERROR]++; return -1; }
  /* refresh the defining planes of every corner from the ring */
  for (int k = 0; k < m; ++k) {
    int km = (k + m - 1) % m;
    G->v2[k].pl[0] = G->sp; G->v2[k].pl[1] = G->e2[km]; G->v2[k].pl[2] = G->e2[k];
  }
  G->n = m;
  memcpy(G->v, G->v2, sizeof(overt) * m);
  memcpy(G->e, G->e2, sizeof(int) * m);
  if (m < 3) { G->n = 0; return 1; }
  return 0;
}

/* ------------------------------------------------------------------------- */
/* one piece P_{a,i}                                                          */
/* ------------------------------------------------------------------------- */
typedef struct {
  opoly* G3; opgon* G2;
  pctx P;
  int64_t* knn_id; double* knn_d; int64_t knn_cap;
} workspace;

typedef struct {
  double meas, m1[3];
  int nf; int32_t flags[PF_MAX]; double fmeas[PF_MAX];
  int status;
} piece_out;

static workspace* ws_new(const orc_ctx* C, int64_t* st) {
  workspace* w = (workspace*)calloc(1, sizeof(workspace));
  if (C->mode == ORC_MODE_3D) w->G3 = (opoly*)malloc(sizeof(opoly));
  else w->G2 = (opgon*)malloc(sizeof(opgon));
  w->P.C = C; w->P.st = st;
  return w;
}

static void ws_free(workspace* w) {
  free(w->G3); free(w->G2); free(w->P.pl); free(w->knn_id); free(w->knn_d); free(w);
}

static int32_t face_flag(const orc_ctx* C, int64_t a, int f) {
  int32_t b = C->adj[a * C->k + f];
  return b < 0 ? ORC_FLAG_BOUNDARY : -(b + 1);
}

static void init_piece(workspace* w, int64_t a, int64_t i) {
  const orc_ctx* C = w->P.C;
  pctx* P = &w->P;
  P->site = i; P->np = 0;
  const int32_t* s = C->simp + a * C->k;
  const double* vi = C->sites + 3 * i;
  if (C->mode == ORC_MODE_3D) {
    opoly* G = w->G3;
    G->nv = 4; G->nf = 4;
    for (int f = 0; f < 4; ++f) {
      int t[3], m = 0;
      for (int k = 0; k < 4; ++k) if (k != f) t[m++] = k;
      const double *A = C->verts + 3 * (int64_t)s[t[0]], *B = C->verts + 3 * (int64_t)s[t[1]],
                   *Cc = C->verts + 3 * (int64_t)s[t[2]], *D = C->verts + 3 * (int64_t)s[f];
      double e1[3], e2[3], cr[3];
      for (int d = 0; d < 3; ++d) { e1[d] = B[d] - A[d]; e2[d] = Cc[d] - A[d]; }
      cr[0] = e1[1] * e2[2] - e1[2] * e2[1];
      cr[1] = e1[2] * e2[0] - e1[0] * e2[2];
      cr[2] = e1[0] * e2[1] - e1[1] * e2[0];
      double side = cr[0] * (D[0] - A[0]) + cr[1] * (D[1] - A[1]) + cr[2] * (D[2] - A[2]);
      oplane p; p.kind = PL_FACE; p.a = s[t[0]]; p.b = s[t[1]]; p.c = s[t[2]];
      p.sgn = side < 0 ? 1.0 : -1.0; p.flag = face_flag(C, a, f);
      add_plane(P, p);  /* plane index f */
      G->fpl[f] = f; G->fn[f] = 3;
      if (p.sgn > 0) { G->fv[f][0] = t[0]; G->fv[f][1] = t[1]; G->fv[f][2] = t[2]; }
      else { G->fv[f][0] = t[0]; G->fv[f][1] = t[2]; G->fv[f][2] = t[1]; }
    }
    for (int k = 0; k < 4; ++k) {
      overt* v = &G->v[k];
      const double* V = C->verts + 3 * (int64_t)s[k];
      double mx = 0;
      for (int d = 0; d < 3; ++d) { v->q[d] = V[d] - vi[d]; if (dabs(v->q[d]) > mx) mx = dabs(v->q[d]); }
      v->qe = 2 * U64 * mx;
      int m = 0;
      for (int f = 0; f < 4; ++f) if (f != k) v->pl[m++] = f;
    }
  } else {
    opgon* G = w->G2;
    /* ring A->B->C, counter-clockwise about n_S = (B-A)x(C-A) */
    oplane sp; sp.kind = PL_FACE; sp.a = s[0]; sp.b = s[1]; sp.c = s[2]; sp.sgn = 1.0;
    sp.flag = ORC_FLAG_BOUNDARY;
    G->sp = add_plane(P, sp);  /* plane 0 */
    G->n = 3;
    for (int k = 0; k < 3; ++k) {
      /* edge k: s[k] -> s[k+1], opposite local vertex k+2 */
      oplane e; e.kind = PL_EDGE; e.a = s[k]; e.b = s[(k + 1) % 3]; e.c = s[(k + 2) % 3];
      e.sgn = 1.0; e.flag = face_flag(C, a, (k + 2) % 3);
      G->e[k] = add_plane(P, e);
    }
    for (int k = 0; k < 3; ++k) {
      overt* v = &G->v[k];
      const double* V = C->verts + 3 * (int64_t)s[k];
      double mx = 0;
      for (int d = 0; d < 3; ++d) { v->q[d] = V[d] - vi[d]; if (dabs(v->q[d]) > mx) mx = dabs(v->q[d]); }
      v->qe = 2 * U64 * mx;
      v->pl[0] = G->sp; v->pl[1] = G->e[(k + 2) % 3]; v->pl[2] = G->e[k];
    }
  }
}

static int piece_empty(const workspace* w) {
  return w->P.C->mode == ORC_MODE_3D ? w->G3->nv == 0 : w->G2->n == 0;
}

/* largest distance from v_i to a corner of the piece (an upper bound) */
static double piece_radius(const workspace* w) {
  double r = 0;
  if (w->P.C->mode == ORC_MODE_3D) {
    for (int v = 0; v < w->G3->nv; ++v) {
      const overt* c = &w->G3->v[v];
      double d = sqrt(c->q[0] * c->q[0] + c->q[1] * c->q[1] + c->q[2] * c->q[2]) + 2 * c->qe;
      if (d > r) r = d;
    }
  } else {
    for (int v = 0; v < w->G2->n; ++v) {
      const overt* c = &w->G2->v[v];
      double d = sqrt(c->q[0] * c->q[0] + c->q[1] * c->q[1] + c->q[2] * c->q[2]) + 2 * c->qe;
      if (d > r) r = d;
    }
  }
  return r;
}

static int clip_by_site(workspace* w, int64_t j) {
  oplane p; p.kind = PL_BIS; p.a = (int32_t)j; p.b = p.c = 0; p.sgn = 1.0; p.flag = (int32_t)j;
  int idx = add_plane(&w->P, p);
  return w->P.C->mode == ORC_MODE_3D ? poly_clip(&w->P, w->G3, idx) : pgon_clip(&w->P, w->G2, idx);
}

/* exact: no sign decision of this piece was a tie or left uncertain, so the
   clipped piece is a simple polytope (polygon) whose every face (edge) has
   positive measure, as has the piece itself -- whatever float64 makes of a
   sliver far below its resolution.  Otherwise the computed measures decide. */
static void integrate(workspace* w, int64_t a, piece_out* o, int exact) {
  const orc_ctx* C = w->P.C;
  o->meas = 0; o->m1[0] = o->m1[1] = o->m1[2] = 0; o->nf = 0;
  if (C->mode == ORC_MODE_3D) {
    opoly* G = w->G3;
    for (int f = 0; f < G->nf; ++f) {
      int n = G->fn[f];
      const double* q0 = G->v[G->fv[f][0]].q;
      double ax = 0, ay = 0, az = 0;
      for (int t = 1; t + 1 < n; ++t) {
        const double* q1 = G->v[G->fv[f][t]].q;
        const double* q2 = G->v[G->fv[f][t + 1]].q;
        double det = q0[0] * (q1[1] * q2[2] - q1[2] * q2[1]) - q0[1] * (q1[0] * q2[2] - q1[2] * q2[0]) +
                     q0[2] * (q1[0] * q2[1] - q1[1] * q2[0]);
        o->meas += det / 6.0;
        for (int d = 0; d < 3; ++d) o->m1[d] += det / 24.0 * (q0[d] + q1[d] + q2[d]);
        double u[3] = {q1[0] - q0[0], q1[1] - q0[1], q1[2] - q0[2]};
        double v[3] = {q2[0] - q0[0], q2[1] - q0[1], q2[2] - q0[2]};
        ax += u[1] * v[2] - u[2] * v[1];
        ay += u[2] * v[0] - u[0] * v[2];
        az += u[0] * v[1] - u[1] * v[0];
      }
      double area = 0.5 * sqrt(ax * ax + ay * ay + az * az);
      if (area > 0 || exact) {
        o->flags[o->nf] = w->P.pl[G->fpl[f]].flag;
        o->fmeas[o->nf] = area;
        o->nf++;
      }
    }
  } else {
    opgon* G = w->G2;
    const int32_t* s = C->simp + a * C->k;
    const double *A = C->verts + 3 * (int64_t)s[0], *B = C->verts + 3 * (int64_t)s[1],
                 *Cc = C->verts + 3 * (int64_t)s[2];
    double e1[3], e2[3], ns[3];
    for (int d = 0; d < 3; ++d) { e1[d] = B[d] - A[d]; e2[d] = Cc[d] - A[d]; }
    ns[0] = e1[1] * e2[2] - e1[2] * e2[1];
    ns[1] = e1[2] * e2[0] - e1[0] * e2[2];
    ns[2] = e1[0] * e2[1] - e1[1] * e2[0];
    double nl = sqrt(ns[0] * ns[0] + ns[1] * ns[1] + ns[2] * ns[2]);
    for (int d = 0; d < 3; ++d) ns[d] /= nl;
    const double* q0 = G->v[0].q;
    for (int t = 1; t + 1 < G->n; ++t) {
      const double* q1 = G->v[t].q;
      const double* q2 = G->v[t + 1].q;
      double u[3] = {q1[0] - q0[0], q1[1] - q0[1], q1[2] - q0[2]};
      double v[3] = {q2[0] - q0[0], q2[1] - q0[1], q2[2] - q0[2]};
      double cr[3] = {u[1] * v[2] - u[2] * v[1], u[2] * v[0] - u[0] * v[2], u[0] * v[1] - u[1] * v[0]};
      double ar = 0.5 * (cr[0] * ns[0] + cr[1] * ns[1] + cr[2] * ns[2]);
      o->meas += ar;
      for (int d = 0; d < 3; ++d) o->m1[d] += ar * (q0[d] + q1[d] + q2[d]) / 3.0;
    }
    for (int k = 0; k < G->n; ++k) {
      const double* p = G->v[k].q;
      const double* r = G->v[(k + 1) % G->n].q;
      double len = sqrt((r[0] - p[0]) * (r[0] - p[0]) + (r[1] - p[1]) * (r[1] - p[1]) +
                        (r[2] - p[2]) * (r[2] - p[2]));
      if (len > 0 || exact) {
        o->flags[o->nf] = w->P.pl[G->e[k]].flag;
        o->fmeas[o->nf] = len;
        o->nf++;
      }
    }
  }
  if (exact && !(o->meas > 0)) {
    /* positive in exact arithmetic, below float64 resolution: the smallest
       normal double as its measure, no moment */
    o->meas = 2.2250738585072014e-308;
    o->m1[0] = o->m1[1] = o->m1[2] = 0;
  }
}

static void compute_piece(workspace* w, int64_t a, int64_t i, piece_out* o) {
  const orc_ctx* C = w->P.C;
  init_piece(w, a, i);
  w->P.st[ST_PIECES]++;
  const int64_t undecided0 = w->P.st[ST_TIE] + w->P.st[ST_UNCERTAIN];
  int rc = 0;
  if (C->brute) {
    for (int64_t j = 0; j < C->n && rc == 0; ++j) {
      if (j == i) continue;
      rc = clip_by_site(w, j);
    }
  } else {
    int64_t k = 32, done_upto = 0;
    const double* vi = C->sites + 3 * i;
    int finished = 0;
    while (!finished) {
      if (k > C->n - 1) k = C->n - 1;
      if (k <= 0) break;
      if (w->knn_cap < k) {
        w->knn_cap = k;
        w->knn_id = (int64_t*)realloc(w->knn_id, 8 * k);
        w->knn_d = (double*)realloc(w->knn_d, 8 * k);
      }
      int64_t got = kd_knn(&C->kd_sites, vi, k, i, w->knn_id, w->knn_d);
      for (int64_t t = done_upto; t < got; ++t) {
        double R = piece_radius(w);
        /* a bisector at distance |v_j - v_i| = D lies at (D^2 - (w_j - w_i)) / (2D) >=
           (D^2 - dw) / (2D) from v_i, dw = wmax - w_i: it cannot cut the piece (inside
           the ball of radius R) once D >= R + sqrt(R^2 + dw); dw = 0 gives D >= 2R */
        double dw = C->w ? C->wmax - C->w[i] : 0.0;
        if (dw < 0) dw = 0;
        if (sqrt(w->knn_d[t]) > (R + sqrt(R * R + dw)) * (1.0 + 1e-9)) { finished = 1; break; }
        rc = clip_by_site(w, w->knn_id[t]);
        if (rc != 0) { finished = 1; break; }
      }
      done_upto = got;
      if (got < k || k >= C->n - 1) break;
      k *= 2;
    }
  }
  o->status = rc < 0 ? -1 : 0;
  if (rc < 0 || piece_empty(w)) { o->meas = 0; o->m1[0] = o->m1[1] = o->m1[2] = 0; o->nf = 0; return; }
  integrate(w, a, o, w->P.st[ST_TIE] + w->P.st[ST_UNCERTAIN] == undecided0);
}

/* ------------------------------------------------------------------------- */
/* adjacency of simplices                                                     */
/* ------------------------------------------------------------------------- */
typedef struct { int32_t v[3]; int64_t s; int f; } facekey;

static int cmp_face(const void* a, const void* b) {
  const facekey* x = (const facekey*)a; const facekey* y = (const facekey*)b;
  for (int d = 0; d < 3; ++d) if (x->v[d] != y->v[d]) return x->v[d] < y->v[d] ? -1 : 1;
  return 0;
}

static void sort3(int32_t* v, int n) {
  for (int i = 1; i < n; ++i)
    for (int j = i; j > 0 && v[j - 1] > v[j]; --j) { int32_t t = v[j]; v[j] = v[j - 1]; v[j - 1] = t; }
}

static void build_adjacency(orc_ctx* C) {
  int64_t nf = C->m * C->k;
  facekey* F = (facekey*)malloc(sizeof(facekey) * (nf ? nf : 1));
  for (int64_t a = 0; a < C->m; ++a)
    for (int f = 0; f < C->k; ++f) {
      facekey* fk = &F[a * C->k + f];
      int m = 0;
      for (int t = 0; t < C->k; ++t) if (t != f) fk->v[m++] = C->simp[a * C->k + t];
      if (m == 2) fk->v[2] = -1;
      sort3(fk->v, m);
      fk->s = a; fk->f = f;
    }
  qsort(F, nf, sizeof(facekey), cmp_face);
  for (int64_t t = 0; t < nf * 1; ++t) C->adj[t] = -1;
  for (int64_t t = 0; t < nf;) {
    int64_t u = t + 1;
    while (u < nf && cmp_face(&F[t], &F[u]) == 0) ++u;
    if (u - t == 2) {
      C->adj[F[t].s * C->k + F[t].f] = (int32_t)F[t + 1].s;
      C->adj[F[t + 1].s * C->k + F[t + 1].f] = (int32_t)F[t].s;
    }
    t = u;
  }
  free(F);
}

/* ------------------------------------------------------------------------- */
/* public API                                                                 */
/* ------------------------------------------------------------------------- */
typedef struct {
  int64_t np;
  int32_t* a; int32_t* i; double* meas; double* m1; int64_t* foff; int32_t* flags; double* fmeas;
  int32_t* status;
  int64_t stats[ST_N];
} orc_result;

orc_ctx* orc_create(int mode, int64_t n, const double* sites, int64_t nv, const double* verts, int64_t m,
                    const int32_t* simp, int brute, int nthreads) {
  orc_ctx* C = (orc_ctx*)calloc(1, sizeof(orc_ctx));
  C->mode = mode; C->k = mode == ORC_MODE_3D ? 4 : 3; C->brute = brute;
  C->nthreads = nthreads > 0 ? nthreads : 1;
  C->n = n; C->nv = nv; C->m = m;
  C->sites = (double*)malloc(sizeof(double) * 3 * (n ? n : 1));
  memcpy(C->sites, sites, sizeof(double) * 3 * n);
  C->verts = (double*)malloc(sizeof(double) * 3 * (nv ? nv : 1));
  memcpy(C->verts, verts, sizeof(double) * 3 * nv);
  C->simp = (int32_t*)malloc(sizeof(int32_t) * C->k * (m ? m : 1));
  memcpy(C->simp, simp, sizeof(int32_t) * C->k * m);
  C->adj = (int32_t*)malloc(sizeof(int32_t) * C->k * (m ? m : 1));
  build_adjacency(C);
  kd_build(&C->kd_sites, C->sites, n);
  C->cent = (double*)malloc(sizeof(double) * 3 * (m ? m : 1));
  for (int64_t a = 0; a < m; ++a)
    for (int d = 0; d < 3; ++d) {
      double s = 0;
      for (int t = 0; t < C->k; ++t) s += C->verts[3 * (int64_t)C->simp[a * C->k + t] + d];
      C->cent[3 * a + d] = s / C->k;
    }
  kd_build(&C->kd_cent, C->cent, m);
  return C;
}

/* power weights for the sites (NULL: back to the Voronoi diagram); copied */
void orc_set_weights(orc_ctx* C, const double* w) {
  free(C->w);
  C->w = NULL;
  if (!w) return;
  C->w = (double*)malloc(sizeof(double) * (C->n ? C->n : 1));
  memcpy(C->w, w, sizeof(double) * C->n);
  C->wmax = -INFINITY;
  for (int64_t i = 0; i < C->n; ++i) if (C->w[i] > C->wmax) C->wmax = C->w[i];
}

void orc_destroy(orc_ctx* C) {
  if (!C) return;
  free(C->w);
  kd_free(&C->kd_sites); kd_free(&C->kd_cent);
  free(C->sites); free(C->verts); free(C->simp); free(C->adj); free(C->cent); free(C);
}

int64_t orc_adjacency(const orc_ctx* C, int32_t* out) {
  memcpy(out, C->adj, sizeof(int32_t) * C->k * C->m);
  return C->m * C->k;
}

/* growable list of pieces produced by one work item */
typedef struct {
  int64_t np, cap, nfl, flcap;
  int32_t *a, *i, *status; double *meas, *m1; int64_t* fcnt; int32_t* flags; double* fmeas;
} plist;

static void pl_add(plist* L, int64_t a, int64_t i, const piece_out* o) {
  if (L->np == L->cap) {
    L->cap = L->cap ? 2 * L->cap : 16;
    L->a = (int32_t*)realloc(L->a, 4 * L->cap); L->i = (int32_t*)realloc(L->i, 4 * L->cap);
    L->status = (int32_t*)realloc(L->status, 4 * L->cap);
    L->meas = (double*)realloc(L->meas, 8 * L->cap); L->m1 = (double*)realloc(L->m1, 24 * L->cap);
    L->fcnt = (int64_t*)realloc(L->fcnt, 8 * L->cap);
  }
  while (L->nfl + o->nf > L->flcap) {
    L->flcap = L->flcap ? 2 * L->flcap : 64;
    L->flags = (int32_t*)realloc(L->flags, 4 * L->flcap);
    L->fmeas = (double*)realloc(L->fmeas, 8 * L->flcap);
  }
  int64_t p = L->np++;
  L->a[p] = (int32_t)a; L->i[p] = (int32_t)i; L->status[p] = o->status; L->meas[p] = o->meas;
  memcpy(L->m1 + 3 * p, o->m1, 24); L->fcnt[p] = o->nf;
  memcpy(L->flags + L->nfl, o->flags, 4 * o->nf); memcpy(L->fmeas + L->nfl, o->fmeas, 8 * o->nf);
  L->nfl += o->nf;
}

static void pl_free(plist* L) {
  free(L->a); free(L->i); free(L->status); free(L->meas); free(L->m1); free(L->fcnt); free(L->flags);
  free(L->fmeas);
}

typedef struct {
  const orc_ctx* C;
  int kind;                 /* 0: pairs, 1: simplices (enumerate), 2: sites (flood) */
  int64_t nitems;
  const int64_t* ia; const int64_t* ib;
  int keep_empty;
  plist* out;               /* one list per item */
  int64_t next;
  pthread_mutex_t mu;
  int64_t stats[ST_N];
} job;

static void item_pairs(job* J, workspace* w, int64_t t) {
  piece_out o;
  compute_piece(w, J->ia[t], J->ib[t], &o);
  pl_add(&J->out[t], J->ia[t], J->ib[t], &o);
}

static void item_simplex(job* J, workspace* w, int64_t a) {
  const orc_ctx* C = J->C;
  piece_out o;
  ivec cand = {0, 0, 0};
  if (C->brute) {
    for (int64_t i = 0; i < C->n; ++i) iv_push(&cand, i);
  } else {
    /* a site can own a point x of T_a only if |c - v_i| <= d_NN(c) + 2 rho, with c the
       centroid and rho the largest centroid-to-corner distance (d_NN is 1-Lipschitz) */
    const double* c = C->cent + 3 * a;
    double rho = 0;
    for (int t = 0; t < C->k; ++t) {
      double d = sqrt(d2(c, C->verts + 3 * (int64_t)C->simp[a * C->k + t]));
      if (d > rho) rho = d;
    }
    int64_t id; double dd;
    kd_knn(&C->kd_sites, c, 1, -1, &id, &dd);
    double R = (sqrt(dd) + 2 * rho) * (1 + 1e-9) + 1e-12;
    if (C->w) {
      /* power diagram: |x - v_i|^2 <= (d_NN(c) + rho)^2 + (w_max - w_min) for x of T_a
         owned by v_i, so |c - v_i| <= rho + sqrt((d_NN + rho)^2 + dw) */
      double wmin = INFINITY;
      for (int64_t u = 0; u < C->n; ++u) if (C->w[u] < wmin) wmin = C->w[u];
      double dn = sqrt(dd) + rho;
      R = (rho + sqrt(dn * dn + (C->wmax - wmin))) * (1 + 1e-9) + 1e-12;
    }
    kd_range_rec(&C->kd_sites, c, R * R, 0, C->kd_sites.n, 0, &cand);
    /* deterministic order */
    for (int64_t u = 1; u < cand.n; ++u)
      for (int64_t v = u; v > 0 && cand.v[v - 1] > cand.v[v]; --v) {
        int64_t tt = cand.v[v]; cand.v[v] = cand.v[v - 1]; cand.v[v - 1] = tt;
      }
  }
  for (int64_t t = 0; t < cand.n; ++t) {
    compute_piece(w, a, cand.v[t], &o);
    if (o.status != 0 || o.meas > 0 || J->keep_empty) pl_add(&J->out[a], a, cand.v[t], &o);
  }
  free(cand.v);
}

static void item_site(job* J, workspace* w, int64_t t) {
  const orc_ctx* C = J->C;
  int64_t i = J->ia[t];
  piece_out o;
  ivec seen = {0, 0, 0}, queue = {0, 0, 0};
  /* seeds: simplices with the nearest centroids; widen until one piece is non-empty */
  int64_t k = 16;
  int found = 0;
  while (!found) {
    if (k > C->m) k = C->m;
    int64_t* ids = (int64_t*)malloc(8 * k);
    double* ds = (double*)malloc(8 * k);
    int64_t got = kd_knn(&C->kd_cent, C->sites + 3 * i, k, -1, ids, ds);
    for (int64_t u = 0; u < got; ++u) {
      int dup = 0;
      for (int64_t s = 0; s < seen.n; ++s) if (seen.v[s] == ids[u]) { dup = 1; break; }
      if (dup) continue;
      iv_push(&seen, ids[u]);
      compute_piece(w, ids[u], i, &o);
      if (o.meas > 0 || o.status != 0) { pl_add(&J->out[t], ids[u], i, &o); iv_push(&queue, ids[u]); found = 1; }
    }
    free(ids); free(ds);
    if (k >= C->m) break;
    k *= 4;
  }
  /* flood across simplex faces of positive measure (the set of simplices met by a
     connected Omega_i intersected with M is connected through such faces) */
  int64_t head = 0;
  while (head < queue.n) {
    int64_t a = queue.v[head++];
    plist* L = &J->out[t];
    int64_t p;
    for (p = 0; p < L->np; ++p) if (L->a[p] == a) break;
    int64_t off = 0;
    for (int64_t r = 0; r < p; ++r) off += L->fcnt[r];
    int64_t nfl = L->fcnt[p];
    int32_t fl[PF_MAX];
    memcpy(fl, L->flags + off, 4 * nfl);
    for (int64_t f = 0; f < nfl; ++f) {
      if (fl[f] >= 0 || fl[f] == ORC_FLAG_BOUNDARY) continue;
      int64_t b = -(int64_t)fl[f] - 1;
      int dup = 0;
      for (int64_t s = 0; s < seen.n; ++s) if (seen.v[s] == b) { dup = 1; break; }
      if (dup) continue;
      iv_push(&seen, b);
      compute_piece(w, b, i, &o);
      if (o.meas > 0 || o.status != 0) { pl_add(&J->out[t], b, i, &o); iv_push(&queue, b); }
    }
  }
  free(seen.v); free(queue.v);
}

static void* worker(void* arg) {
  job* J = (job*)arg;
  int64_t st[ST_N] = {0};
  workspace* w = ws_new(J->C, st);
  for (;;) {
    int64_t t = __atomic_fetch_add(&J->next, 1, __ATOMIC_RELAXED);
    if (t >= J->nitems) break;
    if (J->kind == 0) item_pairs(J, w, t);
    else if (J->kind == 1) item_simplex(J, w, t);
    else item_site(J, w, t);
  }
  ws_free(w);
  pthread_mutex_lock(&J->mu);
  for (int s = 0; s < ST_N; ++s) J->stats[s] += st[s];
  pthread_mutex_unlock(&J->mu);
  return NULL;
}

static orc_result* run_job(job* J) {
  J->out = (plist*)calloc(J->nitems ? J->nitems : 1, sizeof(plist));
  J->next = 0;
  pthread_mutex_init(&J->mu, NULL);
  int nt = J->C->nthreads;
  pthread_t* th = (pthread_t*)malloc(sizeof(pthread_t) * nt);
  for (int t = 0; t < nt; ++t) pthread_create(&th[t], NULL, worker, J);
  for (int t = 0; t < nt; ++t) pthread_join(th[t], NULL);
  free(th);
  pthread_mutex_destroy(&J->mu);
  orc_result* R = (orc_result*)calloc(1, sizeof(orc_result));
  int64_t np = 0, nfl = 0;
  for (int64_t t = 0; t < J->nitems; ++t) { np += J->out[t].np; nfl += J->out[t].nfl; }
  R->np = np;
  R->a = (int32_t*)malloc(4 * (np + 1)); R->i = (int32_t*)malloc(4 * (np + 1));
  R->status = (int32_t*)malloc(4 * (np + 1));
  R->meas = (double*)malloc(8 * (np + 1)); R->m1 = (double*)malloc(24 * (np + 1));
  R->foff = (int64_t*)malloc(8 * (np + 1));
  R->flags = (int32_t*)malloc(4 * (nfl + 1)); R->fmeas = (double*)malloc(8 * (nfl + 1));
  int64_t p = 0, f = 0;
  R->foff[0] = 0;
  for (int64_t t = 0; t < J->nitems; ++t) {
    plist* L = &J->out[t];
    memcpy(R->a + p, L->a, 4 * L->np); memcpy(R->i + p, L->i, 4 * L->np);
    memcpy(R->status + p, L->status, 4 * L->np);
    memcpy(R->meas + p, L->meas, 8 * L->np); memcpy(R->m1 + 3 * p, L->m1, 24 * L->np);
    for (int64_t u = 0; u < L->np; ++u) R->foff[p + u + 1] = R->foff[p + u] + L->fcnt[u];
    memcpy(R->flags + f, L->flags, 4 * L->nfl); memcpy(R->fmeas + f, L->fmeas, 8 * L->nfl);
    p += L->np; f += L->nfl;
    pl_free(L);
  }
  free(J->out);
  memcpy(R->stats, J->stats, sizeof(R->stats));
  return R;
}

/* pieces for an explicit list of (simplex, site) pairs (empty pieces included) */
orc_result* orc_pieces(const orc_ctx* C, int64_t npairs, const int64_t* a, const int64_t* i) {
  job J; memset(&J, 0, sizeof(J));
  J.C = C; J.kind = 0; J.nitems = npairs; J.ia = a; J.ib = i;
  return run_job(&J);
}

/* every non-empty piece, found simplex by simplex from a candidate ball */
orc_result* orc_enumerate(const orc_ctx* C) {
  job J; memset(&J, 0, sizeof(J));
  J.C = C; J.kind = 1; J.nitems = C->m;
  return run_job(&J);
}

/* every non-empty piece of the listed sites (flood over simplex adjacency) */
orc_result* orc_site_pieces(const orc_ctx* C, int64_t nsites, const int64_t* sites) {
  job J; memset(&J, 0, sizeof(J));
  J.C = C; J.kind = 2; J.nitems = nsites; J.ia = sites;
  return run_job(&J);
}

void orc_free_result(orc_result* R) {
  if (!R) return;
  free(R->a); free(R->i); free(R->status); free(R->meas); free(R->m1); free(R->foff); free(R->flags);
  free(R->fmeas); free(R);
}
