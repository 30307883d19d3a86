/*
 * vd_serial.c -- the paper's serial method on the CPU: Alg. 1 (simplex-cell
 * intersection by clipping along real edges) driven by Alg. 2 (per simplex:
 * the first piece from the nearest site of the simplex's first corner, then
 * the other pieces reached through positive face flags, each started from an
 * intermediate polytope G_{a,j} built from the (u, f) tuple of the piece that
 * discovered it).  Single-threaded by design; a CPU baseline of the method,
 * never a fallback of the GPU path.
 *
 * Passages followed:
 *   Sec. 2.1, Eq. 1   the cell Omega_i and the pieces P_{a,i} = T_a ^ Omega_i
 *   Sec. 2.2          face flags: j for the face on bisector B_ij, -(b+1) for a
 *                     face shared with simplex b, INT32_MIN on the boundary
 *   Sec. 3.1          point-in-cell test of a corner: outside iff some site not
 *                     among the corner's own flag sites is strictly closer
 *   Sec. 3.2          edge-based bisector search on p_s p_t (p_s in Omega_i)
 *   Sec. 3.3, Alg. 1  clip along edges with p_s inside and p_t outside until no
 *                     corner is outside; corners known inside are not retested
 *   Sec. 3.4, Alg. 2  per simplex: first piece, queue over positive flags, the
 *                     intermediate polytope G_{a,j} (clips by B_{j,u} and by
 *                     B_{j,w} for the positive flags w of the faces adjacent to f)
 *   Sec. 5.1          improved start point g = p_s + lambda delta (p_t - p_s)/|.|
 *   Sec. 5.2          uniform site grids, 3-4 sites per cell (2-3 in 2D / on
 *                     surfaces); cells much denser than that get a finer grid
 *
 * Representation (this file's own): a convex polytope is a set of corners,
 * each the meeting point of three planes with, per plane, the neighbour across
 * the edge formed by its other two planes.  Polygons (2D, surface) are the same
 * structure with the simplex's supporting plane S among every corner's planes.
 * Geometry is FP64 in the global frame; every sign decision (corner against a
 * plane) is certified: FP64 with a running error bound, then binary128 with a
 * running error bound, else counted as uncertain.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define SRC_S (-100)          /* the triangle's own plane (2D, surface) */
#define MAXPL 128             /* planes per polytope */
#define MAXV 256              /* corner slots per polytope */
#define FLAG_BND ((int32_t)0x80000000)

enum { ST_UNK = 0, ST_IN = 1, ST_OUT = 2 };
enum { M2D = 2, MSURF = 3, M3D = 4 };

/* ---------------------------------------------------------------------------
 * numbers with a bound on their absolute error: FP64 and binary128
 * ------------------------------------------------------------------------- */
typedef struct { double v, e; } e64;
typedef struct { __float128 v, e; } e128;

#define U64 (0x1p-53)
static const __float128 U128 = 1.0 / 10384593717069655257060992658440192.0; /* 2^-113 */

static inline double ad(double x) { return x < 0 ? -x : x; }
static inline __float128 aq(__float128 x) { return x < 0 ? -x : x; }

static inline e64 c64(double x) { e64 r = {x, 0.0}; return r; }
static inline e64 add64(e64 a, e64 b) { double s = a.v + b.v; e64 r = {s, a.e + b.e + U64 * ad(s)}; return r; }
static inline e64 sub64(e64 a, e64 b) { double s = a.v - b.v; e64 r = {s, a.e + b.e + U64 * ad(s)}; return r; }
static inline e64 mul64(e64 a, e64 b) {
  double p = a.v * b.v;
  e64 r = {p, ad(a.v) * b.e + ad(b.v) * a.e + a.e * b.e + U64 * ad(p)};
  return r;
}
static inline e128 c128(double x) { e128 r = {(__float128)x, 0}; return r; }
static inline e128 add128(e128 a, e128 b) { __float128 s = a.v + b.v; e128 r = {s, a.e + b.e + U128 * aq(s)}; return r; }
static inline e128 sub128(e128 a, e128 b) { __float128 s = a.v - b.v; e128 r = {s, a.e + b.e + U128 * aq(s)}; return r; }
static inline e128 mul128(e128 a, e128 b) {
  __float128 p = a.v * b.v;
  e128 r = {p, aq(a.v) * b.e + aq(b.v) * a.e + a.e * b.e + U128 * aq(p)};
  return r;
}

/* ---------------------------------------------------------------------------
 * context
 * ------------------------------------------------------------------------- */
typedef struct {
  int gx, gy, gz;
  double ox, oy, oz, h;
  int32_t* start;       /* [G+1] */
  int32_t* item;        /* [n] site ids by cell */
  int32_t* sub;         /* [G] -1 or index of a finer grid over that cell */
} Grid;

typedef struct sv_ctx {
  int mode, k;
  int64_t n, nv, m;
  double* sites;        /* n*3 */
  double* verts;        /* nv*3 */
  int32_t* simp;        /* m*k */
  int32_t* adj;         /* m*k: simplex across facet f (opposite local vertex f), -1 none */
  double* delta;        /* n: half the distance to the nearest other site (Sec. 5.1) */
  Grid g;
  Grid* fine;           /* finer grids of dense cells */
  int nfine;
  int32_t* stamp;       /* n: last simplex that queued the site */
  int64_t stats[12];
} sv_ctx;

enum { S_TESTS = 0, S_NN = 1, S_CLIPS = 2, S_GCLIPS = 3, S_FACES = 4, S_EXCESS = 5, S_FALLBACK = 6,
       S_F128 = 7, S_UNCERTAIN = 8, S_TIES = 9, S_SEARCH = 10, S_ERROR = 11 };

/* ---------------------------------------------------------------------------
 * site grids (Sec. 5.2)
 * ------------------------------------------------------------------------- */
static int grid_build(Grid* G, const double* sites, const int32_t* ids, int64_t cnt, const double lo[3],
                      const double hi[3], double per_cell, int dims) {
  double ext[3], vol = 1.0;
  for (int d = 0; d < 3; ++d) {
    ext[d] = hi[d] - lo[d];
    if (!(ext[d] > 0)) ext[d] = 1e-12;
  }
  for (int d = 0; d < dims; ++d) vol *= ext[d];
  double h = pow(vol * per_cell / (double)(cnt > 0 ? cnt : 1), 1.0 / dims);
  for (;;) {
    long long g[3];
    for (int d = 0; d < 3; ++d) g[d] = d < dims ? (long long)ceil(ext[d] / h) : 1;
    for (int d = 0; d < 3; ++d) if (g[d] < 1) g[d] = 1;
    if (g[0] * g[1] * g[2] <= (1ll << 26)) { G->gx = (int)g[0]; G->gy = (int)g[1]; G->gz = (int)g[2]; break; }
    h *= 1.25;
  }
  G->h = h; G->ox = lo[0]; G->oy = lo[1]; G->oz = lo[2];
  long long nc = (long long)G->gx * G->gy * G->gz;
  G->start = (int32_t*)calloc((size_t)nc + 1, sizeof(int32_t));
  G->item = (int32_t*)malloc(sizeof(int32_t) * (size_t)(cnt > 0 ? cnt : 1));
  G->sub = (int32_t*)malloc(sizeof(int32_t) * (size_t)nc);
  int32_t* cell = (int32_t*)malloc(sizeof(int32_t) * (size_t)(cnt > 0 ? cnt : 1));
  if (!G->start || !G->item || !G->sub || !cell) { free(cell); return -1; }
  for (long long c = 0; c < nc; ++c) G->sub[c] = -1;
  for (int64_t t = 0; t < cnt; ++t) {
    const double* p = sites + 3 * (size_t)ids[t];
    int c[3];
    double o[3] = {G->ox, G->oy, G->oz};
    int gd[3] = {G->gx, G->gy, G->gz};
    for (int d = 0; d < 3; ++d) {
      long long x = (long long)floor((p[d] - o[d]) / h);
      c[d] = (int)(x < 0 ? 0 : (x >= gd[d] ? gd[d] - 1 : x));
    }
    cell[t] = (c[2] * G->gy + c[1]) * G->gx + c[0];
    G->start[cell[t] + 1]++;
  }
  for (long long c = 0; c < nc; ++c) G->start[c + 1] += G->start[c];
  int32_t* cur = (int32_t*)malloc(sizeof(int32_t) * (size_t)nc);
  if (!cur) { free(cell); return -1; }
  memcpy(cur, G->start, sizeof(int32_t) * (size_t)nc);
  for (int64_t t = 0; t < cnt; ++t) G->item[cur[cell[t]]++] = ids[t];
  free(cur);
  free(cell);
  return 0;
}

static void grid_free(Grid* G) {
  free(G->start); free(G->item); free(G->sub);
  memset(G, 0, sizeof(*G));
}

/* sites of the level-0 cells denser than 8 x the target get a finer grid over
 * the cell (one level: enough for the Gaussian clusters of the tests) */
static int grids_build(sv_ctx* c) {
  int dims = c->mode == M2D ? 2 : 3;
  double per = c->mode == M3D ? 3.5 : 2.5;
  double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
  for (int64_t v = 0; v < c->nv; ++v)
    for (int d = 0; d < 3; ++d) {
      double x = c->verts[3 * v + d];
      if (x < lo[d]) lo[d] = x;
      if (x > hi[d]) hi[d] = x;
    }
  for (int d = 0; d < 3; ++d) { double pad = 1e-3 * (hi[d] - lo[d]) + 1e-9; lo[d] -= pad; hi[d] += pad; }
  int32_t* ids = (int32_t*)malloc(sizeof(int32_t) * (size_t)c->n);
  if (!ids) return -1;
  for (int64_t i = 0; i < c->n; ++i) ids[i] = (int32_t)i;
  if (grid_build(&c->g, c->sites, ids, c->n, lo, hi, per, dims)) { free(ids); return -1; }
  free(ids);
  long long nc = (long long)c->g.gx * c->g.gy * c->g.gz;
  int nf = 0;
  for (long long q = 0; q < nc; ++q) nf += (c->g.start[q + 1] - c->g.start[q]) > 8 * per;
  c->fine = nf ? (Grid*)calloc((size_t)nf, sizeof(Grid)) : NULL;
  c->nfine = 0;
  for (long long q = 0; q < nc && nf; ++q) {
    int cnt = c->g.start[q + 1] - c->g.start[q];
    if (cnt <= 8 * per) continue;
    int x = (int)(q % c->g.gx), y = (int)((q / c->g.gx) % c->g.gy), z = (int)(q / ((long long)c->g.gx * c->g.gy));
    double clo[3] = {c->g.ox + x * c->g.h, c->g.oy + y * c->g.h, c->g.oz + z * c->g.h};
    double chi[3] = {clo[0] + c->g.h, clo[1] + c->g.h, clo[2] + c->g.h};
    if (dims == 2) { clo[2] = c->g.oz; chi[2] = c->g.oz + c->g.h; }
    /* boundary cells also hold sites beyond the grid box: widen to their extent */
    for (int t = c->g.start[q]; t < c->g.start[q + 1]; ++t)
      for (int d = 0; d < 3; ++d) {
        double p = c->sites[3 * (size_t)c->g.item[t] + d];
        if (p < clo[d]) clo[d] = p;
        if (p > chi[d]) chi[d] = p;
      }
    if (grid_build(&c->fine[c->nfine], c->sites, c->g.item + c->g.start[q], cnt, clo, chi, per, dims)) return -1;
    c->g.sub[q] = c->nfine++;
  }
  return 0;
}

/* squared distance from p to the box of cell (x,y,z) of grid G (0 inside) */
static double cell_d2(const Grid* G, int x, int y, int z, const double* p) {
  double lo[3] = {G->ox + x * G->h, G->oy + y * G->h, G->oz + z * G->h}, s = 0;
  int id[3] = {x, y, z}, gd[3] = {G->gx, G->gy, G->gz};
  for (int d = 0; d < 3; ++d) {
    /* boundary cells are open outwards (they hold the sites beyond the box) */
    double a = (id[d] == 0) ? -1e300 : lo[d], b = (id[d] == gd[d] - 1) ? 1e300 : lo[d] + G->h;
    double t = p[d] < a ? a - p[d] : (p[d] > b ? p[d] - b : 0);
    s += t * t;
  }
  return s;
}

/* cell index range of grid G covering the box [p - r, p + r] */
static inline void cell_range(const Grid* G, const double* p, double r, int lo[3], int hi[3]) {
  double o[3] = {G->ox, G->oy, G->oz};
  int gd[3] = {G->gx, G->gy, G->gz};
  for (int d = 0; d < 3; ++d) {
    double a = (p[d] - r - o[d]) / G->h, b = (p[d] + r - o[d]) / G->h;
    long long x0 = (long long)floor(a < -1e9 ? -1e9 : (a > 1e9 ? 1e9 : a));
    long long x1 = (long long)floor(b < -1e9 ? -1e9 : (b > 1e9 ? 1e9 : b));
    lo[d] = (int)(x0 < 0 ? 0 : (x0 >= gd[d] ? gd[d] - 1 : x0));
    hi[d] = (int)(x1 < 0 ? 0 : (x1 >= gd[d] ? gd[d] - 1 : x1));
  }
}

/* FOR_BALL(c, p, r, k, body): body for every site k stored in a grid cell (or a
 * finer grid's cell) within distance r of p -- a superset of the sites within r */
#define FOR_CELLS_(L, G, P_, R_, ...)                                                         \
  do {                                                                                        \
    int lo##L[3], hi##L[3];                                                                   \
    cell_range((G), (P_), (R_), lo##L, hi##L);                                                \
    double r2##L = (R_) * (R_);                                                               \
    for (int z##L = lo##L[2]; z##L <= hi##L[2]; ++z##L)                                       \
      for (int y##L = lo##L[1]; y##L <= hi##L[1]; ++y##L)                                     \
        for (int x##L = lo##L[0]; x##L <= hi##L[0]; ++x##L) {                                 \
          if (cell_d2((G), x##L, y##L, z##L, (P_)) > r2##L) continue;                         \
          long long q##L = ((long long)z##L * (G)->gy + y##L) * (G)->gx + x##L;               \
          __VA_ARGS__                                                                         \
        }                                                                                     \
  } while (0)
#define FOR_CELLS0_(G, P_, R_, ...) FOR_CELLS_(_0, G, P_, R_, __VA_ARGS__)
#define FOR_CELLS1_(G, P_, R_, ...) FOR_CELLS_(_1, G, P_, R_, __VA_ARGS__)

#define FOR_BALL(C, P, R, K, ...)                                                             \
  FOR_CELLS0_(&(C)->g, (P), (R), {                                                            \
    if ((C)->g.sub[q_0] >= 0) {                                                               \
      const Grid* F_ = &(C)->fine[(C)->g.sub[q_0]];                                           \
      FOR_CELLS1_(F_, (P), (R), {                                                             \
        for (int t_ = F_->start[q_1]; t_ < F_->start[q_1 + 1]; ++t_) { int32_t K = F_->item[t_]; __VA_ARGS__ } \
      });                                                                                     \
    } else {                                                                                  \
      for (int t_ = (C)->g.start[q_0]; t_ < (C)->g.start[q_0 + 1]; ++t_) { int32_t K = (C)->g.item[t_]; __VA_ARGS__ } \
    }                                                                                         \
  })

/* cell size where p lies: the finer grid's inside a dense cell */
static double local_h(const sv_ctx* c, const double* p) {
  const Grid* G = &c->g;
  double o[3] = {G->ox, G->oy, G->oz};
  int gd[3] = {G->gx, G->gy, G->gz}, id[3];
  for (int d = 0; d < 3; ++d) {
    double a = (p[d] - o[d]) / G->h;
    long long x = (long long)floor(a < -1e9 ? -1e9 : (a > 1e9 ? 1e9 : a));
    id[d] = (int)(x < 0 ? 0 : (x >= gd[d] ? gd[d] - 1 : x));
  }
  long long q = ((long long)id[2] * G->gy + id[1]) * G->gx + id[0];
  return G->sub[q] >= 0 ? c->fine[G->sub[q]].h : G->h;
}

/* nearest site of p (ties: smaller index), skipping `skip` and the sites ex0,
 * ex1; grows the ball from the local cell size until it holds a site, then
 * rescans the ball of the best distance */
static int nearest_ex(sv_ctx* c, const double* p, int skip, int ex0, int ex1, double* d2) {
  double bd = 1e300;
  int bi = -1;
  const double* S = c->sites;
#define NN_BODY                                                             \
  if (k != skip && k != ex0 && k != ex1) {                                  \
    const double* v = S + 3 * (size_t)k;                                    \
    double dx = v[0] - p[0], dy = v[1] - p[1], dz = v[2] - p[2];            \
    double dd = dx * dx + dy * dy + dz * dz;                                \
    if (dd < bd || (dd == bd && k < bi)) { bd = dd; bi = k; }               \
  }
  double r = local_h(c, p);
  for (int it = 0; it < 64 && bi < 0; ++it, r *= 2) FOR_BALL(c, p, r, k, NN_BODY);
  if (bi < 0) { *d2 = 1e300; return -1; }
  double rb = sqrt(bd) * (1 + 1e-12) + 1e-300;
  if (rb > r / 2) FOR_BALL(c, p, rb, k, NN_BODY);
#undef NN_BODY
  c->stats[S_NN]++;
  *d2 = bd;
  return bi;
}

static int nearest(sv_ctx* c, const double* p, int skip, double* d2) { return nearest_ex(c, p, skip, -2, -2, d2); }

/* ---------------------------------------------------------------------------
 * planes: from their sources, with error bounds, in the frame of site s
 * (exact predicates) or in the global frame (s < 0: geometry)
 * ------------------------------------------------------------------------- */
typedef struct { int src; int a; } PlaneId;  /* src: >= 0 bisector with that site; -1-f facet f; SRC_S */

#define DEFINE_PLANE(T, C, ADD, SUB, MUL)                                                           \
  static void plane_##T(const sv_ctx* c, int s, int a, int src, T n[3], T* cc) {                   \
    T o[3];                                                                                         \
    for (int d = 0; d < 3; ++d) o[d] = s >= 0 ? C(c->sites[3 * (size_t)s + d]) : C(0.0);            \
    if (src >= 0) { /* bisector of s and src: |x - v_s|^2 <= |x - v_src|^2 */                      \
      for (int d = 0; d < 3; ++d) n[d] = SUB(C(c->sites[3 * (size_t)src + d]), C(c->sites[3 * (size_t)s + d])); \
      T w2 = ADD(ADD(MUL(n[0], n[0]), MUL(n[1], n[1])), MUL(n[2], n[2]));                           \
      T half = MUL(w2, C(0.5));                                                                     \
      if (s >= 0) { *cc = half; return; }                                                          \
      return;                                                                                       \
    }                                                                                               \
    const int32_t* sp = c->simp + (size_t)a * c->k;                                                 \
    const double* V[4];                                                                             \
    for (int l = 0; l < c->k; ++l) V[l] = c->verts + 3 * (size_t)sp[l];                             \
    T e1[3], e2[3], tn[3];                                                                          \
    if (c->k == 4 || src == SRC_S) {                                                                \
      int l0 = 0, l1 = 1, l2 = 2, f = -1;                                                           \
      if (src != SRC_S) { f = -1 - src; l0 = f == 0 ? 1 : 0; l1 = f <= 1 ? 2 : 1; l2 = f <= 2 ? 3 : 2; } \
      for (int d = 0; d < 3; ++d) { e1[d] = SUB(C(V[l1][d]), C(V[l0][d])); e2[d] = SUB(C(V[l2][d]), C(V[l0][d])); } \
      tn[0] = SUB(MUL(e1[1], e2[2]), MUL(e1[2], e2[1]));                                            \
      tn[1] = SUB(MUL(e1[2], e2[0]), MUL(e1[0], e2[2]));                                            \
      tn[2] = SUB(MUL(e1[0], e2[1]), MUL(e1[1], e2[0]));                                            \
      double sg = 1.0;                                                                              \
      if (f >= 0) { /* outward: vertex f strictly inside */                                         \
        double t = 0;                                                                               \
        for (int d = 0; d < 3; ++d) t += (double)tn[d].v * (V[f][d] - V[l0][d]);                    \
        sg = t > 0 ? -1.0 : 1.0;                                                                    \
      }                                                                                             \
      for (int d = 0; d < 3; ++d) n[d] = MUL(tn[d], C(sg));                                         \
      *cc = ADD(ADD(MUL(n[0], SUB(C(V[l0][0]), o[0])), MUL(n[1], SUB(C(V[l0][1]), o[1]))),          \
                MUL(n[2], SUB(C(V[l0][2]), o[2])));                                                 \
      return;                                                                                       \
    }                                                                                               \
    /* triangle edge f (opposite local vertex f): contains the edge and the normal */               \
    int f = -1 - src, p0 = f == 0 ? 1 : 0, p1 = f == 2 ? 1 : 2;                                     \
    for (int d = 0; d < 3; ++d) { e1[d] = SUB(C(V[1][d]), C(V[0][d])); e2[d] = SUB(C(V[2][d]), C(V[0][d])); } \
    tn[0] = SUB(MUL(e1[1], e2[2]), MUL(e1[2], e2[1]));                                              \
    tn[1] = SUB(MUL(e1[2], e2[0]), MUL(e1[0], e2[2]));                                              \
    tn[2] = SUB(MUL(e1[0], e2[1]), MUL(e1[1], e2[0]));                                              \
    T ed[3];                                                                                        \
    for (int d = 0; d < 3; ++d) ed[d] = SUB(C(V[p1][d]), C(V[p0][d]));                              \
    n[0] = SUB(MUL(ed[1], tn[2]), MUL(ed[2], tn[1]));                                               \
    n[1] = SUB(MUL(ed[2], tn[0]), MUL(ed[0], tn[2]));                                               \
    n[2] = SUB(MUL(ed[0], tn[1]), MUL(ed[1], tn[0]));                                               \
    double t = 0;                                                                                   \
    for (int d = 0; d < 3; ++d) t += (double)n[d].v * (V[f][d] - V[p0][d]);                         \
    if (t > 0) for (int d = 0; d < 3; ++d) n[d] = MUL(n[d], C(-1.0));                               \
    *cc = ADD(ADD(MUL(n[0], SUB(C(V[p0][0]), o[0])), MUL(n[1], SUB(C(V[p0][1]), o[1]))),            \
              MUL(n[2], SUB(C(V[p0][2]), o[2])));                                                   \
  }

DEFINE_PLANE(e64, c64, add64, sub64, mul64)
DEFINE_PLANE(e128, c128, add128, sub128, mul128)

/* Side of the corner of planes q[0..2] against plane p4, for site s's piece in
 * simplex a: +1 strictly inside (n4.x < c4), -1 strictly outside, 0 on it.
 * With N the matrix of the corner's normals and c their offsets,
 * c4 - n4.x = (c4 det N - n4.adj(N) c) / det N. */
#define DEFINE_SIDE(T, NAME, C, ADD, SUB, MUL, ABS, U)                                              \
  static int NAME(const sv_ctx* c, int s, int a, const int q[3], int p4, int* certain, int* zero) { \
    T n[4][3], cc[4];                                                                               \
    for (int r = 0; r < 3; ++r) plane_##T(c, s, a, q[r], n[r], &cc[r]);                             \
    plane_##T(c, s, a, p4, n[3], &cc[3]);                                                           \
    T x12[3], x20[3], x01[3];                                                                       \
    T* A = n[0]; T* B = n[1]; T* Cn = n[2];                                                         \
    x12[0] = SUB(MUL(B[1], Cn[2]), MUL(B[2], Cn[1])); x12[1] = SUB(MUL(B[2], Cn[0]), MUL(B[0], Cn[2])); \
    x12[2] = SUB(MUL(B[0], Cn[1]), MUL(B[1], Cn[0]));                                               \
    x20[0] = SUB(MUL(Cn[1], A[2]), MUL(Cn[2], A[1])); x20[1] = SUB(MUL(Cn[2], A[0]), MUL(Cn[0], A[2])); \
    x20[2] = SUB(MUL(Cn[0], A[1]), MUL(Cn[1], A[0]));                                               \
    x01[0] = SUB(MUL(A[1], B[2]), MUL(A[2], B[1])); x01[1] = SUB(MUL(A[2], B[0]), MUL(A[0], B[2]));  \
    x01[2] = SUB(MUL(A[0], B[1]), MUL(A[1], B[0]));                                                 \
    T D = ADD(ADD(MUL(A[0], x12[0]), MUL(A[1], x12[1])), MUL(A[2], x12[2]));                        \
    T adjc[3];                                                                                      \
    for (int d = 0; d < 3; ++d) adjc[d] = ADD(ADD(MUL(cc[0], x12[d]), MUL(cc[1], x20[d])), MUL(cc[2], x01[d])); \
    T E = SUB(MUL(cc[3], D), ADD(ADD(MUL(n[3][0], adjc[0]), MUL(n[3][1], adjc[1])), MUL(n[3][2], adjc[2]))); \
    double sf = 1.0 + 1e-9;                                                                         \
    int sD = D.v > D.e * sf ? 1 : (D.v < -D.e * sf ? -1 : 0);                                       \
    int sE = E.v > E.e * sf ? 1 : (E.v < -E.e * sf ? -1 : 0);                                       \
    *zero = E.v == 0;                                                                               \
    *certain = sD != 0 && (sE != 0 || (E.v == 0 && E.e == 0));                                      \
    if (!*certain) { sD = D.v > 0 ? 1 : -1; sE = E.v > 0 ? 1 : (E.v < 0 ? -1 : 0); }                \
    return sD * sE;                                                                                 \
  }

DEFINE_SIDE(e64, side64, c64, add64, sub64, mul64, ad, U64)
DEFINE_SIDE(e128, side128, c128, add128, sub128, mul128, aq, U128)

static int side_exact(sv_ctx* c, int s, int a, const int q[3], int p4) {
  for (int r = 0; r < 3; ++r)
    if (q[r] == p4) return 0;  /* the corner lies on its own planes */
  int cert, zero;
  int sg = side64(c, s, a, q, p4, &cert, &zero);
  if (cert) return sg;
  c->stats[S_F128]++;
  sg = side128(c, s, a, q, p4, &cert, &zero);
  if (!cert) {
    if (zero) c->stats[S_TIES]++;
    else c->stats[S_UNCERTAIN]++;
  }
  return sg;
}

/* ---------------------------------------------------------------------------
 * polytope: corners of three planes with neighbours across their edges
 * ------------------------------------------------------------------------- */
typedef struct {
  double x[3];   /* global coordinates */
  double err;    /* bound on each coordinate's error */
  int p[3];      /* plane slots */
  int nb[3];     /* neighbour across the edge formed by the two planes other than p[k] */
  int alive, st, wit;
} Corner;

typedef struct {
  int a;                 /* simplex */
  int s;                 /* the site whose cell clips it: the frame's origin */
  double o[3];           /* v_s: corner coordinates and planes are relative to it */
  int npl, nc;
  int src[MAXPL];        /* plane sources */
  e64 pn[MAXPL][3], pc[MAXPL];  /* planes in the frame of v_s, with error bounds */
  Corner v[MAXV];
  int err;
} Poly;

/* corner of three planes: Cramer's rule with error bounds (frame of v_s) */
static void corner_make(Poly* P, Corner* q, int p0, int p1, int p2) {
  e64* A = P->pn[p0];
  e64* B = P->pn[p1];
  e64* C = P->pn[p2];
  e64 x12[3] = {sub64(mul64(B[1], C[2]), mul64(B[2], C[1])), sub64(mul64(B[2], C[0]), mul64(B[0], C[2])),
                sub64(mul64(B[0], C[1]), mul64(B[1], C[0]))};
  e64 x20[3] = {sub64(mul64(C[1], A[2]), mul64(C[2], A[1])), sub64(mul64(C[2], A[0]), mul64(C[0], A[2])),
                sub64(mul64(C[0], A[1]), mul64(C[1], A[0]))};
  e64 x01[3] = {sub64(mul64(A[1], B[2]), mul64(A[2], B[1])), sub64(mul64(A[2], B[0]), mul64(A[0], B[2])),
                sub64(mul64(A[0], B[1]), mul64(A[1], B[0]))};
  e64 D = add64(add64(mul64(A[0], x12[0]), mul64(A[1], x12[1])), mul64(A[2], x12[2]));
  double den = ad(D.v) - D.e, emax = 0;
  for (int d = 0; d < 3; ++d) {
    e64 num = add64(add64(mul64(P->pc[p0], x12[d]), mul64(P->pc[p1], x20[d])), mul64(P->pc[p2], x01[d]));
    q->x[d] = num.v / D.v;
    double e = den > 0 ? (num.e + ad(q->x[d]) * D.e) / den + 2 * U64 * ad(q->x[d]) : 1e300;
    if (e > emax) emax = e;
  }
  q->err = emax * (1 + 1e-9);
  q->p[0] = p0; q->p[1] = p1; q->p[2] = p2;
  q->nb[0] = q->nb[1] = q->nb[2] = -1;
  q->alive = 1; q->st = ST_UNK; q->wit = -1;
}

static int add_plane(sv_ctx* c, Poly* P, int src) {
  if (P->npl >= MAXPL) { P->err = 1; return -1; }
  int k = P->npl++;
  P->src[k] = src;
  plane_e64(c, P->s, P->a, src, P->pn[k], &P->pc[k]);
  return k;
}

/* P = T_a: tetrahedron (faces 0..3) or triangle (plane S, edges 0..2); corner k
 * is vertex k, on the facets other than k; across the edge that leaves facet g
 * out lies vertex g */
static void poly_simplex(sv_ctx* c, Poly* P, int a, int s) {
  P->a = a; P->s = s; P->npl = 0; P->nc = 0; P->err = 0;
  for (int d = 0; d < 3; ++d) P->o[d] = c->sites[3 * (size_t)s + d];
  const int32_t* sp = c->simp + (size_t)a * c->k;
  if (c->k == 4) {
    for (int f = 0; f < 4; ++f) add_plane(c, P, -1 - f);
    for (int k = 0; k < 4; ++k) {
      Corner* q = &P->v[P->nc++];
      int pl[3], t = 0;
      for (int f = 0; f < 4; ++f) if (f != k) pl[t++] = f;
      q->p[0] = pl[0]; q->p[1] = pl[1]; q->p[2] = pl[2];
      for (int d = 0; d < 3; ++d) q->x[d] = c->verts[3 * (size_t)sp[k] + d] - P->o[d];
      q->err = U64 * (ad(q->x[0]) + ad(q->x[1]) + ad(q->x[2]));
      q->alive = 1; q->st = ST_UNK; q->wit = -1;
      for (int x = 0; x < 3; ++x) q->nb[x] = pl[x];
    }
  } else {
    add_plane(c, P, SRC_S);
    for (int e = 0; e < 3; ++e) add_plane(c, P, -1 - e);
    for (int k = 0; k < 3; ++k) {
      Corner* q = &P->v[P->nc++];
      int pl[3] = {0, 0, 0}, t = 1;
      for (int e = 0; e < 3; ++e) if (e != k) pl[t++] = 1 + e;
      q->p[0] = pl[0]; q->p[1] = pl[1]; q->p[2] = pl[2];
      for (int d = 0; d < 3; ++d) q->x[d] = c->verts[3 * (size_t)sp[k] + d] - P->o[d];
      q->err = U64 * (ad(q->x[0]) + ad(q->x[1]) + ad(q->x[2]));
      q->alive = 1; q->st = ST_UNK; q->wit = -1;
      q->nb[0] = -1;
      q->nb[1] = pl[1] - 1;
      q->nb[2] = pl[2] - 1;
    }
  }
}

static int srcs_of(const Poly* P, const Corner* q, int out[3]) {
  for (int r = 0; r < 3; ++r) out[r] = P->src[q->p[r]];
  return 0;
}

/* Clip P by plane slot h (the half-space n.x <= c of site P->s).  Corners known
 * inside the cell (st == ST_IN) are inside every bisector of the site and are not
 * tested (Sec. 3.3).  Returns the number of corners removed, -1 if P is gone. */
static int poly_clip(sv_ctx* c, Poly* P, int h) {
  int s = P->s;
  int out[MAXV], nout = 0, nin = 0;
  int hsrc = P->src[h];
  for (int t = 0; t < P->nc; ++t) {
    Corner* q = &P->v[t];
    out[t] = 0;
    if (!q->alive) continue;
    if (q->st != ST_IN) {
      int sr[3];
      srcs_of(P, q, sr);
      out[t] = side_exact(c, s, P->a, sr, hsrc) < 0;
    }
    nout += out[t];
    nin += !out[t];
  }
  if (nout == 0) return 0;
  if (nin == 0) {
    for (int t = 0; t < P->nc; ++t) P->v[t].alive = 0;
    return -1;
  }
  /* new corners on the edges from a kept corner to a removed one */
  int first[MAXPL], second[MAXPL];
  for (int x = 0; x < P->npl; ++x) first[x] = second[x] = -1;
  int made[MAXV], nm = 0, nc0 = P->nc;
  for (int t = 0; t < nc0; ++t) {
    Corner* u = &P->v[t];
    if (!u->alive || out[t]) continue;
    for (int k = 0; k < 3; ++k) {
      int w = u->nb[k];
      if (w < 0 || !out[w]) continue;
      if (P->nc >= MAXV) { P->err = 1; return -1; }
      int e0 = u->p[(k + 1) % 3], e1 = u->p[(k + 2) % 3];
      int nt = P->nc++;
      Corner* q = &P->v[nt];
      out[nt] = 0;
      corner_make(P, q, e0, e1, h);
      q->nb[2] = t;           /* across the edge (e0, e1) */
      u->nb[k] = nt;
      made[nm++] = nt;
      for (int r = 0; r < 2; ++r) {
        int pl = r == 0 ? e0 : e1;
        if (first[pl] < 0) first[pl] = nt;
        else if (second[pl] < 0) second[pl] = nt;
        else P->err = 2;      /* not a simple polytope (degenerate input) */
      }
    }
  }
  /* link the new corners along the new face: corner (e0, e1, h) meets the other
   * new corner on plane e1 across the edge (e1, h), and on e0 across (e0, h) */
  for (int m = 0; m < nm; ++m) {
    Corner* q = &P->v[made[m]];
    for (int r = 0; r < 2; ++r) {
      int pl = q->p[r];       /* nb[0] is across (e1, h): found on plane e1 = p[1], and vice versa */
      int other = first[pl] == made[m] ? second[pl] : first[pl];
      q->nb[1 - r] = other;
    }
  }
  for (int t = 0; t < P->nc; ++t)
    if (out[t]) P->v[t].alive = 0;
  /* compact: keep slot numbers stable only within a clip */
  int map[MAXV], k = 0;
  for (int t = 0; t < P->nc; ++t) map[t] = P->v[t].alive ? k++ : -1;
  for (int t = 0; t < P->nc; ++t) {
    if (map[t] < 0) continue;
    Corner q = P->v[t];
    for (int r = 0; r < 3; ++r) q.nb[r] = q.nb[r] >= 0 ? map[q.nb[r]] : -1;
    P->v[map[t]] = q;
  }
  P->nc = k;
  return nout;
}

/* ---------------------------------------------------------------------------
 * point-in-cell test of a corner (Sec. 3.1)
 * ------------------------------------------------------------------------- */
/* returns ST_IN or ST_OUT; *wit = the certified closer site nearest to the corner.
 * The nearest site other than the corner's own flag sites comes first (a local
 * grid query); when it is certainly closer than v_s the corner is outside.
 * Otherwise every site within |q - v_s| (plus the error margin) is checked, the
 * ambiguous ones by the exact predicate. */
static int corner_test(sv_ctx* c, const Poly* P, const Corner* q, int s, int* wit) {
  double qg[3], ds2 = 0;
  for (int d = 0; d < 3; ++d) {
    qg[d] = q->x[d] + P->o[d];
    ds2 += q->x[d] * q->x[d];
  }
  int ex[3], psrc[3];
  for (int r = 0; r < 3; ++r) {
    psrc[r] = P->src[q->p[r]];
    ex[r] = psrc[r] >= 0 ? psrc[r] : -2;
  }
  const double err = q->err, rs = sqrt(ds2);
  c->stats[S_TESTS]++;
  /* f_k = |q - v_k|^2 - |q - v_s|^2 from the rounded corner, with its bound */
#define F_OF(K, F, BOUND)                                                                  \
  double F, BOUND;                                                                         \
  {                                                                                        \
    const double* v_ = c->sites + 3 * (size_t)(K);                                         \
    double da_ = 0;                                                                        \
    for (int d = 0; d < 3; ++d) {                                                          \
      double t_ = q->x[d] - (v_[d] - P->o[d]);                                             \
      da_ += t_ * t_;                                                                      \
    }                                                                                      \
    F = da_ - ds2;                                                                         \
    BOUND = 2.0 * 1.7320508075688772 * err * (sqrt(da_) + rs) + 3 * err * err + 8 * U64 * (da_ + ds2) + 1e-300; \
  }
  if (rs > 2 * local_h(c, qg)) {  /* far from its site (a simplex corner): the nearest site decides first */
    double d2;
    int k = nearest_ex(c, qg, ex[2], ex[0], ex[1], &d2);
    if (k >= 0 && k != s) {
      F_OF(k, f, bound);
      if (f < -bound) { *wit = k; return ST_OUT; }
    }
  }
  double bestf = 1e300;
  int best = -1;
  double r = rs + 4 * err + 1e-12 * (rs + ad(qg[0]) + ad(qg[1]) + ad(qg[2])) + 1e-300;
  FOR_BALL(c, qg, r, k, {
    if (k != s && k != ex[0] && k != ex[1] && k != ex[2]) {
      F_OF(k, f, bound);
      int closer = f < -bound ? 1 : (f > bound ? 0 : side_exact(c, s, P->a, psrc, k) < 0);
      if (closer && (f < bestf || (f == bestf && k < best))) { bestf = f; best = k; }
    }
  });
#undef F_OF
  *wit = best;
  return best >= 0 ? ST_OUT : ST_IN;
}

/* ---------------------------------------------------------------------------
 * Alg. 1 with the edge-based search of Sec. 3.2 (start point of Sec. 5.1)
 * ------------------------------------------------------------------------- */
/* Target bisector on the edge ps -> pt (ps inside Omega_s, the corner pt outside
 * with certified closer site wit).  ex0, ex1: the sites whose bisectors with s
 * contain the edge (-2: none); a point of the edge nearest to one of them is in
 * Omega_s by the flag rule of Sec. 3.1, so they are left out of its queries. */
static int find_bisector(sv_ctx* c, int s, const double* ps, const double* pt0, int wit, int ex0, int ex1) {
  const double* vs = c->sites + 3 * (size_t)s;
  double pt[3] = {pt0[0], pt0[1], pt0[2]};
  int j = wit;
  /* Sec. 5.1: g = ps + lambda delta dir, lambda = 2, 3, ... while NN(g) = s */
  double dir[3], len = 0;
  for (int d = 0; d < 3; ++d) { dir[d] = pt[d] - ps[d]; len += dir[d] * dir[d]; }
  len = sqrt(len);
  if (len > 0) {
    double del = c->delta[s];
    for (int lam = 2; lam < 66; ++lam) {
      double step = lam * del;
      if (!(step < len)) break;
      double g[3], d2;
      for (int d = 0; d < 3; ++d) g[d] = ps[d] + dir[d] / len * step;
      int k = nearest_ex(c, g, -1, ex0, ex1, &d2);
      if (k != s && k >= 0) { j = k; memcpy(pt, g, sizeof(pt)); break; }
    }
  }
  (void)vs;
  for (int it = 0; it < 256; ++it) {
    const double* vj = c->sites + 3 * (size_t)j;
    double n[3], cc = 0, a = 0, b = 0;
    for (int d = 0; d < 3; ++d) {
      n[d] = vj[d] - c->sites[3 * (size_t)s + d];
      cc += n[d] * (vj[d] + c->sites[3 * (size_t)s + d]);
      a += n[d] * ps[d];
      b += n[d] * (pt[d] - ps[d]);
    }
    cc *= 0.5;
    if (!(b > 0)) { c->stats[S_FALLBACK]++; return wit; }
    double t = (cc - a) / b;
    if (!(t < 1)) return j;
    if (t < 0) t = 0;
    double q[3], d2;
    for (int d = 0; d < 3; ++d) q[d] = ps[d] + t * (pt[d] - ps[d]);
    int k = nearest_ex(c, q, -1, ex0, ex1, &d2);
    c->stats[S_SEARCH]++;
    if (k == s || k == j || k < 0) return j;
    j = k;
    memcpy(pt, q, sizeof(pt));
  }
  c->stats[S_FALLBACK]++;
  return wit;
}

/* clips performed by the last alg1 call, by plane slot (to count the excess) */
static int alg1(sv_ctx* c, Poly* P, int s, unsigned char* clipped) {
  for (int guard = 0; guard < 4 * MAXPL; ++guard) {
    if (P->err) return -1;
    /* an edge p_s p_t with p_s inside and p_t outside: corners next to inside ones
     * are tested as they are met, until one is outside or no untested corner
     * borders an inside one (then every corner is inside: P is connected) */
    int su = -1, tw = -1, grew = 1;
    while (tw < 0 && grew) {
      grew = 0;
      for (int t = 0; t < P->nc && tw < 0; ++t) {
        Corner* u = &P->v[t];
        if (u->st != ST_IN) continue;
        for (int k = 0; k < 3 && tw < 0; ++k) {
          int w = u->nb[k];
          if (w < 0) continue;
          Corner* q = &P->v[w];
          if (q->st == ST_UNK) {
            q->st = corner_test(c, P, q, s, &q->wit);
            grew = 1;
          }
          if (q->st == ST_OUT) { su = t; tw = w; }
        }
      }
    }
    if (tw < 0) return 0;
    Corner* w = &P->v[tw];
    /* the edge's planes: the two planes the corners share (one besides S in a polygon) */
    int ex[2] = {-2, -2}, ne = 0;
    for (int r = 0; r < 3; ++r)
      for (int q2 = 0; q2 < 3; ++q2)
        if (P->v[su].p[r] == w->p[q2] && P->src[w->p[q2]] >= 0 && ne < 2) ex[ne++] = P->src[w->p[q2]];
    double ps[3], pt[3];
    for (int d = 0; d < 3; ++d) { ps[d] = P->v[su].x[d] + P->o[d]; pt[d] = w->x[d] + P->o[d]; }
    int j = find_bisector(c, s, ps, pt, w->wit, ex[0], ex[1]);
    int sr[3];
    srcs_of(P, w, sr);
    if (j < 0 || j == s || side_exact(c, s, P->a, sr, j) >= 0) {  /* must cut p_t: else the witness */
      c->stats[S_FALLBACK]++;
      j = w->wit;
    }
    int h = add_plane(c, P, j);
    if (h < 0) return -1;
    int r = poly_clip(c, P, h);
    c->stats[S_CLIPS]++;
    if (clipped) clipped[h] = 1;
    if (r < 0) return P->err ? -1 : 1;
  }
  P->err = 3;
  return -1;
}

/* ---------------------------------------------------------------------------
 * measures, faces and flags of a finished piece
 * ------------------------------------------------------------------------- */
typedef struct {
  int64_t np, cap, nf, fcap;
  int32_t *a, *i, *flags;
  double *meas, *m1, *fmeas;
  int64_t* foff;
} Out;

static int out_reserve(Out* O, int64_t np, int64_t nf) {
  if (np + 1 > O->cap) {
    int64_t cap = O->cap ? 2 * O->cap : 1024;
    while (cap < np + 1) cap *= 2;
    O->a = (int32_t*)realloc(O->a, sizeof(int32_t) * cap);
    O->i = (int32_t*)realloc(O->i, sizeof(int32_t) * cap);
    O->meas = (double*)realloc(O->meas, sizeof(double) * cap);
    O->m1 = (double*)realloc(O->m1, sizeof(double) * 3 * cap);
    O->foff = (int64_t*)realloc(O->foff, sizeof(int64_t) * (cap + 1));
    O->cap = cap;
    if (!O->a || !O->i || !O->meas || !O->m1 || !O->foff) return -1;
  }
  if (nf > O->fcap) {
    int64_t cap = O->fcap ? 2 * O->fcap : 4096;
    while (cap < nf) cap *= 2;
    O->flags = (int32_t*)realloc(O->flags, sizeof(int32_t) * cap);
    O->fmeas = (double*)realloc(O->fmeas, sizeof(double) * cap);
    O->fcap = cap;
    if (!O->flags || !O->fmeas) return -1;
  }
  return 0;
}

static void cross3(const double* a, const double* b, double* r) {
  r[0] = a[1] * b[2] - a[2] * b[1];
  r[1] = a[2] * b[0] - a[0] * b[2];
  r[2] = a[0] * b[1] - a[1] * b[0];
}

/* corners of the face on plane slot x in cyclic order (a polygon's edge: its
 * two corners); returns their count */
static int face_cycle(const Poly* P, int x, int* cyc) {
  int start = -1, cnt = 0;
  for (int t = 0; t < P->nc && start < 0; ++t)
    if (P->v[t].p[0] == x || P->v[t].p[1] == x || P->v[t].p[2] == x) start = t;
  if (start < 0) return 0;
  int prev = -1, cur = start;
  do {
    if (cnt >= MAXV) return -1;
    cyc[cnt++] = cur;
    const Corner* q = &P->v[cur];
    int nxt = -1;
    for (int k = 0; k < 3 && nxt < 0; ++k) {
      if (q->p[k] == x) continue;  /* that edge leaves the face */
      int w = q->nb[k];
      if (w >= 0 && w != prev) nxt = w;
    }
    prev = cur;
    cur = nxt;
  } while (cur >= 0 && cur != start);
  return cnt;
}

/* measure of the face on every plane slot (area in 3D, length of a polygon's
 * edge; 0 when the plane bounds no face of positive measure).  exact: no sign
 * decision of the piece was a tie or uncertain, so the piece is a simple
 * polytope (polygon) and every plane holding a face cycle bounds a face of
 * positive measure, however small its float64 value (the smallest normal
 * double stands in for one that rounds to zero). */
static void face_measures(const sv_ctx* c, const Poly* P, double* fm, int exact) {
  int cyc[MAXV];
  int polygon = c->k == 3;
  for (int x = 0; x < P->npl; ++x) {
    fm[x] = 0;
    if (polygon && x == 0) continue;  /* the polygon's own plane S */
    int n = face_cycle(P, x, cyc);
    if (polygon) {
      if (n == 2) {
        double l2 = 0;
        for (int d = 0; d < 3; ++d) {
          double t = P->v[cyc[1]].x[d] - P->v[cyc[0]].x[d];
          l2 += t * t;
        }
        fm[x] = sqrt(l2);
      }
    } else if (n >= 3) {
      double sum[3] = {0, 0, 0};
      for (int t = 1; t + 1 < n; ++t) {
        double e1[3], e2[3], cr[3];
        for (int d = 0; d < 3; ++d) {
          e1[d] = P->v[cyc[t]].x[d] - P->v[cyc[0]].x[d];
          e2[d] = P->v[cyc[t + 1]].x[d] - P->v[cyc[0]].x[d];
        }
        cross3(e1, e2, cr);
        for (int d = 0; d < 3; ++d) sum[d] += cr[d];
      }
      fm[x] = 0.5 * sqrt(sum[0] * sum[0] + sum[1] * sum[1] + sum[2] * sum[2]);
    }
    if (exact && !(fm[x] > 0) && n >= (polygon ? 2 : 3)) fm[x] = 2.2250738585072014e-308;
  }
}

static int32_t flag_of(const sv_ctx* c, int a, int src) {
  if (src >= 0) return src;
  int b = c->adj[(size_t)a * c->k + (-1 - src)];
  return b >= 0 ? -(b + 1) : FLAG_BND;
}

/* Record the piece P (site s): measure (area by a triangle fan / volume by a
 * fan of tetrahedra around the corners' mean), first moment in the frame of
 * v_s, and the flags of its faces of positive measure.  clipped[x]: plane x was
 * added by a clip of Alg. 1 (for the count of clips that left no face). */
static double piece_emit(sv_ctx* c, const Poly* P, int s, Out* O, const double* fm, const unsigned char* clipped,
                         int exact) {
  int cyc[MAXV];
  double meas = 0, m1[3] = {0, 0, 0};
  int64_t p = O->np;
  if (out_reserve(O, p + 1, O->nf + MAXPL)) return -1;
  O->foff[p] = O->nf;
  if (c->k == 3) {
    int n = P->nc >= 3 ? face_cycle(P, 0, cyc) : 0;  /* plane 0 (S) holds every corner */
    for (int t = 1; t + 1 < n; ++t) {
      double e1[3], e2[3], cr[3];
      for (int d = 0; d < 3; ++d) {
        e1[d] = P->v[cyc[t]].x[d] - P->v[cyc[0]].x[d];
        e2[d] = P->v[cyc[t + 1]].x[d] - P->v[cyc[0]].x[d];
      }
      cross3(e1, e2, cr);
      double ar = 0.5 * sqrt(cr[0] * cr[0] + cr[1] * cr[1] + cr[2] * cr[2]);
      meas += ar;
      for (int d = 0; d < 3; ++d)
        m1[d] += ar * ((P->v[cyc[0]].x[d] + P->v[cyc[t]].x[d] + P->v[cyc[t + 1]].x[d]) / 3.0);
    }
  } else if (P->nc >= 4) {
    double ref[3] = {0, 0, 0};
    for (int t = 0; t < P->nc; ++t)
      for (int d = 0; d < 3; ++d) ref[d] += P->v[t].x[d] / P->nc;
    for (int x = 0; x < P->npl; ++x) {
      if (!(fm[x] > 0)) continue;
      int n = face_cycle(P, x, cyc);
      for (int t = 1; t + 1 < n; ++t) {
        double a[3], b[3], e[3], cr[3];
        for (int d = 0; d < 3; ++d) {
          a[d] = P->v[cyc[0]].x[d] - ref[d];
          b[d] = P->v[cyc[t]].x[d] - ref[d];
          e[d] = P->v[cyc[t + 1]].x[d] - ref[d];
        }
        cross3(b, e, cr);
        double v = ad(a[0] * cr[0] + a[1] * cr[1] + a[2] * cr[2]) / 6.0;
        meas += v;
        for (int d = 0; d < 3; ++d)
          m1[d] += v * ((ref[d] + P->v[cyc[0]].x[d] + P->v[cyc[t]].x[d] + P->v[cyc[t + 1]].x[d]) / 4.0);
      }
    }
  }
  if (exact && !(meas > 0) && P->nc >= (c->k == 3 ? 3 : 4)) {
    /* positive in exact arithmetic, below float64 resolution */
    meas = 2.2250738585072014e-308;
    m1[0] = m1[1] = m1[2] = 0;
  }
  int nclip = 0, contrib = 0;
  for (int x = 0; x < P->npl; ++x) nclip += clipped[x];
  if (meas > 0) {
    for (int x = 0; x < P->npl; ++x) {
      if (!(fm[x] > 0)) continue;
      O->flags[O->nf] = flag_of(c, P->a, P->src[x]);
      O->fmeas[O->nf] = fm[x];
      O->nf++;
      if (P->src[x] >= 0) c->stats[S_FACES]++;
      contrib += clipped[x];
    }
  }
  c->stats[S_EXCESS] += nclip - contrib;
  O->a[p] = P->a;
  O->i[p] = s;
  O->meas[p] = meas > 0 ? meas : 0;
  for (int d = 0; d < 3; ++d) O->m1[3 * p + d] = meas > 0 ? m1[d] : 0;
  O->np = p + 1;
  O->foff[O->np] = O->nf;
  return meas;
}

/* ---------------------------------------------------------------------------
 * Alg. 2
 * ------------------------------------------------------------------------- */
typedef struct { int j, u, nadj; int adj[MAXPL]; } Job;

/* the tuple (u, f) of the face on plane x of the piece P_{a,u} (flag j): the
 * positive flags w of the faces adjacent to it (planes sharing a corner with it) */
static void job_from_face(const Poly* P, const double* fm, int x, int u, Job* J) {
  J->j = P->src[x];
  J->u = u;
  J->nadj = 0;
  for (int t = 0; t < P->nc; ++t) {
    const Corner* q = &P->v[t];
    if (q->p[0] != x && q->p[1] != x && q->p[2] != x) continue;
    for (int r = 0; r < 3; ++r) {
      int y = q->p[r];
      if (y == x || P->src[y] < 0 || !(fm[y] > 0)) continue;
      int w = P->src[y], dup = 0;
      for (int k = 0; k < J->nadj; ++k) dup |= J->adj[k] == w;
      if (!dup && J->nadj < MAXPL) J->adj[J->nadj++] = w;
    }
  }
}

typedef struct { Job* q; int64_t n, head, cap; } JobQ;

static int queue_faces(sv_ctx* c, const Poly* P, const double* fm, int a, int u, JobQ* Q) {
  for (int x = 0; x < P->npl; ++x) {
    int j = P->src[x];
    if (j < 0 || !(fm[x] > 0) || c->stamp[j] == a) continue;
    c->stamp[j] = a;
    if (Q->n >= Q->cap) {
      Q->cap = Q->cap ? 2 * Q->cap : 256;
      Q->q = (Job*)realloc(Q->q, sizeof(Job) * (size_t)Q->cap);
      if (!Q->q) return -1;
    }
    job_from_face(P, fm, x, u, &Q->q[Q->n++]);
  }
  return 0;
}

/* Alg. 2 on simplex a: the first piece from the nearest site of the first
 * corner, then the queue over positive flags */
static int simplex_pieces(sv_ctx* c, int a, Out* O, Poly* buf, JobQ* Q) {
  Poly* P = &buf[0];
  Poly* G = &buf[1];
  const double* c0 = c->verts + 3 * (size_t)c->simp[(size_t)a * c->k];
  double d2, fm[MAXPL];
  unsigned char clipped[MAXPL];
  int i = nearest(c, c0, -1, &d2);
  if (i < 0) return -1;
  int64_t und = c->stats[S_TIES] + c->stats[S_UNCERTAIN];  /* undecided signs before the piece */
  for (int guard = 0;; ++guard) {  /* the first corner lies in Omega_i (ties: inside) */
    int wit;
    poly_simplex(c, P, a, i);
    if (corner_test(c, P, &P->v[0], i, &wit) == ST_IN) break;
    if (guard == 16 || wit < 0) return -1;
    i = wit;
  }
  P->v[0].st = ST_IN;
  Q->n = Q->head = 0;
  c->stamp[i] = a;
  memset(clipped, 0, sizeof(clipped));
  if (alg1(c, P, i, clipped) < 0) return -1;
  int exact = c->stats[S_TIES] + c->stats[S_UNCERTAIN] == und;
  face_measures(c, P, fm, exact);
  double m = piece_emit(c, P, i, O, fm, clipped, exact);
  if (m < 0) return -1;
  if (m > 0 && queue_faces(c, P, fm, a, i, Q)) return -1;
  while (Q->head < Q->n) {
    Job J = Q->q[Q->head++];
    int j = J.j;
    /* G_{a,j}: T_a clipped by B_{j,u} and by B_{j,w} for the faces adjacent to f */
    und = c->stats[S_TIES] + c->stats[S_UNCERTAIN];
    poly_simplex(c, G, a, j);
    int h = add_plane(c, G, J.u), r = 0, hu = h;
    if (h < 0) return -1;
    r = poly_clip(c, G, h);
    c->stats[S_GCLIPS]++;
    for (int k = 0; k < J.nadj && r >= 0; ++k) {
      if (J.adj[k] == j) continue;
      h = add_plane(c, G, J.adj[k]);
      if (h < 0) return -1;
      r = poly_clip(c, G, h);
      c->stats[S_GCLIPS]++;
    }
    if (G->err) return -1;
    if (r < 0) { c->stats[S_ERROR]++; continue; }  /* G empty: cannot happen for a face of positive measure */
    /* a corner of G on B_{j,u} (a corner of f) lies in Omega_j: Alg. 1 starts there */
    int started = 0;
    for (int t = 0; t < G->nc && !started; ++t) {
      Corner* q = &G->v[t];
      if (q->p[0] != hu && q->p[1] != hu && q->p[2] != hu) continue;
      q->st = corner_test(c, G, q, j, &q->wit);
      started = q->st == ST_IN;
    }
    if (!started) { c->stats[S_ERROR]++; continue; }
    memset(clipped, 0, sizeof(clipped));
    if (alg1(c, G, j, clipped) < 0) return -1;
    exact = c->stats[S_TIES] + c->stats[S_UNCERTAIN] == und;
    face_measures(c, G, fm, exact);
    m = piece_emit(c, G, j, O, fm, clipped, exact);
    if (m < 0) return -1;
    if (m > 0 && queue_faces(c, G, fm, a, j, Q)) return -1;
  }
  return 0;
}

/* ---------------------------------------------------------------------------
 * C interface (paper_2509_07175_b300/serial.py)
 * ------------------------------------------------------------------------- */
typedef struct {
  int64_t np;
  int32_t *a, *i;
  double *meas, *m1;
  int64_t* foff;
  int32_t* flags;
  double* fmeas;
  int64_t stats[12];
  int status;
} sv_result;

typedef struct { int32_t v[3]; int32_t a, f; } FKey;

static int fkey_cmp(const void* x, const void* y) {
  const FKey* p = (const FKey*)x;
  const FKey* q = (const FKey*)y;
  for (int d = 0; d < 3; ++d)
    if (p->v[d] != q->v[d]) return p->v[d] < q->v[d] ? -1 : 1;
  return 0;
}

void sv_destroy(sv_ctx* c);

/* mode 2 (planar triangles, z = 0), 3 (surface triangles), 4 (tetrahedra);
 * arrays are copied.  NULL on a bad mesh (an index out of range, a facet shared
 * by more than two simplices) or no memory. */
sv_ctx* sv_create(int mode, int64_t n, const double* sites, int64_t nv, const double* verts, int64_t m,
                  const int32_t* simp) {
  if (n < 1 || m < 1 || (mode != M2D && mode != MSURF && mode != M3D)) return NULL;
  sv_ctx* c = (sv_ctx*)calloc(1, sizeof(sv_ctx));
  if (!c) return NULL;
  c->mode = mode;
  c->k = mode == M3D ? 4 : 3;
  c->n = n; c->nv = nv; c->m = m;
  c->sites = (double*)malloc(sizeof(double) * 3 * (size_t)n);
  c->verts = (double*)malloc(sizeof(double) * 3 * (size_t)nv);
  c->simp = (int32_t*)malloc(sizeof(int32_t) * (size_t)m * c->k);
  c->adj = (int32_t*)malloc(sizeof(int32_t) * (size_t)m * c->k);
  c->delta = (double*)malloc(sizeof(double) * (size_t)n);
  c->stamp = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
  FKey* F = (FKey*)malloc(sizeof(FKey) * (size_t)m * c->k);
  if (!c->sites || !c->verts || !c->simp || !c->adj || !c->delta || !c->stamp || !F) { free(F); sv_destroy(c); return NULL; }
  memcpy(c->sites, sites, sizeof(double) * 3 * (size_t)n);
  memcpy(c->verts, verts, sizeof(double) * 3 * (size_t)nv);
  memcpy(c->simp, simp, sizeof(int32_t) * (size_t)m * c->k);
  for (int64_t t = 0; t < m * c->k; ++t)
    if (simp[t] < 0 || simp[t] >= nv) { free(F); sv_destroy(c); return NULL; }
  /* simplex adjacency across facets (facet f: the vertices other than f) */
  for (int64_t a = 0; a < m; ++a)
    for (int f = 0; f < c->k; ++f) {
      FKey* q = &F[a * c->k + f];
      int t = 0;
      for (int l = 0; l < c->k; ++l) if (l != f) q->v[t++] = simp[a * c->k + l];
      if (t == 2) q->v[2] = -1;
      for (int x = 0; x < t; ++x)
        for (int y = x + 1; y < t; ++y)
          if (q->v[y] < q->v[x]) { int32_t z = q->v[x]; q->v[x] = q->v[y]; q->v[y] = z; }
      q->a = (int32_t)a; q->f = f;
      c->adj[a * c->k + f] = -1;
    }
  qsort(F, (size_t)m * c->k, sizeof(FKey), fkey_cmp);
  for (int64_t t = 0; t < m * c->k;) {
    int64_t u = t + 1;
    while (u < m * c->k && fkey_cmp(&F[t], &F[u]) == 0) ++u;
    if (u - t > 2) { free(F); sv_destroy(c); return NULL; }
    if (u - t == 2) {
      c->adj[(int64_t)F[t].a * c->k + F[t].f] = F[t + 1].a;
      c->adj[(int64_t)F[t + 1].a * c->k + F[t + 1].f] = F[t].a;
    }
    t = u;
  }
  free(F);
  if (grids_build(c)) { sv_destroy(c); return NULL; }
  for (int64_t i = 0; i < n; ++i) {
    double d2;
    int k = nearest(c, c->sites + 3 * i, (int)i, &d2);
    c->delta[i] = k >= 0 ? 0.5 * sqrt(d2) : 1.0;
    c->stamp[i] = -1;
  }
  memset(c->stats, 0, sizeof(c->stats));
  return c;
}

void sv_destroy(sv_ctx* c) {
  if (!c) return;
  grid_free(&c->g);
  for (int k = 0; k < c->nfine; ++k) grid_free(&c->fine[k]);
  free(c->fine);
  free(c->sites); free(c->verts); free(c->simp); free(c->adj); free(c->delta); free(c->stamp);
  free(c);
}

static sv_result* run_simplices(sv_ctx* c, int64_t a0, int64_t a1, const int64_t* list, int64_t nlist);

/* Alg. 2 over the simplices [a0, a1): a piece for each site reached (empty ones
 * included, with measure 0), with counters */
sv_result* sv_run(sv_ctx* c, int64_t a0, int64_t a1) { return run_simplices(c, a0, a1, NULL, 0); }

/* the same over a list of simplex indices (a sample of the mesh) */
sv_result* sv_run_list(sv_ctx* c, const int64_t* list, int64_t nlist) { return run_simplices(c, 0, 0, list, nlist); }

static sv_result* run_simplices(sv_ctx* c, int64_t a0, int64_t a1, const int64_t* list, int64_t nlist) {
  sv_result* R = (sv_result*)calloc(1, sizeof(sv_result));
  Poly* buf = (Poly*)malloc(2 * sizeof(Poly));
  JobQ Q = {NULL, 0, 0, 0};
  Out O;
  memset(&O, 0, sizeof(O));
  if (!R || !buf) { free(R); free(buf); return NULL; }
  memset(c->stats, 0, sizeof(c->stats));
  for (int64_t i = 0; i < c->n; ++i) c->stamp[i] = -1;  /* visit marks are per simplex and per run */
  if (a0 < 0) a0 = 0;
  if (a1 > c->m) a1 = c->m;
  if (a1 < a0) a1 = a0;
  int status = 0;
  int64_t cnt = list ? nlist : a1 - a0;
  for (int64_t t = 0; t < cnt; ++t) {
    int64_t a = list ? list[t] : a0 + t;
    if (a < 0 || a >= c->m) { status = -1; continue; }
    if (simplex_pieces(c, (int)a, &O, buf, &Q)) { status = -1; c->stats[S_ERROR]++; }
  }
  if (out_reserve(&O, O.np + 1, O.nf + 1)) status = -2;
  if (!O.foff) { O.foff = (int64_t*)calloc(1, sizeof(int64_t)); }
  R->np = O.np;
  R->a = O.a; R->i = O.i; R->meas = O.meas; R->m1 = O.m1; R->foff = O.foff;
  R->flags = O.flags; R->fmeas = O.fmeas;
  memcpy(R->stats, c->stats, sizeof(R->stats));
  R->status = status;
  free(buf);
  free(Q.q);
  return R;
}

void sv_free_result(sv_result* R) {
  if (!R) return;
  free(R->a); free(R->i); free(R->meas); free(R->m1); free(R->foff); free(R->flags); free(R->fmeas);
  free(R);
}
