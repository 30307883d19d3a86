// vd_clip3.cuh -- tetrahedron / Voronoi-cell intersection, one warp per pair.
//
// The working polytope P (Sec. 5.3) is kept as a triangulated dual mesh in the
// warp's shared memory: each plane (tet face or bisector) is a dual vertex,
// each corner of P -- the meeting point of three planes -- is a dual triangle,
// stored with its three neighbours.  Clipping by a bisector removes the
// connected set R_p of outside corners that contains the chosen outside corner
// p, walks the boundary of R_p and fans new corners to the new plane
// (Sec. 5.3).  Alg. 3 drives the clipping: while a corner p lies outside
// Omega_i, find a bisector on the virtual edge v_i -> p (Sec. 3.2, improved
// start point of Sec. 5.1) and clip by it.
//
// Geometry is FP32 in the frame of v_i.  Every corner carries a bound on the
// error of its coordinates; side tests that do not clear their bound are
// settled by the float64 predicate on the defining planes (vd_common.cuh).
//
// The helpers run on every clip (search, clip, integration, nearest-site query)
// are inlined into the pair loop: as out-of-line calls each paid a save and a
// restore of its registers through local memory (10-12 % of the kernel's time
// on the shell, the 100k cube and the 5M box).  Only the float64 paths, which
// run for a few per cent of the decisions, stay out of line.
#pragma once

#include "vd_dev.cuh"

namespace vd {
namespace c3 {

constexpr int MAXP = 48;   // planes
constexpr int MAXT = 96;   // corners (3 x 32 slots)
constexpr float U = 5.9604644775390625e-8f;
constexpr float GAMMA = 64.f * U;   // corner error factor (see corner())
constexpr float SIDEF = 24.f * U;   // side-test error factor

struct Warp3 {
  float4 pn[MAXP];      // n.xyz, c : inside is n.x <= c
  float2 pm[MAXP];      // magnitudes: |n~|_1 and c~ (absolute-value evaluation)
  int psrc[MAXP];       // >= 0: bisector with that site; -1-f: face f of the tetrahedron
  uchar4 tv[MAXT];      // the corner's planes x, y, z (dual triangle, oriented)
  uchar4 tn[MAXT];      // neighbour corners across dual edges x->y, y->z, z->x
  float4 tq[MAXT];      // corner coordinates (frame of v_i), w = coordinate error bound
  int twit[MAXT];       // certified closer site of an outside corner
  mutable int tied;     // this pair met an exact tie or an uncertain sign (see process_pair)
  int stri[MAXP], etri[MAXP];  // boundary loop: new corner starting / ending at a plane
  int pref[MAXP];       // reference corner of each face (integration)
  float parea[MAXP][3]; // face vector areas
  unsigned long long pkey[MAXP];  // smallest corner key of each face (integration)
  unsigned char prank[MAXP];      // rank of each face among the faces by source (integration)
  float4 contrib[MAXT]; // volume / moment terms by corner rank (integration)
  ScanScratch S;
};

// warp-uniform bookkeeping (identical in every lane)
struct Masks {
  unsigned alive[3], in[3], out[3];
  unsigned long long palive;
};

// bit t of a 96-bit mask held as three words (selects, not a run-time array index,
// so that masks in registers stay there)
__device__ __forceinline__ bool bit(const unsigned* m, int t) {
  unsigned w = t < 32 ? m[0] : (t < 64 ? m[1] : m[2]);
  return (w >> (t & 31)) & 1u;
}

__device__ __forceinline__ int nth_set(unsigned m, int k) {
  int pos = 0;
#pragma unroll
  for (int w = 16; w; w >>= 1) {
    unsigned lo = m & ((1u << w) - 1u);
    int c = __popc(lo);
    if (k >= c) { k -= c; m >>= w; pos += w; } else m = lo;
  }
  return pos;
}

// ----- planes --------------------------------------------------------------
// tet face f: the plane through the three vertices other than f, oriented by
// fsgn so that its normal points away from vertex f
__device__ __forceinline__ void face_verts(int f, int& a0, int& a1, int& a2) {
  a0 = f == 0 ? 1 : 0;
  a1 = f <= 1 ? 2 : 1;
  a2 = f <= 2 ? 3 : 2;
}

// pairs whose polytope starts as the box [blo, bhi]: every pair of the box form,
// and the whole-cell pairs (m, i) of the split
__device__ __forceinline__ bool box_pair(const Dev<float>& C, int a) { return C.box || a == C.m; }

// box face f (axis f/2, lower bound for even f): inside is n.x <= c
__device__ __forceinline__ void plane_box(const Dev<float>& C, int f, float3 vi, float4& P, float2& M) {
  int ax = f >> 1;
  float s = (f & 1) ? 1.f : -1.f;
  float b = (f & 1) ? C.bhi[ax] : C.blo[ax];
  float v = ax == 0 ? vi.x : (ax == 1 ? vi.y : vi.z);
  float c = s * (b - v);
  P = make_float4(ax == 0 ? s : 0.f, ax == 1 ? s : 0.f, ax == 2 ? s : 0.f, c);
  M = make_float2(1.f, fabsf(b - v));
}

__device__ void plane_face(const Dev<float>& C, int a, int f, float3 vi, float4& P, float2& M) {
  if (box_pair(C, a)) { plane_box(C, f, vi, P, M); return; }
  int l0, l1, l2;
  face_verts(f, l0, l1, l2);
  const int* s = C.simp + 4 * a;
  const float* A = C.verts + 3 * s[l0];
  const float* B = C.verts + 3 * s[l1];
  const float* Cc = C.verts + 3 * s[l2];
  float sg = (float)C.fsgn[4 * a + f];
  float e1x = B[0] - A[0], e1y = B[1] - A[1], e1z = B[2] - A[2];
  float e2x = Cc[0] - A[0], e2y = Cc[1] - A[1], e2z = Cc[2] - A[2];
  float nx = sg * (e1y * e2z - e1z * e2y), ny = sg * (e1z * e2x - e1x * e2z), nz = sg * (e1x * e2y - e1y * e2x);
  float ax = A[0] - vi.x, ay = A[1] - vi.y, az = A[2] - vi.z;
  float mx = fabsf(e1y * e2z) + fabsf(e1z * e2y), my = fabsf(e1z * e2x) + fabsf(e1x * e2z),
        mz = fabsf(e1x * e2y) + fabsf(e1y * e2x);
  P = make_float4(nx, ny, nz, nx * ax + ny * ay + nz * az);
  M = make_float2(mx + my + mz, mx * fabsf(ax) + my * fabsf(ay) + mz * fabsf(az));
}

__device__ __forceinline__ void plane_bis_at(float sx, float sy, float sz, float3 vi, float4& P, float2& M) {
  float wx = sx - vi.x, wy = sy - vi.y, wz = sz - vi.z;
  float c = 0.5f * (wx * wx + wy * wy + wz * wz);
  P = make_float4(wx, wy, wz, c);
  M = make_float2(fabsf(wx) + fabsf(wy) + fabsf(wz), c);
}

__device__ __forceinline__ void plane_bis(const Dev<float>& C, int j, float3 vi, float4& P, float2& M) {
  plane_bis_at(C.sites[3 * j], C.sites[3 * j + 1], C.sites[3 * j + 2], vi, P, M);
}

// float64 plane from its source, with running error bounds
__device__ __noinline__ ePlane eplane(const Dev<float>& C, int a, int i, int src) {
  ed3 vi{mk(C.sites[3 * i]), mk(C.sites[3 * i + 1]), mk(C.sites[3 * i + 2])};
  ePlane p;
  if (src >= 0) {
    ed3 vj{mk(C.sites[3 * src]), mk(C.sites[3 * src + 1]), mk(C.sites[3 * src + 2])};
    p.n = sub3(vj, vi);
    ed w2 = dot3(p.n, p.n);
    if (C.lift) {  // power bisector: (|v_j - v_i|^2 + h_j^2 - h_i^2) / 2
      ed hj = mk(C.lift[src]), hi = mk(C.lift[i]);
      w2 = w2 + (hj * hj - hi * hi);
    }
    p.c = half(w2);
    return p;
  }
  int f = -1 - src, l0, l1, l2;
  if (box_pair(C, a)) {
    int ax = f >> 1;
    double sg = (f & 1) ? 1.0 : -1.0;
    double b = (f & 1) ? (double)C.bhi[ax] : (double)C.blo[ax];
    ed v = ax == 0 ? vi.x : (ax == 1 ? vi.y : vi.z);
    p.n = ed3{mk(ax == 0 ? sg : 0.0), mk(ax == 1 ? sg : 0.0), mk(ax == 2 ? sg : 0.0)};
    ed d = mk(b) - v;
    p.c = ed{sg * d.v, d.e};
    return p;
  }
  face_verts(f, l0, l1, l2);
  const int* s = C.simp + 4 * a;
  const float* A = C.verts + 3 * s[l0];
  const float* B = C.verts + 3 * s[l1];
  const float* Cc = C.verts + 3 * s[l2];
  ed3 eA{mk(A[0]), mk(A[1]), mk(A[2])}, eB{mk(B[0]), mk(B[1]), mk(B[2])}, eC{mk(Cc[0]), mk(Cc[1]), mk(Cc[2])};
  p.n = scale3(cross3(sub3(eB, eA), sub3(eC, eA)), (double)C.fsgn[4 * a + f]);
  p.c = dot3(p.n, sub3(eA, vi));
  return p;
}

// ----- corners ---------------------------------------------------------------
// Corner of three planes by Cramer's rule.  With D = det N and A = adj(N) c,
// |D^ - D| <= g D~ and |A^ - A| <= g A~, where ~ is the same expression on
// absolute values (bounded here by products of the planes' magnitudes) and g
// covers the rounding of the plane coefficients and of the evaluation; then
// |q^ - q| <= (g A~ + |q| g D~) / (|D^| - g D~) + 2u|q|.  Corners whose D does
// not clear its bound get an infinite error: every test on them is exact.
// Every operation is an explicitly rounded intrinsic (no contraction into fused
// multiply-adds), so each call site rounds a corner identically whatever the
// compiler inlines around it.
__device__ __forceinline__ float4 corner(float4 P0, float2 M0, float4 P1, float2 M1, float4 P2, float2 M2) {
  auto cr = [](float ay, float az, float by, float bz) { return __fsub_rn(__fmul_rn(ay, bz), __fmul_rn(az, by)); };
  auto dot = [](float ax, float ay, float az, float bx, float by, float bz) {
    return __fadd_rn(__fadd_rn(__fmul_rn(ax, bx), __fmul_rn(ay, by)), __fmul_rn(az, bz));
  };
  float3 x12 = make_float3(cr(P1.y, P1.z, P2.y, P2.z), cr(P1.z, P1.x, P2.z, P2.x), cr(P1.x, P1.y, P2.x, P2.y));
  float3 x20 = make_float3(cr(P2.y, P2.z, P0.y, P0.z), cr(P2.z, P2.x, P0.z, P0.x), cr(P2.x, P2.y, P0.x, P0.y));
  float3 x01 = make_float3(cr(P0.y, P0.z, P1.y, P1.z), cr(P0.z, P0.x, P1.z, P1.x), cr(P0.x, P0.y, P1.x, P1.y));
  float D = dot(P0.x, P0.y, P0.z, x12.x, x12.y, x12.z);
  float qx = __fdiv_rn(dot(P0.w, P1.w, P2.w, x12.x, x20.x, x01.x), D);
  float qy = __fdiv_rn(dot(P0.w, P1.w, P2.w, x12.y, x20.y, x01.y), D);
  float qz = __fdiv_rn(dot(P0.w, P1.w, P2.w, x12.z, x20.z, x01.z), D);
  float Dm = __fmul_rn(__fmul_rn(M0.x, M1.x), M2.x);
  float Am = __fadd_rn(__fadd_rn(__fmul_rn(__fmul_rn(M0.y, M1.x), M2.x), __fmul_rn(__fmul_rn(M1.y, M2.x), M0.x)),
                       __fmul_rn(__fmul_rn(M2.y, M0.x), M1.x));
  float qm = fmaxf(fabsf(qx), fmaxf(fabsf(qy), fabsf(qz)));
  float gD = __fmul_rn(GAMMA, Dm);
  float den = __fsub_rn(fabsf(D), gD);
  float e = (den > gD && isfinite(qm))
                ? __fadd_rn(__fdiv_rn(__fadd_rn(__fmul_rn(GAMMA, Am), __fmul_rn(qm, gD)), den), __fmul_rn(2.f * U, qm))
                : 1e30f;
  return make_float4(qx, qy, qz, e);
}

// A corner whose FP32 error bound exceeds 3e-3 |q| is recomputed in float64 (the
// test is explicitly rounded so that every mapping takes the same decision).
__device__ __forceinline__ bool loose(float4 q) {
  float n2 = __fadd_rn(__fadd_rn(__fmul_rn(q.x, q.x), __fmul_rn(q.y, q.y)), __fmul_rn(q.z, q.z));
  return !(q.w <= __fmul_rn(3e-3f, __fsqrt_rn(n2)));
}

// loose FP32 bound: recompute the corner from its exact planes in float64
__device__ __noinline__ float4 refine64(const Dev<float>& C, int a, int i, int s0, int s1, int s2) {
  atomicAdd(C.stats + VD_STAT_FP64, 1ull);
  return corner64(eplane(C, a, i, s0), eplane(C, a, i, s1), eplane(C, a, i, s2));
}

// ----- exact side tests ----------------------------------------------------------
__device__ __noinline__ int exact_side(const Dev<float>& C, const Warp3& W, int a, int i, int t, int src4) {
  ePlane p[4];
  uchar4 v = W.tv[t];
  // the corner lies on each of its own planes: the side value is exactly zero
  if (src4 == W.psrc[v.x] || src4 == W.psrc[v.y] || src4 == W.psrc[v.z]) return 0;
  p[0] = eplane(C, a, i, W.psrc[v.x]);
  p[1] = eplane(C, a, i, W.psrc[v.y]);
  p[2] = eplane(C, a, i, W.psrc[v.z]);
  p[3] = eplane(C, a, i, src4);
  int certain, tie;
  int s = side_from_planes(p, &certain, &tie);
  atomicAdd(C.stats + VD_STAT_FP64, 1ull);
  if (!certain) {
    atomicAdd(C.stats + (tie ? VD_STAT_TIES : VD_STAT_UNCERTAIN), 1ull);
    record_diag(C.stats, a, i, W.psrc[v.x], W.psrc[v.y], W.psrc[v.z], src4, tie, 0);
    return s < 0 ? -2 : 2;  // not certified: +-2 (a tie counts as inside)
  }
  return s;
}

// side of corner t w.r.t. plane P (slot pl): -1 outside, +1 inside, 0 on it; +-2 a
// decision that is a tie (+2, inside) or left uncertain, after which the pair's
// positivity follows the computed measures
__device__ __forceinline__ int side_of(const Dev<float>& C, const Warp3& W, int a, int i, int t, int pl) {
  float4 q = W.tq[t];
  float4 P = W.pn[pl];
  float2 M = W.pm[pl];
  if (q.w < 1e29f && !C.force_exact) {
    float s = P.w - (P.x * q.x + P.y * q.y + P.z * q.z);
    float qm = fmaxf(fabsf(q.x), fmaxf(fabsf(q.y), fabsf(q.z)));
    float b = (fabsf(P.x) + fabsf(P.y) + fabsf(P.z)) * q.w + SIDEF * (M.y + M.x * qm);
    if (s > b) return 1;
    if (s < -b) return -1;
  }
  int r = exact_side(C, W, a, i, t, W.psrc[pl]);
  if (r == 2 || r == -2) W.tied = 1;
  return r;
}

// ----- one pair ------------------------------------------------------------------
struct Counters {
  unsigned nn, corner, clips, lam, search, learned, fallback, list;
  unsigned long long scanned;
};

__device__ __forceinline__ void add_plane(Warp3& W, int slot, float4 P, float2 M, int src, int lane) {
  __syncwarp();
  if (lane == 0) { W.pn[slot] = P; W.pm[slot] = M; W.psrc[slot] = src; }
  __syncwarp();
}

// nearest site through the warp (counted); POW: of the lifted point (x, y, z, u)
template <bool POW = false>
__device__ __forceinline__ int nn_query(const Dev<float>& C, Warp3& W, float x, float y, float z, int lane,
                                        Counters& K, float u = 0.f) {
  float d2;
  int sc = 0;
  int k = warp_nearest<float, POW>(C.G, x, y, z, lane, W.S, d2, &sc, C.lift, u);
  K.nn++;
  K.scanned += sc;
  return k;
}

// nearest site of the search point v_i + s.  Learned form: when 2|s| <= r32 the
// nearest site is v_i or one of v_i's 32 nearest sites (any site at least as close
// to the point as v_i lies within 2|s| of v_i), found with no grid scan.
template <typename NL>
__device__ __forceinline__ int nn_search(const Dev<float>& C, Warp3& W, const NL& L, int i, float3 vi,
                                         float sx, float sy, float sz, int lane, Counters& K, float su = 0.f) {
  float px = vi.x + sx, py = vi.y + sy, pz = vi.z + sz;
  if (NL::pow) return nn_query<true>(C, W, px, py, pz, lane, K, su);
  if (L.r32 > 0.f) {
    float s = sqrtf(sx * sx + sy * sy + sz * sz);
    if (2.f * s * (1.f + 1e-5f) + 4e-7f * (fabsf(px) + fabsf(py) + fabsf(pz)) <= L.r32) {
      float d2 = 1e30f;
      int kk = 0x7fffffff;
      if (L.id >= 0) {
        float dx = L.x - px, dy = L.y - py, dz = L.z - pz;
        d2 = dx * dx + dy * dy + dz * dz;
        kk = L.id;
      }
      float dxi = vi.x - px, dyi = vi.y - py, dzi = vi.z - pz;
      float di2 = dxi * dxi + dyi * dyi + dzi * dzi;
      if (lane == 0 && (di2 < d2 || (di2 == d2 && i < kk))) { d2 = di2; kk = i; }
      warp_argmin(d2, kk);
      K.list++;
      K.nn++;
      return kk;
    }
    // the 64 nearest (each lane also takes its entry among the 33rd..64th)
    if (NL::ext && L.r64 > 0.f && 2.f * s * (1.f + 1e-5f) + 4e-7f * (fabsf(px) + fabsf(py) + fabsf(pz)) <= L.r64) {
      float d2 = 1e30f;
      int kk = 0x7fffffff;
      if (L.id >= 0) {
        float dx = L.x - px, dy = L.y - py, dz = L.z - pz;
        d2 = dx * dx + dy * dy + dz * dz;
        kk = L.id;
      }
      int k2 = C.knn2[(long long)i * 32 + lane];
      if (k2 >= 0) {
        float dx = C.sites[3 * k2] - px, dy = C.sites[3 * k2 + 1] - py, dz = C.sites[3 * k2 + 2] - pz;
        float e2 = dx * dx + dy * dy + dz * dz;
        if (e2 < d2 || (e2 == d2 && k2 < kk)) { d2 = e2; kk = k2; }
      }
      float dxi = vi.x - px, dyi = vi.y - py, dzi = vi.z - pz;
      float di2 = dxi * dxi + dyi * dyi + dzi * dzi;
      if (lane == 0 && (di2 < d2 || (di2 == d2 && i < kk))) { d2 = di2; kk = i; }
      warp_argmin(d2, kk);
      K.list++;
      K.nn++;
      return kk;
    }
  }
  return nn_query<false>(C, W, px, py, pz, lane, K);
}

// Coordinates of site k (warp-uniform k >= 0): shuffled from the lane whose
// listed site it is, else loaded (one of the 33rd..64th nearest, or unlisted).
template <typename NL>
__device__ __forceinline__ void listed_coords(const Dev<float>& C, const NL& L, int k, int lane, float& x, float& y,
                                              float& z) {
  unsigned m = __ballot_sync(FULL, L.id == k && k >= 0);
  if (m) {
    int src = __ffs(m) - 1;
    x = __shfl_sync(FULL, L.x, src);
    y = __shfl_sync(FULL, L.y, src);
    z = __shfl_sync(FULL, L.z, src);
  } else if (k >= 0) {
    x = C.sites[3 * k]; y = C.sites[3 * k + 1]; z = C.sites[3 * k + 2];
  } else {
    x = y = z = 0.f;
  }
}

// Sec. 3.2 with the start point of Sec. 5.1 (and the learned shortcut).
// Returns the bisector site j for the outside corner t.
template <typename NL>
__device__ __forceinline__ int find_bisector(const Dev<float>& C, Warp3& W, const NL& L, int i, float3 vi,
                                          int t, int lane, Counters& K) {
  float4 q = W.tq[t];
  int wit = W.twit[t];
  // power diagram: the virtual edge runs from the lifted site (v_i, h_i) to the
  // corner (p, 0); gu is its lifted component (relative to h_i), 0 otherwise
  const float hi = NL::pow ? (float)L.hi : 0.f;
  float dist = sqrtf(q.x * q.x + q.y * q.y + q.z * q.z + hi * hi);
  float dx = q.x / dist, dy = q.y / dist, dz = q.z / dist, du = -hi / dist;
  float gx = q.x, gy = q.y, gz = q.z, gu = -hi;
  int j = wit;
  float delta = C.delta[i];
  if (__any_sync(FULL, L.cand)) {
    // learned proposal, shortcut: the first crossing of the ray v_i -> p with a
    // candidate bisector (or the witness's); one query there either confirms it as
    // the exit point of Omega_i or restarts the plain search from it (Sec. 3.2)
    float tb = 1.f;
    int cb = 0x7fffffff;
    // the witness joins the candidates in the lane that is not one
    unsigned nc = __ballot_sync(FULL, L.cand);
    int wl = nc == FULL ? -1 : __ffs(~nc) - 1;
    int k = L.cand ? L.id : (lane == wl ? wit : -1);
    // the witness's coordinates: from the lane that lists it (a register shuffle),
    // else from memory
    float wx_, wy_, wz_;
    listed_coords(C, L, wit, lane, wx_, wy_, wz_);
    if (k >= 0 && k != i) {
      float kx = L.cand ? L.x : wx_, ky = L.cand ? L.y : wy_, kz = L.cand ? L.z : wz_;
      float wx = kx - vi.x, wy = ky - vi.y, wz = kz - vi.z;
      float den = wx * q.x + wy * q.y + wz * q.z;
      if (den > 0.f) {
        float tt = 0.5f * (wx * wx + wy * wy + wz * wz) / den;
        if (tt < tb) { tb = tt; cb = k; }
      }
    }
    warp_argmin(tb, cb);
    if (cb != 0x7fffffff) {
      float sx = q.x * tb, sy = q.y * tb, sz = q.z * tb;
      int kk = nn_search(C, W, L, i, vi, sx, sy, sz, lane, K);
      K.search++;
      if (kk == i || kk == cb) { K.learned++; return cb; }
      j = kk;
      gx = sx; gy = sy; gz = sz;
      goto search;
    }
  }
  for (int lam = 2; lam < 2 + C.max_lambda; ++lam) {
    float step = (float)lam * delta;
    if (!(step < dist)) break;
    float sx = dx * step, sy = dy * step, sz = dz * step, su = du * step;
    int k = nn_query<NL::pow>(C, W, vi.x + sx, vi.y + sy, vi.z + sz, lane, K, hi + su);
    K.lam++;
    if (k != i) { gx = sx; gy = sy; gz = sz; gu = su; j = k; break; }
  }
search:
  for (int s = 0; s < C.max_search; ++s) {
    float wx = C.sites[3 * j] - vi.x, wy = C.sites[3 * j + 1] - vi.y, wz = C.sites[3 * j + 2] - vi.z;
    float wu = NL::pow ? C.lift[j] - hi : 0.f;  // the lifted sites' difference
    float den = wx * gx + wy * gy + wz * gz + wu * gu;
    if (!(den > 0.f)) { K.fallback++; return wit; }
    float tt = 0.5f * (wx * wx + wy * wy + wz * wz + wu * wu) / den;
    if (!(tt < 1.f)) return j;   // the bisector meets the segment at its end
    float sx = gx * tt, sy = gy * tt, sz = gz * tt, su = gu * tt;
    int k = nn_search(C, W, L, i, vi, sx, sy, sz, lane, K, hi + su);
    K.search++;
    if (k == i || k == j) return j;
    j = k;
    gx = sx; gy = sy; gz = sz; gu = su;
  }
  K.fallback++;
  return wit;
}

// Clip by the plane in slot pl, removing the component of outside corners that
// contains p.  Returns 0 (clipped), 1 (P became empty), -1 (error, status set).
__device__ __forceinline__ int clip(const Dev<float>& C, Warp3& W, Masks& Mk, int a, int i, int pl, int p, int lane) {
  unsigned om[3], R[3];
#pragma unroll
  for (int r = 0; r < 3; ++r) {
    int t = r * 32 + lane;
    // a corner already proven inside Omega_i lies inside every bisector half-space
    // of v_i (Omega_i is their intersection): no side test (Sec. 3.3)
    bool o = bit(Mk.alive, t) && !bit(Mk.in, t) && side_of(C, W, a, i, t, pl) < 0;
    om[r] = __ballot_sync(FULL, o);
    R[r] = 0;
  }
  if (!bit(om, p)) { set_error(C.status, VD_ERR_LIMIT); return -1; }
  // The corners beyond a plane of a convex polytope are connected through its
  // edges, and every side decision here is exact, so R_p (Sec. 5.3) is the whole
  // outside set: no search over the dual mesh is needed.
  R[0] = om[0]; R[1] = om[1]; R[2] = om[2];
  if (R[0] == Mk.alive[0] && R[1] == Mk.alive[1] && R[2] == Mk.alive[2]) return 1;
  // boundary edges of R: (x -> y) of a removed corner whose neighbour u is kept,
  // packed x | y << 8 | u << 16; counted first, then written straight to shared
  // memory at the lane's offset (lane order, corner slots, edges x->y, y->z, z->x)
  int cnt = 0;
#pragma unroll
  for (int r = 0; r < 3; ++r) {
    int t = r * 32 + lane;
    if (bit(R, t)) {
      uchar4 nb = W.tn[t];
      cnt += (int)!bit(R, nb.x) + (int)!bit(R, nb.y) + (int)!bit(R, nb.z);
    }
  }
  unsigned fr[3] = {~Mk.alive[0] | R[0], ~Mk.alive[1] | R[1], ~Mk.alive[2] | R[2]};
  int nfree = __popc(fr[0]) + __popc(fr[1]) + __popc(fr[2]);
  int inc = warp_incl_scan(cnt, lane);
  int base = inc - cnt;
  int total = __shfl_sync(FULL, inc, 31);
  if (total > nfree || total < 3) { set_error(C.status, total < 3 ? VD_ERR_LIMIT : VD_ERR_CAPACITY); return -1; }
  // Edge k of the boundary (in lane order) takes the k-th free slot; the edges are
  // spread over the lanes through shared memory (the integration scratch, unused
  // until the polytope is final) so that each lane claims and builds one new
  // corner instead of the owner of a removed corner building all of its edges.
  unsigned* ebuf = reinterpret_cast<unsigned*>(W.contrib);
  int* sbuf = reinterpret_cast<int*>(ebuf + MAXT);
  __syncwarp();
  {
    int c = base;
#pragma unroll
    for (int r = 0; r < 3; ++r) {
      int t = r * 32 + lane;
      if (bit(R, t)) {
        uchar4 v = W.tv[t], nb = W.tn[t];
        if (!bit(R, nb.x)) ebuf[c++] = (unsigned)v.x | ((unsigned)v.y << 8) | ((unsigned)nb.x << 16);
        if (!bit(R, nb.y)) ebuf[c++] = (unsigned)v.y | ((unsigned)v.z << 8) | ((unsigned)nb.y << 16);
        if (!bit(R, nb.z)) ebuf[c++] = (unsigned)v.z | ((unsigned)v.x << 8) | ((unsigned)nb.z << 16);
      }
    }
  }
  __syncwarp();
  // reset the loop maps, then claim them
#pragma unroll 1
  for (int k = lane; k < total; k += 32) { unsigned e = ebuf[k]; W.stri[e & 255u] = -1; W.etri[(e >> 8) & 255u] = -1; }
  __syncwarp();
  int c0 = __popc(fr[0]), c1 = __popc(fr[1]);
  bool bad = false;
  unsigned newm[3] = {0, 0, 0};
#pragma unroll 1
  for (int k = lane; k < total; k += 32) {
    unsigned e = ebuf[k];
    int sl = k < c0 ? nth_set(fr[0], k) : (k < c0 + c1 ? 32 + nth_set(fr[1], k - c0) : 64 + nth_set(fr[2], k - c0 - c1));
    sbuf[k] = sl;
    if (atomicExch(&W.stri[e & 255u], sl) != -1) bad = true;
    if (atomicExch(&W.etri[(e >> 8) & 255u], sl) != -1) bad = true;
  }
  if (__any_sync(FULL, bad)) { set_error(C.status, VD_ERR_LIMIT); return -1; }
  __syncwarp();
  // write the new corners (their slots held removed corners or were free)
  float4 Pn = W.pn[pl];
  float2 Mn = W.pm[pl];
#pragma unroll 1
  for (int k = lane; k < total; k += 32) {
    unsigned e = ebuf[k];
    int sl = sbuf[k], x = e & 255u, y = (e >> 8) & 255u, u = e >> 16;
    W.tv[sl] = make_uchar4((unsigned char)x, (unsigned char)y, (unsigned char)pl, 0);
    W.tn[sl] = make_uchar4((unsigned char)u, (unsigned char)W.stri[y], (unsigned char)W.etri[x], 0);
    uchar4 uv = W.tv[u];
    if (uv.x == y && uv.y == x) W.tn[u].x = (unsigned char)sl;
    else if (uv.y == y && uv.z == x) W.tn[u].y = (unsigned char)sl;
    else if (uv.z == y && uv.x == x) W.tn[u].z = (unsigned char)sl;
    else bad = true;
    float4 qc = corner(W.pn[x], W.pm[x], W.pn[y], W.pm[y], Pn, Mn);
    if (loose(qc) || C.force_exact)
      qc = refine64(C, a, i, W.psrc[x], W.psrc[y], W.psrc[pl]);
    W.tq[sl] = qc;
    W.twit[sl] = -1;
    unsigned b = 1u << (sl & 31);
    newm[0] |= sl < 32 ? b : 0u;
    newm[1] |= (sl >> 5) == 1 ? b : 0u;
    newm[2] |= sl >= 64 ? b : 0u;
  }
  __syncwarp();
  if (__any_sync(FULL, bad)) { set_error(C.status, VD_ERR_LIMIT); return -1; }
#pragma unroll
  for (int r = 0; r < 3; ++r) {
    unsigned nm = __reduce_or_sync(FULL, newm[r]);
    Mk.alive[r] = (Mk.alive[r] & ~R[r]) | nm;
    Mk.in[r] &= ~(R[r] | nm);
    Mk.out[r] &= ~(R[r] | nm);
  }
  // planes still referenced by a corner
  unsigned long long pm = 0;
#pragma unroll
  for (int r = 0; r < 3; ++r) {
    int t = r * 32 + lane;
    if (bit(Mk.alive, t)) {
      uchar4 v = W.tv[t];
      pm |= (1ull << v.x) | (1ull << v.y) | (1ull << v.z);
    }
  }
  unsigned lo = __reduce_or_sync(FULL, (unsigned)pm), hi = __reduce_or_sync(FULL, (unsigned)(pm >> 32));
  Mk.palive = ((unsigned long long)hi << 32) | lo;
  __syncwarp();
  return 0;
}

#ifdef VD_CHECK
// Consistency of the dual mesh after a clip (checking builds only): neighbours
// are mutual, and no corner is certifiably outside an alive plane.
__device__ void check_mesh(const Dev<float>& C, Warp3& W, const Masks& Mk, int a, int i, int pl_new, int lane) {
  __syncwarp();
#pragma unroll
  for (int r = 0; r < 3; ++r) {
    int t = r * 32 + lane;
    if (!bit(Mk.alive, t)) continue;
    uchar4 v = W.tv[t], nb = W.tn[t];
    int vv[3] = {v.x, v.y, v.z}, nn[3] = {nb.x, nb.y, nb.z};
    for (int e = 0; e < 3; ++e) {
      int u = nn[e], x = vv[e], y = vv[(e + 1) % 3];
      uchar4 uv = W.tv[u], un = W.tn[u];
      int back = (uv.x == y && uv.y == x) ? un.x : (uv.y == y && uv.z == x) ? un.y : (uv.z == y && uv.x == x) ? un.z : -1;
      if (!bit(Mk.alive, u) || back != t) {
        set_error(C.status, VD_ERR_LIMIT);
        record_diag(C.stats, a, i, t, u, x, y, back, 2);
      }
    }
    for (int x = 0; x < MAXP; ++x) {
      if (!((Mk.palive >> x) & 1ull) || x == v.x || x == v.y || x == v.z) continue;
      float4 q = W.tq[t], P = W.pn[x];
      float2 M = W.pm[x];
      float sd = P.w - (P.x * q.x + P.y * q.y + P.z * q.z);
      float qm = fmaxf(fabsf(q.x), fmaxf(fabsf(q.y), fabsf(q.z)));
      float b = (fabsf(P.x) + fabsf(P.y) + fabsf(P.z)) * q.w + SIDEF * (M.y + M.x * qm);
      if (sd < -b) {
        set_error(C.status, VD_ERR_LIMIT);
        record_diag(C.stats, a, i, t, x, W.psrc[x], pl_new, __float_as_int(q.w), 3);
      }
    }
  }
  __syncwarp();
}
#endif

// Canonical key of a corner: the ranks (among the polytope's faces, ordered by
// source: tet faces first, then bisectors by site) of its three planes, sorted,
// 6 bits each.  Equal for the same corner whatever sequence of clips produced
// it, for any number of sites.
__device__ __forceinline__ unsigned long long corner_key(int r0, int r1, int r2) {
  unsigned a = (unsigned)r0, b = (unsigned)r1, c = (unsigned)r2, t;
  if (a > b) { t = a; a = b; b = t; }
  if (b > c) { t = b; b = c; c = t; }
  if (a > b) { t = a; a = b; b = t; }
  return ((unsigned long long)a << 12) | ((unsigned long long)b << 6) | (unsigned long long)c;
}

// Volume and first-moment terms of one corner A (its three edge terms, faces in
// key order; R = reference corner of the face, B = neighbour across the edge; all
// relative to the origin corner O).  Explicitly rounded operations, so every
// mapping of the clip kernel rounds them identically.
__device__ __forceinline__ float4 corner_terms(float4 A4, float4 O, float4 R0, float4 B0, float4 R1, float4 B1,
                                               float4 R2, float4 B2) {
  float ax = __fsub_rn(A4.x, O.x), ay = __fsub_rn(A4.y, O.y), az = __fsub_rn(A4.z, O.z);
  float v6 = 0.f, mx = 0.f, my = 0.f, mz = 0.f;
  auto edge = [&](float4 R4, float4 B4) {
    float rx = __fsub_rn(R4.x, O.x), ry = __fsub_rn(R4.y, O.y), rz = __fsub_rn(R4.z, O.z);
    float bx = __fsub_rn(B4.x, O.x), by = __fsub_rn(B4.y, O.y), bz = __fsub_rn(B4.z, O.z);
    float cx = __fsub_rn(__fmul_rn(ay, bz), __fmul_rn(az, by));
    float cy = __fsub_rn(__fmul_rn(az, bx), __fmul_rn(ax, bz));
    float cz = __fsub_rn(__fmul_rn(ax, by), __fmul_rn(ay, bx));
    float det = __fadd_rn(__fadd_rn(__fmul_rn(rx, cx), __fmul_rn(ry, cy)), __fmul_rn(rz, cz));
    v6 = __fadd_rn(v6, det);
    mx = __fadd_rn(mx, __fmul_rn(det, __fadd_rn(__fadd_rn(rx, ax), bx)));
    my = __fadd_rn(my, __fmul_rn(det, __fadd_rn(__fadd_rn(ry, ay), by)));
    mz = __fadd_rn(mz, __fmul_rn(det, __fadd_rn(__fadd_rn(rz, az), bz)));
  };
  edge(R0, B0);
  edge(R1, B1);
  edge(R2, B2);
  return make_float4(v6, mx, my, mz);
}

// volume and first moment (frame of v_i) from the summed terms S = (6V, M_x, M_y, M_z)
// of the corner fan around O; sigma = +-1 (orientation)
__device__ __forceinline__ float4 finish_moments(float sigma, float4 S, float4 O) {
  float vol = __fdiv_rn(__fmul_rn(sigma, S.x), 6.f);
  float s24 = __fdiv_rn(sigma, 24.f);
  return make_float4(vol, __fadd_rn(__fmul_rn(s24, S.y), __fmul_rn(vol, O.x)),
                     __fadd_rn(__fmul_rn(s24, S.z), __fmul_rn(vol, O.y)),
                     __fadd_rn(__fmul_rn(s24, S.w), __fmul_rn(vol, O.z)));
}

// Integrate volume, first moment (frame of v_i) and face areas of the final
// polytope, independently of the clip history: every corner is recomputed from
// its three planes taken in key order (tet vertices directly from the mesh), the
// reference corner of each face and the origin are the smallest-key corners, and
// the terms are summed in corner-key order.  sigma is +-1 (orientation of the
// dual mesh against space).
__device__ __forceinline__ void integrate(const Dev<float>& C, Warp3& W, const Masks& Mk, int a, int i, float3 vi,
                                       float sigma, int lane, float& vol, float3& m1) {
  for (int x = lane; x < MAXP; x += 32) {
    W.pref[x] = 0x7fffffff;
    W.pkey[x] = ~0ull;
    W.parea[x][0] = W.parea[x][1] = W.parea[x][2] = 0.f;
    int rk = 0;
    if ((Mk.palive >> x) & 1ull) {
      int sx = W.psrc[x];
      for (unsigned long long m = Mk.palive; m; m &= m - 1) rk += W.psrc[__ffsll((long long)m) - 1] < sx;
    }
    W.prank[x] = (unsigned char)rk;
  }
  __syncwarp();
  unsigned long long key[3];
#pragma unroll 1
  for (int r = 0; r < 3; ++r) {
    int t = r * 32 + lane;
    key[r] = ~0ull;
    if (!bit(Mk.alive, t)) continue;
    uchar4 v = W.tv[t];
    int pl[3] = {v.x, v.y, v.z};
    int sr[3] = {W.psrc[v.x], W.psrc[v.y], W.psrc[v.z]};
    // planes in key order
    for (int u = 0; u < 2; ++u)
      for (int w = 0; w < 2 - u; ++w)
        if (sr[w] + 4 > sr[w + 1] + 4) { int tt = sr[w]; sr[w] = sr[w + 1]; sr[w + 1] = tt; tt = pl[w]; pl[w] = pl[w + 1]; pl[w + 1] = tt; }
    float4 q;
    if (sr[2] < 0) {
      float qx, qy, qz;
      if (box_pair(C, a)) {  // box vertex: one face per axis
        float b[3];
        for (int u = 0; u < 3; ++u) {
          int f = -1 - sr[u];
          b[f >> 1] = (f & 1) ? C.bhi[f >> 1] : C.blo[f >> 1];
        }
        qx = b[0] - vi.x; qy = b[1] - vi.y; qz = b[2] - vi.z;
      } else {
        int k = 6 - (-1 - sr[0]) - (-1 - sr[1]) - (-1 - sr[2]);  // tet vertex off the three faces
        const float* V = C.verts + 3 * C.simp[4 * a + k];
        qx = V[0] - vi.x; qy = V[1] - vi.y; qz = V[2] - vi.z;
      }
      q = make_float4(qx, qy, qz, 2.f * U * fmaxf(fabsf(qx), fmaxf(fabsf(qy), fabsf(qz))));
    } else {
      q = corner(W.pn[pl[0]], W.pm[pl[0]], W.pn[pl[1]], W.pm[pl[1]], W.pn[pl[2]], W.pm[pl[2]]);
      if (loose(q) || C.force_exact) q = refine64(C, a, i, sr[0], sr[1], sr[2]);
    }
    W.tq[t] = q;
    key[r] = corner_key(W.prank[pl[0]], W.prank[pl[1]], W.prank[pl[2]]);
    atomicMin(&W.pkey[v.x], key[r]); atomicMin(&W.pkey[v.y], key[r]); atomicMin(&W.pkey[v.z], key[r]);
  }
  __syncwarp();
  // rank of each corner among all corners (keys are distinct for distinct corners)
  int rank[3] = {0, 0, 0};
#pragma unroll 1
  for (int j = 0; j < 32; ++j) {
    unsigned long long k0 = __shfl_sync(FULL, key[0], j), k1 = __shfl_sync(FULL, key[1], j),
                       k2 = __shfl_sync(FULL, key[2], j);
#pragma unroll
    for (int r = 0; r < 3; ++r) {
      int tr = r * 32 + lane;
      rank[r] += (k0 < key[r] || (k0 == key[r] && j < tr)) + (k1 < key[r] || (k1 == key[r] && 32 + j < tr)) +
                 (k2 < key[r] || (k2 == key[r] && 64 + j < tr));
    }
  }
  int o = -1;
#pragma unroll
  for (int r = 0; r < 3; ++r) {
    int t = r * 32 + lane;
    if (key[r] == ~0ull) continue;
    uchar4 v = W.tv[t];
    if (W.pkey[v.x] == key[r]) W.pref[v.x] = t;
    if (W.pkey[v.y] == key[r]) W.pref[v.y] = t;
    if (W.pkey[v.z] == key[r]) W.pref[v.z] = t;
    if (rank[r] == 0) o = t;
  }
  o = __reduce_max_sync(FULL, (unsigned)(o + 1)) - 1;
  __syncwarp();
  float4 O = W.tq[o];
  int nalive = __popc(Mk.alive[0]) + __popc(Mk.alive[1]) + __popc(Mk.alive[2]);
#pragma unroll 1
  for (int r = 0; r < 3; ++r) {
    int t = r * 32 + lane;
    if (key[r] == ~0ull) continue;
    uchar4 v = W.tv[t], nb = W.tn[t];
    float4 A4 = W.tq[t];
    float ax = A4.x - O.x, ay = A4.y - O.y, az = A4.z - O.z;
    // the corner's three edge terms, faces in key order
    int fx[3] = {v.x, v.y, v.z}, fn[3] = {nb.x, nb.y, nb.z};
    int sr[3] = {W.psrc[v.x] + 4, W.psrc[v.y] + 4, W.psrc[v.z] + 4};
    int ord[3] = {0, 1, 2};
    for (int u = 0; u < 2; ++u)
      for (int w = 0; w < 2 - u; ++w)
        if (sr[ord[w]] > sr[ord[w + 1]]) { int tt = ord[w]; ord[w] = ord[w + 1]; ord[w + 1] = tt; }
    float4 Rq[3], Bq[3];
#pragma unroll
    for (int e3 = 0; e3 < 3; ++e3) {
      int e = ord[e3];
      int x = fx[e];
      Rq[e3] = W.tq[W.pref[x]];
      Bq[e3] = W.tq[fn[e]];
      float rx = Rq[e3].x - O.x, ry = Rq[e3].y - O.y, rz = Rq[e3].z - O.z;
      float bx = Bq[e3].x - O.x, by = Bq[e3].y - O.y, bz = Bq[e3].z - O.z;
      float ux = ax - rx, uy = ay - ry, uz = az - rz, wx = bx - rx, wy = by - ry, wz = bz - rz;
      atomicAdd(&W.parea[x][0], uy * wz - uz * wy);
      atomicAdd(&W.parea[x][1], uz * wx - ux * wz);
      atomicAdd(&W.parea[x][2], ux * wy - uy * wx);
    }
    W.contrib[rank[r]] = corner_terms(A4, O, Rq[0], Bq[0], Rq[1], Bq[1], Rq[2], Bq[2]);
  }
  __syncwarp();
  float v6 = 0.f, mx = 0.f, my = 0.f, mz = 0.f;
#pragma unroll
  for (int r = 0; r < 3; ++r) {
    int k = r * 32 + lane;
    if (k < nalive) {
      float4 c4 = W.contrib[k];
      v6 += c4.x; mx += c4.y; my += c4.z; mz += c4.w;
    }
  }
  v6 = warp_sum(v6);
  mx = warp_sum(mx); my = warp_sum(my); mz = warp_sum(mz);
  float4 F = finish_moments(sigma, make_float4(v6, mx, my, mz), O);
  vol = F.x;
  m1 = make_float3(F.y, F.z, F.w);
  __syncwarp();
}

// the corner table of a tetrahedron: corner k (vertex k) is where the three faces
// other than f = k meet; dual triangles oriented as the boundary of a simplex
__constant__ unsigned char TET_TV[4][3] = {{1, 2, 3}, {0, 3, 2}, {0, 1, 3}, {0, 2, 1}};

// the dual mesh of the box: corner k = (x, y, z sides in bits 0, 1, 2) where one
// face of each axis meets, oriented by the parity of k; across the dual edge
// between two faces lies the corner that differs on the third axis
__device__ void init_box(const Dev<float>& C, Warp3& W, Masks& Mk, float3 vi, int lane) {
  if (lane < 6) {
    float4 P;
    float2 M;
    plane_box(C, lane, vi, P, M);
    W.pn[lane] = P; W.pm[lane] = M; W.psrc[lane] = -1 - lane;
  }
  if (lane < 8) {
    int k = lane, sx = k & 1, sy = (k >> 1) & 1, sz = (k >> 2) & 1;
    float qx = (sx ? C.bhi[0] : C.blo[0]) - vi.x, qy = (sy ? C.bhi[1] : C.blo[1]) - vi.y,
          qz = (sz ? C.bhi[2] : C.blo[2]) - vi.z;
    W.tq[k] = make_float4(qx, qy, qz, 2.f * U * fmaxf(fabsf(qx), fmaxf(fabsf(qy), fabsf(qz))));
    unsigned char fx = (unsigned char)sx, fy = (unsigned char)(2 + sy), fz = (unsigned char)(4 + sz);
    if (((sx + sy + sz) & 1) == 0) {
      W.tv[k] = make_uchar4(fx, fy, fz, 0);
      W.tn[k] = make_uchar4((unsigned char)(k ^ 4), (unsigned char)(k ^ 1), (unsigned char)(k ^ 2), 0);
    } else {
      W.tv[k] = make_uchar4(fx, fz, fy, 0);
      W.tn[k] = make_uchar4((unsigned char)(k ^ 2), (unsigned char)(k ^ 1), (unsigned char)(k ^ 4), 0);
    }
    W.twit[k] = -1;
  }
  Mk.alive[0] = 0xFFu; Mk.alive[1] = Mk.alive[2] = 0;
  Mk.in[0] = Mk.in[1] = Mk.in[2] = 0;
  Mk.out[0] = Mk.out[1] = Mk.out[2] = 0;
  Mk.palive = 0x3Full;
  __syncwarp();
}

__device__ void init_tet(const Dev<float>& C, Warp3& W, Masks& Mk, int a, int i, float3 vi, int lane) {
  if (box_pair(C, a)) { init_box(C, W, Mk, vi, lane); return; }
  if (lane < 4) {
    float4 P;
    float2 M;
    plane_face(C, a, lane, vi, P, M);
    W.pn[lane] = P; W.pm[lane] = M; W.psrc[lane] = -1 - lane;
    int k = lane;
    const float* V = C.verts + 3 * C.simp[4 * a + k];
    float qx = V[0] - vi.x, qy = V[1] - vi.y, qz = V[2] - vi.z;
    float qm = fmaxf(fabsf(qx), fmaxf(fabsf(qy), fabsf(qz)));
    W.tq[k] = make_float4(qx, qy, qz, 2.f * U * qm);
    unsigned char x = TET_TV[k][0], y = TET_TV[k][1], z = TET_TV[k][2];
    W.tv[k] = make_uchar4(x, y, z, 0);
    // across dual edge (x,y) lies the corner at the tet vertex that is neither k, x nor y
    unsigned char n0 = (unsigned char)(6 - k - x - y), n1 = (unsigned char)(6 - k - y - z),
                  n2 = (unsigned char)(6 - k - z - x);
    W.tn[k] = make_uchar4(n0, n1, n2, 0);
    W.twit[k] = -1;
  }
  Mk.alive[0] = 0xFu; Mk.alive[1] = Mk.alive[2] = 0;
  Mk.in[0] = Mk.in[1] = Mk.in[2] = 0;
  Mk.out[0] = Mk.out[1] = Mk.out[2] = 0;
  Mk.palive = 0xFull;
  __syncwarp();
}

#ifdef VD_PROFILE
#define PROF_T0() long long _t0 = clock64()
#define PROF_ADD(k) do { long long _t1 = clock64(); if (lane == 0) atomicAdd(C.stats + VD_STAT_DIAG + (k), (unsigned long long)(_t1 - _t0)); _t0 = _t1; } while (0)
#else
#define PROF_T0() do {} while (0)
#define PROF_ADD(k) do {} while (0)
#endif

template <bool EXT, bool POW = false>
__device__ void process_pair(const Dev<float>& C, Warp3& W, int a, int i, long long slot, int lane) {
  Counters K = {0, 0, 0, 0, 0, 0, 0, 0, 0};
  const NbrList<float, EXT, POW> L = load_nbrs<float, EXT, POW>(C, i, lane);
  // power diagram: B_ij on u = 0 is n.x <= (|w|^2 + h_j^2 - h_i^2) / 2 (Sec. 6.3)
  auto lifted = [&](int j, float4& P, float2& M) {
    if (POW) {
      float hj = C.lift[j], h = (float)L.hi;
      P.w += 0.5f * (hj * hj - h * h);
      M.y += 0.5f * (hj * hj + h * h);
    }
  };
  PROF_T0();
  float3 vi = make_float3(C.sites[3 * i], C.sites[3 * i + 1], C.sites[3 * i + 2]);
  Masks Mk;
  init_tet(C, W, Mk, a, i, vi, lane);
  // orientation of the dual mesh against space: with the corner table below, the
  // edge-term sum of integrate() has the sign of the tet's orientation
  const bool bx = box_pair(C, a);
  if (lane == 0) W.tied = 0;
  __syncwarp();
  float sigma = 1.f;  // the box's dual mesh is oriented like a positive tet
  if (!bx) {
    sigma = (float)C.tsgn[a];
  }
  bool empty = false;
  int nclip = 0;
  PROF_ADD(0);
  for (;;) {
    // first corner (in slot order) outside Omega_i; each corner is tested once
    int p = -1;
    for (;;) {
      unsigned c0 = Mk.alive[0] & ~Mk.in[0], c1 = Mk.alive[1] & ~Mk.in[1], c2 = Mk.alive[2] & ~Mk.in[2];
      int t = c0 ? __ffs(c0) - 1 : (c1 ? 31 + __ffs(c1) : (c2 ? 63 + __ffs(c2) : -1));
      if (t < 0) break;
      if (bit(Mk.out, t)) { p = t; break; }
      float4 q = W.tq[t];
      uchar4 v = W.tv[t];
      int ex[3];
      ex[0] = W.psrc[v.x]; ex[1] = W.psrc[v.y]; ex[2] = W.psrc[v.z];
      for (int u = 0; u < 3; ++u) if (ex[u] < 0) ex[u] = -2;  // tet faces exclude no site
      bool uns = false;
      auto exact = [&](int k) {
        int r = exact_side(C, W, a, i, t, k);
        uns |= r == 2 || r == -2;
        return r;
      };
      int wit;
      int sc = 0, ls = 0;
      int out = corner_outside(C, i, vi.x, vi.y, vi.z, q.x, q.y, q.z, q.w, ex, lane, W.S, L, exact, &wit, &sc, &ls);
      // a corner found inside with a tie (or an uncertain sign) lies on that
      // site's bisector: the polytope may be degenerate there
      if (__any_sync(FULL, uns) && !out && lane == 0) W.tied = 1;
      K.corner++;
      K.nn++;
      K.scanned += sc;
      K.list += ls;
      if (out) {
        Mk.out[t >> 5] |= 1u << (t & 31);
        if (lane == 0) W.twit[t] = wit;
        __syncwarp();
        p = t;
        break;
      }
      Mk.in[t >> 5] |= 1u << (t & 31);
    }
    PROF_ADD(1);
    if (p < 0) break;
    if (++nclip > C.max_clips) { set_error(C.status, VD_ERR_LIMIT); return; }
    if (*(volatile int*)C.status) return;
    int j = find_bisector(C, W, L, i, vi, p, lane, K);
    PROF_ADD(2);
    // free plane slot for B_ij
    unsigned long long freep = ~Mk.palive & ((1ull << MAXP) - 1ull);
    if (!freep) { set_error(C.status, VD_ERR_CAPACITY); return; }
    int pl = __ffsll((long long)freep) - 1;
    float4 P;
    float2 M;
    {
      float jx, jy, jz;
      listed_coords(C, L, j, lane, jx, jy, jz);
      plane_bis_at(jx, jy, jz, vi, P, M);
      lifted(j, P, M);
    }
    add_plane(W, pl, P, M, j, lane);
    if (side_of(C, W, a, i, p, pl) >= 0) {
      // FP32 search landed on a bisector that does not cut p: use the certified closer site
      K.fallback++;
      j = W.twit[p];
      plane_bis(C, j, vi, P, M);
      lifted(j, P, M);
      add_plane(W, pl, P, M, j, lane);
    }
    int rc = clip(C, W, Mk, a, i, pl, p, lane);
    K.clips++;
    PROF_ADD(3);
    if (rc < 0) return;
#ifdef VD_CHECK
    if (rc == 0) check_mesh(C, W, Mk, a, i, pl, lane);
#endif
    if (rc == 1) { empty = true; break; }
  }
  float vol = 0.f;
  float3 m1 = make_float3(0.f, 0.f, 0.f);
  if (!empty) integrate(C, W, Mk, a, i, vi, sigma, lane, vol, m1);
  // Positive measure (Sec. 2.2) is decided from the exact structure: every side
  // decision was certified, so with no exact tie (or uncertain sign) in this pair
  // the piece (at least four corners) and each of its faces (at least three) has
  // positive measure however FP32 rounds a face far below the cell's size (its
  // corners can round to one point).  After a tie the computed measures decide.
  __syncwarp();
  const bool exact_faces = W.tied == 0;
  bool nonempty = !empty && (vol > 0.f || exact_faces);
  if (nonempty && !(vol > 0.f)) {  // a sliver below FP32 resolution: positive, negligible
    vol = 1.17549435e-38f;
    m1 = make_float3(0.f, 0.f, 0.f);
  }
  // faces of positive area: output flags and propagate (Alg. 4 / Alg. 5 rules)
  int nflag = 0;
  int myflag[2];
  bool has[2] = {false, false}, bis[2] = {false, false};
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    int x = lane + 32 * h;
    if (nonempty && x < MAXP && ((Mk.palive >> x) & 1ull)) {
      float ax = W.parea[x][0], ay = W.parea[x][1], az = W.parea[x][2];
      if (exact_faces || ax * ax + ay * ay + az * az > 0.f) {
        int src = W.psrc[x];
        bis[h] = src >= 0;
        if (src >= 0) {
          myflag[h] = src;
          // the box form seeds every site itself; the split propagates through
          // negative flags only (Alg. 5)
          if (!bx && !C.split) push_pair(C, a, src);
        } else if (bx) {
          myflag[h] = FLAG_BOUNDARY;
        } else {
          int b = C.adj[4 * a + (-1 - src)];
          myflag[h] = b >= 0 ? -(b + 1) : FLAG_BOUNDARY;
          if (b >= 0) push_pair(C, b, i);
        }
        has[h] = true;
      }
    }
  }
  unsigned b0 = __ballot_sync(FULL, has[0]), b1 = __ballot_sync(FULL, has[1]);
  nflag = __popc(b0) + __popc(b1);
  // bisector faces of the final piece: each clip that contributed left one (Sec. 3.3)
  unsigned nbis = C.want_stats ? __popc(__ballot_sync(FULL, bis[0])) + __popc(__ballot_sync(FULL, bis[1])) : 0u;
  long long fbase = 0;
  if (lane == 0 && nflag) fbase = (long long)atomicAdd(C.ctr + CTR_FLAGS, (unsigned long long)nflag);
  fbase = __shfl_sync(FULL, fbase, 0);
  if (fbase + nflag > C.fcap) { set_error(C.status, VD_ERR_CAPACITY); return; }
  unsigned lt = (1u << lane) - 1u;
  if (has[0]) C.pflags[fbase + __popc(b0 & lt)] = myflag[0];
  if (has[1]) C.pflags[fbase + __popc(b0) + __popc(b1 & lt)] = myflag[1];
  PROF_ADD(4);
  if (lane == 0) {
    C.pmeas[slot] = nonempty ? vol : 0.f;
    C.pm1[3 * slot] = nonempty ? m1.x : 0.f;
    C.pm1[3 * slot + 1] = nonempty ? m1.y : 0.f;
    C.pm1[3 * slot + 2] = nonempty ? m1.z : 0.f;
    C.pfoff[slot] = fbase;
    C.pfcnt[slot] = nflag;
    if (C.want_stats) {
      stat_add(C, VD_STAT_NN_QUERIES, K.nn);
      stat_add(C, VD_STAT_CORNER_TESTS, K.corner);
      stat_add(C, VD_STAT_CLIPS, K.clips);
      stat_add(C, VD_STAT_LAMBDA_STEPS, K.lam);
      stat_add(C, VD_STAT_SEARCH_STEPS, K.search);
      stat_add(C, VD_STAT_SITES_SCANNED, K.scanned);
      stat_add(C, VD_STAT_FALLBACK, K.fallback);
      stat_add(C, VD_STAT_LEARNED_HITS, K.learned);
      stat_add(C, VD_STAT_LIST_TESTS, K.list);
      stat_add(C, VD_STAT_BISECTOR_FACES, nbis);
      stat_add(C, VD_STAT_EXCESS_CLIPS, K.clips > nbis ? K.clips - nbis : 0u);
    }
  }
  __syncwarp();
}

}  // namespace c3
}  // namespace vd
