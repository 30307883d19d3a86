// vd_clippoly.cuh -- triangle / Voronoi-cell intersection (2D and surface), one
// warp per pair.
//
// The piece is a convex polygon in the plane S of its triangle: a ring of at
// most 32 corners (one per lane), corner k between the edge planes e[k-1] and
// e[k].  A corner is the meeting point of S and two planes (triangle edges, or
// bisectors cut by S), so the side tests and their float64 fallback are the
// same as in 3D.  In 2D the sites and the triangles lie in z = 0.  Alg. 3 with
// the search of Sec. 3.2 / 5.1 drives the clipping, exactly as in vd_clip3.cuh;
// removing the outside run of the ring that contains p is R_p of Sec. 5.3.
#pragma once

#include "vd_dev.cuh"

namespace vd {
namespace cp {

constexpr int MAXV = 32;
constexpr int MAXPL = 48;

template <typename T>
struct Vec {
  using V4 = typename Prec<T>::V4;
};

template <typename T>
struct WarpP {
  using V4 = typename Prec<T>::V4;
  V4 pn[MAXPL];    // n.xyz, c : inside is n.x <= c (S: the triangle's plane)
  T pmx[MAXPL];    // |n~|_1
  T pmc[MAXPL];    // c~
  int psrc[MAXPL]; // >= 0 bisector site; -1: S; -2-e: triangle edge e (local vertex e -> e+1)
  V4 vq[MAXV];     // corner (frame of v_i), w = coordinate error bound
  int ve[MAXV];    // plane of the edge from corner k to corner k+1
  int vst[MAXV];   // 0 untested, 1 inside, 2 outside
  int vwit[MAXV];
  mutable int tied;  // this pair met an exact tie or an uncertain sign
  ScanScratch S;
};

template <typename T> __device__ __forceinline__ T gam() { return T(64) * Prec<T>::U; }
template <typename T> __device__ __forceinline__ T sidef() { return T(24) * Prec<T>::U; }

template <typename T> __device__ __forceinline__ const T* vtx(const Dev<T>& C, int a, int l) {
  return C.verts + 3 * C.simp[3 * a + l];
}

// S: n = (B-A) x (C-A), through A
template <typename T>
__device__ void plane_S(const Dev<T>& C, int a, const T* vi, typename Prec<T>::V4& P, T& mx, T& mc) {
  const T *A = vtx(C, a, 0), *B = vtx(C, a, 1), *Cc = vtx(C, a, 2);
  T e1x = B[0] - A[0], e1y = B[1] - A[1], e1z = B[2] - A[2];
  T e2x = Cc[0] - A[0], e2y = Cc[1] - A[1], e2z = Cc[2] - A[2];
  T nx = e1y * e2z - e1z * e2y, ny = e1z * e2x - e1x * e2z, nz = e1x * e2y - e1y * e2x;
  T ax = A[0] - vi[0], ay = A[1] - vi[1], az = A[2] - vi[2];
  T m0 = fabs(e1y * e2z) + fabs(e1z * e2y), m1 = fabs(e1z * e2x) + fabs(e1x * e2z),
    m2 = fabs(e1x * e2y) + fabs(e1y * e2x);
  P = Prec<T>::mk4(nx, ny, nz, nx * ax + ny * ay + nz * az);
  mx = m0 + m1 + m2;
  mc = m0 * fabs(ax) + m1 * fabs(ay) + m2 * fabs(az);
}

// edge e (local vertex e -> e+1): n = (V_{e+1} - V_e) x n_S (outward for the ring
// A -> B -> C, which turns counter-clockwise about n_S), through V_e
template <typename T>
__device__ void plane_E(const Dev<T>& C, int a, int e, const T* vi, typename Prec<T>::V4& P, T& mx, T& mc) {
  const T *A = vtx(C, a, 0), *B = vtx(C, a, 1), *Cc = vtx(C, a, 2);
  T e1x = B[0] - A[0], e1y = B[1] - A[1], e1z = B[2] - A[2];
  T e2x = Cc[0] - A[0], e2y = Cc[1] - A[1], e2z = Cc[2] - A[2];
  T sx = e1y * e2z - e1z * e2y, sy = e1z * e2x - e1x * e2z, sz = e1x * e2y - e1y * e2x;
  T s0 = fabs(e1y * e2z) + fabs(e1z * e2y), s1 = fabs(e1z * e2x) + fabs(e1x * e2z),
    s2 = fabs(e1x * e2y) + fabs(e1y * e2x);
  const T* P0 = vtx(C, a, e);
  const T* P1 = vtx(C, a, (e + 1) % 3);
  T dx = P1[0] - P0[0], dy = P1[1] - P0[1], dz = P1[2] - P0[2];
  T nx = dy * sz - dz * sy, ny = dz * sx - dx * sz, nz = dx * sy - dy * sx;
  T m0 = fabs(dy) * s2 + fabs(dz) * s1, m1 = fabs(dz) * s0 + fabs(dx) * s2, m2 = fabs(dx) * s1 + fabs(dy) * s0;
  T ax = P0[0] - vi[0], ay = P0[1] - vi[1], az = P0[2] - vi[2];
  P = Prec<T>::mk4(nx, ny, nz, nx * ax + ny * ay + nz * az);
  mx = m0 + m1 + m2;
  mc = m0 * fabs(ax) + m1 * fabs(ay) + m2 * fabs(az);
}

template <typename T>
__device__ void plane_B(const Dev<T>& C, int j, const T* vi, typename Prec<T>::V4& P, T& mx, T& mc) {
  T wx = C.sites[3 * j] - vi[0], wy = C.sites[3 * j + 1] - vi[1], wz = C.sites[3 * j + 2] - vi[2];
  T c = T(0.5) * (wx * wx + wy * wy + wz * wz);
  P = Prec<T>::mk4(wx, wy, wz, c);
  mx = fabs(wx) + fabs(wy) + fabs(wz);
  mc = c;
}

template <typename T>
__device__ __noinline__ ePlane eplane(const Dev<T>& C, int a, int i, int src) {
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
  const T *A = vtx(C, a, 0), *B = vtx(C, a, 1), *Cc = vtx(C, a, 2);
  ed3 eA{mk(A[0]), mk(A[1]), mk(A[2])}, eB{mk(B[0]), mk(B[1]), mk(B[2])}, eC{mk(Cc[0]), mk(Cc[1]), mk(Cc[2])};
  ed3 nS = cross3(sub3(eB, eA), sub3(eC, eA));
  if (src == -1) {
    p.n = nS;
    p.c = dot3(nS, sub3(eA, vi));
    return p;
  }
  int e = -2 - src;
  const T* P0 = vtx(C, a, e);
  const T* P1 = vtx(C, a, (e + 1) % 3);
  ed3 e0{mk(P0[0]), mk(P0[1]), mk(P0[2])}, e1{mk(P1[0]), mk(P1[1]), mk(P1[2])};
  p.n = cross3(sub3(e1, e0), nS);
  p.c = dot3(p.n, sub3(e0, vi));
  return p;
}

// corner of three planes (Cramer), with the error bound of vd_clip3.cuh
template <typename T>
__device__ typename Prec<T>::V4 corner(const WarpP<T>& W, int p0, int p1, int p2) {
  typename Prec<T>::V4 P0 = W.pn[p0], P1 = W.pn[p1], P2 = W.pn[p2];
  T x12x = P1.y * P2.z - P1.z * P2.y, x12y = P1.z * P2.x - P1.x * P2.z, x12z = P1.x * P2.y - P1.y * P2.x;
  T x20x = P2.y * P0.z - P2.z * P0.y, x20y = P2.z * P0.x - P2.x * P0.z, x20z = P2.x * P0.y - P2.y * P0.x;
  T x01x = P0.y * P1.z - P0.z * P1.y, x01y = P0.z * P1.x - P0.x * P1.z, x01z = P0.x * P1.y - P0.y * P1.x;
  T D = P0.x * x12x + P0.y * x12y + P0.z * x12z;
  T qx = (P0.w * x12x + P1.w * x20x + P2.w * x01x) / D;
  T qy = (P0.w * x12y + P1.w * x20y + P2.w * x01y) / D;
  T qz = (P0.w * x12z + P1.w * x20z + P2.w * x01z) / D;
  T Dm = W.pmx[p0] * W.pmx[p1] * W.pmx[p2];
  T Am = W.pmc[p0] * W.pmx[p1] * W.pmx[p2] + W.pmc[p1] * W.pmx[p2] * W.pmx[p0] + W.pmc[p2] * W.pmx[p0] * W.pmx[p1];
  T qm = fmax(fabs(qx), fmax(fabs(qy), fabs(qz)));
  T g = gam<T>();
  T den = fabs(D) - g * Dm;
  T e = (den > g * Dm && isfinite(qm)) ? (g * Am + qm * g * Dm) / den + T(2) * Prec<T>::U * qm : T(1e30);
  return Prec<T>::mk4(qx, qy, qz, e);
}

// a corner whose FP32 error bound is loose is recomputed from its exact planes
template <typename T>
__device__ __noinline__ typename Prec<T>::V4 refine(const Dev<T>& C, const WarpP<T>& W, int a, int i,
                                                       typename Prec<T>::V4 q, int p1, int p2) {
  if (sizeof(T) == 8) return q;
  if (q.w <= T(3e-3) * sqrt(q.x * q.x + q.y * q.y + q.z * q.z)) return q;
  float4 r = corner64(eplane(C, a, i, -1), eplane(C, a, i, W.psrc[p1]), eplane(C, a, i, W.psrc[p2]));
  atomicAdd(C.stats + VD_STAT_FP64, 1ull);
  return Prec<T>::mk4((T)r.x, (T)r.y, (T)r.z, (T)r.w);
}

template <typename T>
__device__ __noinline__ int exact_side(const Dev<T>& C, const WarpP<T>& W, int a, int i, int k, int nv, int src4) {
  int km = (k + nv - 1) % nv;
  // the corner lies on each of its own planes: the side value is exactly zero
  if (src4 == -1 || src4 == W.psrc[W.ve[km]] || src4 == W.psrc[W.ve[k]]) return 0;
  ePlane p[4];
  p[0] = eplane(C, a, i, -1);
  p[1] = eplane(C, a, i, W.psrc[W.ve[km]]);
  p[2] = eplane(C, a, i, W.psrc[W.ve[k]]);
  p[3] = eplane(C, a, i, src4);
  int certain, tie;
  int s = side_from_planes(p, &certain, &tie);
  atomicAdd(C.stats + VD_STAT_FP64, 1ull);
  if (!certain) {
    atomicAdd(C.stats + (tie ? VD_STAT_TIES : VD_STAT_UNCERTAIN), 1ull);
    record_diag(C.stats, a, i, -1, W.psrc[W.ve[km]], W.psrc[W.ve[k]], src4, tie, 0);
    return s < 0 ? -2 : 2;  // not certified: +-2 (a tie counts as inside)
  }
  return s;
}

template <typename T>
__device__ __forceinline__ int side_of(const Dev<T>& C, const WarpP<T>& W, int a, int i, int k, int nv, int pl) {
  typename Prec<T>::V4 q = W.vq[k], P = W.pn[pl];
  if (q.w < T(1e29) && !C.force_exact) {
    T s = P.w - (P.x * q.x + P.y * q.y + P.z * q.z);
    T qm = fmax(fabs(q.x), fmax(fabs(q.y), fabs(q.z)));
    T b = (fabs(P.x) + fabs(P.y) + fabs(P.z)) * q.w + sidef<T>() * (W.pmc[pl] + W.pmx[pl] * qm);
    if (s > b) return 1;
    if (s < -b) return -1;
  }
  int r = exact_side(C, W, a, i, k, nv, W.psrc[pl]);
  if (r == 2 || r == -2) W.tied = 1;
  return r;
}

struct Counters {
  unsigned long long nn, corner, clips, lam, search, scanned, fallback, learned, list;
};

template <typename T, bool POW = false>
__device__ __noinline__ int nn_query(const Dev<T>& C, WarpP<T>& W, T x, T y, T z, int lane, Counters& K,
                                     T u = T(0)) {
  T d2;
  int sc = 0;
  int k = warp_nearest<T, POW>(C.G, x, y, z, lane, W.S, d2, &sc, C.lift, u);
  K.nn++;
  K.scanned += sc;
  return k;
}

// nearest site of v_i + s; learned form: from the 32-NN list when 2|s| <= r32
template <typename T, typename NL>
__device__ __forceinline__ int nn_search(const Dev<T>& C, WarpP<T>& W, const NL& L, int i, const T* vi,
                                         T sx, T sy, T sz, int lane, Counters& K, T su = T(0)) {
  T px = vi[0] + sx, py = vi[1] + sy, pz = vi[2] + sz;
  if (NL::pow) return nn_query<T, true>(C, W, px, py, pz, lane, K, su);
  if (L.r32 > 0.f) {
    T s = sqrt(sx * sx + sy * sy + sz * sz);
    if ((float)(T(2) * s) * (1.f + 2e-5f) + 4e-7f * (float)(fabs(px) + fabs(py) + fabs(pz)) <= L.r32) {
      T d2 = T(1e30);
      int kk = 0x7fffffff;
      if (L.id >= 0) {
        T dx = L.x - px, dy = L.y - py, dz = L.z - pz;
        d2 = dx * dx + dy * dy + dz * dz;
        kk = L.id;
      }
      T dxi = vi[0] - px, dyi = vi[1] - py, dzi = vi[2] - pz;
      T di2 = dxi * dxi + dyi * dyi + dzi * dzi;
      if (lane == 0 && (di2 < d2 || (di2 == d2 && i < kk))) { d2 = di2; kk = i; }
      warp_argmin(d2, kk);
      K.nn++;
      K.list++;
      return kk;
    }
    // the 64 nearest (each lane also takes its entry among the 33rd..64th)
    if (NL::ext && L.r64 > 0.f &&
        (float)(T(2) * s) * (1.f + 2e-5f) + 4e-7f * (float)(fabs(px) + fabs(py) + fabs(pz)) <= L.r64) {
      T d2 = T(1e30);
      int kk = 0x7fffffff;
      if (L.id >= 0) {
        T dx = L.x - px, dy = L.y - py, dz = L.z - pz;
        d2 = dx * dx + dy * dy + dz * dz;
        kk = L.id;
      }
      int k2 = C.knn2[(long long)i * 32 + lane];
      if (k2 >= 0) {
        T dx = C.sites[3 * k2] - px, dy = C.sites[3 * k2 + 1] - py, dz = C.sites[3 * k2 + 2] - pz;
        T e2 = dx * dx + dy * dy + dz * dz;
        if (e2 < d2 || (e2 == d2 && k2 < kk)) { d2 = e2; kk = k2; }
      }
      T dxi = vi[0] - px, dyi = vi[1] - py, dzi = vi[2] - pz;
      T di2 = dxi * dxi + dyi * dyi + dzi * dzi;
      if (lane == 0 && (di2 < d2 || (di2 == d2 && i < kk))) { d2 = di2; kk = i; }
      warp_argmin(d2, kk);
      K.nn++;
      K.list++;
      return kk;
    }
  }
  return nn_query<T, false>(C, W, px, py, pz, lane, K);
}

template <typename T, typename NL>
__device__ __noinline__ int find_bisector(const Dev<T>& C, WarpP<T>& W, const NL& L, int i, const T* vi,
                                          int k, int lane, Counters& K) {
  typename Prec<T>::V4 q = W.vq[k];
  int wit = W.vwit[k];
  // power diagram: the virtual edge from the lifted site (v_i, h_i) to (p, 0)
  const T hi = NL::pow ? L.hi : T(0);
  T dist = sqrt(q.x * q.x + q.y * q.y + q.z * q.z + hi * hi);
  T dx = q.x / dist, dy = q.y / dist, dz = q.z / dist, du = -hi / dist;
  T gx = q.x, gy = q.y, gz = q.z, gu = -hi;
  int j = wit;
  T delta = C.delta[i];
  if (__any_sync(FULL, L.cand)) {
    // learned proposal: first crossing of the ray v_i -> p with a candidate
    // bisector (or the witness's), confirmed by one query (as in 3D)
    T tb = T(1);
    int cb = 0x7fffffff;
    unsigned nc = __ballot_sync(FULL, L.cand);
    int wl = nc == FULL ? -1 : __ffs(~nc) - 1;
    int kc = L.cand ? L.id : (lane == wl ? wit : -1);
    if (kc >= 0 && kc != i) {
      T kx = L.cand ? L.x : C.sites[3 * kc], ky = L.cand ? L.y : C.sites[3 * kc + 1],
        kz = L.cand ? L.z : C.sites[3 * kc + 2];
      T wx = kx - vi[0], wy = ky - vi[1], wz = kz - vi[2];
      T den = wx * q.x + wy * q.y + wz * q.z;
      if (den > T(0)) {
        T tt = T(0.5) * (wx * wx + wy * wy + wz * wz) / den;
        if (tt < tb) { tb = tt; cb = kc; }
      }
    }
    warp_argmin(tb, cb);
    if (cb != 0x7fffffff) {
      T sx = q.x * tb, sy = q.y * tb, sz = q.z * tb;
      int kk = nn_search(C, W, L, i, vi, sx, sy, sz, lane, K);
      K.search++;
      if (kk == i || kk == cb) { K.learned++; return cb; }
      j = kk;
      gx = sx; gy = sy; gz = sz;
      goto search;
    }
  }
  for (int lam = 2; lam < 2 + C.max_lambda; ++lam) {
    T step = T(lam) * delta;
    if (!(step < dist)) break;
    T sx = dx * step, sy = dy * step, sz = dz * step, su = du * step;
    int kk = nn_query<T, NL::pow>(C, W, vi[0] + sx, vi[1] + sy, vi[2] + sz, lane, K, hi + su);
    K.lam++;
    if (kk != i) { gx = sx; gy = sy; gz = sz; gu = su; j = kk; break; }
  }
search:
  for (int s = 0; s < C.max_search; ++s) {
    T wx = C.sites[3 * j] - vi[0], wy = C.sites[3 * j + 1] - vi[1], wz = C.sites[3 * j + 2] - vi[2];
    T wu = NL::pow ? (T)C.lift[j] - hi : T(0);
    T den = wx * gx + wy * gy + wz * gz + wu * gu;
    if (!(den > T(0))) { K.fallback++; return wit; }
    T tt = T(0.5) * (wx * wx + wy * wy + wz * wz + wu * wu) / den;
    if (!(tt < T(1))) return j;
    T sx = gx * tt, sy = gy * tt, sz = gz * tt, su = gu * tt;
    int kk = nn_search(C, W, L, i, vi, sx, sy, sz, lane, K, hi + su);
    K.search++;
    if (kk == i || kk == j) return j;
    j = kk;
    gx = sx; gy = sy; gz = sz; gu = su;
  }
  K.fallback++;
  return wit;
}

// clip the ring by plane pl, removing the outside run that contains corner p.
// returns 0 clipped, 1 empty, -1 error.  nv is updated.
template <typename T>
__device__ __forceinline__ int clip(const Dev<T>& C, WarpP<T>& W, int a, int i, int pl, int p, int& nv, int lane) {
  // a corner already proven inside Omega_i stays (inside every bisector half-space of v_i)
  bool o = lane < nv && W.vst[lane] != 1 && side_of(C, W, a, i, lane, nv, pl) < 0;
  unsigned om = __ballot_sync(FULL, o);
  if (!((om >> p) & 1u)) { set_error(C.status, VD_ERR_LIMIT); return -1; }
  int s = p, e = p, run = 1;
  while (run < nv && ((om >> ((s + nv - 1) % nv)) & 1u)) { s = (s + nv - 1) % nv; ++run; }
  while (run < nv && ((om >> ((e + 1) % nv)) & 1u)) { e = (e + 1) % nv; ++run; }
  if (run >= nv) return 1;
  int keep = nv - run, m = keep + 2;
  if (m > MAXV) { set_error(C.status, VD_ERR_CAPACITY); return -1; }
  int sm = (s + nv - 1) % nv;
  int eX = W.ve[sm], eY = W.ve[e];
  // gather kept corners (ring order starting after the run), then X and Y
  typename Prec<T>::V4 q;
  int ve = 0, st = 0, wt = -1;
  int src = -1;
  if (lane < keep) {
    src = (e + 1 + lane) % nv;
    q = W.vq[src]; ve = W.ve[src]; st = W.vst[src]; wt = W.vwit[src];
  }
  typename Prec<T>::V4 X, Y;
  if (lane == keep) {
    X = corner(W, 0, eX, pl);
    if (sizeof(T) == 4 && (C.force_exact || !(X.w <= T(3e-3) * sqrt(X.x * X.x + X.y * X.y + X.z * X.z)))) X = refine(C, W, a, i, X, eX, pl);
  }
  if (lane == keep + 1) {
    Y = corner(W, 0, pl, eY);
    if (sizeof(T) == 4 && (C.force_exact || !(Y.w <= T(3e-3) * sqrt(Y.x * Y.x + Y.y * Y.y + Y.z * Y.z)))) Y = refine(C, W, a, i, Y, pl, eY);
  }
  __syncwarp();
  if (lane < keep) { W.vq[lane] = q; W.ve[lane] = ve; W.vst[lane] = st; W.vwit[lane] = wt; }
  if (lane == keep) { W.vq[lane] = X; W.ve[lane] = pl; W.vst[lane] = 0; W.vwit[lane] = -1; }
  if (lane == keep + 1) { W.vq[lane] = Y; W.ve[lane] = eY; W.vst[lane] = 0; W.vwit[lane] = -1; }
  nv = m;
  __syncwarp();
  return 0;
}

template <typename T, bool EXT, bool POW = false>
__device__ void process_pair(const Dev<T>& C, WarpP<T>& W, int a, int i, long long slot, int lane) {
  using V4 = typename Prec<T>::V4;
  Counters K = {0, 0, 0, 0, 0, 0, 0, 0, 0};
  T vi[3] = {C.sites[3 * i], C.sites[3 * i + 1], C.sites[3 * i + 2]};
  const NbrList<T, EXT, POW> L = load_nbrs<T, EXT, POW>(C, i, lane);
  // power diagram: B_ij in the lifted space meets u = 0 in the power bisector (Sec. 6.3)
  auto lifted = [&](int j, V4& P, T& mx, T& mc) {
    if (POW) {
      T hj = (T)C.lift[j];
      P.w += T(0.5) * (hj * hj - L.hi * L.hi);
      mc += T(0.5) * (hj * hj + L.hi * L.hi);
    }
  };
  int np = 4, nv = 3;
  if (lane == 0) W.tied = 0;
  if (lane < 4) {
    V4 P;
    T mx, mc;
    if (lane == 0) plane_S(C, a, vi, P, mx, mc);
    else plane_E(C, a, lane - 1, vi, P, mx, mc);
    W.pn[lane] = P; W.pmx[lane] = mx; W.pmc[lane] = mc; W.psrc[lane] = lane == 0 ? -1 : -1 - lane;
  }
  if (lane < 3) {
    const T* V = vtx(C, a, lane);
    T qx = V[0] - vi[0], qy = V[1] - vi[1], qz = V[2] - vi[2];
    T qm = fmax(fabs(qx), fmax(fabs(qy), fabs(qz)));
    W.vq[lane] = Prec<T>::mk4(qx, qy, qz, T(2) * Prec<T>::U * qm);
    W.ve[lane] = 1 + lane;
    W.vst[lane] = 0;
    W.vwit[lane] = -1;
  }
  __syncwarp();
  bool empty = false;
  int nclip = 0;
  for (;;) {
    int p = -1;
    for (int k = 0; k < nv; ++k) {
      int st = W.vst[k];
      if (st == 1) continue;
      if (st == 2) { p = k; break; }
      V4 q = W.vq[k];
      int km = (k + nv - 1) % nv;
      int ex[3] = {W.psrc[W.ve[km]], W.psrc[W.ve[k]], -2};
      if (ex[0] < 0) ex[0] = -2;
      if (ex[1] < 0) ex[1] = -2;
      int nvv = nv, kk = k;
      bool uns = false;
      auto exact = [&](int site) {
        int r = exact_side(C, W, a, i, kk, nvv, site);
        uns |= r == 2 || r == -2;
        return r;
      };
      int wit, sc = 0, ls = 0;
      int out = corner_outside(C, i, vi[0], vi[1], vi[2], q.x, q.y, q.z, q.w, ex, lane, W.S, L, exact, &wit, &sc, &ls);
      // a corner found inside with a tie (or an uncertain sign) lies on that
      // site's bisector: the polygon may be degenerate there
      if (__any_sync(FULL, uns) && !out && lane == 0) W.tied = 1;
      K.corner++;
      K.nn++;
      K.scanned += sc;
      K.list += ls;
      if (*(volatile int*)C.status) return;
      __syncwarp();
      if (lane == 0) { W.vst[k] = out ? 2 : 1; W.vwit[k] = wit; }
      __syncwarp();
      if (out) { p = k; break; }
    }
    if (p < 0) break;
    if (++nclip > C.max_clips) { set_error(C.status, VD_ERR_LIMIT); return; }
    int j = find_bisector(C, W, L, i, vi, p, lane, K);
    if (np >= MAXPL) { set_error(C.status, VD_ERR_CAPACITY); return; }
    int pl = np++;
    {
      V4 P;
      T mx, mc;
      plane_B(C, j, vi, P, mx, mc);
      lifted(j, P, mx, mc);
      if (lane == 0) { W.pn[pl] = P; W.pmx[pl] = mx; W.pmc[pl] = mc; W.psrc[pl] = j; }
      __syncwarp();
      if (side_of(C, W, a, i, p, nv, pl) >= 0) {
        K.fallback++;
        j = W.vwit[p];
        plane_B(C, j, vi, P, mx, mc);
        lifted(j, P, mx, mc);
        __syncwarp();
        if (lane == 0) { W.pn[pl] = P; W.pmx[pl] = mx; W.pmc[pl] = mc; W.psrc[pl] = j; }
        __syncwarp();
      }
    }
    int rc = clip(C, W, a, i, pl, p, nv, lane);
    K.clips++;
    if (rc < 0) return;
    if (rc == 1) { empty = true; break; }
  }
  // integrate: area and first moment by a fan in the plane S, independently of
  // the clip history: corners recomputed from their planes in source order
  // (triangle vertices directly from the mesh), the fan starts at the corner with
  // the smallest key (sorted sources of its two edge planes) and runs in ring order
  T area = 0, mx = 0, my = 0, mz = 0;
  bool nonempty = false;
  if (!empty) {
    unsigned khi = 0xffffffffu, klo = 0xffffffffu;
    if (lane < nv) {
      int km = (lane + nv - 1) % nv;
      int pa = W.ve[km], pb = W.ve[lane];
      int sa = W.psrc[pa], sb = W.psrc[pb];
      V4 q;
      if (sa < -1 && sb < -1) {
        const T* V = vtx(C, a, -2 - sb);  // edge e starts at local vertex e
        T qx = V[0] - vi[0], qy = V[1] - vi[1], qz = V[2] - vi[2];
        q = Prec<T>::mk4(qx, qy, qz, T(2) * Prec<T>::U * fmax(fabs(qx), fmax(fabs(qy), fabs(qz))));
      } else {
        if (sa + 8 > sb + 8) { int t = pa; pa = pb; pb = t; }
        q = corner(W, 0, pa, pb);
        if (sizeof(T) == 4 && (C.force_exact || !(q.w <= T(3e-3) * sqrt(q.x * q.x + q.y * q.y + q.z * q.z)))) q = refine(C, W, a, i, q, pa, pb);
      }
      unsigned ua = (unsigned)(sa + 8), ub = (unsigned)(sb + 8);
      khi = min(ua, ub);
      klo = max(ua, ub);
      __syncwarp(__activemask());
      W.vq[lane] = q;
    }
    __syncwarp();
    unsigned mh = __reduce_min_sync(FULL, khi);
    unsigned ml = __reduce_min_sync(FULL, khi == mh ? klo : 0xffffffffu);
    int st = (int)__reduce_min_sync(FULL, (khi == mh && klo == ml) ? (unsigned)lane : 0xffffffffu);
    V4 S = W.pn[0];
    T sl = sqrt(S.x * S.x + S.y * S.y + S.z * S.z);
    T nx = S.x / sl, ny = S.y / sl, nz = S.z / sl;
    V4 O = W.vq[st];
    if (lane >= 1 && lane + 1 < nv) {
      V4 A = W.vq[(st + lane) % nv], B = W.vq[(st + lane + 1) % nv];
      T ax = A.x - O.x, ay = A.y - O.y, az = A.z - O.z;
      T bx = B.x - O.x, by = B.y - O.y, bz = B.z - O.z;
      T cx = ay * bz - az * by, cy = az * bx - ax * bz, cz = ax * by - ay * bx;
      area = T(0.5) * (nx * cx + ny * cy + nz * cz);
      mx = area * (ax + bx) / T(3);
      my = area * (ay + by) / T(3);
      mz = area * (az + bz) / T(3);
    }
    area = warp_sum(area);
    mx = warp_sum(mx) + area * O.x;
    my = warp_sum(my) + area * O.y;
    mz = warp_sum(mz) + area * O.z;
    nonempty = area > T(0);
  }
  // positive measure from the exact structure when no tie was met (as in 3D):
  // a polygon of at least three corners and each of its edges
  __syncwarp();
  const bool exact_faces = W.tied == 0;
  if (!empty && !nonempty && exact_faces) {
    nonempty = true;
    area = sizeof(T) == 4 ? T(1.17549435e-38) : T(2.2250738585072014e-308);
    mx = my = mz = T(0);
  }
  // edges of positive length: flags and propagation
  bool has = false, bis = false;
  int flag = 0;
  if (nonempty && lane < nv) {
    V4 A = W.vq[lane], B = W.vq[(lane + 1) % nv];
    T lx = B.x - A.x, ly = B.y - A.y, lz = B.z - A.z;
    if (exact_faces || lx * lx + ly * ly + lz * lz > T(0)) {
      int src = W.psrc[W.ve[lane]];
      bis = src >= 0;
      if (src >= 0) {
        flag = src;
        push_pair(C, a, src);
      } else {
        int ed = -2 - src;  // edge ed is opposite local vertex ed+2
        int b = C.adj[3 * a + (ed + 2) % 3];
        flag = b >= 0 ? -(b + 1) : FLAG_BOUNDARY;
        if (b >= 0) push_pair(C, b, i);
      }
      has = true;
    }
  }
  unsigned bm = __ballot_sync(FULL, has);
  int nflag = __popc(bm);
  unsigned nbis = C.want_stats ? __popc(__ballot_sync(FULL, bis)) : 0u;
  long long fbase = 0;
  if (lane == 0 && nflag) fbase = (long long)atomicAdd(C.ctr + CTR_FLAGS, (unsigned long long)nflag);
  fbase = __shfl_sync(FULL, fbase, 0);
  if (fbase + nflag > C.fcap) { set_error(C.status, VD_ERR_CAPACITY); return; }
  if (has) C.pflags[fbase + __popc(bm & ((1u << lane) - 1u))] = flag;
  if (lane == 0) {
    C.pmeas[slot] = nonempty ? area : T(0);
    C.pm1[3 * slot] = nonempty ? mx : T(0);
    C.pm1[3 * slot + 1] = nonempty ? my : T(0);
    C.pm1[3 * slot + 2] = nonempty ? mz : T(0);
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

}  // namespace cp
}  // namespace vd
