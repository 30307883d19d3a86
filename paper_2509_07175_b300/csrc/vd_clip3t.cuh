// vd_clip3t.cuh -- tetrahedron / Voronoi-cell intersection, one thread per pair.
//
// The same computation as vd_clip3.cuh (Alg. 3 on the dual-mesh polytope of
// Sec. 5.3, point-in-cell tests of Sec. 3.1, search of Sec. 3.2 / 5.1, the
// learned proposal), mapped one (tetrahedron, site) pair per thread as in the
// paper's own GPU form: every lane of a warp works on its own pair, so nothing
// waits on a reduction or a shuffle, at the cost of a per-thread polytope in
// local memory and sequential nearest-site scans.  Which mapping is faster
// depends on the workload; the autotuner of the host side times both.
//
// Results are bit-identical to the warp form: sign decisions are exact, and the
// final integration recomputes the corners from key-sorted planes and sums the
// per-corner terms in the same order and with the same summation tree as the
// warp form (32 lane partials over corner ranks r, r+32, r+64, then the
// butterfly of the warp sum).
#pragma once

#include "vd_clip3.cuh"

namespace vd {
namespace c3t {

using c3::GAMMA;
using c3::MAXP;
using c3::MAXT;
using c3::SIDEF;
using c3::U;

// per-thread polytope (local memory)
struct Poly {
  float4 pn[MAXP];
  float2 pm[MAXP];
  int psrc[MAXP];
  unsigned tv[MAXT];   // planes x | y << 8 | z << 16 (dual triangle, oriented)
  unsigned tn[MAXT];   // neighbours across x->y, y->z, z->x, same packing
  float4 tq[MAXT];     // corner (frame of v_i), w = coordinate error bound
  int twit[MAXT];      // certified closer site of an outside corner
  mutable int tied;    // this pair met an exact tie or an uncertain sign
};

struct Masks {
  unsigned alive[3], in[3], out[3];
  unsigned long long palive;
};

__device__ __forceinline__ int b0(unsigned p) { return (int)(p & 255u); }
__device__ __forceinline__ int b1(unsigned p) { return (int)((p >> 8) & 255u); }
__device__ __forceinline__ int b2(unsigned p) { return (int)((p >> 16) & 255u); }
__device__ __forceinline__ unsigned pack3(int x, int y, int z) {
  return (unsigned)x | ((unsigned)y << 8) | ((unsigned)z << 16);
}
__device__ __forceinline__ bool bit(const unsigned* m, int t) { return (m[t >> 5] >> (t & 31)) & 1u; }
__device__ __forceinline__ void setb(unsigned* m, int t) { m[t >> 5] |= 1u << (t & 31); }

// learned-form view of site i's 32 nearest sites / candidate list, read on demand
struct TList {
  const int* ids;    // 32 ids (knn form) or ncand ids (explicit candidates); null: plain
  unsigned cmask;    // knn form: candidate slots
  int n;             // slots
  bool explicit_cand;
  float r32;         // certified radius of the 32-NN list (0: no list certificate)
};

__device__ __forceinline__ TList load_list(const Dev<float>& C, int i) {
  TList L;
  L.ids = nullptr; L.cmask = 0; L.n = 0; L.explicit_cand = false; L.r32 = 0.f;
  if (C.knn) {
    L.ids = C.knn + (long long)i * 32;
    L.n = 32;
    float d32 = C.knn_d2[(long long)i * 32 + 31];
    int k32 = L.ids[31];
    L.r32 = (d32 > 0.f && k32 >= 0) ? sqrtf(d32 * (1.f - 1e-6f)) : 0.f;
    L.cmask = C.cmask[i];
  } else if (C.ncand > 0) {
    L.ids = C.cand + (long long)i * C.ncand;
    L.n = C.ncand < 32 ? C.ncand : 32;
    L.explicit_cand = true;
  }
  return L;
}

// slot s: site id (-1 none) and whether it is a ranked candidate
__device__ __forceinline__ int slot_id(const TList& L, int s, int i, bool& cand) {
  int k = L.ids[s];
  cand = L.explicit_cand ? (k >= 0 && k != i) : (k >= 0 && ((L.cmask >> s) & 1u));
  return k;
}

__device__ __forceinline__ bool any_cand(const TList& L, int i) {
  if (!L.ids) return false;
  for (int s = 0; s < L.n; ++s) {
    bool c;
    slot_id(L, s, i, c);
    if (c) return true;
  }
  return false;
}

struct Counters {
  unsigned nn, corner, clips, lam, search, learned, fallback, list;
  unsigned long long scanned;
  unsigned bisf, excess;  // bisector faces of the final pieces; clips that left none
};

// ----- nearest-site queries -------------------------------------------------------
__device__ int t_nearest(const Dev<float>& C, float qx, float qy, float qz, Counters& K) {
  const GridView<float>& G = C.G;
  float bd = 1e30f;
  int bi = 0x7fffffff;
  unsigned seen = 0;
  auto visit = [&](const float4& s) {
    float dx = s.x - qx, dy = s.y - qy, dz = s.z - qz;
    float d = dx * dx + dy * dy + dz * dz;
    int id = site_id(s);
    ++seen;
    if (d < bd || (d == bd && id < bi)) { bd = d; bi = id; }
  };
  for (int lev = G.query_level(qx, qy, qz); lev >= 0; --lev) {
    int cx, cy, cz;
    G.cell_at(lev, qx, qy, qz, cx, cy, cz);
    bool done = false;
    for (int r = 1;; ++r) {
      thread_scan_ring(G, lev, cx, cy, cz, r, visit);
      float m = G.cover(lev, cx, cy, cz, r, qx, qy, qz);
      if (m >= 1e29f || (m > 0.f && bd <= m * m)) { done = true; break; }
      if (lev > 0 ? r >= HASH_MAX_RING : r >= G.max_ring()) break;
    }
    if (done || lev == 0) break;
  }
  K.nn++;
  K.scanned += seen;
  return bi;
}

// nearest site of v_i + s; from the 32-NN list when 2|s| <= r32 (as the warp form)
__device__ int t_nn_search(const Dev<float>& C, const TList& L, int i, float3 vi, float sx, float sy, float sz,
                           Counters& K) {
  float px = vi.x + sx, py = vi.y + sy, pz = vi.z + sz;
  if (L.r32 > 0.f) {
    float s = sqrtf(sx * sx + sy * sy + sz * sz);
    if (2.f * s * (1.f + 1e-5f) + 4e-7f * (fabsf(px) + fabsf(py) + fabsf(pz)) <= L.r32) {
      float dxi = vi.x - px, dyi = vi.y - py, dzi = vi.z - pz;
      float bd = dxi * dxi + dyi * dyi + dzi * dzi;
      int bk = i;
      for (int t = 0; t < 32; ++t) {
        int k = L.ids[t];
        if (k < 0) continue;
        float dx = C.sites[3 * k] - px, dy = C.sites[3 * k + 1] - py, dz = C.sites[3 * k + 2] - pz;
        float d2 = dx * dx + dy * dy + dz * dz;
        if (d2 < bd || (d2 == bd && k < bk)) { bd = d2; bk = k; }
      }
      K.list++;
      K.nn++;
      return bk;
    }
  }
  return t_nearest(C, px, py, pz, K);
}

// ----- exact side test -------------------------------------------------------------
__device__ __noinline__ int t_exact_side(const Dev<float>& C, const Poly& P, int a, int i, int t, int src4) {
  unsigned v = P.tv[t];
  int s0 = P.psrc[b0(v)], s1 = P.psrc[b1(v)], s2 = P.psrc[b2(v)];
  if (src4 == s0 || src4 == s1 || src4 == s2) return 0;
  ePlane p[4];
  p[0] = c3::eplane(C, a, i, s0);
  p[1] = c3::eplane(C, a, i, s1);
  p[2] = c3::eplane(C, a, i, s2);
  p[3] = c3::eplane(C, a, i, src4);
  int certain, tie;
  int s = side_from_planes(p, &certain, &tie);
  atomicAdd(C.stats + VD_STAT_FP64, 1ull);
  if (!certain) {
    atomicAdd(C.stats + (tie ? VD_STAT_TIES : VD_STAT_UNCERTAIN), 1ull);
    record_diag(C.stats, a, i, s0, s1, s2, src4, tie, 0);
    return s < 0 ? -2 : 2;  // not certified: +-2 (a tie counts as inside)
  }
  return s;
}

__device__ __forceinline__ int t_side_of(const Dev<float>& C, const Poly& P, int a, int i, int t, int pl) {
  float4 q = P.tq[t];
  float4 Pl = P.pn[pl];
  float2 M = P.pm[pl];
  if (q.w < 1e29f && !C.force_exact) {
    float s = Pl.w - (Pl.x * q.x + Pl.y * q.y + Pl.z * q.z);
    float qm = fmaxf(fabsf(q.x), fmaxf(fabsf(q.y), fabsf(q.z)));
    float b = (fabsf(Pl.x) + fabsf(Pl.y) + fabsf(Pl.z)) * q.w + SIDEF * (M.y + M.x * qm);
    if (s > b) return 1;
    if (s < -b) return -1;
  }
  int r = t_exact_side(C, P, a, i, t, P.psrc[pl]);
  if (r == 2 || r == -2) P.tied = 1;
  return r;
}

// ----- point-in-cell test of a corner (Sec. 3.1; same criterion as the warp form) ---
__device__ __noinline__ int t_corner_outside(const Dev<float>& C, const Poly& P, const TList& L, int a, int i,
                                            float3 vi, int t, int* wit, Counters& K) {
  float4 q = P.tq[t];
  unsigned v = P.tv[t];
  int e0 = P.psrc[b0(v)], e1 = P.psrc[b1(v)], e2 = P.psrc[b2(v)];
  if (e0 < 0) e0 = -2;
  if (e1 < 0) e1 = -2;
  if (e2 < 0) e2 = -2;
  const float Uf = Prec<float>::U;
  float gx = vi.x + q.x, gy = vi.y + q.y, gz = vi.z + q.z;
  float di2;
  {
    float dx = vi.x - gx, dy = vi.y - gy, dz = vi.z - gz;
    di2 = dx * dx + dy * dy + dz * dz;
  }
  float di = sqrtf(di2);
  float gmax = fmaxf(fabsf(gx), fmaxf(fabsf(gy), fabsf(gz)));
  float delta = 1.7320508075688772f * (q.w + 2.f * Uf * gmax);
  float D = 1.2f * di + delta;
  float B = 4.5f * D * delta + 2.5f * delta * delta + 16.f * Uf * D * D;
  bool well = delta <= 0.03f * di;
  float R = di * (1.f + 1e-5f) + 2.f * delta + 4.f * Uf * gmax;
  float amb = well ? B : (R * R - di2) + B;
  if (!well && C.want_stats) atomicAdd(C.stats + VD_STAT_ILLCOND, 1ull);
  K.corner++;
  K.nn++;
  // a tie (or an uncertain sign) met by a corner found inside puts it on that
  // site's bisector: the pair's polytope may be degenerate there
  bool uns = false;
  auto exact = [&](int k) {
    int r = t_exact_side(C, P, a, i, t, k);
    uns |= r == 2 || r == -2;
    return r;
  };
  // 32-NN list certificate (learned form)
  if (L.r32 > 0.f && (double)L.r32 >= 2.0 * ((double)di + (double)delta) * (1.0 + 1e-5) + 1e-30) {
    K.list++;
    float ld = 1e30f, lo = 1e30f;
    int lk = 0x7fffffff, lok = 0x7fffffff;
    for (int s = 0; s < 32; ++s) {
      int k = L.ids[s];
      if (k < 0 || k == e0 || k == e1 || k == e2) continue;
      float dx = C.sites[3 * k] - gx, dy = C.sites[3 * k + 1] - gy, dz = C.sites[3 * k + 2] - gz;
      float d2 = dx * dx + dy * dy + dz * dz;
      float f = d2 - di2;
      if (f < -B) {
        if (d2 < ld || (d2 == ld && k < lk)) { ld = d2; lk = k; }
      } else if (f <= B && (d2 < lo || (d2 == lo && k < lok)) && exact(k) < 0) {
        lo = d2; lok = k;
      }
    }
    if (lk != 0x7fffffff) { *wit = lk; return 1; }
    if (lok != 0x7fffffff) { *wit = lok; return 1; }
    if (uns) P.tied = 1;
    *wit = -1;
    return 0;
  }
  // ranked-candidate outside certificate (learned proposal)
  if (L.ids) {
    float cd = 1e30f;
    int ck = 0x7fffffff;
    bool anyc = false;
    for (int s = 0; s < L.n; ++s) {
      bool c;
      int k = slot_id(L, s, i, c);
      if (!c) continue;
      anyc = true;
      if (k == i || k == e0 || k == e1 || k == e2) continue;
      float dx = C.sites[3 * k] - gx, dy = C.sites[3 * k + 1] - gy, dz = C.sites[3 * k + 2] - gz;
      float d2 = dx * dx + dy * dy + dz * dz;
      if (d2 - di2 < -B && (d2 < cd || (d2 == cd && k < ck))) { cd = d2; ck = k; }
    }
    if (anyc && ck != 0x7fffffff) { *wit = ck; K.list++; return 1; }
  }
  float bd = 1e30f, od = 1e30f;
  int bk = 0x7fffffff, ok = 0x7fffffff;
  unsigned seen = 0;
  auto visit = [&](const float4& s) {
    ++seen;
    int k = site_id(s);
    if (k == i || k == e0 || k == e1 || k == e2) return;
    float dx = s.x - gx, dy = s.y - gy, dz = s.z - gz;
    float d2 = dx * dx + dy * dy + dz * dz;
    float f = d2 - di2;
    if (d2 < bd || (d2 == bd && k < bk)) { bd = d2; bk = k; }
    if (f >= -B && f <= amb && (d2 < od || (d2 == od && k < ok)) && exact(k) < 0) {
      od = d2; ok = k;
    }
  };
  const GridView<float>& G = C.G;
  for (int lev = G.query_level(gx, gy, gz); lev >= 0; --lev) {
    int cx, cy, cz;
    G.cell_at(lev, gx, gy, gz, cx, cy, cz);
    bool done = false;
    for (int r = 1;; ++r) {
      thread_scan_ring(G, lev, cx, cy, cz, r, visit);
      if (bd - di2 < -B) { done = true; break; }
      float m = G.cover(lev, cx, cy, cz, r, gx, gy, gz);
      if (m >= 1e29f || m >= R) { done = true; break; }
      if (lev > 0 ? r >= HASH_MAX_RING : r >= G.max_ring()) break;
    }
    if (done) break;
  }
  K.scanned += seen;
  if (bd - di2 < -B) { *wit = bk; return 1; }
  if (ok != 0x7fffffff) { *wit = ok; return 1; }
  if (uns) P.tied = 1;
  *wit = -1;
  return 0;
}

// ----- bisector search (Sec. 3.2, start point of Sec. 5.1, learned shortcut) ----------
__device__ __noinline__ int t_find_bisector(const Dev<float>& C, const Poly& P, const TList& L, int i, float3 vi,
                                            int t, Counters& K) {
  float4 q = P.tq[t];
  int wit = P.twit[t];
  float dist = sqrtf(q.x * q.x + q.y * q.y + q.z * q.z);
  float dx = q.x / dist, dy = q.y / dist, dz = q.z / dist;
  float gx = q.x, gy = q.y, gz = q.z;
  int j = wit;
  float delta = C.delta[i];
  if (L.ids) {
    // candidates of the ranking, plus the witness when some slot is not a candidate
    float tb = 1.f;
    int cb = 0x7fffffff;
    int ncand = 0;
    auto consider = [&](int k, float kx, float ky, float kz) {
      if (k < 0 || k == i) return;
      float wx = kx - vi.x, wy = ky - vi.y, wz = kz - vi.z;
      float den = wx * q.x + wy * q.y + wz * q.z;
      if (den > 0.f) {
        float tt = 0.5f * (wx * wx + wy * wy + wz * wz) / den;
        if (tt < 1.f && (tt < tb || (tt == tb && k < cb))) { tb = tt; cb = k; }
      }
    };
    for (int s = 0; s < 32; ++s) {
      bool c = false;
      int k = s < L.n ? slot_id(L, s, i, c) : -1;
      if (!c) continue;
      ++ncand;
      consider(k, C.sites[3 * k], C.sites[3 * k + 1], C.sites[3 * k + 2]);
    }
    if (ncand > 0) {
      if (ncand < 32 && wit >= 0) consider(wit, C.sites[3 * wit], C.sites[3 * wit + 1], C.sites[3 * wit + 2]);
      if (cb != 0x7fffffff) {
        float sx = q.x * tb, sy = q.y * tb, sz = q.z * tb;
        int kk = t_nn_search(C, L, i, vi, sx, sy, sz, K);
        K.search++;
        if (kk == i || kk == cb) { K.learned++; return cb; }
        j = kk;
        gx = sx; gy = sy; gz = sz;
        goto search;
      }
    }
  }
  for (int lam = 2; lam < 2 + C.max_lambda; ++lam) {
    float step = (float)lam * delta;
    if (!(step < dist)) break;
    float sx = dx * step, sy = dy * step, sz = dz * step;
    int k = t_nearest(C, vi.x + sx, vi.y + sy, vi.z + sz, K);
    K.lam++;
    if (k != i) { gx = sx; gy = sy; gz = sz; j = k; break; }
  }
search:
  for (int s = 0; s < C.max_search; ++s) {
    float wx = C.sites[3 * j] - vi.x, wy = C.sites[3 * j + 1] - vi.y, wz = C.sites[3 * j + 2] - vi.z;
    float den = wx * gx + wy * gy + wz * gz;
    if (!(den > 0.f)) { K.fallback++; return wit; }
    float tt = 0.5f * (wx * wx + wy * wy + wz * wz) / den;
    if (!(tt < 1.f)) return j;
    float sx = gx * tt, sy = gy * tt, sz = gz * tt;
    int k = t_nn_search(C, L, i, vi, sx, sy, sz, K);
    K.search++;
    if (k == i || k == j) return j;
    j = k;
    gx = sx; gy = sy; gz = sz;
  }
  K.fallback++;
  return wit;
}

// ----- clip (Sec. 5.3: remove the component R_p of outside corners holding p) ------
// Returns 0 (clipped), 1 (P became empty), -1 (error, status set).
__device__ __noinline__ int t_clip(const Dev<float>& C, Poly& P, Masks& Mk, int a, int i, int pl, int p) {
  unsigned om[3] = {0, 0, 0}, R[3] = {0, 0, 0};
  for (int r = 0; r < 3; ++r) {
    unsigned m = Mk.alive[r] & ~Mk.in[r];  // corners proven inside Omega_i stay (Sec. 3.3)
    while (m) {
      int b = __ffs(m) - 1;
      m &= m - 1;
      int t = 32 * r + b;
      if (t_side_of(C, P, a, i, t, pl) < 0) om[r] |= 1u << b;
    }
  }
  if (!bit(om, p)) { set_error(C.status, VD_ERR_LIMIT); return -1; }
  // connected component of p among the outside corners (depth-first, explicit stack)
  unsigned char stk[MAXT];
  int sp = 0;
  setb(R, p);
  stk[sp++] = (unsigned char)p;
  while (sp > 0) {
    int t = stk[--sp];
    unsigned nb = P.tn[t];
    int nn[3] = {b0(nb), b1(nb), b2(nb)};
    for (int e = 0; e < 3; ++e) {
      int u = nn[e];
      if (bit(om, u) && !bit(R, u)) { setb(R, u); stk[sp++] = (unsigned char)u; }
    }
  }
  if (R[0] == Mk.alive[0] && R[1] == Mk.alive[1] && R[2] == Mk.alive[2]) return 1;
  // boundary edges of R (x -> y of a removed corner whose neighbour u is kept)
  unsigned edge[MAXT];
  int cnt = 0;
  for (int r = 0; r < 3; ++r) {
    unsigned m = R[r];
    while (m) {
      int b = __ffs(m) - 1;
      m &= m - 1;
      int t = 32 * r + b;
      unsigned v = P.tv[t], nb = P.tn[t];
      int vv[3] = {b0(v), b1(v), b2(v)}, nn[3] = {b0(nb), b1(nb), b2(nb)};
      for (int e = 0; e < 3; ++e)
        if (!bit(R, nn[e])) {
          if (cnt >= MAXT) { set_error(C.status, VD_ERR_CAPACITY); return -1; }
          edge[cnt++] = pack3(vv[e], vv[(e + 1) % 3], nn[e]);
        }
    }
  }
  unsigned fr[3] = {~Mk.alive[0] | R[0], ~Mk.alive[1] | R[1], ~Mk.alive[2] | R[2]};
  int nfree = __popc(fr[0]) + __popc(fr[1]) + __popc(fr[2]);
  if (cnt > nfree || cnt < 3) { set_error(C.status, cnt < 3 ? VD_ERR_LIMIT : VD_ERR_CAPACITY); return -1; }
  signed char stri[MAXP], etri[MAXP];
  for (int x = 0; x < MAXP; ++x) stri[x] = etri[x] = -1;
  unsigned char slot[MAXT];
  {
    int r = 0;
    unsigned m = fr[0];
    for (int c = 0; c < cnt; ++c) {
      while (!m) m = fr[++r];
      int b = __ffs(m) - 1;
      m &= m - 1;
      int sl = 32 * r + b;
      slot[c] = (unsigned char)sl;
      int x = b0(edge[c]), y = b1(edge[c]);
      if (stri[x] != -1 || etri[y] != -1) { set_error(C.status, VD_ERR_LIMIT); return -1; }
      stri[x] = (signed char)sl;
      etri[y] = (signed char)sl;
    }
  }
  float4 Pn = P.pn[pl];
  float2 Mn = P.pm[pl];
  unsigned newm[3] = {0, 0, 0};
  for (int c = 0; c < cnt; ++c) {
    int sl = slot[c], x = b0(edge[c]), y = b1(edge[c]), u = b2(edge[c]);
    if (stri[y] < 0 || etri[x] < 0) { set_error(C.status, VD_ERR_LIMIT); return -1; }  // boundary not a loop
    P.tv[sl] = pack3(x, y, pl);
    P.tn[sl] = pack3(u, stri[y], etri[x]);
    unsigned uv = P.tv[u], un = P.tn[u];
    if (b0(uv) == y && b1(uv) == x) un = (un & ~0xFFu) | (unsigned)sl;
    else if (b1(uv) == y && b2(uv) == x) un = (un & ~0xFF00u) | ((unsigned)sl << 8);
    else if (b2(uv) == y && b0(uv) == x) un = (un & ~0xFF0000u) | ((unsigned)sl << 16);
    else { set_error(C.status, VD_ERR_LIMIT); return -1; }
    P.tn[u] = un;
    float4 qc = c3::corner(P.pn[x], P.pm[x], P.pn[y], P.pm[y], Pn, Mn);
    if (c3::loose(qc) || C.force_exact)
      qc = c3::refine64(C, a, i, P.psrc[x], P.psrc[y], P.psrc[pl]);
    P.tq[sl] = qc;
    P.twit[sl] = -1;
    setb(newm, sl);
  }
  for (int r = 0; r < 3; ++r) {
    Mk.alive[r] = (Mk.alive[r] & ~R[r]) | newm[r];
    Mk.in[r] &= ~(R[r] | newm[r]);
    Mk.out[r] &= ~(R[r] | newm[r]);
  }
  unsigned long long pmask = 0;
  for (int r = 0; r < 3; ++r) {
    unsigned m = Mk.alive[r];
    while (m) {
      int b = __ffs(m) - 1;
      m &= m - 1;
      unsigned v = P.tv[32 * r + b];
      pmask |= (1ull << b0(v)) | (1ull << b1(v)) | (1ull << b2(v));
    }
  }
  Mk.palive = pmask;
  return 0;
}

// ----- canonical integration (bit-identical to c3::integrate) -------------------------
__device__ __noinline__ void t_integrate(const Dev<float>& C, Poly& P, const Masks& Mk, int a, int i, float3 vi,
                                         float sigma, float& vol, float3& m1, unsigned long long& posarea) {
  unsigned long long pkey[MAXP];
  unsigned char pref[MAXP], prank[MAXP];
  for (int x = 0; x < MAXP; ++x) {
    pkey[x] = ~0ull;
    int rk = 0;
    if ((Mk.palive >> x) & 1ull) {
      int sx = P.psrc[x];
      for (unsigned long long m = Mk.palive; m; m &= m - 1) rk += P.psrc[__ffsll((long long)m) - 1] < sx;
    }
    prank[x] = (unsigned char)rk;
  }
  unsigned long long key[MAXT];
  unsigned char list[MAXT];
  int nalive = 0;
  for (int r = 0; r < 3; ++r) {
    unsigned m = Mk.alive[r];
    while (m) {
      int b = __ffs(m) - 1;
      m &= m - 1;
      int t = 32 * r + b;
      list[nalive++] = (unsigned char)t;
      unsigned v = P.tv[t];
      int pl[3] = {b0(v), b1(v), b2(v)};
      int sr[3] = {P.psrc[pl[0]], P.psrc[pl[1]], P.psrc[pl[2]]};
      for (int u = 0; u < 2; ++u)
        for (int w = 0; w < 2 - u; ++w)
          if (sr[w] + 4 > sr[w + 1] + 4) {
            int tt = sr[w]; sr[w] = sr[w + 1]; sr[w + 1] = tt;
            tt = pl[w]; pl[w] = pl[w + 1]; pl[w + 1] = tt;
          }
      float4 q;
      if (sr[2] < 0) {
        int k = 6 - (-1 - sr[0]) - (-1 - sr[1]) - (-1 - sr[2]);
        const float* V = C.verts + 3 * C.simp[4 * a + k];
        float qx = V[0] - vi.x, qy = V[1] - vi.y, qz = V[2] - vi.z;
        q = make_float4(qx, qy, qz, 2.f * U * fmaxf(fabsf(qx), fmaxf(fabsf(qy), fabsf(qz))));
      } else {
        q = c3::corner(P.pn[pl[0]], P.pm[pl[0]], P.pn[pl[1]], P.pm[pl[1]], P.pn[pl[2]], P.pm[pl[2]]);
        if (c3::loose(q) || C.force_exact) q = c3::refine64(C, a, i, sr[0], sr[1], sr[2]);
      }
      P.tq[t] = q;
      unsigned long long kk = c3::corner_key(prank[pl[0]], prank[pl[1]], prank[pl[2]]);
      key[t] = kk;
      int vx = b0(v), vy = b1(v), vz = b2(v);
      if (kk < pkey[vx]) pkey[vx] = kk;
      if (kk < pkey[vy]) pkey[vy] = kk;
      if (kk < pkey[vz]) pkey[vz] = kk;
    }
  }
  // order the corners by key (insertion sort of the slot list; keys are distinct)
  for (int u = 1; u < nalive; ++u) {
    unsigned char t = list[u];
    unsigned long long kt = key[t];
    int w = u - 1;
    while (w >= 0 && (key[list[w]] > kt || (key[list[w]] == kt && list[w] > t))) { list[w + 1] = list[w]; --w; }
    list[w + 1] = t;
  }
  for (int u = 0; u < nalive; ++u) {
    int t = list[u];
    unsigned v = P.tv[t];
    if (pkey[b0(v)] == key[t]) pref[b0(v)] = (unsigned char)t;
    if (pkey[b1(v)] == key[t]) pref[b1(v)] = (unsigned char)t;
    if (pkey[b2(v)] == key[t]) pref[b2(v)] = (unsigned char)t;
  }
  float4 O = P.tq[list[0]];
  float parea[MAXP][3];
  for (int x = 0; x < MAXP; ++x) parea[x][0] = parea[x][1] = parea[x][2] = 0.f;
  // lane partials of the warp form: lane l holds ranks l, l+32, l+64 summed in that order
  float4 part[32];
  for (int l = 0; l < 32; ++l) part[l] = make_float4(0.f, 0.f, 0.f, 0.f);
  for (int rank = 0; rank < nalive; ++rank) {
    int t = list[rank];
    unsigned v = P.tv[t], nb = P.tn[t];
    float4 A4 = P.tq[t];
    float ax = A4.x - O.x, ay = A4.y - O.y, az = A4.z - O.z;
    int fx[3] = {b0(v), b1(v), b2(v)}, fn[3] = {b0(nb), b1(nb), b2(nb)};
    int sr[3] = {P.psrc[fx[0]] + 4, P.psrc[fx[1]] + 4, P.psrc[fx[2]] + 4};
    int ord[3] = {0, 1, 2};
    for (int u = 0; u < 2; ++u)
      for (int w = 0; w < 2 - u; ++w)
        if (sr[ord[w]] > sr[ord[w + 1]]) { int tt = ord[w]; ord[w] = ord[w + 1]; ord[w + 1] = tt; }
    float4 Rq[3], Bq[3];
    for (int e3 = 0; e3 < 3; ++e3) {
      int e = ord[e3];
      int x = fx[e];
      Rq[e3] = P.tq[pref[x]];
      Bq[e3] = P.tq[fn[e]];
      float rx = Rq[e3].x - O.x, ry = Rq[e3].y - O.y, rz = Rq[e3].z - O.z;
      float bx = Bq[e3].x - O.x, by = Bq[e3].y - O.y, bz = Bq[e3].z - O.z;
      float ux = ax - rx, uy = ay - ry, uz = az - rz, wx = bx - rx, wy = by - ry, wz = bz - rz;
      parea[x][0] += uy * wz - uz * wy;
      parea[x][1] += uz * wx - ux * wz;
      parea[x][2] += ux * wy - uy * wx;
    }
    float4 c4 = c3::corner_terms(A4, O, Rq[0], Bq[0], Rq[1], Bq[1], Rq[2], Bq[2]);
    float4& pt = part[rank & 31];
    pt.x += c4.x; pt.y += c4.y; pt.z += c4.z; pt.w += c4.w;
  }
  // butterfly of the warp sum (xor offsets 16, 8, 4, 2, 1)
  for (int o = 16; o > 0; o >>= 1)
    for (int l = 0; l < 32; ++l)
      if (l < (l ^ o)) {
        float4 A = part[l], Bv = part[l ^ o];
        float4 S = make_float4(A.x + Bv.x, A.y + Bv.y, A.z + Bv.z, A.w + Bv.w);
        part[l] = S;
        part[l ^ o] = S;
      }
  float4 F = c3::finish_moments(sigma, part[0], O);
  vol = F.x;
  m1 = make_float3(F.y, F.z, F.w);
  unsigned long long pa = 0;
  for (int x = 0; x < MAXP; ++x)
    if ((Mk.palive >> x) & 1ull) {
      float ax = parea[x][0], ay = parea[x][1], az = parea[x][2];
      // exact structure without a tie: every alive plane is a face of positive area
      if (!P.tied || ax * ax + ay * ay + az * az > 0.f) pa |= 1ull << x;
    }
  posarea = pa;
}

__device__ void t_init_tet(const Dev<float>& C, Poly& P, Masks& Mk, int a, float3 vi) {
  for (int k = 0; k < 4; ++k) {
    float4 Pl;
    float2 M;
    c3::plane_face(C, a, k, vi, Pl, M);
    P.pn[k] = Pl; P.pm[k] = M; P.psrc[k] = -1 - k;
    const float* V = C.verts + 3 * C.simp[4 * a + k];
    float qx = V[0] - vi.x, qy = V[1] - vi.y, qz = V[2] - vi.z;
    float qm = fmaxf(fabsf(qx), fmaxf(fabsf(qy), fabsf(qz)));
    P.tq[k] = make_float4(qx, qy, qz, 2.f * U * qm);
    int x = c3::TET_TV[k][0], y = c3::TET_TV[k][1], z = c3::TET_TV[k][2];
    P.tv[k] = pack3(x, y, z);
    P.tn[k] = pack3(6 - k - x - y, 6 - k - y - z, 6 - k - z - x);
    P.twit[k] = -1;
  }
  Mk.alive[0] = 0xFu; Mk.alive[1] = Mk.alive[2] = 0;
  Mk.in[0] = Mk.in[1] = Mk.in[2] = 0;
  Mk.out[0] = Mk.out[1] = Mk.out[2] = 0;
  Mk.palive = 0xFull;
}

// One pair; counters accumulate into K (flushed by the caller).
__device__ void process_pair(const Dev<float>& C, Poly& P, int a, int i, long long slot, Counters& K) {
  const TList L = load_list(C, i);
  float3 vi = make_float3(C.sites[3 * i], C.sites[3 * i + 1], C.sites[3 * i + 2]);
  Masks Mk;
  t_init_tet(C, P, Mk, a, vi);
  P.tied = 0;
  float sigma;
  {
    sigma = (float)C.tsgn[a];
  }
  bool empty = false;
  int nclip = 0;
  unsigned pclips = 0;
  for (;;) {
    int p = -1;
    for (;;) {
      unsigned c0 = Mk.alive[0] & ~Mk.in[0], c1 = Mk.alive[1] & ~Mk.in[1], c2 = Mk.alive[2] & ~Mk.in[2];
      int t = c0 ? __ffs(c0) - 1 : (c1 ? 31 + __ffs(c1) : (c2 ? 63 + __ffs(c2) : -1));
      if (t < 0) break;
      if (bit(Mk.out, t)) { p = t; break; }
      int wit;
      if (t_corner_outside(C, P, L, a, i, vi, t, &wit, K)) {
        setb(Mk.out, t);
        P.twit[t] = wit;
        p = t;
        break;
      }
      setb(Mk.in, t);
    }
    if (p < 0) break;
    if (++nclip > C.max_clips) { set_error(C.status, VD_ERR_LIMIT); return; }
    if (*(volatile int*)C.status) return;
    int j = t_find_bisector(C, P, L, i, vi, p, K);
    unsigned long long freep = ~Mk.palive & ((1ull << MAXP) - 1ull);
    if (!freep) { set_error(C.status, VD_ERR_CAPACITY); return; }
    int pl = __ffsll((long long)freep) - 1;
    float4 Pl;
    float2 M;
    c3::plane_bis(C, j, vi, Pl, M);
    P.pn[pl] = Pl; P.pm[pl] = M; P.psrc[pl] = j;
    if (t_side_of(C, P, a, i, p, pl) >= 0) {
      K.fallback++;
      j = P.twit[p];
      c3::plane_bis(C, j, vi, Pl, M);
      P.pn[pl] = Pl; P.pm[pl] = M; P.psrc[pl] = j;
    }
    int rc = t_clip(C, P, Mk, a, i, pl, p);
    K.clips++;
    ++pclips;
    if (rc < 0) return;
    if (rc == 1) { empty = true; break; }
  }
  float vol = 0.f;
  float3 m1 = make_float3(0.f, 0.f, 0.f);
  unsigned long long posarea = 0;
  if (!empty) t_integrate(C, P, Mk, a, i, vi, sigma, vol, m1, posarea);
  bool nonempty = !empty && (vol > 0.f || !P.tied);
  if (nonempty && !(vol > 0.f)) {  // a sliver below FP32 resolution (as in the warp form)
    vol = 1.17549435e-38f;
    m1 = make_float3(0.f, 0.f, 0.f);
  }
  int nflag = nonempty ? __popcll(posarea) : 0;
  long long fbase = nflag ? (long long)atomicAdd(C.ctr + CTR_FLAGS, (unsigned long long)nflag) : 0;
  if (fbase + nflag > C.fcap) { set_error(C.status, VD_ERR_CAPACITY); return; }
  unsigned nbis = 0;
  if (nflag) {
    int w = 0;
    unsigned long long m = posarea;
    while (m) {
      int x = __ffsll((long long)m) - 1;
      m &= m - 1;
      int src = P.psrc[x], flag;
      nbis += src >= 0;
      if (src >= 0) {
        flag = src;
        push_pair(C, a, src);
      } else {
        int b = C.adj[4 * a + (-1 - src)];
        flag = b >= 0 ? -(b + 1) : FLAG_BOUNDARY;
        if (b >= 0) push_pair(C, b, i);
      }
      C.pflags[fbase + w++] = flag;
    }
  }
  C.pmeas[slot] = nonempty ? vol : 0.f;
  C.pm1[3 * slot] = nonempty ? m1.x : 0.f;
  C.pm1[3 * slot + 1] = nonempty ? m1.y : 0.f;
  C.pm1[3 * slot + 2] = nonempty ? m1.z : 0.f;
  C.pfoff[slot] = fbase;
  C.pfcnt[slot] = nflag;
  K.bisf += nbis;
  K.excess += pclips > nbis ? pclips - nbis : 0u;
}

}  // namespace c3t
}  // namespace vd
