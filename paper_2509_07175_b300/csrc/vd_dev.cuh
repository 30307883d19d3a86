// vd_dev.cuh -- device context, (simplex, site) pair set and work queue, and
// the certified point-in-cell test on polytope corners (Sec. 3.1).
#pragma once

#include "vd_grid.cuh"

namespace vd {

// counters in Dev::ctr
enum { CTR_TAIL = 0, CTR_HEAD = 1, CTR_DONE = 2, CTR_FLAGS = 3, CTR_SEEDS = 4, CTR_OUT = 5, CTR_MARK = 6, CTR_OWNED = 7, CTR_N = 8 };

template <typename T>
struct Dev {
  int mode;              // VD_MODE_*
  int n, m, k;           // sites, simplices, vertices per simplex
  const T* sites;        // [n*3] original order (z = 0 in 2D)
  const T* verts;        // [nv*3]
  const int* simp;       // [m*k]
  const int* adj;        // [m*k] neighbour across the face opposite local vertex f, -1: boundary
  const signed char* fsgn;  // [m*k] +-1: orientation making the face normal point outward
  const signed char* tsgn;  // [m] 3D: +-1, the sign of the tetrahedron's orientation determinant
  const T* delta;        // [n] half the distance to the nearest other site (Sec. 5.1)
  GridView<T> G;
  // learned proposal: candidate bisector neighbours of each site (ranked)
  const int* cand;       // [n*ncand] candidate neighbours, -1 unused
  int ncand;             // 0: plain search (Sec. 3.2 / 5.1 only)
  const int* knn;        // [n*32] nearest other sites, ascending (learned form), or null
  const float* knn_d2;   // [n*32] their squared distances (FP32); 32nd < 0: list not certified
  const unsigned* cmask; // [n] learned form: which of the 32 nearest are ranked candidates
  const int* knn2;       // [n*32] the 33rd..64th nearest (any order, -1 unused), or null
  const float* knn_r64;  // [n] certified radius of the 64 nearest (0: not certified)
  // power diagrams (Sec. 6.3): site i lifted to (v_i, h_i), h_i = sqrt(eta - w_i);
  // distances are taken to the lifted sites (null: Voronoi diagram)
  const float* lift;     // [n] h_i
  float lift_max;        // max_i h_i
  // pair set and queue
  unsigned long long* hash;
  unsigned long long hmask;
  unsigned long long* queue;
  long long qcap;
  unsigned long long* ctr;  // CTR_*
  // per queue slot output
  T* pmeas;
  T* pm1;                // [qcap*3] first moment, frame of the site
  long long* pfoff;      // start of the slot's flags in pflags
  int* pfcnt;            // number of flags
  int* pflags;
  long long fcap;
  // status
  int* status;
  unsigned long long* stats;  // [VD_STAT_N]
  int want_stats;
  int max_clips, max_search, max_lambda;
  long long wait_ns;
  // box domain (Sec. 4.2, a convex domain with few corners): one piece per site,
  // the box [blo, bhi] clipped by the site's bisectors; faces 0..5 = -x, +x, -y,
  // +y, -z, +z
  int box;
  float blo[3], bhi[3];
  // split (Alg. 5, 3D): pairs (m, i) are whole cells, the box [blo, bhi] (the mesh's
  // bounding box) clipped by the site's bisectors; the pieces of per-tetrahedron
  // pairs propagate through negative flags only
  int split;
  int force_exact;       // 1: every clip decision and new corner through the float64 path
  // partition of one diagram across ranks (site ownership): pairs of sites this
  // rank does not own are recorded in the outbox for their owner instead of being
  // queued (null owner: one rank owns every site)
  const int* owner;      // [n] rank of each site, or null
  int rank;
  int* own_order;        // [n] grid-order positions of the rank's own sites (CTR_OWNED of them), or null
  unsigned long long* outbox;
  long long ocap;
};

template <typename T>
__device__ __forceinline__ bool owned(const Dev<T>& C, int i) {
  return !C.owner || C.owner[i] == C.rank;
}

__device__ __forceinline__ unsigned long long pair_key(int a, int i) {
  return ((unsigned long long)(unsigned)a << 32) | (unsigned)i;
}
__device__ __forceinline__ unsigned long long mix64(unsigned long long x) {
  x ^= x >> 30; x *= 0xbf58476d1ce4e5b9ull;
  x ^= x >> 27; x *= 0x94d049bb133111ebull;
  x ^= x >> 31;
  return x;
}

// Insert (a,i) into the pair set ("label it in atomic", Alg. 4); a new pair is
// appended to the queue.  Returns 1 if new.
template <typename T>
__device__ int push_pair(const Dev<T>& C, int a, int i) {
  unsigned long long key = pair_key(a, i);
  unsigned long long h = mix64(key) & C.hmask;
  for (unsigned long long probe = 0; probe <= C.hmask; ++probe) {
    unsigned long long prev = atomicCAS(C.hash + h, EMPTY_KEY, key);
    if (prev == key) return 0;
    if (prev == EMPTY_KEY) {
      if (!owned(C, i)) {  // another rank's pair: to the outbox, once (the pair set dedups)
        unsigned long long o = atomicAdd(C.ctr + CTR_OUT, 1ull);
        if ((long long)o >= C.ocap) { set_error(C.status, VD_ERR_CAPACITY); return 0; }
        C.outbox[o] = key;
        return 0;
      }
      unsigned long long pos = atomicAdd(C.ctr + CTR_TAIL, 1ull);
      if ((long long)pos >= C.qcap) { set_error(C.status, VD_ERR_CAPACITY); return 0; }
      C.queue[pos] = key;
      __threadfence();
      return 1;
    }
    h = (h + 1) & C.hmask;
  }
  set_error(C.status, VD_ERR_CAPACITY);
  return 0;
}

// Wait until queue slot h holds a pair, or the flood is over.  Lane 0 waits;
// all lanes get the key (EMPTY_KEY: stop).  The wait is bounded by wall time.
template <typename T>
__device__ unsigned long long wait_item(const Dev<T>& C, long long h, int lane) {
  unsigned long long key = EMPTY_KEY;
  if (lane == 0) {
    unsigned long long t0;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t0));
    volatile unsigned long long* q = C.queue;
    volatile unsigned long long* ctr = C.ctr;
    volatile int* st = C.status;
    for (;;) {
      if (h < C.qcap) {
        key = q[h];
        if (key != EMPTY_KEY) break;
      }
      unsigned long long done = ctr[CTR_DONE];
      __threadfence();
      unsigned long long tail = ctr[CTR_TAIL];
      if (done >= tail || *st != 0) { key = EMPTY_KEY; break; }
      unsigned long long t1;
      asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t1));
      if ((long long)(t1 - t0) > C.wait_ns) { set_error(C.status, VD_ERR_LIMIT); key = EMPTY_KEY; break; }
      __nanosleep(128);
    }
  }
  return __shfl_sync(FULL, key, 0);
}

// Single-thread form of wait_item (thread-per-pair kernels).
template <typename T>
__device__ unsigned long long wait_item_one(const Dev<T>& C, long long h) {
  unsigned long long t0;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t0));
  volatile unsigned long long* q = C.queue;
  volatile unsigned long long* ctr = C.ctr;
  volatile int* st = C.status;
  for (;;) {
    if (h < C.qcap) {
      unsigned long long key = q[h];
      if (key != EMPTY_KEY) return key;
    }
    unsigned long long done = ctr[CTR_DONE];
    __threadfence();
    unsigned long long tail = ctr[CTR_TAIL];
    if (done >= tail || *st != 0) return EMPTY_KEY;
    unsigned long long t1;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t1));
    if ((long long)(t1 - t0) > C.wait_ns) { set_error(C.status, VD_ERR_LIMIT); return EMPTY_KEY; }
    __nanosleep(256);
  }
}

template <typename T>
__device__ __forceinline__ void stat_add(const Dev<T>& C, int slot, unsigned long long v) {
  if (v) atomicAdd(C.stats + slot, v);
}

// ---------------------------------------------------------------------------
// Learned form: the 32 nearest sites of v_i, one per lane, loaded once per pair.
// cand marks the ranked candidates; r32 (> 0) is a certified lower bound on the
// distance from v_i to every site that is not in the list.  r64 (> 0) is the
// same for the list extended by the 33rd..64th nearest, which are loaded only
// by the tests that need them.
// ---------------------------------------------------------------------------
// EXT: the clip kernel is compiled with the 64-site tests (a separate
// instantiation, so that workloads that do not need them keep the lean code).
// POW: power diagram -- distances to the lifted sites (x, u) -> (v_k, h_k) with
// the domain at u = 0; the lists are not used (the plain search only).
template <typename T, bool EXT = false, bool POW = false>
struct NbrList {
  static constexpr bool ext = EXT;
  static constexpr bool pow = POW;
  int id;       // this lane's site (-1: none)
  T x, y, z;
  bool cand;
  float r32, r64;
  T hi;         // power diagram: the lift h_i of the pair's site (0 otherwise)
};

template <typename T, bool EXT = false, bool POW = false>
__device__ __forceinline__ NbrList<T, EXT, POW> load_nbrs(const Dev<T>& C, int i, int lane) {
  NbrList<T, EXT, POW> L;
  L.id = -1; L.x = L.y = L.z = T(0); L.cand = false; L.r32 = 0.f; L.r64 = 0.f; L.hi = T(0);
  if (POW) {
    L.hi = (T)C.lift[i];
    return L;
  }
  if (C.knn) {
    L.id = C.knn[(long long)i * 32 + lane];
    float d32 = C.knn_d2[(long long)i * 32 + 31];
    int k32 = C.knn[(long long)i * 32 + 31];
    L.r32 = (d32 > 0.f && k32 >= 0) ? sqrtf(d32 * (1.f - 1e-6f)) : 0.f;
    if (EXT && C.knn2 && L.r32 > 0.f) L.r64 = C.knn_r64[i];
    L.cand = L.id >= 0 && ((C.cmask[i] >> lane) & 1u);
  } else if (C.ncand > 0) {
    L.id = lane < C.ncand ? C.cand[(long long)i * C.ncand + lane] : -1;
    L.cand = L.id >= 0 && L.id != i;
  }
  if (L.id >= 0) { L.x = C.sites[3 * L.id]; L.y = C.sites[3 * L.id + 1]; L.z = C.sites[3 * L.id + 2]; }
  return L;
}

// ---------------------------------------------------------------------------
// Point-in-cell test of a polytope corner (Sec. 3.1).
//
// q (frame of v_i) is a corner with coordinate error bound e; excl[] holds the
// sites whose bisectors pass through it (its positive flags F_q).  The corner is
// outside Omega_i iff some site k, not i and not in F_q, is strictly closer to
// q than v_i (Eq. 1 with the flag rule of Sec. 3.1).  The grid is scanned ring
// by ring around q; each candidate's difference of squared distances
// f_k = |q - v_k|^2 - |q - v_i|^2 is compared with a bound B on its rounding
// error (from e and the unit roundoff).  f_k < -B certifies "outside" and ends
// the scan; |f_k| <= B is settled on the spot by the exact predicate `exact(k)`
// (float64 on the defining planes) in the lane that met the site.  Without a
// certified closer site the scan must cover the ball of radius |q - v_i| (plus
// the error margin).  Returns 1 if outside; *wit gets the closer site with the
// smallest (f_k, k) among the certified ones.
// ---------------------------------------------------------------------------
template <typename T, typename NL, typename Exact>
__device__ int corner_outside(const Dev<T>& C, int i, T vix, T viy, T viz, T qx, T qy, T qz, T e,
                              const int* excl, int lane, ScanScratch& S, const NL& L, Exact& exact,
                              int* wit, int* scanned, int* listed) {
  const T U = Prec<T>::U;
  T gx = vix + qx, gy = viy + qy, gz = viz + qz;
  T di2;
  {
    T dx = vix - gx, dy = viy - gy, dz = viz - gz;
    di2 = dx * dx + dy * dy + dz * dz;
  }
  // power diagram: the corner (q, 0) against the lifted site (v_i, h_i); every
  // site closer to it in 4D is closer in 3D too, so the 3D scan radius below
  // (from the 4D distance) covers them
  if (NL::pow) di2 += L.hi * L.hi;
  T di = sqrt(di2);
  T gmax = fmax(fabs(gx), fmax(fabs(gy), fabs(gz)));
  T delta = T(1.7320508075688772) * (e + T(2) * U * gmax);
  T D = T(1.2) * di + delta;
  T B = T(4.5) * D * delta + T(2.5) * delta * delta + T(16) * U * D * D;
  if (NL::pow) B += T(8) * U * (L.hi * L.hi + (T)C.lift_max * (T)C.lift_max);
  bool well = delta <= T(0.03) * di;
  T R = di * (T(1) + T(1e-5)) + T(2) * delta + T(4) * U * gmax;
  // ill-conditioned corner: every site that could be closer goes to the exact test
  T amb = well ? B : (R * R - di2) + B;
  if (!well && lane == 0 && C.want_stats) atomicAdd(C.stats + VD_STAT_ILLCOND, 1ull);
  int e0 = excl[0], e1 = excl[1], e2 = excl[2];
  // minimum of the squared distance d_k^2 (>= 0) over the candidates; f = d_k^2 - d_i^2
  T bd = T(1e30), od = T(1e30);
  int bk = 0x7fffffff, ok = 0x7fffffff;
  auto visit = [&](const typename Prec<T>::V4& s) {
    int k = site_id(s);
    if (k == i || k == e0 || k == e1 || k == e2) return;
    T dx = s.x - gx, dy = s.y - gy, dz = s.z - gz;
    T d2 = dx * dx + dy * dy + dz * dz;
    if (NL::pow) {
      T hk = (T)C.lift[k];
      d2 += hk * hk;
    }
    T f = d2 - di2;
    if (d2 < bd || (d2 == bd && k < bk)) { bd = d2; bk = k; }
    if (f >= -B && f <= amb && (d2 < od || (d2 == od && k < ok)) && exact(k) < 0) { od = d2; ok = k; }
  };
  // learned form: when the ball of radius |q - v_i| around q lies inside the ball
  // holding v_i's 32 nearest sites (2 |q - v_i| <= r32), every site that could be
  // closer to q than v_i is in the list, which settles the test exactly
  // (float arithmetic: its rounding, below 1e-6 relative, is inside the 2e-5 margin)
  if (L.r32 > 0.f && L.r32 >= 2.f * (float)(di + delta) * (1.f + 2e-5f)) {
    *listed += 1;
    T ld = T(1e30), lo = T(1e30);
    int lk = 0x7fffffff, lok = 0x7fffffff;
    int k = L.id;
    if (k >= 0 && k != e0 && k != e1 && k != e2) {
      T dx = L.x - gx, dy = L.y - gy, dz = L.z - gz;
      T d2 = dx * dx + dy * dy + dz * dz;
      T f = d2 - di2;
      if (f < -B) { ld = d2; lk = k; }
      else if (f <= B && exact(k) < 0) { lo = d2; lok = k; }
    }
    if (__any_sync(FULL, lk != 0x7fffffff)) {
      warp_argmin(ld, lk);
      *wit = lk;
      return 1;
    }
    if (__any_sync(FULL, lok != 0x7fffffff)) {
      warp_argmin(lo, lok);
      *wit = lok;
      return 1;
    }
    *wit = -1;
    return 0;
  }
  // the same with the 64 nearest, when their radius covers the ball: each lane
  // also tests its entry among the 33rd..64th (loaded here, rarely needed)
  if (NL::ext && L.r64 > 0.f && L.r64 >= 2.f * (float)(di + delta) * (1.f + 2e-5f)) {
    *listed += 1;
    T ld = T(1e30), lo = T(1e30);
    int lk = 0x7fffffff, lok = 0x7fffffff;
    auto test = [&](int k, T x, T y, T z) {
      if (k < 0 || k == e0 || k == e1 || k == e2) return;
      T dx = x - gx, dy = y - gy, dz = z - gz;
      T d2 = dx * dx + dy * dy + dz * dz;
      T f = d2 - di2;
      if (f < -B) {
        if (d2 < ld || (d2 == ld && k < lk)) { ld = d2; lk = k; }
      } else if (f <= B && (d2 < lo || (d2 == lo && k < lok)) && exact(k) < 0) {
        lo = d2; lok = k;
      }
    };
    test(L.id, L.x, L.y, L.z);
    int k2 = C.knn2[(long long)i * 32 + lane];
    if (k2 >= 0) test(k2, C.sites[3 * k2], C.sites[3 * k2 + 1], C.sites[3 * k2 + 2]);
    if (__any_sync(FULL, lk != 0x7fffffff)) {
      warp_argmin(ld, lk);
      *wit = lk;
      return 1;
    }
    if (__any_sync(FULL, lok != 0x7fffffff)) {
      warp_argmin(lo, lok);
      *wit = lok;
      return 1;
    }
    *wit = -1;
    return 0;
  }
  // learned proposal, outside certificate: a listed site (a ranked candidate or
  // one of the other nearest sites) certified closer than v_i settles "outside"
  // with no grid scan (same exact criterion as the scan)
  if (__any_sync(FULL, L.id >= 0)) {
    T cd = T(1e30);
    int ck = 0x7fffffff;
    int k = L.id;
    if (k >= 0 && k != i && k != e0 && k != e1 && k != e2) {
      T dx = L.x - gx, dy = L.y - gy, dz = L.z - gz;
      T d2 = dx * dx + dy * dy + dz * dz;
      if (d2 - di2 < -B) { cd = d2; ck = k; }
    }
    warp_argmin(cd, ck);
    if (ck != 0x7fffffff) { *wit = ck; *listed += 1; return 1; }
  }
  for (int lev = C.G.query_level(gx, gy, gz); lev >= 0; --lev) {
    int cx, cy, cz;
    C.G.cell_at(lev, gx, gy, gz, cx, cy, cz);
    bool done = false;
    for (int r = 1;; ++r) {
      *scanned += warp_scan_ring(C.G, lev, cx, cy, cz, r, lane, S, visit);
      warp_argmin(bd, bk);
      if (bd - di2 < -B) { done = true; break; }  // a certified closer site: outside, no need to cover the ball
      T m = C.G.cover(lev, cx, cy, cz, r, gx, gy, gz);
      if (m >= T(1e29) || m >= R) { done = true; break; }
      if (lev > 0 ? r >= HASH_MAX_RING : r >= C.G.max_ring()) break;
    }
    if (done) break;
  }
  if (bd - di2 < -B) { *wit = bk; return 1; }
  warp_argmin(od, ok);
  if (ok != 0x7fffffff) { *wit = ok; return 1; }
  *wit = -1;
  return 0;
}

}  // namespace vd
