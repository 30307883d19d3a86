// vd_grid.cuh -- site grids and nearest-site queries (Sec. 5.2).
//
// Level 0 is the uniform grid of Sec. 5.2 over the mesh box, sized for a few
// sites per cell at the average density; its sites are counting-sorted by cell
// (x fastest), so the cells of one x-row of a block form one contiguous range.
// For strongly clustered sites (where a level-0 cell can hold thousands of
// sites) levels 1.. are spatial-hash grids with the cell edge halved per level;
// every level holds all the sites.  A query starts at the level that level 0
// assigns to its cell (about the same few sites per cell at the query's own
// density) and falls back to coarser levels when a few rings do not settle it.
//
// A ring scan visits the sites of the block of Chebyshev radius r around a
// cell minus the block of radius r-1.  In the warp form the block's segments
// (level 0: x-rows, hashed levels: single cells) are prefix-summed across the
// lanes and the flattened site list is dealt out 32 sites at a time, so the
// lanes stay busy however unevenly the sites fill the cells.
#pragma once

#include "vd_common.cuh"

namespace vd {

constexpr int MAX_LEVELS = 6;
constexpr int HASH_MAX_RING = 2;  // rings tried on a hashed level before the next coarser one

template <typename T>
struct Level {
  using V4 = typename Prec<T>::V4;
  const V4* gs;        // sites sorted by bucket: x, y, z, original index (bit-packed)
  const int* start;    // [buckets+1] first sorted position of each bucket
  unsigned mask;       // hashed levels: buckets - 1 (a power of two); level 0: unused
  T h, ih;             // cell edge and its inverse
};

__device__ __forceinline__ unsigned cell_hash(int x, int y, int z) {
  unsigned h = (unsigned)x * 0x8da6b343u ^ (unsigned)y * 0xd8163841u ^ (unsigned)z * 0xcb1ab31fu;
  h ^= h >> 15;
  h *= 0x2c1b3c6du;
  h ^= h >> 12;
  return h;
}

template <typename T>
struct GridView {
  using V4 = typename Prec<T>::V4;
  int gx, gy, gz;              // level-0 dimensions
  T ox, oy, oz;                // lower corner of the level-0 box (origin of every level)
  int nlev;
  const unsigned char* qlev;   // [gx*gy*gz] query level of each level-0 cell
  Level<T> L[MAX_LEVELS];

  __device__ __forceinline__ static int clampi(int v, int hi) { return v < 0 ? 0 : (v > hi ? hi : v); }
  // level-0 cell (clamped into the box; far-away values are clamped before the conversion)
  __device__ __forceinline__ void cell0(T x, T y, T z, int& cx, int& cy, int& cz) const {
    T ih = L[0].ih;
    T fx = (x - ox) * ih, fy = (y - oy) * ih, fz = (z - oz) * ih;
    fx = fx < T(-1) ? T(-1) : (fx > T(gx) ? T(gx) : fx);
    fy = fy < T(-1) ? T(-1) : (fy > T(gy) ? T(gy) : fy);
    fz = fz < T(-1) ? T(-1) : (fz > T(gz) ? T(gz) : fz);
    cx = clampi((int)floor(fx), gx - 1);
    cy = clampi((int)floor(fy), gy - 1);
    cz = clampi((int)floor(fz), gz - 1);
  }
  __device__ __forceinline__ void cell_at(int lev, T x, T y, T z, int& cx, int& cy, int& cz) const {
    if (lev == 0) { cell0(x, y, z, cx, cy, cz); return; }
    T ih = L[lev].ih;
    T lim = T(1 << 30);
    T fx = fmin(fmax((x - ox) * ih, -lim), lim), fy = fmin(fmax((y - oy) * ih, -lim), lim),
      fz = fmin(fmax((z - oz) * ih, -lim), lim);
    cx = (int)floor(fx); cy = (int)floor(fy); cz = (int)floor(fz);
  }
  __device__ __forceinline__ int query_level(T x, T y, T z) const {
    if (nlev <= 1) return 0;
    int cx, cy, cz;
    cell0(x, y, z, cx, cy, cz);
    return qlev[(cz * gy + cy) * gx + cx];
  }
  // distance from q to the outside of the block of radius r around (cx,cy,cz);
  // on level 0 sides lying on the box boundary do not bound it (no site lies
  // beyond them: sites outside the box are stored in the boundary cells).
  // +1e30: the block covers the whole level-0 grid.
  __device__ __forceinline__ T cover(int lev, int cx, int cy, int cz, int r, T qx, T qy, T qz) const {
    T h = L[lev].h;
    T m = T(1e30);
    bool hashed = lev > 0;
    if (hashed || cx - r > 0) m = fmin(m, qx - (ox + T(cx - r) * h));
    if (hashed || cx + r < gx - 1) m = fmin(m, (ox + T(cx + r + 1) * h) - qx);
    if (hashed || cy - r > 0) m = fmin(m, qy - (oy + T(cy - r) * h));
    if (hashed || cy + r < gy - 1) m = fmin(m, (oy + T(cy + r + 1) * h) - qy);
    if (hashed || cz - r > 0) m = fmin(m, qz - (oz + T(cz - r) * h));
    if (hashed || cz + r < gz - 1) m = fmin(m, (oz + T(cz + r + 1) * h) - qz);
    return m;
  }
  __device__ __forceinline__ int max_ring() const { return max(gx, max(gy, gz)); }
};

// Per-warp scratch for the segment table of a ring scan.
struct ScanScratch {
  int seg_b[WARP];
  int seg_i[WARP];
};

// number of segment slots of ring r on a level
__device__ __forceinline__ int ring_slots(int lev, int r) {
  int side = 2 * r + 1;
  return lev == 0 ? 2 * side * side : side * side * side;
}

// Segment `slot` of ring r (r == 1: the whole 3x3x3 block).  Returns [b, e).
template <typename T>
__device__ __forceinline__ void ring_segment(const GridView<T>& G, int lev, int cx, int cy, int cz, int r,
                                             int slot, int& b, int& e) {
  b = e = 0;
  int side = 2 * r + 1;
  if (lev > 0) {
    // hashed level: one cell per slot; cells inside ring r-1 are skipped
    if (slot >= side * side * side) return;
    int dx = slot % side - r, t = slot / side;
    int dy = t % side - r, dz = t / side - r;
    if (r > 1 && dx > -r && dx < r && dy > -r && dy < r && dz > -r && dz < r) return;
    const Level<T>& Lv = G.L[lev];
    unsigned k = cell_hash(cx + dx, cy + dy, cz + dz) & Lv.mask;
    b = __ldg(Lv.start + k);
    e = __ldg(Lv.start + k + 1);
    return;
  }
  int row = slot >> 1, half = slot & 1;
  int dy = row % side - r, dz = row / side - r;
  int y = cy + dy, z = cz + dz;
  if (row >= side * side || y < 0 || y >= G.gy || z < 0 || z >= G.gz) return;
  bool full = (r == 1) || dy == r || dy == -r || dz == r || dz == -r;
  int x0, x1;
  if (full) {
    if (half) return;
    x0 = cx - r; x1 = cx + r;
  } else {
    x0 = x1 = half ? cx + r : cx - r;
  }
  x0 = x0 < 0 ? 0 : x0;
  x1 = x1 > G.gx - 1 ? G.gx - 1 : x1;
  if (x0 > x1) return;
  int base = (z * G.gy + y) * G.gx;
  b = __ldg(G.L[0].start + base + x0);
  e = __ldg(G.L[0].start + base + x1 + 1);
}

// Ring 1 (the 3x3x3 block), the common case, without a prefix sum: on level 0
// three lanes share each of the 9 x-rows (sites strided by 3), on a hashed
// level each of 27 lanes takes one cell.  Loads are independent across lanes.
template <typename T, typename Visit>
__device__ __forceinline__ int warp_scan_block(const GridView<T>& G, int lev, int cx, int cy, int cz, int lane,
                                               Visit& visit) {
  const typename Prec<T>::V4* gs = G.L[lev].gs;
  int b = 0, e = 0, step = 1;
  if (lane < 27) {
    if (lev == 0) {
      int row = lane / 3, j = lane - 3 * row;
      int y = cy + row % 3 - 1, z = cz + row / 3 - 1;
      if (y >= 0 && y < G.gy && z >= 0 && z < G.gz) {
        int x0 = cx > 0 ? cx - 1 : 0, x1 = cx + 1 < G.gx ? cx + 1 : G.gx - 1;
        int base = (z * G.gy + y) * G.gx;
        b = __ldg(G.L[0].start + base + x0) + j;
        e = __ldg(G.L[0].start + base + x1 + 1);
        step = 3;
      }
    } else {
      int dx = lane % 3 - 1, t = lane / 3;
      unsigned k = cell_hash(cx + dx, cy + t % 3 - 1, cz + t / 3 - 1) & G.L[lev].mask;
      b = __ldg(G.L[lev].start + k);
      e = __ldg(G.L[lev].start + k + 1);
    }
  }
  int seen = e > b ? (e - b + step - 1) / step : 0;
  for (int p = b; p < e; p += step) visit(gs[p]);
  return __reduce_add_sync(FULL, (unsigned)seen);
}

// Rings r >= 2: segments prefix-summed across the lanes, flattened list.  Inlined:
// as an out-of-line call its register save and restore cost more than the
// larger code (clip kernel 13-17 % faster inlined, despite a few more spills).
template <typename T, typename Visit>
__device__ __forceinline__ int warp_scan_shell(const GridView<T>& G, int lev, int cx, int cy, int cz, int r,
                                            int lane, ScanScratch& S, Visit& visit) {
  int nslots = ring_slots(lev, r);
  const typename Prec<T>::V4* gs = G.L[lev].gs;
  int seen = 0;
  for (int base = 0; base < nslots; base += WARP) {
    int b = 0, e = 0;
    if (base + lane < nslots) ring_segment(G, lev, cx, cy, cz, r, base + lane, b, e);
    int incl = warp_incl_scan(e - b, lane);
    int total = __shfl_sync(FULL, incl, 31);
    if (total == 0) continue;
    __syncwarp();
    S.seg_b[lane] = b;
    S.seg_i[lane] = incl;
    __syncwarp();
    for (int f0 = 0; f0 < total; f0 += WARP) {
      int f = f0 + lane;
      if (f < total) {
        int lo = 0, hi = WARP - 1;
        while (lo < hi) {
          int mid = (lo + hi) >> 1;
          if (S.seg_i[mid] > f) hi = mid; else lo = mid + 1;
        }
        int excl = lo ? S.seg_i[lo - 1] : 0;
        visit(gs[S.seg_b[lo] + (f - excl)]);
      }
    }
    seen += total;
  }
  __syncwarp();
  return seen;
}

// Warp-cooperative visit of every site of ring r on a level; visit(site4) runs
// on the lane that owns the site.  Returns the number of sites visited.
template <typename T, typename Visit>
__device__ __forceinline__ int warp_scan_ring(const GridView<T>& G, int lev, int cx, int cy, int cz, int r,
                                              int lane, ScanScratch& S, Visit& visit) {
  if (r == 1) return warp_scan_block(G, lev, cx, cy, cz, lane, visit);
  return warp_scan_shell(G, lev, cx, cy, cz, r, lane, S, visit);
}

// Nearest site of q (ties: smaller index), warp-cooperative ring search.
// Returns the index; d2 receives the squared distance.  All lanes get the result.
// POW: q = (qx, qy, qz, qu) in the lifted space of a power diagram, site k at
// (v_k, lift[k]); the 3D ring cover still bounds the search (4D distances are
// never shorter than 3D ones).
template <typename T, bool POW = false>
__device__ int warp_nearest(const GridView<T>& G, T qx, T qy, T qz, int lane, ScanScratch& S, T& d2out,
                            int* scanned, const float* lift = nullptr, T qu = T(0)) {
  T bd = T(1e30);
  int bi = 0x7fffffff;
  auto visit = [&](const typename Prec<T>::V4& s) {
    T dx = s.x - qx, dy = s.y - qy, dz = s.z - qz;
    T d = dx * dx + dy * dy + dz * dz;
    int id = site_id(s);
    if (POW) {
      T du = qu - (T)lift[id];
      d += du * du;
    }
    if (d < bd || (d == bd && id < bi)) { bd = d; bi = id; }
  };
  int seen = 0;
  for (int lev = G.query_level(qx, qy, qz); lev >= 0; --lev) {
    int cx, cy, cz;
    G.cell_at(lev, qx, qy, qz, cx, cy, cz);
    bool done = false;
    for (int r = 1;; ++r) {
      seen += warp_scan_ring(G, lev, cx, cy, cz, r, lane, S, visit);
      warp_argmin(bd, bi);
      T m = G.cover(lev, cx, cy, cz, r, qx, qy, qz);
      if (m >= T(1e29) || (m > 0 && bd <= m * m)) { done = true; break; }
      if (lev > 0 ? r >= HASH_MAX_RING : r >= G.max_ring()) break;
    }
    if (done || lev == 0) break;
  }
  if (scanned) *scanned += seen;
  d2out = bd;
  return bi;
}

// Single-thread scan of ring r on a level (same segments as the warp form).
template <typename T, typename Visit>
__device__ __forceinline__ void thread_scan_ring(const GridView<T>& G, int lev, int cx, int cy, int cz, int r,
                                                 Visit& visit) {
  int nslots = ring_slots(lev, r);
  const typename Prec<T>::V4* gs = G.L[lev].gs;
  for (int slot = 0; slot < nslots; ++slot) {
    int b, e;
    ring_segment(G, lev, cx, cy, cz, r, slot, b, e);
    for (int p = b; p < e; ++p) visit(gs[p]);
  }
}

// Single-thread nearest site (seeding, nearest-neighbour distances); `skip` is
// excluded.  lift (power diagrams): the nearest lifted site to (q, 0).
template <typename T>
__device__ int thread_nearest(const GridView<T>& G, T qx, T qy, T qz, int skip, T& d2out,
                              const float* lift = nullptr) {
  T bd = T(1e30);
  int bi = 0x7fffffff;
  auto visit = [&](const typename Prec<T>::V4& s) {
    int id = site_id(s);
    if (id == skip) return;
    T dx = s.x - qx, dy = s.y - qy, dz = s.z - qz;
    T d = dx * dx + dy * dy + dz * dz;
    if (lift) d += (T)lift[id] * (T)lift[id];
    if (d < bd || (d == bd && id < bi)) { bd = d; bi = id; }
  };
  for (int lev = G.query_level(qx, qy, qz); lev >= 0; --lev) {
    int cx, cy, cz;
    G.cell_at(lev, qx, qy, qz, cx, cy, cz);
    bool done = false;
    for (int r = 1;; ++r) {
      thread_scan_ring(G, lev, cx, cy, cz, r, visit);
      T m = G.cover(lev, cx, cy, cz, r, qx, qy, qz);
      if (m >= T(1e29) || (m > 0 && bd <= m * m)) { done = true; break; }
      if (lev > 0 ? r >= HASH_MAX_RING : r >= G.max_ring()) break;
    }
    if (done || lev == 0) break;
  }
  d2out = bd;
  return bi;
}

}  // namespace vd
