// vd_grid.cuh -- uniform site grid and nearest-site queries (Sec. 5.2).
//
// Sites are counting-sorted by cell (x fastest), so the cells of one x-row of
// a block are one contiguous range of the sorted array.  A ring scan visits
// the sites of the block of Chebyshev radius r around a cell minus the block
// of radius r-1: at most 2 (2r+1)^2 contiguous segments.  In the warp form the
// segments' lengths are prefix-summed across lanes and the flattened site list
// is dealt out 32 sites at a time, so the lanes stay busy however the sites are
// spread over the cells.
#pragma once

#include "vd_common.cuh"

namespace vd {

template <typename T>
struct GridView {
  using V4 = typename Prec<T>::V4;
  const V4* gs;        // sites sorted by cell: x, y, z, original index (bit-packed)
  const int* cstart;   // [G+1] first sorted position of each cell
  int gx, gy, gz;
  T ox, oy, oz;        // lower corner of the grid box
  T h, ih;             // cell edge and its inverse

  __device__ __forceinline__ int clampi(int v, int hi) const { return v < 0 ? 0 : (v > hi ? hi : v); }
  __device__ __forceinline__ void cell_of(T x, T y, T z, int& cx, int& cy, int& cz) const {
    // floor of a value far outside the grid is clamped before the int conversion
    T fx = (x - ox) * ih, fy = (y - oy) * ih, fz = (z - oz) * ih;
    fx = fx < T(-1) ? T(-1) : (fx > T(gx) ? T(gx) : fx);
    fy = fy < T(-1) ? T(-1) : (fy > T(gy) ? T(gy) : fy);
    fz = fz < T(-1) ? T(-1) : (fz > T(gz) ? T(gz) : fz);
    cx = clampi((int)floor(fx), gx - 1);
    cy = clampi((int)floor(fy), gy - 1);
    cz = clampi((int)floor(fz), gz - 1);
  }
  // distance from q to the outside of the block of radius r around (cx,cy,cz);
  // sides lying on the grid boundary do not bound it (no site lies beyond them,
  // sites outside the box are stored in the boundary cells).  +inf: whole grid.
  __device__ __forceinline__ T cover(int cx, int cy, int cz, int r, T qx, T qy, T qz) const {
    T m = T(1e30);
    if (cx - r > 0) m = fmin(m, qx - (ox + T(cx - r) * h));
    if (cx + r < gx - 1) m = fmin(m, (ox + T(cx + r + 1) * h) - qx);
    if (cy - r > 0) m = fmin(m, qy - (oy + T(cy - r) * h));
    if (cy + r < gy - 1) m = fmin(m, (oy + T(cy + r + 1) * h) - qy);
    if (cz - r > 0) m = fmin(m, qz - (oz + T(cz - r) * h));
    if (cz + r < gz - 1) m = fmin(m, (oz + T(cz + r + 1) * h) - qz);
    return m;
  }
  __device__ __forceinline__ int max_ring() const { return max(gx, max(gy, gz)); }
};

// Per-warp scratch for the segment table of a ring scan.
struct ScanScratch {
  int seg_b[WARP];
  int seg_i[WARP];
};

// Segment `slot` of ring r (r == 1: the whole 3x3x3 block).  Returns [b, e).
template <typename T>
__device__ __forceinline__ void ring_segment(const GridView<T>& G, int cx, int cy, int cz, int r, int slot,
                                             int& b, int& e) {
  b = e = 0;
  int side = 2 * r + 1;
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
  b = __ldg(G.cstart + base + x0);
  e = __ldg(G.cstart + base + x1 + 1);
}

// Warp-cooperative visit of every site of ring r; visit(site4) runs on the lane
// that owns the site.  Returns the number of sites visited.
template <typename T, typename Visit>
__device__ __forceinline__ int warp_scan_ring(const GridView<T>& G, int cx, int cy, int cz, int r, int lane,
                                              ScanScratch& S, Visit& visit) {
  int side = 2 * r + 1;
  int nslots = 2 * side * side;
  int seen = 0;
  for (int base = 0; base < nslots; base += WARP) {
    int b = 0, e = 0;
    if (base + lane < nslots) ring_segment(G, cx, cy, cz, r, base + lane, b, e);
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
        visit(G.gs[S.seg_b[lo] + (f - excl)]);
      }
    }
    seen += total;
  }
  __syncwarp();
  return seen;
}

// Nearest site of q (ties: smaller index), warp-cooperative ring search.
// Returns the index; d2 receives the squared distance.  All lanes get the result.
template <typename T>
__device__ int warp_nearest(const GridView<T>& G, T qx, T qy, T qz, int lane, ScanScratch& S, T& d2out,
                            int* scanned) {
  int cx, cy, cz;
  G.cell_of(qx, qy, qz, cx, cy, cz);
  T bd = T(1e30);
  int bi = 0x7fffffff;
  auto visit = [&](const typename Prec<T>::V4& s) {
    T dx = s.x - qx, dy = s.y - qy, dz = s.z - qz;
    T d = dx * dx + dy * dy + dz * dz;
    int id = site_id(s);
    if (d < bd || (d == bd && id < bi)) { bd = d; bi = id; }
  };
  int r = 1, seen = 0;
  seen += warp_scan_ring(G, cx, cy, cz, r, lane, S, visit);
  for (;;) {
    warp_argmin(bd, bi);
    T m = G.cover(cx, cy, cz, r, qx, qy, qz);
    if (m >= T(1e29) || (m > 0 && bd <= m * m) || r >= G.max_ring()) break;
    ++r;
    seen += warp_scan_ring(G, cx, cy, cz, r, lane, S, visit);
  }
  if (scanned) *scanned += seen;
  d2out = bd;
  return bi;
}

// Single-thread nearest site (used by seeding and the nearest-neighbour
// distance of each site).  `skip` is excluded.
template <typename T>
__device__ int thread_nearest(const GridView<T>& G, T qx, T qy, T qz, int skip, T& d2out) {
  int cx, cy, cz;
  G.cell_of(qx, qy, qz, cx, cy, cz);
  T bd = T(1e30);
  int bi = 0x7fffffff;
  int maxr = G.max_ring();
  for (int r = 0; r <= maxr; ++r) {
    for (int z = cz - r; z <= cz + r; ++z) {
      if (z < 0 || z >= G.gz) continue;
      for (int y = cy - r; y <= cy + r; ++y) {
        if (y < 0 || y >= G.gy) continue;
        bool full = r == 0 || z == cz - r || z == cz + r || y == cy - r || y == cy + r;
        int base = (z * G.gy + y) * G.gx;
        for (int pass = 0; pass < (full ? 1 : 2); ++pass) {
          int x0, x1;
          if (full) { x0 = cx - r; x1 = cx + r; }
          else { x0 = x1 = pass ? cx + r : cx - r; }
          x0 = x0 < 0 ? 0 : x0;
          x1 = x1 > G.gx - 1 ? G.gx - 1 : x1;
          if (x0 > x1) continue;
          int b = __ldg(G.cstart + base + x0), e = __ldg(G.cstart + base + x1 + 1);
          for (int p = b; p < e; ++p) {
            typename Prec<T>::V4 s = G.gs[p];
            int id = site_id(s);
            if (id == skip) continue;
            T dx = s.x - qx, dy = s.y - qy, dz = s.z - qz;
            T d = dx * dx + dy * dy + dz * dz;
            if (d < bd || (d == bd && id < bi)) { bd = d; bi = id; }
          }
        }
      }
    }
    T m = G.cover(cx, cy, cz, r, qx, qy, qz);
    if (m >= T(1e29) || (m > 0 && bd <= m * m)) break;
  }
  d2out = bd;
  return bi;
}

}  // namespace vd
