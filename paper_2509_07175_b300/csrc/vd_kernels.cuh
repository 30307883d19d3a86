// vd_kernels.cuh -- the kernels of one diagram computation, in launch order:
//   grid build (counting sort, Sec. 5.2), nearest-neighbour distances (Sec. 5.1),
//   pair seeding (Alg. 4 / Alg. 5), the persistent clip-and-flood kernel (Alg. 3
//   per pair, pairs discovered through face flags), and the per-site reduction
//   (measure, centroid, neighbour CSR), plus Lloyd's update (Sec. 6.4).
#pragma once

#include <type_traits>

#include "vd_clip3.cuh"
#include "vd_clip3t.cuh"
#include "vd_clippoly.cuh"

namespace vd {

// ---------------------------------------------------------------------------
// exclusive scan (3 phases: block scan with block sums, scan of the sums, add)
// ---------------------------------------------------------------------------
constexpr int SCAN_T = 512, SCAN_IPT = 8, SCAN_TILE = SCAN_T * SCAN_IPT;

template <typename In, typename Out>
__global__ void __launch_bounds__(SCAN_T) k_scan_tile(const In* in, Out* out, Out* bsum, long long n) {
  __shared__ Out wsum[SCAN_T / WARP];
  long long base = (long long)blockIdx.x * SCAN_TILE + (long long)threadIdx.x * SCAN_IPT;
  Out v[SCAN_IPT];
  Out s = 0;
#pragma unroll
  for (int k = 0; k < SCAN_IPT; ++k) {
    v[k] = (base + k < n) ? (Out)in[base + k] : (Out)0;
    s += v[k];
  }
  int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  Out inc = s;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    Out t = __shfl_up_sync(FULL, inc, o);
    if (lane >= o) inc += t;
  }
  if (lane == 31) wsum[w] = inc;
  __syncthreads();
  if (w == 0) {
    Out x = lane < SCAN_T / WARP ? wsum[lane] : (Out)0;
    Out xi = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      Out t = __shfl_up_sync(FULL, xi, o);
      if (lane >= o) xi += t;
    }
    if (lane < SCAN_T / WARP) wsum[lane] = xi - x;
    if (lane == SCAN_T / WARP - 1 && bsum) bsum[blockIdx.x] = xi;
  }
  __syncthreads();
  Out run = wsum[w] + inc - s;
#pragma unroll
  for (int k = 0; k < SCAN_IPT; ++k) {
    if (base + k < n) out[base + k] = run;
    run += v[k];
  }
}

template <typename Out>
__global__ void k_scan_add(Out* out, const Out* boff, long long n) {
  long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] += boff[i / SCAN_TILE];
}

// ---------------------------------------------------------------------------
// site grids (counting sort by bucket: level-0 cell, x fastest, or hashed cell)
// ---------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ int bucket_of(const GridView<T>& G, int lev, T x, T y, T z) {
  int cx, cy, cz;
  G.cell_at(lev, x, y, z, cx, cy, cz);
  if (lev == 0) return (cz * G.gy + cy) * G.gx + cx;
  return (int)(cell_hash(cx, cy, cz) & G.L[lev].mask);
}

template <typename T>
__global__ void k_cell_count(Dev<T> C, int lev, int* cellid, int* count) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= C.n) return;
  int c = bucket_of(C.G, lev, C.sites[3 * i], C.sites[3 * i + 1], C.sites[3 * i + 2]);
  cellid[i] = c;
  atomicAdd(count + c, 1);
}

template <typename T>
__global__ void k_cell_scatter(Dev<T> C, const int* cellid, const int* cstart, int* cursor,
                               typename Prec<T>::V4* gs) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= C.n) return;
  int c = cellid[i];
  int pos = cstart[c] + atomicAdd(cursor + c, 1);
  gs[pos] = Prec<T>::mk4(C.sites[3 * i], C.sites[3 * i + 1], C.sites[3 * i + 2], pack_id(T(0), i));
}

// query level of every level-0 cell: the level whose cells hold about rho sites
// at the cell's own density (each level halves the cell edge).  qlev_nbr: the
// same for the densest cell of the 3x3x3 block around it, for queries that lie
// mostly off the sites (the boundary pass of the split queries points on the
// domain's boundary, where a sparse cell can border a dense cluster whose sites
// its level-0 ring would scan one by one).
__global__ void k_query_level(int gx, int gy, int gz, const int* cstart0, unsigned char* qlev,
                              unsigned char* qlev_nbr, int nlev, float rho) {
  int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= gx * gy * gz) return;
  auto level = [&](int cnt) {
    int l = 0;
    if ((float)cnt > rho) l = (int)ceilf(log2f((float)cnt / rho) / 3.f - 0.15f);
    return (unsigned char)min(l, nlev - 1);
  };
  qlev[c] = level(cstart0[c + 1] - cstart0[c]);
  if (qlev_nbr) {
    int x = c % gx, y = (c / gx) % gy, z = c / (gx * gy), mx = 0;
    for (int dz = -1; dz <= 1; ++dz)
      for (int dy = -1; dy <= 1; ++dy)
        for (int dx = -1; dx <= 1; ++dx) {
          int xx = x + dx, yy = y + dy, zz = z + dz;
          if (xx < 0 || yy < 0 || zz < 0 || xx >= gx || yy >= gy || zz >= gz) continue;
          int cc = (zz * gy + yy) * gx + xx;
          mx = max(mx, cstart0[cc + 1] - cstart0[cc]);
        }
    qlev_nbr[c] = level(mx);
  }
}

// delta_i = half the distance from v_i to its nearest other site (Sec. 5.1)
template <typename T>
__global__ void k_delta(const __grid_constant__ Dev<T> C, T* delta) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= C.n) return;
  // sites in the grid's cell order: neighbouring threads query neighbouring cells
  const typename Prec<T>::V4 s = C.G.L[0].gs[t];
  int i = site_id(s);
  T d2;
  int k = thread_nearest(C.G, s.x, s.y, s.z, i, d2);
  if (k >= 0 && k < C.n && d2 == T(0)) set_error(C.status, VD_ERR_DUPLICATE);  // coincident sites
  delta[i] = (k >= 0 && k < C.n) ? T(0.5) * sqrt(d2) : T(1);
}

// ---------------------------------------------------------------------------
// seeding: (T_a, nearest site of T_a's centroid) for every simplex (Alg. 4), and
// (simplex containing v_i, i) for every site inside the mesh
// ---------------------------------------------------------------------------
template <typename T>
__global__ void k_seed_simplex(const __grid_constant__ Dev<T> C) {
  int a = blockIdx.x * blockDim.x + threadIdx.x;
  if (a >= C.m) return;
  T c[3] = {0, 0, 0};
  for (int l = 0; l < C.k; ++l)
    for (int d = 0; d < 3; ++d) c[d] += C.verts[3 * C.simp[C.k * a + l] + d];
  for (int d = 0; d < 3; ++d) c[d] /= T(C.k);
  T d2;
  // power diagrams: the nearest lifted site, whose power cell contains the centroid
  int i = thread_nearest(C.G, c[0], c[1], c[2], -1, d2, C.lift);
  if (i >= 0 && i < C.n && owned(C, i)) push_pair(C, a, i);  // each rank seeds its own sites
}

// ---------------------------------------------------------------------------
// power diagrams in the plane by lifting: p_i = (x_i, y_i, sqrt(eta - w_i)) with
// eta = max w, so |x - p_i|^2 = |x - v_i|^2 - w_i + eta for x in the plane z = 0
// ---------------------------------------------------------------------------
__device__ __forceinline__ int ordered_bits(float f) {
  int b = __float_as_int(f);
  return b >= 0 ? b : b ^ 0x7fffffff;  // monotone in f as a signed integer
}
__device__ __forceinline__ float from_ordered(int b) { return __int_as_float(b >= 0 ? b : b ^ 0x7fffffff); }

__global__ void k_power_max(const float* w, long long n, int* best) {
  int m = ordered_bits(-3.0e38f);
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x)
    m = max(m, ordered_bits(w[t]));
  m = __reduce_max_sync(FULL, m);
  if ((threadIdx.x & 31) == 0) atomicMax(best, m);
}

__global__ void k_power_lift(const float* xy, const float* w, long long n, const int* best, float* out, int* bad) {
  long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n) return;
  float eta = from_ordered(*best), wt = w[t];
  if (!(wt <= eta) || !isfinite(wt)) { atomicExch(bad, 1); wt = eta; }
  out[3 * t] = xy[2 * t];
  out[3 * t + 1] = xy[2 * t + 1];
  out[3 * t + 2] = sqrtf(eta - wt);
}

// power diagrams in 3D and on surfaces (Sec. 6.3): the lift h_i = sqrt(eta - w_i),
// eta = max w (from k_power_max); best[1] collects max h (ordered bits), bad flags
// a weight that is not finite
__global__ void k_power_heights(const float* w, long long n, int* best, float* lift, int* bad) {
  long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  float h = 0.f;
  if (t < n) {
    float eta = from_ordered(best[0]), wt = w[t];
    if (!(wt <= eta) || !isfinite(wt)) { atomicExch(bad, 1); wt = eta; }
    h = sqrtf(eta - wt);
    lift[t] = h;
  }
  int m = __reduce_max_sync(FULL, ordered_bits(h));
  if ((threadIdx.x & 31) == 0) atomicMax(best + 1, m);
}

// box domain: every site's cell is one piece, (0, i); no pair set is needed.  The
// queue follows the grid's cell order, so that pairs processed at the same time
// are neighbours and share their grid cells and lists in the caches.
__global__ void k_seed_box(Dev<float> C) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (!C.owner) {
    if (t >= C.n) return;
    if (t == 0) atomicAdd(C.ctr + CTR_TAIL, (unsigned long long)C.n);
    if ((long long)t >= C.qcap) { set_error(C.status, VD_ERR_CAPACITY); return; }
    C.queue[t] = pair_key(0, site_id(C.G.L[0].gs[t]));
    return;
  }
  // partitioned: this rank's sites only, compacted a warp at a time (grid order
  // within each warp)
  int i = t < C.n ? site_id(C.G.L[0].gs[t]) : -1;
  bool mine = i >= 0 && owned(C, i);
  unsigned m = __ballot_sync(FULL, mine);
  if (!m) return;
  int lane = threadIdx.x & 31;
  unsigned long long base = 0;
  if (lane == 0) base = atomicAdd(C.ctr + CTR_TAIL, (unsigned long long)__popc(m));
  base = __shfl_sync(FULL, base, 0);
  if (!mine) return;
  long long pos = (long long)base + __popc(m & ((1u << lane) - 1u));
  if (pos >= C.qcap) { set_error(C.status, VD_ERR_CAPACITY); return; }
  C.queue[pos] = pair_key(0, i);
}

// vd_resume: the queue continues from its tail (claims past it by the finished
// flood are void), the outbox starts empty and the tail before the new pairs is
// kept to count them
__global__ void k_resume_prep(unsigned long long* ctr) {
  unsigned long long t = ctr[CTR_TAIL];
  ctr[CTR_HEAD] = t;
  ctr[CTR_DONE] = t;
  ctr[CTR_OUT] = 0;
  ctr[CTR_MARK] = t;
}

// pairs received from the other ranks: into the pair set (new ones are queued)
template <typename T>
__global__ void k_push_keys(const __grid_constant__ Dev<T> C, const unsigned long long* keys, long long count) {
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < count; t += (long long)gridDim.x * blockDim.x) {
    unsigned long long key = keys[t];
    long long a = (long long)(key >> 32), i = (long long)(key & 0xffffffffull);
    // a simplex of the domain (the box form: 0; the split's whole cell: m) and a site
    bool ok = i < C.n && (C.box ? a == 0 : (a < C.m || (a == C.m && C.split)));
    if (!ok) { set_error(C.status, VD_ERR_ARG); continue; }
    push_pair(C, (int)a, (int)i);
  }
}

struct Locator {
  const int* start;   // [B+1]
  const int* items;   // simplex ids
  int bx, by, bz;
  double ox, oy, oz, ih;
};

template <typename R>
__device__ __forceinline__ R orient3(const R* a, const R* b, const R* c, const R* p) {
  R ux = b[0] - a[0], uy = b[1] - a[1], uz = b[2] - a[2];
  R vx = c[0] - a[0], vy = c[1] - a[1], vz = c[2] - a[2];
  R wx = p[0] - a[0], wy = p[1] - a[1], wz = p[2] - a[2];
  return ux * (vy * wz - vz * wy) - uy * (vx * wz - vz * wx) + uz * (vx * wy - vy * wx);
}
template <typename R>
__device__ __forceinline__ R orient2(const R* a, const R* b, const R* p) {
  return (b[0] - a[0]) * (p[1] - a[1]) - (b[1] - a[1]) * (p[0] - a[0]);
}

// The simplex containing each site seeds (simplex, site).  Any simplex that meets
// the site's cell is a valid seed (the output does not depend on the seeds), so
// the barycentric test runs in the context's precision with a tolerance of 1e-5
// of the simplex for FP32: a site within that of a face may seed either side.
template <typename T>
__global__ void k_seed_site(const __grid_constant__ Dev<T> C, Locator L) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= C.n) return;
  const typename Prec<T>::V4 s4 = C.G.L[0].gs[t];  // grid cell order (see k_seed_box)
  int i = site_id(s4);
  if (!owned(C, i)) return;
  T p[3] = {s4.x, s4.y, s4.z};
  int bx = (int)floor(((double)p[0] - L.ox) * L.ih), by = (int)floor(((double)p[1] - L.oy) * L.ih),
      bz = (int)floor(((double)p[2] - L.oz) * L.ih);
  if (bx < 0 || by < 0 || bz < 0 || bx >= L.bx || by >= L.by || bz >= L.bz) return;
  const T tol = sizeof(T) == 4 ? T(1e-5) : T(0);
  int b = (bz * L.by + by) * L.bx + bx;
  for (int t = L.start[b]; t < L.start[b + 1]; ++t) {
    int a = L.items[t];
    T V[4][3];
    for (int l = 0; l < C.k; ++l)
      for (int d = 0; d < 3; ++d) V[l][d] = C.verts[3 * C.simp[C.k * a + l] + d];
    bool in;
    // barycentric signs: p substituted for each vertex keeps the orientation
    if (C.k == 4) {
      T o = orient3(V[0], V[1], V[2], V[3]);
      T s0 = orient3(p, V[1], V[2], V[3]), s1 = orient3(V[0], p, V[2], V[3]);
      T s2 = orient3(V[0], V[1], p, V[3]), s3 = orient3(V[0], V[1], V[2], p);
      T lim = -tol * fabs(o);
      if (o < 0) { s0 = -s0; s1 = -s1; s2 = -s2; s3 = -s3; }
      in = s0 >= lim && s1 >= lim && s2 >= lim && s3 >= lim;
    } else {
      T o = orient2(V[0], V[1], V[2]);
      T s0 = orient2(p, V[1], V[2]), s1 = orient2(V[0], p, V[2]), s2 = orient2(V[0], V[1], p);
      T lim = -tol * fabs(o);
      if (o < 0) { s0 = -s0; s1 = -s1; s2 = -s2; }
      in = s0 >= lim && s1 >= lim && s2 >= lim;
    }
    if (in) { push_pair(C, a, i); return; }
  }
}

// ---------------------------------------------------------------------------
// persistent clip-and-flood: one warp per (simplex, site) pair, pairs taken
// from the queue in order, new pairs appended by the flag rules
// ---------------------------------------------------------------------------
template <typename T, int MODE>
struct WarpOf {
  using type = cp::WarpP<T>;
};
template <>
struct WarpOf<float, VD_MODE_3D> {
  using type = c3::Warp3;
};

constexpr int FLOOD_WARPS = 4;
// resident blocks per SM the register allocation aims at: 4 (128 registers) for
// the 3D form, 5-6 % faster than 3 on the 100k cube and the 5M box and 1 % on
// the shell despite its spills; 3 (168 registers) for the polygon forms, which
// lose 4-10 % with fewer registers
template <int MODE>
constexpr int flood_min_blocks() { return MODE == VD_MODE_3D ? 4 : 3; }

// Warp per pair: each warp claims `chunk` consecutive queue slots at a time.
// EXT: point-in-cell tests and searches may use the 33rd..64th nearest (learned
// form with the extended list).
template <typename T, int MODE, bool EXT = false, bool POW = false>
__global__ void __launch_bounds__(FLOOD_WARPS * 32, flood_min_blocks<MODE>()) k_flood(const __grid_constant__ Dev<T> C, int chunk) {
  using W = typename WarpOf<T, MODE>::type;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  W& w = reinterpret_cast<W*>(smem_raw)[threadIdx.x >> 5];
  int lane = threadIdx.x & 31;
  for (;;) {
    unsigned long long h0 = 0;
    if (lane == 0) h0 = atomicAdd(C.ctr + CTR_HEAD, (unsigned long long)chunk);
    h0 = __shfl_sync(FULL, h0, 0);
    bool stop = false;
    for (int c = 0; c < chunk; ++c) {
      unsigned long long h = h0 + (unsigned long long)c;
#ifdef VD_PROFILE
      long long tw = clock64();
#endif
      unsigned long long key = wait_item(C, (long long)h, lane);
#ifdef VD_PROFILE
      if (lane == 0) atomicAdd(C.stats + VD_STAT_DIAG + 5, (unsigned long long)(clock64() - tw));
#endif
      if (key == EMPTY_KEY) { stop = true; break; }
      int a = (int)(key >> 32), i = (int)(key & 0xffffffffull);
      if constexpr (MODE == VD_MODE_3D) c3::process_pair<EXT, POW>(C, w, a, i, (long long)h, lane);
      else cp::process_pair<T, EXT, POW>(C, w, a, i, (long long)h, lane);
      __syncwarp();
      if (lane == 0) {
        __threadfence();
        atomicAdd(C.ctr + CTR_DONE, 1ull);
      }
    }
    if (stop) break;
  }
}

// Thread per pair (3D): the threads of a warp that need work claim together
// (one atomic for all of them), `chunk` consecutive queue slots each.
#ifndef FLOOD_T_THREADS
#define FLOOD_T_THREADS 128
#endif
#ifndef FLOOD_T_MIN_BLOCKS
#define FLOOD_T_MIN_BLOCKS 4
#endif

__global__ void __launch_bounds__(FLOOD_T_THREADS, FLOOD_T_MIN_BLOCKS) k_flood_thread(const __grid_constant__ Dev<float> C, int chunk) {
  c3t::Poly P;
  c3t::Counters K = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
  const int lane = threadIdx.x & 31;
  for (;;) {
    unsigned m = __activemask();
    int leader = __ffs(m) - 1;
    unsigned rank = __popc(m & ((1u << lane) - 1u));
    unsigned long long base = 0;
    if (lane == leader) base = atomicAdd(C.ctr + CTR_HEAD, (unsigned long long)__popc(m) * (unsigned)chunk);
    base = __shfl_sync(m, base, leader);
    unsigned long long h0 = base + (unsigned long long)rank * (unsigned)chunk;
    bool stop = false;
    for (int c = 0; c < chunk; ++c) {
      unsigned long long h = h0 + (unsigned long long)c;
      unsigned long long key = wait_item_one(C, (long long)h);
      if (key == EMPTY_KEY) { stop = true; break; }
      int a = (int)(key >> 32), i = (int)(key & 0xffffffffull);
      c3t::process_pair(C, P, a, i, (long long)h, K);
      __threadfence();
      atomicAdd(C.ctr + CTR_DONE, 1ull);
    }
    if (stop) break;
  }
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
    stat_add(C, VD_STAT_BISECTOR_FACES, K.bisf);
    stat_add(C, VD_STAT_EXCESS_CLIPS, K.excess);
  }
}

// ---------------------------------------------------------------------------
// the 32 nearest other sites of every site (features of the learned proposal)
// ---------------------------------------------------------------------------
constexpr int KNN = 32;
constexpr int KNN_SLOTS = 32;  // stored sites per lane (1024 per site)
constexpr int KNN_WARPS = 4;

struct KnnScratch {
  float d2[KNN_SLOTS][WARP];  // [slot][lane]: each lane appends to its own column
  int id[KNN_SLOTS][WARP];
  ScanScratch ss;             // segment table of rings beyond ring 1
};

// Ring r of level 0 or a hashed level (r = 1: the 3x3x3 block), flattened over
// the lanes like the rings of the clip kernel's scans, restricted to the cells that meet
// the ball of squared radius r2 around q (a ring cell or row farther away cannot
// hold one of the 32 nearest once 32 sites within sqrt(r2) are known).  Cell
// bounds are widened by 1e-4 of the edge, and the outer side of a level-0
// boundary row is open (sites beyond the grid box are kept in boundary cells).
// Inlined into k_knn: the pass is 40 % faster than with an out-of-line call.
template <typename T, typename Visit>
__device__ __forceinline__ void knn_scan_shell(const GridView<T>& G, int lev, int cx, int cy, int cz, int r, int lane,
                                            ScanScratch& S, Visit& visit, T qx, T qy, T qz, T r2) {
  const T h = G.L[lev].h, slack = T(1e-4) * h;
  auto gap = [&](T q, T lo, bool has_lo, bool has_hi) {
    T g = T(0);
    if (has_lo) g = fmax(g, (lo - slack) - q);
    if (has_hi) g = fmax(g, q - (lo + h + slack));
    return g;
  };
  int nslots = ring_slots(lev, r);
  const typename Prec<T>::V4* gs = G.L[lev].gs;
  for (int base = 0; base < nslots; base += WARP) {
    int b = 0, e = 0;
    int slot = base + lane;
    if (slot < nslots) {
      int side = 2 * r + 1;
      if (lev > 0) {
        int dx = slot % side - r, t = slot / side;
        int dy = t % side - r, dz = t / side - r;
        bool inner = r > 1 && dx > -r && dx < r && dy > -r && dy < r && dz > -r && dz < r;
        if (slot < side * side * side && !inner) {
          T gx_ = gap(qx, G.ox + T(cx + dx) * h, true, true), gy_ = gap(qy, G.oy + T(cy + dy) * h, true, true),
            gz_ = gap(qz, G.oz + T(cz + dz) * h, true, true);
          if (gx_ * gx_ + gy_ * gy_ + gz_ * gz_ <= r2) {
            unsigned k = cell_hash(cx + dx, cy + dy, cz + dz) & G.L[lev].mask;
            b = __ldg(G.L[lev].start + k);
            e = __ldg(G.L[lev].start + k + 1);
          }
        }
      } else {
        int row = slot >> 1, half = slot & 1;
        int dy = row % side - r, dz = row / side - r;
        int y = cy + dy, z = cz + dz;
        if (row < side * side && y >= 0 && y < G.gy && z >= 0 && z < G.gz) {
          bool full = r == 1 || dy == r || dy == -r || dz == r || dz == -r;
          int x0 = -1, x1 = -2;
          if (full) { if (!half) { x0 = cx - r; x1 = cx + r; } }
          else x0 = x1 = half ? cx + r : cx - r;
          x0 = x0 < 0 ? 0 : x0;
          x1 = x1 > G.gx - 1 ? G.gx - 1 : x1;
          T gy_ = gap(qy, G.oy + T(y) * h, y > 0, y < G.gy - 1), gz_ = gap(qz, G.oz + T(z) * h, z > 0, z < G.gz - 1);
          T rem = r2 - gy_ * gy_ - gz_ * gz_;
          if (x0 <= x1 && rem >= T(0)) {
            T w = sqrt(rem) + slack;
            T fa = (qx - w - G.ox) * G.L[0].ih, fb = (qx + w - G.ox) * G.L[0].ih;
            if (fa > T(x0)) x0 = fa >= T(x1 + 1) ? x1 + 1 : (int)floor(fa);
            if (fb < T(x1)) x1 = fb < T(x0) ? x0 - 1 : (int)floor(fb);
            if (x0 <= x1) {
              int rb = (z * G.gy + y) * G.gx;
              b = __ldg(G.L[0].start + rb + x0);
              e = __ldg(G.L[0].start + rb + x1 + 1);
            }
          }
        }
      }
    }
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
  }
  __syncwarp();
}

// Warp per site: collect the sites of growing rings around v_i (each lane keeps
// the sites it meets in its own column of shared memory), then merge the lanes'
// sorted columns into the 32 (or 64) nearest (ties: smaller index).  Once that
// many collected sites lie within some radius, the radius bounds the rest of the
// scan.
// delta (optional): also writes delta_i (Sec. 5.1) from the list's first entry when
// the scan certifies it as the nearest site, with the checks of k_delta; a site whose
// nearest is not certified by the scan gets its own nearest-site query.
// knn2, r64 (optional): the 33rd..64th nearest (ids) and the certified radius of
// the 64 (0 when the scan does not certify them).
// grid-order positions of the rank's own sites (partitioned context), a warp's
// positions in order, for the nearest-list pass
template <typename T>
__global__ void k_own_order(const __grid_constant__ Dev<T> C, int* order) {
  for (long long t0 = (long long)blockIdx.x * blockDim.x; t0 < C.n; t0 += (long long)gridDim.x * blockDim.x) {
    long long t = t0 + threadIdx.x;
    bool mine = t < C.n && owned(C, site_id(C.G.L[0].gs[t]));
    unsigned m = __ballot_sync(FULL, mine);
    if (!m) continue;
    int lane = threadIdx.x & 31;
    unsigned long long base = 0;
    if (lane == 0) base = atomicAdd(C.ctr + CTR_OWNED, (unsigned long long)__popc(m));
    base = __shfl_sync(FULL, base, 0);
    if (mine) order[base + __popc(m & ((1u << lane) - 1u))] = (int)t;
  }
}

template <typename T>
__global__ void __launch_bounds__(KNN_WARPS * 32) k_knn(const __grid_constant__ Dev<T> C, int* knn, float* knn_d2,
                                                        T* delta, int* knn2, float* r64) {
  const int want = knn2 ? 2 * KNN : KNN;
  __shared__ KnnScratch sh[KNN_WARPS];
  KnnScratch& S = sh[threadIdx.x >> 5];
  int lane = threadIdx.x & 31;
  // each block takes a contiguous range of the sites in the grid's cell order, its
  // warps interleaved, so that a block's warps scan neighbouring cells.  A
  // partitioned context without the split (own_order set) lists its own sites
  // only: the others' pairs are clipped by other ranks, and nothing here reads
  // their lists but the candidate ranking, which bounds every id it reads.
  const long long N = C.own_order ? (long long)C.ctr[CTR_OWNED] : (long long)C.n;
  long long per = (N + gridDim.x - 1) / gridDim.x;
  long long t0 = (long long)blockIdx.x * per, t1 = t0 + per < N ? t0 + per : N;
  for (long long t = t0 + (threadIdx.x >> 5); t < t1; t += KNN_WARPS) {
    const typename Prec<T>::V4 s4 = C.G.L[0].gs[C.own_order ? (long long)C.own_order[t] : t];
    const int i = site_id(s4);
    T qx = s4.x, qy = s4.y, qz = s4.z;
    int cnt = 0;
    bool over = false;
    T bound2 = T(1e36);  // squared radius already holding `want` collected sites
    auto visit = [&](const typename Prec<T>::V4& s) {
      int k = site_id(s);
      if (k == i) return;
      T dx = s.x - qx, dy = s.y - qy, dz = s.z - qz;
      T d = dx * dx + dy * dy + dz * dz;
      if (d > bound2) return;  // cannot be one of the `want` nearest
      if (cnt < KNN_SLOTS) {
        S.d2[cnt][lane] = (float)d;
        S.id[cnt][lane] = k;
        ++cnt;
      } else {
        over = true;
      }
    };
    auto count_below = [&](float lim) {
      int c = 0;
      for (int t = 0; t < cnt; ++t) c += S.d2[t][lane] <= lim;
      return (int)__reduce_add_sync(FULL, (unsigned)c);
    };
    int lev = C.G.query_level(qx, qy, qz), cx, cy, cz;
    C.G.cell_at(lev, qx, qy, qz, cx, cy, cz);
    // certified: every site within `cover` of v_i was stored and at least 32 of
    // the stored distances are below cover^2 (so no unseen site can be nearer
    // than the 32nd); otherwise the list is kept for the features but flagged.
    // certified2: the same for the 64 nearest.
    bool certified = false, certified2 = false;
    T covered = T(0);    // every site within this distance of v_i has been collected
    for (int r = 1;; ++r) {
      knn_scan_shell(C.G, lev, cx, cy, cz, r, lane, S.ss, visit, qx, qy, qz, bound2);
      __syncwarp();
      if (__any_sync(FULL, over)) break;
      T m = C.G.cover(lev, cx, cy, cz, r, qx, qy, qz);
      covered = r == 1 || bound2 > m * m ? m : sqrt(bound2);
      if (m >= T(1e29)) { certified = certified2 = true; break; }
      int total = (int)__reduce_add_sync(FULL, (unsigned)cnt);
      if (total >= KNN) {
        float m2 = (float)(m * m) * (1.f - 1e-5f);
        int below = count_below(m2);
        if (below >= KNN) certified = true;  // the first 32 stay certified: later rings lie beyond m
        if (below >= want) { certified2 = true; break; }
        // a radius with `want` collected sites within it bounds the rest of the
        // scan (cells beyond it are skipped, sites beyond it are not stored): grow
        // a guess from the cover until the count reaches it (at worst the largest
        // collected distance)
        if (total < want) { if (r >= 4) break; continue; }
        float top = 0.f;
        for (int t = 0; t < cnt; ++t) top = fmaxf(top, S.d2[t][lane]);
        top = __uint_as_float(__reduce_max_sync(FULL, __float_as_uint(top)));
        float g = m2 > 0.f ? m2 : top;
        while (g < top && count_below(g) < want) g = fminf(top, 2.f * g);
        T nb = (T)g * T(1.0001);
        bound2 = nb < bound2 ? nb : bound2;
      }
      if (r >= 4) break;
    }
    __syncwarp();
    // each lane sorts its column (insertion sort; ties by index), then one round
    // of a warp-wide minimum over the column heads per output entry
    for (int u = 1; u < cnt; ++u) {
      float du = S.d2[u][lane];
      int iu = S.id[u][lane];
      int v = u - 1;
      while (v >= 0 && (S.d2[v][lane] > du || (S.d2[v][lane] == du && S.id[v][lane] > iu))) {
        S.d2[v + 1][lane] = S.d2[v][lane];
        S.id[v + 1][lane] = S.id[v][lane];
        --v;
      }
      S.d2[v + 1][lane] = du;
      S.id[v + 1][lane] = iu;
    }
    int head = 0;
    float near2 = 3.0e38f;
    int near = 0x7fffffff;
    // entry k is kept by lane k % 32 and written with the others of its half
    int mine = -1;
    float mined = 0.f;
    for (int k = 0; k < want; ++k) {
      float bd = head < cnt ? S.d2[head][lane] : 3.0e38f;
      int bi = head < cnt ? S.id[head][lane] : 0x7fffffff;
      float d0 = bd;
      int i0 = bi;
      warp_argmin(bd, bi);
      if (d0 == bd && i0 == bi && head < cnt) ++head;
      if (k == 0) { near2 = bd; near = bi; }
      if (lane == (k & (KNN - 1))) { mine = bi == 0x7fffffff ? -1 : bi; mined = bd; }
      if (k == KNN - 1) {
        knn[(long long)i * KNN + lane] = mine;
        // a negative 32nd distance marks a list that is not certified complete
        knn_d2[(long long)i * KNN + lane] = (lane == KNN - 1 && !certified) ? -1.f : mined;
      } else if (k == 2 * KNN - 1) {
        knn2[(long long)i * KNN + lane] = mine;
        if (lane == KNN - 1) r64[i] = (certified2 && mine >= 0) ? sqrtf(mined * (1.f - 1e-6f)) : 0.f;
      }
    }
    if (delta && lane == 0) {
      // the first entry is the nearest site when nothing nearer can be unseen
      bool known = certified || (near != 0x7fffffff && (double)near2 <= (double)covered * (double)covered * (1.0 - 1e-5));
      if (known && near != 0x7fffffff) {
        if (near2 == 0.f) set_error(C.status, VD_ERR_DUPLICATE);  // coincident sites
        delta[i] = T(0.5) * sqrt((T)near2);
      } else if (known) {
        delta[i] = T(1);  // no other site
      } else {
        T d2;
        int k = thread_nearest(C.G, qx, qy, qz, i, d2);
        if (k >= 0 && k < C.n && d2 == T(0)) set_error(C.status, VD_ERR_DUPLICATE);
        delta[i] = (k >= 0 && k < C.n) ? T(0.5) * sqrt(d2) : T(1);
      }
    }
    __syncwarp();
  }
}

// candidates ranked by distance: the first k of the 32 nearest
__global__ void k_cand_by_distance(int n, int k, unsigned* cmask) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) cmask[i] = k >= 32 ? 0xffffffffu : ((1u << k) - 1u);
}

// ---------------------------------------------------------------------------
// per-site reduction, deterministic: the pieces of a site are summed in order
// of their simplex index whatever order the flood produced them in
// ---------------------------------------------------------------------------
// The kernels that read the flood's per-slot outputs (split marks, per-site
// reduction, export) run after it.  A device-side error leaves the outputs of
// unfinished pairs unwritten (stale offsets and counts), so each of them
// returns at once when the status is set.
template <typename T>
__device__ __forceinline__ bool failed(const Dev<T>& C) { return *(volatile const int*)C.status != 0; }

template <typename T>
__device__ __forceinline__ long long npairs(const Dev<T>& C) {
  unsigned long long t = C.ctr[CTR_TAIL];
  return (long long)(t < (unsigned long long)C.qcap ? t : (unsigned long long)C.qcap);
}

// ---------------------------------------------------------------------------
// Split of the sites for 3D clipped diagrams (Alg. 5).  The restricted diagram
// on the domain's boundary triangles (the surface form of the same clip kernel,
// run first on the same pair set) finds the boundary sites: those whose cells
// meet the boundary surface in positive area.  Every other site's cell lies
// inside M when the site does (Omega_i is convex and does not cross the
// boundary), and misses M when it does not.
// ---------------------------------------------------------------------------
// Boundary pass results (queue slots [0, tail) of S): mark the boundary sites and
// collect the 3D seeds (tetrahedron incident to the triangle, site); CTR_SEEDS
// counts them.
__global__ void k_split_mark(const __grid_constant__ Dev<float> S, const int* btet, int* bnd,
                             unsigned long long* seeds) {
  if (failed(S)) return;
  long long np = npairs(S);
  long long stride = (long long)gridDim.x * blockDim.x;
  for (long long p0 = (long long)blockIdx.x * blockDim.x; p0 < np; p0 += stride) {
    long long p = p0 + threadIdx.x;
    bool first = false;
    if (p < np && S.pmeas[p] > 0.f) {
      unsigned long long key = S.queue[p];
      int b = (int)(key >> 32), j = (int)(key & 0xffffffffull);
      first = atomicExch(bnd + j, 1) == 0;
      unsigned long long t = atomicAdd(S.ctr + CTR_SEEDS, 1ull);
      seeds[t] = pair_key(btet[b], j);
    }
    unsigned f = __ballot_sync(FULL, first);
    if ((threadIdx.x & 31) == 0 && f) atomicAdd(S.stats + VD_STAT_BOUNDARY_SITES, (unsigned long long)__popc(f));
  }
}

__global__ void k_split_push(const __grid_constant__ Dev<float> C, const unsigned long long* seeds) {
  long long ns = (long long)C.ctr[CTR_SEEDS];
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < ns; t += (long long)gridDim.x * blockDim.x) {
    unsigned long long key = seeds[t];
    if (owned(C, (int)(key & 0xffffffffull))) push_pair(C, (int)(key >> 32), (int)(key & 0xffffffffull));
  }
}

// Sign of the orientation determinant of (a, b, c, d) (the volume of the
// tetrahedron, times 6), evaluated in float64 from float32 coordinates; 0 when
// it does not clear an error bound of 1e-12 times the permanent (the same
// products on absolute values), several thousand times the standard forward
// bound of this evaluation order, so a nonzero sign is certain.
__device__ int orient3_sign(const float* a, const float* b, const float* c, const float* d) {
  double adx = (double)a[0] - d[0], ady = (double)a[1] - d[1], adz = (double)a[2] - d[2];
  double bdx = (double)b[0] - d[0], bdy = (double)b[1] - d[1], bdz = (double)b[2] - d[2];
  double cdx = (double)c[0] - d[0], cdy = (double)c[1] - d[1], cdz = (double)c[2] - d[2];
  double det = adx * (bdy * cdz - bdz * cdy) + bdx * (cdy * adz - cdz * ady) + cdx * (ady * bdz - adz * bdy);
  double perm = fabs(adx) * (fabs(bdy * cdz) + fabs(bdz * cdy)) + fabs(bdx) * (fabs(cdy * adz) + fabs(cdz * ady)) +
                fabs(cdx) * (fabs(ady * bdz) + fabs(adz * bdy));
  double eb = 1e-12 * perm;
  return det > eb ? 1 : (det < -eb ? -1 : 0);
}

// The same determinant in float32 with its permanent: Shewchuk's forward bound for
// this evaluation from float inputs is below 5e-7 of the permanent, so a value
// beyond 1e-5 of it has a certain sign.
__device__ __forceinline__ float orient3f(const float* a, const float* b, const float* c, const float* d,
                                          float& perm) {
  float adx = a[0] - d[0], ady = a[1] - d[1], adz = a[2] - d[2];
  float bdx = b[0] - d[0], bdy = b[1] - d[1], bdz = b[2] - d[2];
  float cdx = c[0] - d[0], cdy = c[1] - d[1], cdz = c[2] - d[2];
  perm = fabsf(adx) * (fabsf(bdy * cdz) + fabsf(bdz * cdy)) + fabsf(bdx) * (fabsf(cdy * adz) + fabsf(cdz * ady)) +
         fabsf(cdx) * (fabsf(ady * bdz) + fabsf(adz * bdy));
  return adx * (bdy * cdz - bdz * cdy) + bdx * (cdy * adz - cdz * ady) + cdx * (ady * bdz - adz * bdy);
}

// Where site i lies w.r.t. tetrahedron a: 2 strictly inside (certain), 0 certainly
// not inside, 1 undecided (on or within rounding of its boundary).  The point
// replaces each vertex in turn; it is inside iff every such determinant has the
// tetrahedron's orientation sign.  Float32 first, float64 where float32 cannot
// certify the sign.
__device__ __forceinline__ int tet_holds(const Dev<float>& C, int a, const float* p) {
  float V[4][3];
#pragma unroll
  for (int l = 0; l < 4; ++l) {
    const float* q = C.verts + 3 * C.simp[4 * a + l];
    V[l][0] = q[0]; V[l][1] = q[1]; V[l][2] = q[2];
  }
#pragma unroll
  for (int d = 0; d < 3; ++d) {  // bounding box first (exact comparisons)
    float lo = fminf(fminf(V[0][d], V[1][d]), fminf(V[2][d], V[3][d]));
    float hi = fmaxf(fmaxf(V[0][d], V[1][d]), fmaxf(V[2][d], V[3][d]));
    if (p[d] < lo || p[d] > hi) return 0;
  }
  // orient3f(a, b, c, d) = det[a - d, b - d, c - d] has the sign opposite to the
  // volume of (a, b, c, d), whose sign is tsgn
  const int o = -C.tsgn[a];
  bool all = true;
#pragma unroll
  for (int f = 0; f < 4; ++f) {
    const float* A = f == 0 ? p : V[0];
    const float* B = f == 1 ? p : V[1];
    const float* Cc = f == 2 ? p : V[2];
    const float* D = f == 3 ? p : V[3];
    float pm;
    float x = orient3f(A, B, Cc, D, pm);
    int sg = x > 1e-5f * pm ? 1 : (x < -1e-5f * pm ? -1 : orient3_sign(A, B, Cc, D));
    if (sg == -o) return 0;
    all = all && sg == o;
  }
  return all ? 2 : 1;
}

// Seeds of every site: a site that is not a boundary site and lies strictly in a
// tetrahedron gets the whole-cell pair (m, i); any other site seeds every
// tetrahedron that may hold it (with the boundary seeds these reach every piece
// of a boundary site through negative flags).  A non-boundary site in no
// tetrahedron has an empty cell and no pair.
__global__ void k_split_site(const __grid_constant__ Dev<float> C, Locator L, const int* bnd) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  bool whole = false;
  if (t < C.n) {
    const int i = site_id(C.G.L[0].gs[t]);  // grid cell order (see k_seed_box)
    const float* p = C.sites + 3 * i;
    int bx = (int)floor(((double)p[0] - L.ox) * L.ih), by = (int)floor(((double)p[1] - L.oy) * L.ih),
        bz = (int)floor(((double)p[2] - L.oz) * L.ih);
    if (owned(C, i) && bx >= 0 && by >= 0 && bz >= 0 && bx < L.bx && by < L.by && bz < L.bz) {
      int b = (bz * L.by + by) * L.bx + bx;
      int t0 = L.start[b], t1 = L.start[b + 1];
      if (!bnd[i])
        for (int t = t0; t < t1 && !whole; ++t) whole = tet_holds(C, L.items[t], p) == 2;
      if (whole) {
        push_pair(C, C.m, i);
      } else {
        for (int t = t0; t < t1; ++t)
          if (tet_holds(C, L.items[t], p)) push_pair(C, L.items[t], i);
      }
    }
  }
  unsigned w = __ballot_sync(FULL, whole);
  if ((threadIdx.x & 31) == 0 && w) atomicAdd(C.stats + VD_STAT_WHOLE_CELLS, (unsigned long long)__popc(w));
}

template <typename T>
__global__ void k_site_count(Dev<T> C, int* scnt) {
  if (failed(C)) return;
  long long np = npairs(C);
  for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < np; p += (long long)gridDim.x * blockDim.x)
    if (C.pmeas[p] > T(0)) atomicAdd(scnt + (int)(C.queue[p] & 0xffffffffull), 1);
}

template <typename T>
__global__ void k_site_fill(Dev<T> C, const int* soff, int* scur, int* slist) {
  if (failed(C)) return;
  long long np = npairs(C);
  for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < np; p += (long long)gridDim.x * blockDim.x)
    if (C.pmeas[p] > T(0)) {
      int i = (int)(C.queue[p] & 0xffffffffull);
      slist[soff[i] + atomicAdd(scur + i, 1)] = (int)p;
    }
}

template <typename T>
__global__ void k_site_reduce(Dev<T> C, const int* soff, int* slist, T* measure, T* centroid, int* fc) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= C.n || failed(C)) return;
  int b = soff[i], e = soff[i + 1];
  for (int u = b + 1; u < e; ++u) {  // insertion sort by simplex index
    int pu = slist[u];
    unsigned au = (unsigned)(C.queue[pu] >> 32);
    int v = u - 1;
    while (v >= b && (unsigned)(C.queue[slist[v]] >> 32) > au) { slist[v + 1] = slist[v]; --v; }
    slist[v + 1] = pu;
  }
  T m = 0, mx = 0, my = 0, mz = 0;
  int nf = 0;
  for (int u = b; u < e; ++u) {
    int p = slist[u];
    m += C.pmeas[p];
    mx += C.pm1[3 * p];
    my += C.pm1[3 * p + 1];
    mz += C.pm1[3 * p + 2];
    nf += C.pfcnt[p];
  }
  measure[i] = m;
  T cx = C.sites[3 * i], cy = C.sites[3 * i + 1], cz = C.sites[3 * i + 2];
  if (m > T(0)) { cx += mx / m; cy += my / m; cz += mz / m; }
  centroid[3 * i] = cx;
  centroid[3 * i + 1] = cy;
  centroid[3 * i + 2] = cz;
  fc[i] = nf;
}

template <typename T>
__global__ void k_site_nbr(Dev<T> C, const int* soff, const int* slist, const int* foff, int* tmp, int* ucnt) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= C.n || failed(C)) return;
  int base = foff[i], c = 0;
  for (int u = soff[i]; u < soff[i + 1]; ++u) {
    int p = slist[u];
    long long fo = C.pfoff[p];
    for (int f = 0; f < C.pfcnt[p]; ++f) {
      int x = C.pflags[fo + f];
      if (x < 0) continue;
      int v = c - 1;  // insertion into the sorted prefix, skipping duplicates
      bool dup = false;
      while (v >= 0 && tmp[base + v] >= x) {
        if (tmp[base + v] == x) { dup = true; break; }
        --v;
      }
      if (dup) continue;
      for (int w = c; w > v + 1; --w) tmp[base + w] = tmp[base + w - 1];
      tmp[base + v + 1] = x;
      ++c;
    }
  }
  ucnt[i] = c;
}

__global__ void k_site_nbr_copy(int n, const int* foff, const int* tmp, const long long* noff, int* nidx,
                                const int* status) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n || *(volatile const int*)status != 0) return;
  long long o = noff[i];
  int c = (int)(noff[i + 1] - o);
  for (int k = 0; k < c; ++k) nidx[o + k] = tmp[foff[i] + k];
}

// v_i <- centroid_i (Sec. 6.4); after a failed compute the sites stay as they are
// (the reduction did not run, so measure and centroid are not this iterate's)
template <typename T>
__global__ void k_lloyd(int n, T* sites, const T* measure, const T* centroid, const int* status) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n || *(volatile const int*)status != 0 || !(measure[i] > T(0))) return;
  sites[3 * i] = centroid[3 * i];
  sites[3 * i + 1] = centroid[3 * i + 1];
  sites[3 * i + 2] = centroid[3 * i + 2];
}

// piece export: simplex / site of every processed pair and its flags as a CSR.
// limit: the piece count the host checked the output buffers against; the
// kernels never write past it even if the device count were larger.
template <typename T>
__global__ void k_export_ids(Dev<T> C, int* ps, int* pi, long long limit) {
  long long np = npairs(C);
  np = np < limit ? np : limit;
  for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < np; p += (long long)gridDim.x * blockDim.x) {
    unsigned long long key = C.queue[p];
    ps[p] = (int)(key >> 32);
    pi[p] = (int)(key & 0xffffffffull);
  }
}

template <typename T>
__global__ void k_export_flags(Dev<T> C, const long long* xoff, int* xflags, long long limit) {
  long long np = npairs(C);
  np = np < limit ? np : limit;
  for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < np; p += (long long)gridDim.x * blockDim.x)
    for (int f = 0; f < C.pfcnt[p]; ++f) xflags[xoff[p] + f] = C.pflags[C.pfoff[p] + f];
}

// input conversion: n x dim (dim 2 or 3) of type S into n x 3 of type T
template <typename S, typename T>
__global__ void k_widen(const S* in, T* out, long long n, int dim) {
  long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  out[3 * i] = (T)in[dim * i];
  out[3 * i + 1] = (T)in[dim * i + 1];
  out[3 * i + 2] = dim == 3 ? (T)in[dim * i + 2] : T(0);
}

}  // namespace vd
