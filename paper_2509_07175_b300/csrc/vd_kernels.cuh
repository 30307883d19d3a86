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
// at the cell's own density (each level halves the cell edge)
__global__ void k_query_level(int G0, const int* cstart0, unsigned char* qlev, int nlev, float rho) {
  int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= G0) return;
  float cnt = (float)(cstart0[c + 1] - cstart0[c]);
  int l = 0;
  if (cnt > rho) l = (int)ceilf(log2f(cnt / rho) / 3.f - 0.15f);
  qlev[c] = (unsigned char)min(l, nlev - 1);
}

// delta_i = half the distance from v_i to its nearest other site (Sec. 5.1)
template <typename T>
__global__ void k_delta(const __grid_constant__ Dev<T> C, T* delta) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= C.n) return;
  T d2;
  int k = thread_nearest(C.G, C.sites[3 * i], C.sites[3 * i + 1], C.sites[3 * i + 2], i, d2);
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
  int i = thread_nearest(C.G, c[0], c[1], c[2], -1, d2);
  if (i >= 0 && i < C.n) push_pair(C, a, i);
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

// box domain: every site's cell is one piece, (0, i); no pair set is needed
__global__ void k_seed_box(Dev<float> C) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= C.n) return;
  C.queue[i] = pair_key(0, i);
  if (i == 0) atomicAdd(C.ctr + CTR_TAIL, (unsigned long long)C.n);
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
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= C.n) return;
  T p[3] = {C.sites[3 * i], C.sites[3 * i + 1], C.sites[3 * i + 2]};
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
#ifndef FLOOD_MIN_BLOCKS
#define FLOOD_MIN_BLOCKS 3
#endif

// Warp per pair: each warp claims `chunk` consecutive queue slots at a time.
template <typename T, int MODE>
__global__ void __launch_bounds__(FLOOD_WARPS * 32, FLOOD_MIN_BLOCKS) k_flood(const __grid_constant__ Dev<T> C, int chunk) {
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
      if constexpr (MODE == VD_MODE_3D) c3::process_pair(C, w, a, i, (long long)h, lane);
      else cp::process_pair<T>(C, w, a, i, (long long)h, lane);
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
  c3t::Counters K = {0, 0, 0, 0, 0, 0, 0, 0, 0};
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
  }
}

// ---------------------------------------------------------------------------
// the 32 nearest other sites of every site (features of the learned proposal)
// ---------------------------------------------------------------------------
constexpr int KNN = 32;
constexpr int KNN_CAP = 1024;
constexpr int KNN_WARPS = 4;

struct KnnScratch {
  float d2[KNN_CAP];
  int id[KNN_CAP];
  int cnt;
  ScanScratch ss;  // segment table of rings beyond ring 1
};

// warp per site: collect the sites of growing rings around v_i, then select the
// 32 smallest squared distances (ties: smaller index) once the 32nd is covered
template <typename T>
__global__ void __launch_bounds__(KNN_WARPS * 32) k_knn(const __grid_constant__ Dev<T> C, int* knn, float* knn_d2) {
  __shared__ KnnScratch sh[KNN_WARPS];
  KnnScratch& S = sh[threadIdx.x >> 5];
  int lane = threadIdx.x & 31;
  int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, nw = (gridDim.x * blockDim.x) >> 5;
  for (int i = gw; i < C.n; i += nw) {
    T qx = C.sites[3 * i], qy = C.sites[3 * i + 1], qz = C.sites[3 * i + 2];
    if (lane == 0) S.cnt = 0;
    __syncwarp();
    auto visit = [&](const typename Prec<T>::V4& s) {
      int k = site_id(s);
      if (k == i) return;
      T dx = s.x - qx, dy = s.y - qy, dz = s.z - qz;
      int slot = atomicAdd(&S.cnt, 1);
      if (slot < KNN_CAP) { S.d2[slot] = (float)(dx * dx + dy * dy + dz * dz); S.id[slot] = k; }
    };
    int lev = C.G.query_level(qx, qy, qz), cx, cy, cz;
    C.G.cell_at(lev, qx, qy, qz, cx, cy, cz);
    // certified: every site within `cover` of v_i was stored and at least 32 of
    // the stored distances are below cover^2 (so no unseen site can be nearer
    // than the 32nd); otherwise the list is kept for the features but flagged
    bool certified = false;
    for (int r = 1;; ++r) {
      warp_scan_ring(C.G, lev, cx, cy, cz, r, lane, S.ss, visit);
      __syncwarp();
      int cnt = min(S.cnt, KNN_CAP);
      T m = C.G.cover(lev, cx, cy, cz, r, qx, qy, qz);
      if (S.cnt > KNN_CAP) break;
      if (m >= T(1e29)) { certified = true; break; }
      if (cnt >= KNN) {
        float m2 = (float)(m * m) * (1.f - 1e-5f);
        int below = 0;
        for (int t = lane; t < cnt; t += 32) below += S.d2[t] <= m2;
        below = __reduce_add_sync(FULL, below);
        if (below >= KNN) { certified = true; break; }
      }
      if (r >= 4) break;
    }
    int cnt = min(S.cnt, KNN_CAP);
    __syncwarp();
    // selection of the 32 nearest, in order
    for (int k = 0; k < KNN; ++k) {
      float bd = 3.0e38f;
      int bi = 0x7fffffff, bs = -1;
      for (int t = lane; t < cnt; t += 32) {
        float d = S.d2[t];
        int id = S.id[t];
        if (d < bd || (d == bd && id < bi)) { bd = d; bi = id; bs = t; }
      }
      float d0 = bd;
      int i0 = bi;
      warp_argmin(bd, bi);
      if (d0 == bd && i0 == bi && bs >= 0) S.d2[bs] = 3.0e38f;
      if (lane == 0) {
        knn[(long long)i * KNN + k] = bi == 0x7fffffff ? -1 : bi;
        // a negative 32nd distance marks a list that is not certified complete
        knn_d2[(long long)i * KNN + k] = (k == KNN - 1 && !certified) ? -1.f : bd;
      }
      __syncwarp();
    }
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
    push_pair(C, (int)(key >> 32), (int)(key & 0xffffffffull));
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
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  bool whole = false;
  if (i < C.n) {
    const float* p = C.sites + 3 * i;
    int bx = (int)floor(((double)p[0] - L.ox) * L.ih), by = (int)floor(((double)p[1] - L.oy) * L.ih),
        bz = (int)floor(((double)p[2] - L.oz) * L.ih);
    if (bx >= 0 && by >= 0 && bz >= 0 && bx < L.bx && by < L.by && bz < L.bz) {
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
  long long np = npairs(C);
  for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < np; p += (long long)gridDim.x * blockDim.x)
    if (C.pmeas[p] > T(0)) atomicAdd(scnt + (int)(C.queue[p] & 0xffffffffull), 1);
}

template <typename T>
__global__ void k_site_fill(Dev<T> C, const int* soff, int* scur, int* slist) {
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
  if (i >= C.n) return;
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
  if (i >= C.n) return;
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

__global__ void k_site_nbr_copy(int n, const int* foff, const int* tmp, const long long* noff, int* nidx) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  long long o = noff[i];
  int c = (int)(noff[i + 1] - o);
  for (int k = 0; k < c; ++k) nidx[o + k] = tmp[foff[i] + k];
}

template <typename T>
__global__ void k_lloyd(int n, T* sites, const T* measure, const T* centroid) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n || !(measure[i] > T(0))) return;
  sites[3 * i] = centroid[3 * i];
  sites[3 * i + 1] = centroid[3 * i + 1];
  sites[3 * i + 2] = centroid[3 * i + 2];
}

// piece export: simplex / site of every processed pair and its flags as a CSR
template <typename T>
__global__ void k_export_ids(Dev<T> C, int* ps, int* pi) {
  long long np = npairs(C);
  for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < np; p += (long long)gridDim.x * blockDim.x) {
    unsigned long long key = C.queue[p];
    ps[p] = (int)(key >> 32);
    pi[p] = (int)(key & 0xffffffffull);
  }
}

template <typename T>
__global__ void k_export_flags(Dev<T> C, const long long* xoff, int* xflags) {
  long long np = npairs(C);
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
