// vd.cu -- libvd host side: the C ABI declared in include/vd.h.
//
// One context holds one site set and one domain on one device.  vd_compute
// enqueues, on the context stream and without host synchronisation until its
// final status read: grid build -> nearest-neighbour distances -> seeding ->
// persistent clip-and-flood -> per-site reduction.  The same sequence (plus the
// Lloyd update) is what vd_lloyd captures into a CUDA graph.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>
#include <type_traits>
#include <vector>

#include "vd_kernels.cuh"
#include "vd_mlp.cuh"

using namespace vd;

namespace {

struct Buf {
  void* p = nullptr;
  size_t bytes = 0;
};

constexpr int MLP_RANK_BLOCKS = 3;    // inference blocks per SM (61 KB of shared memory each)
constexpr int TUNE_CHUNKS = 5;        // queue chunks the autotuner tries per mapping
constexpr int kTuneChunks[TUNE_CHUNKS] = {1, 2, 4, 8, 16};
constexpr int MLP_MAX_EPOCHS = 1024;  // per-epoch loss slots of vd_mlp_train
constexpr int kLloydGraphIters = 10;  // Lloyd iterations captured in one graph

}  // namespace

struct vd_ctx {
  int dim = 3, dtype = VD_F32, mode = 0, k = 0;
  long long n = 0, nv = 0, m = 0;
  cudaStream_t stream = nullptr;
  cudaStream_t own_stream = nullptr;
  int device = 0, nsm = 0;
  vd_options opt;
  std::vector<void*> allocs;      // everything owned, freed by vd_destroy
  std::vector<void*> dom_allocs;  // owned by the current domain
  void* sites = nullptr;          // n*3 (T)
  void* stage = nullptr;          // n*dim (T) upload staging
  void* verts = nullptr;
  int* simp = nullptr;
  int* adj = nullptr;
  signed char* fsgn = nullptr;
  signed char* tsgn = nullptr;    // [m] 3D: orientation sign of each tetrahedron
  int* loc_start = nullptr;
  int* loc_items = nullptr;
  Locator L{};
  int gx = 0, gy = 0, gz = 0;
  double ox = 0, oy = 0, oz = 0, h = 1;
  long long G = 0;
  int *cellid = nullptr, *ccount = nullptr, *cstart = nullptr, *ccur = nullptr;
  int nlev = 1;                       // grid levels (level 0 dense, 1.. hashed)
  float rho = 3.5f;                   // target sites per cell at the query level
  int* lstart[MAX_LEVELS] = {};       // hashed levels: bucket starts
  void* lgs[MAX_LEVELS] = {};         // hashed levels: sorted sites
  long long lbuckets[MAX_LEVELS] = {};
  unsigned char* qlev = nullptr;      // [G] query level of each level-0 cell
  unsigned char* qlev_nbr = nullptr;  // [G] the same for the densest cell around it (split's boundary pass)
  void* gs = nullptr;
  void* delta = nullptr;
  unsigned long long *hash = nullptr, *queue = nullptr, *ctr = nullptr;
  unsigned long long hmask = 0;
  long long qcap = 0, fcap = 0;
  void *pmeas = nullptr, *pm1 = nullptr;
  long long* pfoff = nullptr;
  int *pfcnt = nullptr, *pflags = nullptr;
  int *scnt = nullptr, *soff = nullptr, *scur = nullptr, *slist = nullptr, *fc = nullptr, *foff = nullptr,
      *tmp = nullptr, *ucnt = nullptr, *nidx = nullptr;
  long long* noff = nullptr;
  void *measure = nullptr, *centroid = nullptr;
  int* status = nullptr;
  unsigned long long* stats = nullptr;
  void* scan_tmp = nullptr;
  int *xs = nullptr, *xi = nullptr, *xflags = nullptr;
  long long* xoff = nullptr;
  int* cand = nullptr;            // candidates set by the caller (vd_set_candidates)
  int ncand = 0;
  int* knn = nullptr;             // [n*32] nearest sites (learned proposal)
  float* knn_d2 = nullptr;
  int* knn2 = nullptr;            // [n*32] the 33rd..64th nearest
  float* knn_r64 = nullptr;       // [n] certified radius of the 64 nearest
  unsigned* cmask = nullptr;      // [n] ranked candidates among the 32 nearest
  bool knn_fresh = false;         // knn holds the lists of the last compute's sites
  bool sites_fresh = false;       // sites unchanged since the last compute
  // learned proposal network: FP32 master weights, Adam moments, gradient, bf16 copy
  float *mlp_p = nullptr, *mlp_m = nullptr, *mlp_v = nullptr, *mlp_g = nullptr, *mlp_loss = nullptr;
  mlp::bf16* mlp_wb = nullptr;
  long long mlp_step = 0;
  bool mlp_ready = false;
  int flood_grid = 0;
  size_t flood_smem = 0;
  int flood_grid_t = 0;           // thread-per-pair kernel (3D FP32)
  int knn_grid = 0;               // resident blocks of k_knn on the device
  int cur_mapping = 1, cur_chunk = 1;  // used by the next enqueue
  bool cur_list64 = true;         // learned form: the 64-site lists (next enqueue)
  bool tuned = false;             // autotuned choice cached for the current domain and options
  int tuned_mapping = 1, tuned_chunk = 1;
  bool tuned_list64 = true;
  float tune_list_ms[2] = {-1.f, -1.f};  // delta + seed + clip with 32 / 64-site lists
  float tune_ms[2 * TUNE_CHUNKS + 2] = {0};  // clip-phase time of each candidate of the last autotune,
                                            // then the list comparison (tune_list_ms)
  bool have_domain = false;
  bool box = false;               // box domain (vd_set_box)
  float blo[3] = {0, 0, 0}, bhi[3] = {0, 0, 0};
  // split (Alg. 5, 3D tetrahedra FP32): the boundary triangles of the mesh, the
  // tetrahedron each belongs to, their edge adjacency, the mesh's bounding box
  bool split_ok = false;
  long long mb = 0;
  int *bsimp = nullptr, *badj = nullptr, *btet = nullptr;
  int* bnd = nullptr;             // [n] 1: boundary site (set by the boundary pass)
  float mlo[3] = {0, 0, 0}, mhi[3] = {0, 0, 0};
  int flood_grid_s = 0;           // boundary pass: surface form of the clip kernel
  size_t flood_smem_s = 0;
  long long last_pairs = 0, last_nnz = 0, last_nonempty = 0;
  int last_status = 0;
  int last_where = 0;          // source line of the first device-side error
  unsigned long long last_stats[VD_STAT_N] = {0};
  bool computed = false;
  bool pending = false;        // vd_compute_async enqueued work whose status is not read yet
  // power diagram (vd_set_weights): lift h_i of every site, its maximum, on / off
  float* lift = nullptr;
  int* lift_scratch = nullptr;  // [3]: ordered max weight, ordered max lift, bad-weight flag
  float lift_max = 0.f;
  bool lift_on = false;
  // partition of one diagram across ranks (vd_set_partition)
  int* owner = nullptr;            // [n] rank of each site
  int part_rank = 0;
  bool part_on = false;
  unsigned long long* outbox = nullptr;
  long long ocap = 0;
  long long last_out = 0;          // pairs in the outbox after the last compute / resume
  int* own_order = nullptr;        // [n] grid positions of the own sites (nearest-list pass)
  cudaGraphExec_t gexec = nullptr;
  int graph_iters = 0;         // Lloyd iterations held by the captured graph
  cudaGraph_t graph = nullptr;
  cudaEvent_t ev[VD_PHASE_N + 1] = {};
  bool timing_now = false;     // events recorded by the current enqueue
  int launches = 0;            // kernels enqueued by the current enqueue
  double last_phase_ms[VD_PHASE_N] = {0};
};

#define CK(x)                                   \
  do {                                          \
    cudaError_t e_ = (x);                       \
    if (e_ != cudaSuccess) {                    \
      return e_ == cudaErrorMemoryAllocation ? VD_ERR_OOM : VD_ERR_CUDA; \
    }                                           \
  } while (0)

static vd_options default_options() {
  vd_options o;
  std::memset(&o, 0, sizeof(o));
  o.mapping = 1;
  return o;
}

static void resolve_options(vd_options& o) {
  if (o.max_clips <= 0) o.max_clips = 256;
  if (o.max_search <= 0) o.max_search = 256;
  if (o.max_lambda <= 0) o.max_lambda = 64;
  if (o.topk <= 0) o.topk = 24;
  if (o.topk > 32) o.topk = 32;
  if (!(o.wait_limit_s > 0)) o.wait_limit_s = 10.0;
}

template <typename P>
static int dalloc(vd_ctx* c, P*& p, size_t count, bool domain) {
  void* q = nullptr;
  cudaError_t e = cudaMalloc(&q, std::max<size_t>(count, 1) * sizeof(P));
  if (e != cudaSuccess) return VD_ERR_OOM;
  (domain ? c->dom_allocs : c->allocs).push_back(q);
  p = static_cast<P*>(q);
  return VD_OK;
}

#define DALLOC(ptr, T_, count, dom)                          \
  do {                                                       \
    T_* tmp_ = nullptr;                                      \
    int rc_ = dalloc(c, tmp_, (size_t)(count), dom);         \
    if (rc_) return rc_;                                     \
    ptr = tmp_;                                              \
  } while (0)

static size_t tsize(int dtype) { return dtype == VD_F64 ? 8 : 4; }

static void free_domain(vd_ctx* c) {
  if (c->gexec) { cudaGraphExecDestroy(c->gexec); c->gexec = nullptr; }
  if (c->graph) { cudaGraphDestroy(c->graph); c->graph = nullptr; }
  for (void* p : c->dom_allocs) cudaFree(p);
  c->dom_allocs.clear();
  c->have_domain = false;
  c->split_ok = false;
  c->bsimp = c->badj = c->btet = c->bnd = nullptr;
  c->qlev_nbr = nullptr;
  c->computed = false;
  c->sites_fresh = c->knn_fresh = false;
  c->tuned = false;
}

// ---------------------------------------------------------------------------
// device context view
// ---------------------------------------------------------------------------
static bool split_active(const vd_ctx* c) {
  // power cells need not contain their sites: the split's premise does not hold
  return c->opt.split && c->split_ok && !c->box && c->mode == VD_MODE_3D && c->dtype == VD_F32 && !c->lift_on;
}

// the learned form's nearest lists (3D distances; power diagrams run the plain search)
static bool lists_active(const vd_ctx* c) { return c->opt.learned && !c->cand && !c->lift_on; }

template <typename T>
static Dev<T> make_dev(vd_ctx* c) {
  Dev<T> D;
  std::memset(&D, 0, sizeof(D));
  D.mode = c->mode; D.n = (int)c->n; D.m = (int)c->m; D.k = c->k;
  D.sites = (const T*)c->sites; D.verts = (const T*)c->verts; D.simp = c->simp; D.adj = c->adj; D.fsgn = c->fsgn;
  D.tsgn = c->tsgn;
  D.delta = (const T*)c->delta;
  D.G.gx = c->gx; D.G.gy = c->gy; D.G.gz = c->gz;
  D.G.ox = (T)c->ox; D.G.oy = (T)c->oy; D.G.oz = (T)c->oz;
  D.G.nlev = c->nlev;
  D.G.qlev = c->qlev;
  for (int l = 0; l < c->nlev; ++l) {
    double h = c->h / (double)(1 << l);
    D.G.L[l].gs = (const typename Prec<T>::V4*)(l == 0 ? c->gs : c->lgs[l]);
    D.G.L[l].start = l == 0 ? c->cstart : c->lstart[l];
    D.G.L[l].mask = l == 0 ? 0u : (unsigned)(c->lbuckets[l] - 1);
    D.G.L[l].h = (T)h;
    D.G.L[l].ih = (T)(1.0 / h);
  }
  if (c->cand) { D.cand = c->cand; D.ncand = c->ncand; }
  else { D.cand = nullptr; D.ncand = 0; }
  D.knn = lists_active(c) ? c->knn : nullptr;
  D.lift = c->lift_on ? c->lift : nullptr;
  D.lift_max = c->lift_on ? c->lift_max : 0.f;
  D.knn_d2 = c->knn_d2;
  D.knn2 = (D.knn && c->cur_list64) ? c->knn2 : nullptr;
  D.knn_r64 = c->knn_r64;
  D.cmask = c->cmask;
  D.hash = c->hash; D.hmask = c->hmask; D.queue = c->queue; D.qcap = c->qcap; D.ctr = c->ctr;
  D.pmeas = (T*)c->pmeas; D.pm1 = (T*)c->pm1; D.pfoff = c->pfoff; D.pfcnt = c->pfcnt; D.pflags = c->pflags;
  D.fcap = c->fcap;
  D.status = c->status; D.stats = c->stats; D.want_stats = c->opt.stats;
  D.max_clips = c->opt.max_clips; D.max_search = c->opt.max_search; D.max_lambda = c->opt.max_lambda;
  D.wait_ns = (long long)(c->opt.wait_limit_s * 1e9);
  D.box = c->box ? 1 : 0;
  for (int d = 0; d < 3; ++d) { D.blo[d] = c->blo[d]; D.bhi[d] = c->bhi[d]; }
  D.split = split_active(c) ? 1 : 0;
  if (D.split)
    for (int d = 0; d < 3; ++d) { D.blo[d] = c->mlo[d]; D.bhi[d] = c->mhi[d]; }
  D.force_exact = c->opt.force_exact ? 1 : 0;
  D.owner = c->part_on ? c->owner : nullptr;
  D.rank = c->part_rank;
  D.own_order = (c->part_on && !D.split) ? c->own_order : nullptr;
  D.outbox = c->outbox;
  D.ocap = c->ocap;
  return D;
}

static inline unsigned nblk(long long n, int t) { return (unsigned)std::max<long long>(1, (n + t - 1) / t); }

template <typename In, typename Out>
static void scan_excl(cudaStream_t s, const In* in, Out* out, long long n, Out* tmp) {
  long long nb = (n + SCAN_TILE - 1) / SCAN_TILE;
  if (nb <= 1) {
    k_scan_tile<In, Out><<<1, SCAN_T, 0, s>>>(in, out, nullptr, n);
    return;
  }
  Out* bs = tmp;
  Out* bo = tmp + nb;
  k_scan_tile<In, Out><<<(unsigned)nb, SCAN_T, 0, s>>>(in, out, bs, n);
  scan_excl<Out, Out>(s, bs, bo, nb, tmp + 2 * nb);
  k_scan_add<Out><<<nblk(n, 256), 256, 0, s>>>(out, bo, n);
}

static int scan_launches(long long n) {
  long long nb = (n + SCAN_TILE - 1) / SCAN_TILE;
  return nb <= 1 ? 1 : 2 + scan_launches(nb);
}

static size_t scan_tmp_elems(long long n) {
  size_t t = 0;
  long long nb = (n + SCAN_TILE - 1) / SCAN_TILE;
  while (nb > 1) { t += 2 * nb; nb = (nb + SCAN_TILE - 1) / SCAN_TILE; }
  return t + 16;
}

// everything of one diagram computation, enqueued on c->stream (graph-capturable)
static inline void mark(vd_ctx* c, int k) {
  if (c->timing_now) cudaEventRecord(c->ev[k], c->stream);
}

// the clip kernel over the queue (persistent; mapping and list size as resolved)
template <typename T, int MODE>
static void enqueue_flood(vd_ctx* c, const Dev<T>& D) {
  cudaStream_t s = c->stream;
  bool thread_form = false;
  if constexpr (MODE == VD_MODE_3D && std::is_same<T, float>::value) thread_form = c->cur_mapping == 2;
  if (thread_form) {
    if constexpr (MODE == VD_MODE_3D && std::is_same<T, float>::value)
      k_flood_thread<<<c->flood_grid_t, FLOOD_T_THREADS, 0, s>>>(D, c->cur_chunk);
  } else {
    bool power = false;
    if constexpr (std::is_same<T, float>::value && MODE != VD_MODE_2D) {
      if (D.lift) {
        k_flood<T, MODE, false, true><<<c->flood_grid, FLOOD_WARPS * 32, c->flood_smem, s>>>(D, c->cur_chunk);
        power = true;
      }
    }
    if (power) {
    } else if (D.knn2) {
      k_flood<T, MODE, true><<<c->flood_grid, FLOOD_WARPS * 32, c->flood_smem, s>>>(D, c->cur_chunk);
    } else {
      k_flood<T, MODE><<<c->flood_grid, FLOOD_WARPS * 32, c->flood_smem, s>>>(D, c->cur_chunk);
    }
  }
  c->launches += 1;
}

// per-site reduction of the pieces and the neighbour CSR
template <typename T, int MODE>
static void enqueue_reduce(vd_ctx* c, const Dev<T>& D) {
  cudaStream_t s = c->stream;
  cudaMemsetAsync(c->scnt, 0, sizeof(int) * (c->n + 1), s);
  cudaMemsetAsync(c->scur, 0, sizeof(int) * c->n, s);
  cudaMemsetAsync(c->fc, 0, sizeof(int) * (c->n + 1), s);
  cudaMemsetAsync(c->ucnt, 0, sizeof(int) * (c->n + 1), s);
  unsigned pg = (unsigned)std::max(1, c->nsm * 8);
  k_site_count<T><<<pg, 256, 0, s>>>(D, c->scnt);
  scan_excl<int, int>(s, c->scnt, c->soff, c->n + 1, (int*)c->scan_tmp);
  k_site_fill<T><<<pg, 256, 0, s>>>(D, c->soff, c->scur, c->slist);
  unsigned bs = nblk(c->n, 128);
  k_site_reduce<T><<<bs, 128, 0, s>>>(D, c->soff, c->slist, (T*)c->measure, (T*)c->centroid, c->fc);
  scan_excl<int, int>(s, c->fc, c->foff, c->n + 1, (int*)c->scan_tmp);
  k_site_nbr<T><<<bs, 128, 0, s>>>(D, c->soff, c->slist, c->foff, c->tmp, c->ucnt);
  scan_excl<int, long long>(s, c->ucnt, c->noff, c->n + 1, (long long*)c->scan_tmp);
  k_site_nbr_copy<<<bs, 128, 0, s>>>((int)c->n, c->foff, c->tmp, c->noff, c->nidx, c->status);
  c->launches += 5 + 3 * scan_launches(c->n + 1);
}

template <typename T, int MODE>
static void enqueue_compute(vd_ctx* c) {
  cudaStream_t s = c->stream;
  Dev<T> D = make_dev<T>(c);
  c->launches = 0;
  mark(c, 0);
  cudaMemsetAsync(c->stats, 0, sizeof(unsigned long long) * VD_STAT_N, s);
  cudaMemsetAsync(c->ctr, 0, sizeof(unsigned long long) * CTR_N, s);
  cudaMemsetAsync(c->hash, 0xFF, sizeof(unsigned long long) * (c->hmask + 1), s);
  cudaMemsetAsync(c->queue, 0xFF, sizeof(unsigned long long) * c->qcap, s);
  unsigned bn = nblk(c->n, 256);
  for (int l = 0; l < c->nlev; ++l) {
    long long nb = l == 0 ? c->G : c->lbuckets[l];
    int* start = l == 0 ? c->cstart : c->lstart[l];
    void* gs = l == 0 ? c->gs : c->lgs[l];
    cudaMemsetAsync(c->ccount, 0, sizeof(int) * (nb + 1), s);
    cudaMemsetAsync(c->ccur, 0, sizeof(int) * nb, s);
    k_cell_count<T><<<bn, 256, 0, s>>>(D, l, c->cellid, c->ccount);
    scan_excl<int, int>(s, c->ccount, start, nb + 1, (int*)c->scan_tmp);
    k_cell_scatter<T><<<bn, 256, 0, s>>>(D, c->cellid, start, c->ccur, (typename Prec<T>::V4*)gs);
    c->launches += 2 + scan_launches(nb + 1);
    if (l == 0 && c->nlev > 1) {
      k_query_level<<<nblk(c->G, 256), 256, 0, s>>>(c->gx, c->gy, c->gz, c->cstart, c->qlev,
                                                    split_active(c) ? c->qlev_nbr : nullptr, c->nlev, c->rho);
      c->launches += 1;
    }
  }
  mark(c, 1);
  // learned form (FP32): the 32-nearest pass also yields delta_i
  const bool fused = lists_active(c) && std::is_same<T, float>::value;
  if (!fused) {
    k_delta<T><<<nblk(c->n, 128), 128, 0, s>>>(D, (T*)c->delta);
    c->launches += 1;
  }
  if (lists_active(c)) {
    // learned proposal: the 32 nearest sites, ranked into the candidate list
    if (D.own_order) {
      k_own_order<T><<<std::min<unsigned>(nblk(c->n, 256), (unsigned)c->nsm * 16), 256, 0, s>>>(D, D.own_order);
      c->launches += 1;
    }
    k_knn<T><<<c->knn_grid, KNN_WARPS * 32, 0, s>>>(D, c->knn, c->knn_d2, fused ? (T*)c->delta : nullptr,
                                                     c->cur_list64 ? c->knn2 : nullptr, c->knn_r64);
    if (c->opt.proposal == VD_PROPOSAL_MLP)
      mlp::k_mlp_rank<T><<<c->nsm * MLP_RANK_BLOCKS, 128, sizeof(mlp::RankSmem), s>>>(
          D, c->knn, (const T*)c->delta, c->mlp_wb, c->mlp_p, c->opt.topk, c->cmask);
    else
      k_cand_by_distance<<<nblk(c->n, 256), 256, 0, s>>>((int)c->n, c->opt.topk, c->cmask);
    c->launches += 2;
  }
  mark(c, 2);
  bool seeded = false;
  if constexpr (MODE == VD_MODE_3D && std::is_same<T, float>::value) {
    if (c->box) {
      k_seed_box<<<nblk(c->n, 256), 256, 0, s>>>(D);
      c->launches += 1;
      seeded = true;
    } else if (D.split) {
      // Alg. 5: the restricted diagram on the boundary triangles (surface form of
      // the clip kernel on the same pair set, counters off), then the 3D seeds
      Dev<float> S = D;
      S.mode = VD_MODE_SURFACE; S.m = (int)c->mb; S.k = 3; S.simp = c->bsimp; S.adj = c->badj;
      S.fsgn = nullptr; S.tsgn = nullptr; S.want_stats = 0; S.split = 0; S.box = 0;
      S.owner = nullptr;  // every rank runs the whole boundary pass; seeds are filtered below
      if (c->nlev > 1) S.G.qlev = c->qlev_nbr;  // boundary points: level of the densest neighbour
      unsigned pg = (unsigned)std::max(1, c->nsm * 8);
      unsigned long long* seeds = (unsigned long long*)c->pm1;  // free until the 3D flood writes it
      cudaMemsetAsync(c->bnd, 0, sizeof(int) * c->n, s);
      k_seed_simplex<float><<<nblk(c->mb, 128), 128, 0, s>>>(S);
      if (S.knn2)
        k_flood<float, VD_MODE_SURFACE, true><<<c->flood_grid_s, FLOOD_WARPS * 32, c->flood_smem_s, s>>>(S, 1);
      else
        k_flood<float, VD_MODE_SURFACE><<<c->flood_grid_s, FLOOD_WARPS * 32, c->flood_smem_s, s>>>(S, 1);
      k_split_mark<<<pg, 256, 0, s>>>(S, c->btet, c->bnd, seeds);
      cudaMemsetAsync(c->hash, 0xFF, sizeof(unsigned long long) * (c->hmask + 1), s);
      cudaMemsetAsync(c->queue, 0xFF, sizeof(unsigned long long) * c->qcap, s);
      cudaMemsetAsync(c->ctr, 0, sizeof(unsigned long long) * CTR_SEEDS, s);  // keeps the seed count
      k_split_push<<<pg, 256, 0, s>>>(D, seeds);
      k_split_site<<<nblk(c->n, 128), 128, 0, s>>>(D, c->L, c->bnd);
      c->launches += 5;
      seeded = true;
    }
  }
  if (!seeded) {
    k_seed_simplex<T><<<nblk(c->m, 128), 128, 0, s>>>(D);
    if (MODE != VD_MODE_SURFACE) k_seed_site<T><<<nblk(c->n, 128), 128, 0, s>>>(D, c->L);
    c->launches += MODE != VD_MODE_SURFACE ? 2 : 1;
  }
  mark(c, 3);
  enqueue_flood<T, MODE>(c, D);
  mark(c, 4);
  enqueue_reduce<T, MODE>(c, D);
  mark(c, 5);
}

template <typename T, int MODE>
static void enqueue_resume(vd_ctx* c, const unsigned long long* keys, long long count) {
  Dev<T> D = make_dev<T>(c);
  c->launches = 0;
  k_resume_prep<<<1, 1, 0, c->stream>>>(c->ctr);
  if (count > 0)
    k_push_keys<T><<<std::min<unsigned>(nblk(count, 256), (unsigned)c->nsm * 8), 256, 0, c->stream>>>(D, keys, count);
  c->launches += count > 0 ? 2 : 1;
  enqueue_flood<T, MODE>(c, D);
  enqueue_reduce<T, MODE>(c, D);
}

static void enqueue_any(vd_ctx* c) {
  if (c->dtype == VD_F64) {
    enqueue_compute<double, VD_MODE_2D>(c);  // checked at vd_set_domain: FP64 runs the 2D path
  } else if (c->mode == VD_MODE_3D) {
    enqueue_compute<float, VD_MODE_3D>(c);
  } else if (c->mode == VD_MODE_SURFACE) {
    enqueue_compute<float, VD_MODE_SURFACE>(c);
  } else {
    enqueue_compute<float, VD_MODE_2D>(c);
  }
}

static void enqueue_lloyd(vd_ctx* c) {
  unsigned bn = nblk(c->n, 256);
  if (c->dtype == VD_F64)
    k_lloyd<double><<<bn, 256, 0, c->stream>>>((int)c->n, (double*)c->sites, (const double*)c->measure,
                                              (const double*)c->centroid, c->status);
  else
    k_lloyd<float><<<bn, 256, 0, c->stream>>>((int)c->n, (float*)c->sites, (const float*)c->measure,
                                             (const float*)c->centroid, c->status);
}

template <typename T, int MODE>
static int flood_config(vd_ctx* c) {
  using W = typename WarpOf<T, MODE>::type;
  c->flood_smem = sizeof(W) * FLOOD_WARPS;
  CK(cudaFuncSetAttribute(k_flood<T, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)c->flood_smem));
  CK(cudaFuncSetAttribute(k_flood<T, MODE, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)c->flood_smem));
  int per_sm = 0, per_sm_x = 0;
  CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_flood<T, MODE>, FLOOD_WARPS * 32, c->flood_smem));
  CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm_x, k_flood<T, MODE, true>, FLOOD_WARPS * 32,
                                                   c->flood_smem));
  per_sm = std::min(per_sm, per_sm_x);
  if constexpr (std::is_same<T, float>::value && MODE != VD_MODE_2D) {
    int per_sm_p = 0;
    CK(cudaFuncSetAttribute(k_flood<T, MODE, false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                            (int)c->flood_smem));
    CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm_p, k_flood<T, MODE, false, true>, FLOOD_WARPS * 32,
                                                     c->flood_smem));
    per_sm = std::min(per_sm, per_sm_p);
  }
  c->flood_grid = std::max(1, per_sm) * c->nsm;
  int per_sm_k = 0;
  CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm_k, k_knn<T>, KNN_WARPS * 32, 0));
  c->knn_grid = std::max(1, per_sm_k) * c->nsm;
  c->flood_grid_t = 0;
  c->flood_grid_s = 0;
  if constexpr (MODE == VD_MODE_3D && std::is_same<T, float>::value) {
    int per_sm_t = 0;
    CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm_t, k_flood_thread, FLOOD_T_THREADS, 0));
    c->flood_grid_t = std::max(1, per_sm_t) * c->nsm;
    // the split's boundary pass runs the surface form
    using WS = typename WarpOf<float, VD_MODE_SURFACE>::type;
    c->flood_smem_s = sizeof(WS) * FLOOD_WARPS;
    CK(cudaFuncSetAttribute(k_flood<float, VD_MODE_SURFACE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                            (int)c->flood_smem_s));
    CK(cudaFuncSetAttribute(k_flood<float, VD_MODE_SURFACE, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                            (int)c->flood_smem_s));
    int per_sm_s = 0;
    CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm_s, k_flood<float, VD_MODE_SURFACE>, FLOOD_WARPS * 32,
                                                     c->flood_smem_s));
    c->flood_grid_s = std::max(1, per_sm_s) * c->nsm;
  }
  return VD_OK;
}

// learned form: whether the lists carry the 64 nearest (the caller's choice, else
// the autotuned one, 64 until tuned)
static bool list64_choice(const vd_ctx* c) {
  if (!lists_active(c)) return false;
  if (c->opt.nearest == 32) return false;
  if (c->opt.nearest == 64) return true;
  return c->tuned ? c->tuned_list64 : true;
}

// mapping of the clip kernel for the next enqueue: the caller's choice, else the
// cached autotuned one (warp per pair with chunk 1 until tuned)
static void resolve_mapping(vd_ctx* c) {
  int m = c->opt.mapping, ch = c->opt.chunk;
  if (m == 0) {
    m = c->tuned ? c->tuned_mapping : 1;
    if (ch <= 0) ch = c->tuned ? c->tuned_chunk : 1;
  }
  if (m == 2 && (c->flood_grid_t == 0 || c->box || split_active(c) || c->lift_on)) m = 1;  // thread per pair: 3D FP32 tetrahedra only
  c->cur_mapping = m;
  c->cur_list64 = list64_choice(c);
  c->cur_chunk = std::max(1, std::min(ch <= 0 ? 1 : ch, 64));
}

static int read_status(vd_ctx* c) {
  unsigned long long ctr[CTR_N];
  int st = 0, where = 0;
  long long nnz = 0;
  int nonempty = 0;
  CK(cudaStreamSynchronize(c->stream));
  CK(cudaMemcpy(ctr, c->ctr, sizeof(ctr), cudaMemcpyDeviceToHost));
  CK(cudaMemcpy(&st, c->status, sizeof(int), cudaMemcpyDeviceToHost));
  CK(cudaMemcpy(&where, c->status + 1, sizeof(int), cudaMemcpyDeviceToHost));
  c->last_where = where;
  CK(cudaMemcpy(c->last_stats, c->stats, sizeof(c->last_stats), cudaMemcpyDeviceToHost));
  CK(cudaMemcpy(&nnz, c->noff + c->n, sizeof(long long), cudaMemcpyDeviceToHost));
  CK(cudaMemcpy(&nonempty, c->soff + c->n, sizeof(int), cudaMemcpyDeviceToHost));
  c->last_pairs = (long long)std::min<unsigned long long>(ctr[CTR_TAIL], (unsigned long long)c->qcap);
  c->last_out = c->part_on ? (long long)std::min<unsigned long long>(ctr[CTR_OUT], (unsigned long long)c->ocap) : 0;
  c->last_nnz = nnz;
  c->last_nonempty = nonempty;
  c->last_stats[VD_STAT_PAIRS] = (unsigned long long)c->last_pairs;
  c->last_stats[VD_STAT_NONEMPTY] = (unsigned long long)nonempty;
  if (st == 0 && ctr[CTR_TAIL] > (unsigned long long)c->qcap) st = VD_ERR_CAPACITY;
  c->last_status = st;
  c->computed = true;
  c->last_stats[VD_STAT_LAUNCHES] = (unsigned long long)c->launches;
  c->last_stats[VD_STAT_MAPPING] =
      (unsigned long long)(c->cur_mapping | (c->cur_chunk << 8) | ((c->cur_list64 ? 64 : 32) << 16));
  for (int k = 0; k < VD_PHASE_N; ++k) c->last_phase_ms[k] = 0;
  if (c->timing_now) {
    const int map[5] = {VD_PHASE_GRID, VD_PHASE_DELTA, VD_PHASE_SEED, VD_PHASE_CLIP, VD_PHASE_REDUCE};
    for (int k = 0; k < 5; ++k) {
      float ms = 0;
      if (cudaEventElapsedTime(&ms, c->ev[k], c->ev[k + 1]) == cudaSuccess) c->last_phase_ms[map[k]] = ms;
    }
  }
  return st;
}

static void fill_result(vd_ctx* c, vd_result* out) {
  if (!out) return;
  out->n = c->n;
  out->nnz = c->last_nnz;
  out->n_pieces = c->last_nonempty;
  out->dtype = c->dtype;
  out->measure = c->measure;
  out->centroid = c->centroid;
  out->nbr_off = (const int64_t*)c->noff;
  out->nbr_idx = c->nidx;
  std::memcpy(out->stats, c->last_stats, sizeof(out->stats));
  out->status = c->last_status;
  out->stats[VD_STAT_ERROR_LINE] = c->last_where;
  for (int k = 0; k < VD_PHASE_N; ++k) out->phase_ms[k] = c->last_phase_ms[k];
}

// ---------------------------------------------------------------------------
// host-side domain preparation (once per domain)
// ---------------------------------------------------------------------------
namespace {

struct FaceKey {
  int v[3];
  long long s;
  int f;
  bool operator<(const FaceKey& o) const {
    if (v[0] != o.v[0]) return v[0] < o.v[0];
    if (v[1] != o.v[1]) return v[1] < o.v[1];
    return v[2] < o.v[2];
  }
  bool same(const FaceKey& o) const { return v[0] == o.v[0] && v[1] == o.v[1] && v[2] == o.v[2]; }
};

}  // namespace

static int build_adjacency(int k, long long m, const std::vector<int>& simp, std::vector<int>& adj,
                           bool strict = true) {
  std::vector<FaceKey> F((size_t)(m * k));
  for (long long a = 0; a < m; ++a)
    for (int f = 0; f < k; ++f) {
      FaceKey& q = F[(size_t)(a * k + f)];
      int c = 0;
      for (int t = 0; t < k; ++t)
        if (t != f) q.v[c++] = simp[(size_t)(a * k + t)];
      if (c == 2) q.v[2] = -1;
      std::sort(q.v, q.v + c);
      q.s = a;
      q.f = f;
    }
  std::sort(F.begin(), F.end());
  adj.assign((size_t)(m * k), -1);
  for (size_t t = 0; t < F.size();) {
    size_t u = t + 1;
    while (u < F.size() && F[t].same(F[u])) ++u;
    if (u - t > 2 && strict) return VD_ERR_DOMAIN;
    if (u - t == 2) {
      adj[(size_t)(F[t].s * k + F[t].f)] = (int)F[t + 1].s;
      adj[(size_t)(F[t + 1].s * k + F[t + 1].f)] = (int)F[t].s;
    }
    t = u;
  }
  return VD_OK;
}

extern "C" {

const char* vd_strerror(int code) {
  switch (code) {
    case VD_OK: return "ok";
    case VD_ERR_ARG: return "invalid argument";
    case VD_ERR_CUDA: return "CUDA runtime error";
    case VD_ERR_OOM: return "device allocation failed";
    case VD_ERR_CAPACITY: return "capacity exceeded (polytope, queue, pair set or flag buffer)";
    case VD_ERR_LIMIT: return "bounded loop or wait hit its limit";
    case VD_ERR_DOMAIN: return "invalid domain mesh";
    case VD_ERR_UNCERTAIN: return "sign not certified in FP64";
    case VD_ERR_STATE: return "call out of order";
    case VD_ERR_DUPLICATE: return "two sites coincide";
    case VD_ERR_IO: return "model file could not be read or written, or is not a model file";
    default: return "unknown error";
  }
}

int vd_create(vd_ctx** out, const void* sites, int64_t n, int dim, int dtype) {
  if (!out || !sites || n < 1 || n > (int64_t)0x3fffffff || (dim != 2 && dim != 3) ||
      (dtype != VD_F32 && dtype != VD_F64))
    return VD_ERR_ARG;
  vd_ctx* c = new (std::nothrow) vd_ctx();
  if (!c) return VD_ERR_OOM;
  c->n = n; c->dim = dim; c->dtype = dtype;
  c->opt = default_options();
  resolve_options(c->opt);
  cudaError_t e = cudaGetDevice(&c->device);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&c->nsm, cudaDevAttrMultiProcessorCount, c->device);
  if (e != cudaSuccess) { delete c; return VD_ERR_CUDA; }
  size_t ts = tsize(dtype);
  int rc = VD_OK;
  {
    char* p = nullptr;
    rc = dalloc(c, p, (size_t)n * 3 * ts, false);
    c->sites = p;
    if (!rc) { rc = dalloc(c, p, (size_t)n * dim * ts, false); c->stage = p; }
    if (!rc) { int* st = nullptr; rc = dalloc(c, st, 2, false); c->status = st; }
    if (!rc) { unsigned long long* s = nullptr; rc = dalloc(c, s, VD_STAT_N, false); c->stats = s; }
  }
  if (rc) { vd_destroy(c); return rc; }
  *out = c;
  rc = vd_update_sites(c, sites);
  if (rc) { vd_destroy(c); *out = nullptr; return rc; }
  cudaStreamSynchronize(c->stream);
  return VD_OK;
}

int vd_create_power2d(vd_ctx** out, const float* xy, const float* w, int64_t n) {
  if (!out || !xy || !w || n < 1 || n > (int64_t)0x3fffffff) return VD_ERR_ARG;
  *out = nullptr;
  float* lifted = nullptr;
  int* scratch = nullptr;  // [0] ordered max weight, [1] bad-weight flag
  if (cudaMalloc(&lifted, sizeof(float) * 3 * n) != cudaSuccess) return VD_ERR_OOM;
  if (cudaMalloc(&scratch, 2 * sizeof(int)) != cudaSuccess) { cudaFree(lifted); return VD_ERR_OOM; }
  int init[2] = {(int)0x80000000, 0};
  int host[2] = {0, 0};
  int rc = VD_OK;
  if (cudaMemcpy(scratch, init, sizeof(init), cudaMemcpyHostToDevice) != cudaSuccess) rc = VD_ERR_CUDA;
  if (!rc) {
    k_power_max<<<std::max(1u, std::min(nblk(n, 256), 1024u)), 256>>>(w, n, scratch);
    k_power_lift<<<nblk(n, 256), 256>>>(xy, w, n, scratch, lifted, scratch + 1);
    if (cudaGetLastError() != cudaSuccess || cudaDeviceSynchronize() != cudaSuccess ||
        cudaMemcpy(host, scratch, sizeof(host), cudaMemcpyDeviceToHost) != cudaSuccess)
      rc = VD_ERR_CUDA;
    else if (host[1])
      rc = VD_ERR_ARG;  // a weight that is not finite
  }
  if (!rc) rc = vd_create(out, lifted, n, 3, VD_F32);
  cudaFree(lifted);
  cudaFree(scratch);
  return rc;
}

int vd_set_weights(vd_ctx* c, const float* w) {
  if (!c) return VD_ERR_ARG;
  if (c->gexec) { cudaGraphExecDestroy(c->gexec); c->gexec = nullptr; }
  if (c->graph) { cudaGraphDestroy(c->graph); c->graph = nullptr; }
  c->tuned = false;
  c->sites_fresh = c->knn_fresh = false;
  if (!w) { c->lift_on = false; return VD_OK; }
  if (c->dtype != VD_F32 || c->dim != 3) return VD_ERR_ARG;
  if (!c->lift) {
    DALLOC(c->lift, float, c->n, false);
    DALLOC(c->lift_scratch, int, 3, false);
  }
  cudaStream_t s = c->stream;
  // ordered bits of -3e38 (weights' maximum starts below any finite weight), of 0
  // (the lifts' maximum), and the bad-weight flag
  int init[3] = {(int)0x80000000 ^ 0x7fffffff, 0, 0};
  {
    float lo = -3.0e38f;
    int b;
    std::memcpy(&b, &lo, 4);
    init[0] = b >= 0 ? b : b ^ 0x7fffffff;
  }
  CK(cudaMemcpyAsync(c->lift_scratch, init, sizeof(init), cudaMemcpyHostToDevice, s));
  k_power_max<<<std::max(1u, std::min(nblk(c->n, 256), 1024u)), 256, 0, s>>>(w, c->n, c->lift_scratch);
  k_power_heights<<<nblk(c->n, 256), 256, 0, s>>>(w, c->n, c->lift_scratch, c->lift, c->lift_scratch + 2);
  CK(cudaGetLastError());
  int back[3];
  CK(cudaMemcpyAsync(back, c->lift_scratch, sizeof(back), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  if (back[2]) { c->lift_on = false; return VD_ERR_ARG; }
  int b = back[1] >= 0 ? back[1] : back[1] ^ 0x7fffffff;
  std::memcpy(&c->lift_max, &b, 4);
  c->lift_on = true;
  return VD_OK;
}

int vd_update_sites(vd_ctx* c, const void* sites) {
  if (!c || !sites) return VD_ERR_ARG;
  c->sites_fresh = c->knn_fresh = false;
  unsigned bn = nblk(c->n, 256);
  if (c->dtype == VD_F64) k_widen<double, double><<<bn, 256, 0, c->stream>>>((const double*)sites, (double*)c->sites, c->n, c->dim);
  else k_widen<float, float><<<bn, 256, 0, c->stream>>>((const float*)sites, (float*)c->sites, c->n, c->dim);
  CK(cudaGetLastError());
  return VD_OK;
}

int vd_update_sites_host(vd_ctx* c, const void* host) {
  if (!c || !host) return VD_ERR_ARG;
  size_t bytes = (size_t)c->n * c->dim * tsize(c->dtype);
  CK(cudaMemcpyAsync(c->stage, host, bytes, cudaMemcpyHostToDevice, c->stream));
  return vd_update_sites(c, c->stage);
}

int vd_get_sites(vd_ctx* c, void* out) {
  if (!c || !out) return VD_ERR_ARG;
  CK(cudaMemcpyAsync(out, c->sites, (size_t)c->n * 3 * tsize(c->dtype), cudaMemcpyDeviceToDevice, c->stream));
  return VD_OK;
}

int vd_set_stream(vd_ctx* c, void* s) {
  if (!c) return VD_ERR_ARG;
  c->stream = (cudaStream_t)s;
  return VD_OK;
}

int vd_set_options(vd_ctx* c, const vd_options* o) {
  if (!c) return VD_ERR_ARG;
  c->opt = o ? *o : default_options();
  resolve_options(c->opt);
  c->tuned = false;
  if (c->gexec) { cudaGraphExecDestroy(c->gexec); c->gexec = nullptr; }
  if (c->graph) { cudaGraphDestroy(c->graph); c->graph = nullptr; }
  return VD_OK;
}

int vd_set_domain(vd_ctx* c, const void* verts, int64_t nv, const int32_t* simplices, int64_t m, int sv) {
  if (!c || !verts || !simplices || nv < 3 || m < 1 || m > (int64_t)0x3fffffff) return VD_ERR_ARG;
  int mode;
  if (c->dim == 2 && sv == 3) mode = VD_MODE_2D;
  else if (c->dim == 3 && sv == 3) mode = VD_MODE_SURFACE;
  else if (c->dim == 3 && sv == 4) mode = VD_MODE_3D;
  else return VD_ERR_ARG;
  if (c->dtype == VD_F64 && mode != VD_MODE_2D) return VD_ERR_ARG;  // FP64 path: planar only
  free_domain(c);
  c->box = false;
  c->mode = mode; c->k = sv; c->nv = nv; c->m = m;
  size_t ts = tsize(c->dtype);
  // host copies for validation and set-up
  std::vector<double> hv((size_t)nv * 3, 0.0);
  {
    std::vector<char> raw((size_t)nv * c->dim * ts);
    CK(cudaStreamSynchronize(c->stream));
    CK(cudaMemcpy(raw.data(), verts, raw.size(), cudaMemcpyDeviceToHost));
    for (long long v = 0; v < nv; ++v)
      for (int d = 0; d < c->dim; ++d)
        hv[(size_t)(3 * v + d)] = c->dtype == VD_F64 ? ((double*)raw.data())[v * c->dim + d]
                                                     : (double)((float*)raw.data())[v * c->dim + d];
  }
  std::vector<int> hs((size_t)(m * sv));
  CK(cudaMemcpy(hs.data(), simplices, hs.size() * sizeof(int), cudaMemcpyDeviceToHost));
  for (int x : hs)
    if (x < 0 || x >= nv) return VD_ERR_DOMAIN;
  double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
  for (long long v = 0; v < nv; ++v)
    for (int d = 0; d < 3; ++d) { lo[d] = std::min(lo[d], hv[3 * v + d]); hi[d] = std::max(hi[d], hv[3 * v + d]); }
  double measure = 0;
  std::vector<signed char> fs((size_t)(m * sv), 1), orient((size_t)m, 1);
  for (long long a = 0; a < m; ++a) {
    const double* P[4];
    for (int l = 0; l < sv; ++l) P[l] = &hv[3 * (size_t)hs[(size_t)(a * sv + l)]];
    if (sv == 4) {
      double u[3], v[3], w[3];
      for (int d = 0; d < 3; ++d) { u[d] = P[1][d] - P[0][d]; v[d] = P[2][d] - P[0][d]; w[d] = P[3][d] - P[0][d]; }
      double det = u[0] * (v[1] * w[2] - v[2] * w[1]) - u[1] * (v[0] * w[2] - v[2] * w[0]) + u[2] * (v[0] * w[1] - v[1] * w[0]);
      if (!(std::fabs(det) > 0)) return VD_ERR_DOMAIN;
      measure += std::fabs(det) / 6.0;
      orient[(size_t)a] = det > 0 ? 1 : -1;
      for (int f = 0; f < 4; ++f) {
        int l0 = f == 0 ? 1 : 0, l1 = f <= 1 ? 2 : 1, l2 = f <= 2 ? 3 : 2;
        double e1[3], e2[3], dd[3];
        for (int d = 0; d < 3; ++d) { e1[d] = P[l1][d] - P[l0][d]; e2[d] = P[l2][d] - P[l0][d]; dd[d] = P[f][d] - P[l0][d]; }
        double nx = e1[1] * e2[2] - e1[2] * e2[1], ny = e1[2] * e2[0] - e1[0] * e2[2], nz = e1[0] * e2[1] - e1[1] * e2[0];
        fs[(size_t)(4 * a + f)] = (nx * dd[0] + ny * dd[1] + nz * dd[2]) < 0 ? 1 : -1;
      }
    } else {
      double u[3], v[3];
      for (int d = 0; d < 3; ++d) { u[d] = P[1][d] - P[0][d]; v[d] = P[2][d] - P[0][d]; }
      double cx = u[1] * v[2] - u[2] * v[1], cy = u[2] * v[0] - u[0] * v[2], cz = u[0] * v[1] - u[1] * v[0];
      double ar = 0.5 * std::sqrt(cx * cx + cy * cy + cz * cz);
      if (!(ar > 0)) return VD_ERR_DOMAIN;
      measure += ar;
    }
  }
  std::vector<int> hadj;
  int rc = build_adjacency(sv, m, hs, hadj);
  if (rc) return rc;
  // split (Alg. 5): the boundary triangles (tetrahedron faces without a neighbour)
  // with the tetrahedron each belongs to, and their edge adjacency (edges shared by
  // more than two boundary triangles are left unpaired: every boundary triangle is
  // seeded on its own, so the boundary pass covers it without them)
  std::vector<int> bs, bt, badj;
  c->split_ok = false;
  if (mode == VD_MODE_3D && c->dtype == VD_F32) {
    for (long long a = 0; a < m; ++a)
      for (int f = 0; f < 4; ++f)
        if (hadj[(size_t)(4 * a + f)] < 0) {
          for (int l = 0; l < 4; ++l)
            if (l != f) bs.push_back(hs[(size_t)(4 * a + l)]);
          bt.push_back((int)a);
        }
    c->mb = (long long)bt.size();
    if (c->mb > 0) {
      build_adjacency(3, c->mb, bs, badj, /*strict=*/false);
      c->split_ok = true;
    }
    for (int d = 0; d < 3; ++d) { c->mlo[d] = (float)lo[d]; c->mhi[d] = (float)hi[d]; }
  }
  // device copies of the mesh
  {
    char* p = nullptr;
    rc = dalloc(c, p, (size_t)nv * 3 * ts, true); if (rc) return rc;
    c->verts = p;
    if (c->dtype == VD_F64) k_widen<double, double><<<nblk(nv, 256), 256, 0, c->stream>>>((const double*)verts, (double*)p, nv, c->dim);
    else k_widen<float, float><<<nblk(nv, 256), 256, 0, c->stream>>>((const float*)verts, (float*)p, nv, c->dim);
    CK(cudaGetLastError());
  }
  DALLOC(c->simp, int, m * sv, true);
  DALLOC(c->adj, int, m * sv, true);
  DALLOC(c->fsgn, signed char, m * sv, true);
  CK(cudaMemcpy(c->simp, hs.data(), hs.size() * sizeof(int), cudaMemcpyHostToDevice));
  CK(cudaMemcpy(c->adj, hadj.data(), hadj.size() * sizeof(int), cudaMemcpyHostToDevice));
  CK(cudaMemcpy(c->fsgn, fs.data(), fs.size(), cudaMemcpyHostToDevice));
  DALLOC(c->tsgn, signed char, m, true);
  CK(cudaMemcpy(c->tsgn, orient.data(), orient.size(), cudaMemcpyHostToDevice));
  if (c->split_ok) {
    DALLOC(c->bsimp, int, bs.size(), true);
    DALLOC(c->badj, int, badj.size(), true);
    DALLOC(c->btet, int, bt.size(), true);
    DALLOC(c->bnd, int, c->n, true);
    CK(cudaMemcpy(c->bsimp, bs.data(), bs.size() * sizeof(int), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(c->badj, badj.data(), badj.size() * sizeof(int), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(c->btet, bt.data(), bt.size() * sizeof(int), cudaMemcpyHostToDevice));
  }
  // simplex locator: bins over the mesh box, each listing the simplices whose box meets it
  if (mode != VD_MODE_SURFACE) {
    int dims = mode == VD_MODE_2D ? 2 : 3;
    double ext[3] = {hi[0] - lo[0], hi[1] - lo[1], hi[2] - lo[2]};
    double vol = 1;
    for (int d = 0; d < dims; ++d) vol *= std::max(ext[d], 1e-30);
    double bs = std::pow(vol / std::max<double>(1, (double)m), 1.0 / dims);
    int nb[3] = {1, 1, 1};
    for (int d = 0; d < dims; ++d) nb[d] = std::max(1, std::min(1024, (int)std::ceil(ext[d] / bs)));
    double bh = 0;
    for (int d = 0; d < dims; ++d) bh = std::max(bh, ext[d] / nb[d]);
    bh *= 1.000001;
    std::vector<std::vector<int>> bins((size_t)nb[0] * nb[1] * nb[2]);
    for (long long a = 0; a < m; ++a) {
      double blo[3] = {1e300, 1e300, 1e300}, bhi[3] = {-1e300, -1e300, -1e300};
      for (int l = 0; l < sv; ++l)
        for (int d = 0; d < 3; ++d) {
          double x = hv[3 * (size_t)hs[(size_t)(a * sv + l)] + d];
          blo[d] = std::min(blo[d], x); bhi[d] = std::max(bhi[d], x);
        }
      int i0[3], i1[3];
      for (int d = 0; d < 3; ++d) {
        if (d >= dims) { i0[d] = i1[d] = 0; continue; }
        i0[d] = std::max(0, (int)std::floor((blo[d] - lo[d]) / bh) - (blo[d] > lo[d] ? 0 : 0));
        i1[d] = std::min(nb[d] - 1, (int)std::floor((bhi[d] - lo[d]) / bh));
        if ((blo[d] - lo[d]) / bh - i0[d] < 1e-9 && i0[d] > 0) i0[d]--;
        if (i1[d] < nb[d] - 1 && (i1[d] + 1) - (bhi[d] - lo[d]) / bh < 1e-9) i1[d]++;
      }
      for (int z = i0[2]; z <= i1[2]; ++z)
        for (int y = i0[1]; y <= i1[1]; ++y)
          for (int x = i0[0]; x <= i1[0]; ++x) bins[((size_t)z * nb[1] + y) * nb[0] + x].push_back((int)a);
    }
    std::vector<int> st(bins.size() + 1, 0), items;
    for (size_t b = 0; b < bins.size(); ++b) {
      st[b + 1] = st[b] + (int)bins[b].size();
      items.insert(items.end(), bins[b].begin(), bins[b].end());
    }
    DALLOC(c->loc_start, int, st.size(), true);
    DALLOC(c->loc_items, int, items.size() + 1, true);
    CK(cudaMemcpy(c->loc_start, st.data(), st.size() * sizeof(int), cudaMemcpyHostToDevice));
    if (!items.empty()) CK(cudaMemcpy(c->loc_items, items.data(), items.size() * sizeof(int), cudaMemcpyHostToDevice));
    c->L.start = c->loc_start; c->L.items = c->loc_items;
    c->L.bx = nb[0]; c->L.by = nb[1]; c->L.bz = nb[2];
    c->L.ox = lo[0]; c->L.oy = lo[1]; c->L.oz = lo[2]; c->L.ih = 1.0 / bh;
  }
  // site grid: the mesh box, padded; about 3.5 sites per cell in 3D, 2.5 in 2D and
  // on surfaces (Sec. 5.2), sized from the mesh measure
  {
    double pad[3];
    for (int d = 0; d < 3; ++d) pad[d] = 1e-3 * (hi[d] - lo[d]) + 1e-6;
    double rho = c->opt.grid_density > 0 ? c->opt.grid_density : 3.0;
    double hh = mode == VD_MODE_3D ? std::cbrt(measure * rho / (double)c->n) : std::sqrt(measure * rho / (double)c->n);
    double e[3];
    for (int d = 0; d < 3; ++d) e[d] = hi[d] - lo[d] + 2 * pad[d];
    for (;;) {
      long long g[3];
      for (int d = 0; d < 3; ++d) g[d] = std::max<long long>(1, (long long)std::ceil(e[d] / hh));
      if (mode == VD_MODE_2D) g[2] = 1;
      if (g[0] * g[1] * g[2] <= (1ll << 28)) {
        c->gx = (int)g[0]; c->gy = (int)g[1]; c->gz = (int)g[2];
        break;
      }
      hh *= 1.25;
    }
    c->h = hh;
    c->rho = (float)rho;
    c->ox = lo[0] - pad[0]; c->oy = lo[1] - pad[1]; c->oz = lo[2] - pad[2];
    if (mode == VD_MODE_2D) { c->oz = -0.5 * hh; }
    c->G = (long long)c->gx * c->gy * c->gz;
    // levels for clustered sites: the densest level-0 cell of the current sites
    // decides how many halvings of the cell edge are needed (3D and surface)
    c->nlev = 1;
    if (mode != VD_MODE_2D) {
      std::vector<char> raw((size_t)c->n * 3 * ts);
      CK(cudaMemcpy(raw.data(), c->sites, raw.size(), cudaMemcpyDeviceToHost));
      std::vector<int> cnt((size_t)c->G, 0);
      int mx = 0;
      for (long long i = 0; i < c->n; ++i) {
        double p[3];
        for (int d = 0; d < 3; ++d)
          p[d] = c->dtype == VD_F64 ? ((double*)raw.data())[3 * i + d] : (double)((float*)raw.data())[3 * i + d];
        long long g[3] = {c->gx, c->gy, c->gz};
        double o[3] = {c->ox, c->oy, c->oz};
        long long ci[3];
        for (int d = 0; d < 3; ++d) ci[d] = std::min<long long>(g[d] - 1, std::max<long long>(0, (long long)std::floor((p[d] - o[d]) / hh)));
        int& k = cnt[(size_t)((ci[2] * c->gy + ci[1]) * c->gx + ci[0])];
        mx = std::max(mx, ++k);
      }
      if (mx > 4 * rho) c->nlev = std::min(MAX_LEVELS, 1 + (int)std::ceil(std::log2((double)mx / rho) / 3.0));
    }
  }
  // per-computation buffers
  long long n = c->n;
  c->qcap = c->opt.queue_capacity > 0 ? c->opt.queue_capacity : 8 * (n + m) + 4096;
  unsigned long long hc = 1;
  while (hc < 2ull * (unsigned long long)c->qcap) hc <<= 1;
  c->hmask = hc - 1;
  c->fcap = 8 * c->qcap;
  long long nbmax = c->G;
  for (int l = 1; l < c->nlev; ++l) {
    long long nb = 1;
    while (nb < 2 * n) nb <<= 1;
    c->lbuckets[l] = nb;
    nbmax = std::max(nbmax, nb);
    DALLOC(c->lstart[l], int, nb + 1, true);
    char* p = nullptr;
    rc = dalloc(c, p, (size_t)n * 4 * ts, true); if (rc) return rc;
    c->lgs[l] = p;
  }
  DALLOC(c->qlev, unsigned char, c->G, true);
  if (c->split_ok) DALLOC(c->qlev_nbr, unsigned char, c->G, true);
  DALLOC(c->knn, int, n * KNN, true);
  DALLOC(c->knn_d2, float, n * KNN, true);
  DALLOC(c->knn2, int, n * KNN, true);
  DALLOC(c->knn_r64, float, n, true);
  DALLOC(c->cmask, unsigned, n, true);
  DALLOC(c->cellid, int, n, true);
  DALLOC(c->ccount, int, nbmax + 1, true);
  DALLOC(c->cstart, int, c->G + 1, true);
  DALLOC(c->ccur, int, nbmax + 1, true);
  {
    char* p = nullptr;
    rc = dalloc(c, p, (size_t)n * 4 * ts, true); if (rc) return rc; c->gs = p;
    rc = dalloc(c, p, (size_t)n * ts, true); if (rc) return rc; c->delta = p;
    rc = dalloc(c, p, (size_t)c->qcap * ts, true); if (rc) return rc; c->pmeas = p;
    rc = dalloc(c, p, (size_t)c->qcap * 3 * ts, true); if (rc) return rc; c->pm1 = p;
    rc = dalloc(c, p, (size_t)n * ts, true); if (rc) return rc; c->measure = p;
    rc = dalloc(c, p, (size_t)n * 3 * ts, true); if (rc) return rc; c->centroid = p;
  }
  DALLOC(c->hash, unsigned long long, hc, true);
  DALLOC(c->queue, unsigned long long, c->qcap, true);
  DALLOC(c->ctr, unsigned long long, CTR_N, true);
  DALLOC(c->pfoff, long long, c->qcap, true);
  DALLOC(c->pfcnt, int, c->qcap + 1, true);
  DALLOC(c->pflags, int, c->fcap, true);
  DALLOC(c->scnt, int, n + 1, true);
  DALLOC(c->soff, int, n + 1, true);
  DALLOC(c->scur, int, n, true);
  DALLOC(c->slist, int, c->qcap, true);
  DALLOC(c->fc, int, n + 1, true);
  DALLOC(c->foff, int, n + 1, true);
  DALLOC(c->tmp, int, c->fcap, true);
  DALLOC(c->ucnt, int, n + 1, true);
  DALLOC(c->noff, long long, n + 1, true);
  DALLOC(c->nidx, int, c->fcap, true);
  {
    long long L = std::max<long long>(nbmax + 1, std::max<long long>(n + 1, c->qcap + 1));
    long long* p = nullptr;
    rc = dalloc(c, p, scan_tmp_elems(L), true); if (rc) return rc;
    c->scan_tmp = p;
  }
  c->xs = c->xi = c->xflags = nullptr;
  c->xoff = nullptr;
  if (c->dtype == VD_F64) rc = flood_config<double, VD_MODE_2D>(c);
  else if (mode == VD_MODE_3D) rc = flood_config<float, VD_MODE_3D>(c);
  else if (mode == VD_MODE_SURFACE) rc = flood_config<float, VD_MODE_SURFACE>(c);
  else rc = flood_config<float, VD_MODE_2D>(c);
  if (rc) return rc;
  CK(cudaStreamSynchronize(c->stream));
  c->have_domain = true;
  return VD_OK;
}

static bool wants_network(const vd_ctx* c) {
  return lists_active(c) && c->opt.proposal == VD_PROPOSAL_MLP;
}

// Autotuner of the clip kernel's mapping: runs the whole compute on the current
// sites once per candidate (warp or thread per pair x queue chunk), times its
// clip phase with CUDA events on the context stream and caches the fastest for
// the current domain and options.  Every candidate produces the same diagram.
static int autotune(vd_ctx* c) {
  // candidates: mapping (1 warp, 2 thread per pair) x queue chunk; slot of each
  // in tune_ms: (mapping - 1) * TUNE_CHUNKS + index of the chunk
  int cand_m[2 * TUNE_CHUNKS], cand_c[2 * TUNE_CHUNKS], cand_s[2 * TUNE_CHUNKS], nc = 0;
  for (int m = 1; m <= 2; ++m) {
    if (m == 2 && (c->flood_grid_t == 0 || c->box || split_active(c) || c->lift_on)) continue;
    for (int k = 0; k < TUNE_CHUNKS; ++k) {
      int ch = c->opt.chunk > 0 ? std::min(c->opt.chunk, 64) : kTuneChunks[k];
      cand_m[nc] = m; cand_c[nc] = ch; cand_s[nc++] = (m - 1) * TUNE_CHUNKS + k;
      if (c->opt.chunk > 0) {  // the caller's chunk: one candidate per mapping, in its slot if listed
        cand_s[nc - 1] = -1;
        for (int q = 0; q < TUNE_CHUNKS; ++q)
          if (kTuneChunks[q] == ch) cand_s[nc - 1] = (m - 1) * TUNE_CHUNKS + q;
        break;
      }
    }
  }
  if (!c->ev[0])
    for (int k = 0; k <= VD_PHASE_N; ++k) CK(cudaEventCreate(&c->ev[k]));
  // learned form: lists of 32 or 64 nearest, compared on the phases they change
  // (the list pass, the seeding and the clip) with one warp per pair, chunk 1
  c->tune_list_ms[0] = c->tune_list_ms[1] = -1.f;
  bool list64 = list64_choice(c);
  if (lists_active(c) && c->opt.nearest == 0) {
    for (int e = 0; e < 2; ++e) {
      c->cur_mapping = 1;
      c->cur_chunk = 1;
      c->cur_list64 = e == 1;
      CK(cudaMemsetAsync(c->status, 0, 2 * sizeof(int), c->stream));
      c->timing_now = true;
      enqueue_any(c);
      cudaError_t err = cudaGetLastError();
      int st = read_status(c);
      c->timing_now = false;
      if (err != cudaSuccess) return VD_ERR_CUDA;
      if (st) return st;
      c->tune_list_ms[e] = (float)(c->last_phase_ms[VD_PHASE_DELTA] + c->last_phase_ms[VD_PHASE_SEED] +
                                   c->last_phase_ms[VD_PHASE_CLIP]);
    }
    list64 = c->tune_list_ms[1] < c->tune_list_ms[0];
  }
  c->cur_list64 = list64;
  int best = 0;
  double best_ms = 1e300;
  for (int k = 0; k < 2 * TUNE_CHUNKS; ++k) c->tune_ms[k] = -1.f;
  double best_warp = 1e300, thread1 = -1.0;
  for (int k = 0; k < nc; ++k) {
    // the thread mapping at other chunks only if its first chunk beat every warp candidate
    if (cand_m[k] == 2 && cand_c[k] != 1 && thread1 >= 0 && thread1 >= best_warp) continue;
    c->cur_mapping = cand_m[k];
    c->cur_chunk = cand_c[k];
    CK(cudaMemsetAsync(c->status, 0, 2 * sizeof(int), c->stream));
    c->timing_now = true;
    enqueue_any(c);
    cudaError_t e = cudaGetLastError();
    int st = read_status(c);
    c->timing_now = false;
    if (e != cudaSuccess) return VD_ERR_CUDA;
    if (st) return st;
    double ms = c->last_phase_ms[VD_PHASE_CLIP];
    if (cand_s[k] >= 0) c->tune_ms[cand_s[k]] = (float)ms;
    if (cand_m[k] == 1) best_warp = std::min(best_warp, ms);
    else if (cand_c[k] == 1) thread1 = ms;
    if (ms < best_ms) { best_ms = ms; best = k; }
  }
  c->sites_fresh = true;
  c->knn_fresh = lists_active(c) && !(c->part_on && !split_active(c));  // partitioned: own sites only
  c->tuned = true;
  c->tuned_mapping = cand_m[best];
  c->tuned_chunk = cand_c[best];
  c->tuned_list64 = list64;
  c->tune_ms[2 * TUNE_CHUNKS] = c->tune_list_ms[0];
  c->tune_ms[2 * TUNE_CHUNKS + 1] = c->tune_list_ms[1];
  return VD_OK;
}

int vd_set_box(vd_ctx* c, const double* lo, const double* hi) {
  if (!c || !lo || !hi || c->dim != 3 || c->dtype != VD_F32) return VD_ERR_ARG;
  float l[3], h[3];
  for (int d = 0; d < 3; ++d) {
    l[d] = (float)lo[d];
    h[d] = (float)hi[d];
    if (!(l[d] < h[d]) || !std::isfinite(l[d]) || !std::isfinite(h[d])) return VD_ERR_ARG;
  }
  // the same box as 6 tetrahedra around its main diagonal: sizes the site grid and
  // the buffers exactly like vd_set_domain (the clip kernel uses the box itself)
  float v[8][3];
  for (int k = 0; k < 8; ++k)
    for (int d = 0; d < 3; ++d) v[k][d] = ((k >> d) & 1) ? h[d] : l[d];
  const int tets[6][4] = {{0, 1, 3, 7}, {0, 1, 5, 7}, {0, 2, 3, 7}, {0, 2, 6, 7}, {0, 4, 5, 7}, {0, 4, 6, 7}};
  float* dv = nullptr;
  int* dt = nullptr;
  CK(cudaMalloc(&dv, sizeof(v)));
  cudaError_t e = cudaMalloc(&dt, sizeof(tets));
  if (e != cudaSuccess) { cudaFree(dv); return VD_ERR_OOM; }
  int rc = VD_OK;
  if (cudaMemcpy(dv, v, sizeof(v), cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(dt, tets, sizeof(tets), cudaMemcpyHostToDevice) != cudaSuccess)
    rc = VD_ERR_CUDA;
  if (!rc) rc = vd_set_domain(c, dv, 8, dt, 6, 4);
  cudaFree(dv);
  cudaFree(dt);
  if (rc) return rc;
  c->box = true;
  for (int d = 0; d < 3; ++d) { c->blo[d] = l[d]; c->bhi[d] = h[d]; }
  return VD_OK;
}

int vd_compute(vd_ctx* c, vd_result* out) {
  if (!c) return VD_ERR_ARG;
  if (!c->have_domain) return VD_ERR_STATE;
  if (wants_network(c) && !c->mlp_ready) return VD_ERR_STATE;
  if (c->opt.mapping == 0 && !c->tuned) {
    int rc = autotune(c);
    if (rc) return rc;
  }
  resolve_mapping(c);
  CK(cudaMemsetAsync(c->status, 0, 2 * sizeof(int), c->stream));
  if (c->opt.timing && !c->ev[0])
    for (int k = 0; k <= VD_PHASE_N; ++k) CK(cudaEventCreate(&c->ev[k]));
  c->timing_now = c->opt.timing != 0;
  enqueue_any(c);
  CK(cudaGetLastError());
  int st = read_status(c);
  c->timing_now = false;
  c->pending = false;
  c->sites_fresh = true;
  c->knn_fresh = lists_active(c) && !(c->part_on && !split_active(c));  // partitioned: own sites only
  fill_result(c, out);
  return st;
}

int vd_compute_async(vd_ctx* c) {
  if (!c) return VD_ERR_ARG;
  if (!c->have_domain) return VD_ERR_STATE;
  if (wants_network(c) && !c->mlp_ready) return VD_ERR_STATE;
  if (c->opt.mapping == 0 && !c->tuned) return VD_ERR_STATE;  // tuning synchronises: not here
  resolve_mapping(c);
  CK(cudaMemsetAsync(c->status, 0, 2 * sizeof(int), c->stream));
  c->timing_now = false;  // no event records: the work stays capturable as it is
  enqueue_any(c);
  CK(cudaGetLastError());
  c->pending = true;
  c->sites_fresh = true;
  c->knn_fresh = lists_active(c) && !(c->part_on && !split_active(c));  // partitioned: own sites only
  return VD_OK;
}

int vd_get_status(vd_ctx* c, int* status) {
  if (!c || !status) return VD_ERR_ARG;
  if (!c->pending && !c->computed) return VD_ERR_STATE;
  int st = read_status(c);
  if (st == VD_ERR_CUDA || st == VD_ERR_OOM) return st;  // the read itself failed
  c->pending = false;
  *status = st;
  return VD_OK;
}

int vd_get_result(vd_ctx* c, vd_result* out) {
  if (!c || !out) return VD_ERR_ARG;
  if (!c->computed) return VD_ERR_STATE;
  fill_result(c, out);
  return VD_OK;
}

// ---------------------------------------------------------------------------
// partition of one diagram across ranks
// ---------------------------------------------------------------------------
int vd_set_partition(vd_ctx* c, const int32_t* owner, int rank) {
  if (!c) return VD_ERR_ARG;
  if (c->pending) return VD_ERR_STATE;
  c->computed = false;
  if (!owner) { c->part_on = false; return VD_OK; }
  if (rank < 0 || !c->have_domain) return rank < 0 ? VD_ERR_ARG : VD_ERR_STATE;
  if (!c->owner) DALLOC(c->owner, int, c->n, false);
  if (!c->own_order) DALLOC(c->own_order, int, c->n, false);
  if (!c->outbox || c->ocap < c->qcap) {
    DALLOC(c->outbox, unsigned long long, c->qcap, false);
    c->ocap = c->qcap;
  }
  CK(cudaMemcpyAsync(c->owner, owner, sizeof(int) * c->n, cudaMemcpyDeviceToDevice, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  c->part_rank = rank;
  c->part_on = true;
  return VD_OK;
}

int vd_get_outbox(vd_ctx* c, const uint64_t** keys, int64_t* count) {
  if (!c || !keys || !count) return VD_ERR_ARG;
  if (!c->computed || c->pending) return VD_ERR_STATE;
  *keys = (const uint64_t*)c->outbox;
  *count = c->part_on ? c->last_out : 0;
  return VD_OK;
}

int vd_resume(vd_ctx* c, const uint64_t* keys, int64_t count, int64_t* added, vd_result* out) {
  if (!c || count < 0 || (count > 0 && !keys)) return VD_ERR_ARG;
  if (!c->computed || c->pending || c->last_status != VD_OK) return VD_ERR_STATE;
  CK(cudaMemsetAsync(c->status, 0, 2 * sizeof(int), c->stream));
  c->timing_now = false;
  const unsigned long long* k = (const unsigned long long*)keys;
  if (c->dtype == VD_F64) enqueue_resume<double, VD_MODE_2D>(c, k, count);
  else if (c->mode == VD_MODE_3D) enqueue_resume<float, VD_MODE_3D>(c, k, count);
  else if (c->mode == VD_MODE_SURFACE) enqueue_resume<float, VD_MODE_SURFACE>(c, k, count);
  else enqueue_resume<float, VD_MODE_2D>(c, k, count);
  CK(cudaGetLastError());
  int st = read_status(c);
  unsigned long long ctr[CTR_N];
  CK(cudaMemcpy(ctr, c->ctr, sizeof(ctr), cudaMemcpyDeviceToHost));
  if (added) *added = (int64_t)(std::min<unsigned long long>(ctr[CTR_TAIL], (unsigned long long)c->qcap) - ctr[CTR_MARK]);
  fill_result(c, out);
  return st;
}

int vd_lloyd_step(vd_ctx* c) {
  if (!c) return VD_ERR_ARG;
  if (!c->computed || c->pending || c->last_status != VD_OK) return VD_ERR_STATE;
  enqueue_lloyd(c);
  CK(cudaGetLastError());
  CK(cudaStreamSynchronize(c->stream));
  c->sites_fresh = c->knn_fresh = false;
  c->computed = false;
  return VD_OK;
}

int vd_autotune(vd_ctx* c, int* mapping, int* chunk, float* times_ms) {
  if (!c) return VD_ERR_ARG;
  if (!c->have_domain) return VD_ERR_STATE;
  if (wants_network(c) && !c->mlp_ready) return VD_ERR_STATE;
  int rc = autotune(c);
  if (rc) return rc;
  if (mapping) *mapping = c->tuned_mapping;
  if (chunk) *chunk = c->tuned_chunk;
  if (times_ms) std::memcpy(times_ms, c->tune_ms, sizeof(c->tune_ms));
  return VD_OK;
}

int vd_copy_result_host(vd_ctx* c, void* measure, void* centroid, int64_t* nbr_off, int32_t* nbr_idx) {
  if (!c) return VD_ERR_ARG;
  if (!c->computed) return VD_ERR_STATE;
  size_t ts = tsize(c->dtype);
  if (measure) CK(cudaMemcpyAsync(measure, c->measure, (size_t)c->n * ts, cudaMemcpyDeviceToHost, c->stream));
  if (centroid) CK(cudaMemcpyAsync(centroid, c->centroid, (size_t)c->n * 3 * ts, cudaMemcpyDeviceToHost, c->stream));
  if (nbr_off) CK(cudaMemcpyAsync(nbr_off, c->noff, (size_t)(c->n + 1) * 8, cudaMemcpyDeviceToHost, c->stream));
  if (nbr_off && nbr_idx && c->last_nnz)
    CK(cudaMemcpyAsync(nbr_idx, c->nidx, (size_t)c->last_nnz * 4, cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  return VD_OK;
}

int vd_lloyd(vd_ctx* c, int iters, int use_graph) {
  if (!c || iters < 0) return VD_ERR_ARG;
  if (!c->have_domain) return VD_ERR_STATE;
  if (c->part_on) return VD_ERR_STATE;  // a partitioned iteration exchanges pairs and sites between ranks
  if (wants_network(c) && !c->mlp_ready) return VD_ERR_STATE;
  if (iters == 0) return VD_OK;
  if (c->opt.mapping == 0 && !c->tuned) {
    // tune on the current sites before any capture (the tuning computes leave the sites as they are)
    int rc = autotune(c);
    if (rc) return rc;
  }
  resolve_mapping(c);
  c->sites_fresh = c->knn_fresh = false;
  CK(cudaMemsetAsync(c->status, 0, 2 * sizeof(int), c->stream));
  if (use_graph) {
    // one graph holds up to kLloydGraphIters whole iterations (compute + update);
    // it is replayed iters / k times and the rest runs eagerly on the same stream
    const int k = std::min(iters, kLloydGraphIters);
    if (c->gexec && c->graph_iters != k) {
      cudaGraphExecDestroy(c->gexec); c->gexec = nullptr;
      cudaGraphDestroy(c->graph); c->graph = nullptr;
    }
    if (!c->gexec) {
      cudaStream_t cap = c->stream;
      if (!cap) {
        if (!c->own_stream) CK(cudaStreamCreateWithFlags(&c->own_stream, cudaStreamNonBlocking));
        cap = c->own_stream;
      }
      cudaStream_t saved = c->stream;
      CK(cudaStreamSynchronize(saved));
      c->stream = cap;
      CK(cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal));
      for (int t = 0; t < k; ++t) {
        enqueue_any(c);
        enqueue_lloyd(c);
      }
      cudaGraph_t g = nullptr;
      cudaError_t e = cudaStreamEndCapture(cap, &g);
      c->stream = saved;
      if (e != cudaSuccess) return VD_ERR_CUDA;
      c->graph = g;
      c->graph_iters = k;
      CK(cudaGraphInstantiate(&c->gexec, g, 0));
    }
    cudaStream_t run = c->stream ? c->stream : c->own_stream;
    if (run != c->stream) { CK(cudaStreamSynchronize(c->stream)); }
    for (int t = 0; t < iters / k; ++t) CK(cudaGraphLaunch(c->gexec, run));
    if (iters % k) {
      cudaStream_t saved = c->stream;
      c->stream = run;
      for (int t = 0; t < iters % k; ++t) {
        enqueue_any(c);
        enqueue_lloyd(c);
      }
      c->stream = saved;
    }
    if (run != c->stream) { CK(cudaStreamSynchronize(run)); }
  } else {
    for (int t = 0; t < iters; ++t) {
      enqueue_any(c);
      enqueue_lloyd(c);
    }
  }
  CK(cudaGetLastError());
  return read_status(c);
}

int vd_get_pieces(vd_ctx* c, vd_pieces* out) {
  if (!c || !out) return VD_ERR_ARG;
  if (!c->computed || c->last_status != VD_OK) return VD_ERR_STATE;  // failed: per-slot outputs incomplete
  long long np = c->last_pairs;
  if (!c->xs) {
    DALLOC(c->xs, int, c->qcap, true);
    DALLOC(c->xi, int, c->qcap, true);
    DALLOC(c->xoff, long long, c->qcap + 1, true);
    DALLOC(c->xflags, int, c->fcap, true);
  }
  cudaStream_t s = c->stream;
  CK(cudaMemsetAsync(c->pfcnt + np, 0, sizeof(int), s));
  if (c->dtype == VD_F64) {
    Dev<double> D = make_dev<double>(c);
    k_export_ids<double><<<c->nsm * 8, 256, 0, s>>>(D, c->xs, c->xi, np);
    scan_excl<int, long long>(s, c->pfcnt, c->xoff, np + 1, (long long*)c->scan_tmp);
    k_export_flags<double><<<c->nsm * 8, 256, 0, s>>>(D, c->xoff, c->xflags, np);
  } else {
    Dev<float> D = make_dev<float>(c);
    k_export_ids<float><<<c->nsm * 8, 256, 0, s>>>(D, c->xs, c->xi, np);
    scan_excl<int, long long>(s, c->pfcnt, c->xoff, np + 1, (long long*)c->scan_tmp);
    k_export_flags<float><<<c->nsm * 8, 256, 0, s>>>(D, c->xoff, c->xflags, np);
  }
  CK(cudaGetLastError());
  CK(cudaStreamSynchronize(s));
  out->n_pieces = np;
  out->simplex = c->xs;
  out->site = c->xi;
  out->measure = c->pmeas;
  out->moment = c->pm1;
  out->flag_off = (const int64_t*)c->xoff;
  out->flags = c->xflags;
  return VD_OK;
}

int vd_set_candidates(vd_ctx* c, const int32_t* cand, int k) {
  if (!c || k < 0 || (k > 0 && !cand)) return VD_ERR_ARG;
  if (c->cand) {
    auto it = std::find(c->allocs.begin(), c->allocs.end(), (void*)c->cand);
    if (it != c->allocs.end()) c->allocs.erase(it);
    cudaFree(c->cand);
    c->cand = nullptr;
  }
  c->ncand = k;
  c->tuned = false;
  if (k == 0) return VD_OK;
  int* p = nullptr;
  int rc = dalloc(c, p, (size_t)c->n * k, false);
  if (rc) return rc;
  c->cand = p;
  CK(cudaMemcpyAsync(p, cand, (size_t)c->n * k * sizeof(int), cudaMemcpyDeviceToDevice, c->stream));
  if (c->gexec) { cudaGraphExecDestroy(c->gexec); c->gexec = nullptr; }
  if (c->graph) { cudaGraphDestroy(c->graph); c->graph = nullptr; }
  return VD_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Piece export without device allocation (vd_get_pieces_noalloc).
//
// The prefix sum over the per-piece flag counts needs block sums; here they live
// in a fixed file-scope device array instead of context scratch.  Host code may
// not use the array's name as a device address: the address is looked up once
// per device with cudaGetSymbolAddress, with that device current.
// ---------------------------------------------------------------------------
namespace {
constexpr long long NOALLOC_MAX_PIECES = (1ll << 26) - 1;
constexpr size_t NOALLOC_SCRATCH = 40960;  // int64: block sums of a scan over <= 2^26 entries
static __device__ __align__(256) long long g_noalloc_scratch[NOALLOC_SCRATCH];
std::mutex g_noalloc_mu;
long long* g_noalloc_addr[1024] = {};

int noalloc_scratch(int device, long long** out) {
  if (device < 0 || device >= 1024) return VD_ERR_ARG;
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (!g_noalloc_addr[device]) {
    int prev = 0;
    CK(cudaGetDevice(&prev));
    if (prev != device) CK(cudaSetDevice(device));
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (prev != device) cudaSetDevice(prev);
    if (e != cudaSuccess || !p) return VD_ERR_CUDA;
    g_noalloc_addr[device] = static_cast<long long*>(p);
  }
  *out = g_noalloc_addr[device];
  return VD_OK;
}
}  // namespace

extern "C" {

int vd_get_pieces_noalloc(vd_ctx* c, int32_t* simplex, int32_t* site, int64_t* flag_off, int32_t* flags,
                          void* measure, void* moment, int64_t pieces_capacity, int64_t flags_capacity,
                          int64_t* n_pieces, int64_t* n_flags) {
  if (!c || !simplex || !site || !flag_off || !n_pieces || !n_flags || pieces_capacity < 0 || flags_capacity < 0)
    return VD_ERR_ARG;
  if (!c->computed || c->last_status != VD_OK) return VD_ERR_STATE;
  static_assert(NOALLOC_MAX_PIECES + 1 <= (1ll << 26), "scan size");
  if (scan_tmp_elems(NOALLOC_MAX_PIECES + 1) > NOALLOC_SCRATCH) return VD_ERR_CAPACITY;
  long long np = c->last_pairs;
  if (np > NOALLOC_MAX_PIECES || np > pieces_capacity) return VD_ERR_CAPACITY;
  // the scratch address below is the one of the context's device: kernels launched
  // with another device current would be handed a foreign address
  int cur = -1;
  CK(cudaGetDevice(&cur));
  if (cur != c->device) return VD_ERR_ARG;
  long long* scratch = nullptr;
  int rc = noalloc_scratch(c->device, &scratch);
  if (rc) return rc;
  cudaStream_t s = c->stream;
  long long* off = reinterpret_cast<long long*>(flag_off);
  CK(cudaMemsetAsync(c->pfcnt + np, 0, sizeof(int), s));
  if (c->dtype == VD_F64) k_export_ids<double><<<c->nsm * 8, 256, 0, s>>>(make_dev<double>(c), simplex, site, np);
  else k_export_ids<float><<<c->nsm * 8, 256, 0, s>>>(make_dev<float>(c), simplex, site, np);
  scan_excl<int, long long>(s, c->pfcnt, off, np + 1, scratch);
  long long total = 0;
  CK(cudaMemcpyAsync(&total, off + np, sizeof(long long), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  if (total > flags_capacity || (total > 0 && !flags)) return VD_ERR_CAPACITY;
  if (c->dtype == VD_F64) k_export_flags<double><<<c->nsm * 8, 256, 0, s>>>(make_dev<double>(c), off, flags, np);
  else k_export_flags<float><<<c->nsm * 8, 256, 0, s>>>(make_dev<float>(c), off, flags, np);
  size_t ts = tsize(c->dtype);
  if (measure && np) CK(cudaMemcpyAsync(measure, c->pmeas, (size_t)np * ts, cudaMemcpyDeviceToDevice, s));
  if (moment && np) CK(cudaMemcpyAsync(moment, c->pm1, (size_t)np * 3 * ts, cudaMemcpyDeviceToDevice, s));
  CK(cudaGetLastError());
  CK(cudaStreamSynchronize(s));
  *n_pieces = np;
  *n_flags = total;
  return VD_OK;
}

void vd_destroy(vd_ctx* c) {
  if (!c) return;
  if (c->stream) cudaStreamSynchronize(c->stream);
  else cudaDeviceSynchronize();
  free_domain(c);
  for (void* p : c->allocs) cudaFree(p);
  for (int k = 0; k <= VD_PHASE_N; ++k)
    if (c->ev[k]) cudaEventDestroy(c->ev[k]);
  if (c->own_stream) cudaStreamDestroy(c->own_stream);
  delete c;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Learned proposal network (vd_mlp_*): state, training data, training.
// ---------------------------------------------------------------------------
namespace {

int mlp_alloc(vd_ctx* c) {
  if (c->mlp_p) return VD_OK;
  DALLOC(c->mlp_p, float, mlp::NPARAM, false);
  DALLOC(c->mlp_m, float, mlp::NPARAM, false);
  DALLOC(c->mlp_v, float, mlp::NPARAM, false);
  DALLOC(c->mlp_g, float, mlp::NPARAM, false);
  DALLOC(c->mlp_loss, float, MLP_MAX_EPOCHS, false);
  DALLOC(c->mlp_wb, mlp::bf16, mlp::NPARAM, false);
  const int rank_smem = (int)sizeof(mlp::RankSmem), train_smem = (int)sizeof(mlp::TrainSmem);
  CK(cudaFuncSetAttribute(mlp::k_mlp_rank<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, rank_smem));
  CK(cudaFuncSetAttribute(mlp::k_mlp_rank<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, rank_smem));
  CK(cudaFuncSetAttribute(mlp::k_mlp_forward, cudaFuncAttributeMaxDynamicSharedMemorySize, rank_smem));
  CK(cudaFuncSetAttribute(mlp::k_mlp_train, cudaFuncAttributeMaxDynamicSharedMemorySize, train_smem));
  return VD_OK;
}

// blocks of the training kernel: about 8 tiles of 16 rows per block
unsigned train_grid(const vd_ctx* c, long long count) {
  long long tiles = (count + 15) / 16;
  return (unsigned)std::max<long long>(1, std::min<long long>(c->nsm, (tiles + 7) / 8));
}

unsigned long long host_mix(unsigned long long x) {
  x ^= x >> 30; x *= 0xbf58476d1ce4e5b9ull;
  x ^= x >> 27; x *= 0x94d049bb133111ebull;
  x ^= x >> 31;
  return x;
}

unsigned long long gcd_u64(unsigned long long a, unsigned long long b) {
  while (b) { unsigned long long t = a % b; a = b; b = t; }
  return a;
}

template <typename T>
int mlp_features_t(vd_ctx* c, void* x, uint32_t* labels) {
  cudaStream_t s = c->stream;
  Dev<T> D = make_dev<T>(c);
  D.own_order = nullptr;  // the training data lists every site
  if (!c->knn_fresh) {
    k_knn<T><<<c->knn_grid, KNN_WARPS * 32, 0, s>>>(D, c->knn, c->knn_d2, nullptr, nullptr, nullptr);
    c->knn_fresh = true;
  }
  if (x)
    mlp::k_features<T><<<nblk(c->n * 32, 256), 256, 0, s>>>(D, c->knn, (const T*)c->delta, (mlp::bf16*)x);
  if (labels) mlp::k_labels<<<nblk(c->n, 128), 128, 0, s>>>((int)c->n, c->knn, c->noff, c->nidx, labels);
  CK(cudaGetLastError());
  return VD_OK;
}

}  // namespace

extern "C" {

int vd_mlp_init(vd_ctx* c, uint64_t seed) {
  if (!c) return VD_ERR_ARG;
  int rc = mlp_alloc(c);
  if (rc) return rc;
  mlp::k_mlp_init<<<nblk(mlp::NPARAM, 256), 256, 0, c->stream>>>(c->mlp_p, c->mlp_m, c->mlp_v, c->mlp_wb,
                                                                   (unsigned long long)seed);
  CK(cudaGetLastError());
  c->mlp_step = 0;
  c->mlp_ready = true;
  return VD_OK;
}

int vd_mlp_set_state(vd_ctx* c, const float* params, const float* adam_m, const float* adam_v, int64_t step) {
  if (!c || !params || step < 0) return VD_ERR_ARG;
  int rc = mlp_alloc(c);
  if (rc) return rc;
  const size_t bytes = sizeof(float) * mlp::NPARAM;
  cudaStream_t s = c->stream;
  CK(cudaMemcpyAsync(c->mlp_p, params, bytes, cudaMemcpyDeviceToDevice, s));
  if (adam_m) CK(cudaMemcpyAsync(c->mlp_m, adam_m, bytes, cudaMemcpyDeviceToDevice, s));
  else CK(cudaMemsetAsync(c->mlp_m, 0, bytes, s));
  if (adam_v) CK(cudaMemcpyAsync(c->mlp_v, adam_v, bytes, cudaMemcpyDeviceToDevice, s));
  else CK(cudaMemsetAsync(c->mlp_v, 0, bytes, s));
  mlp::k_to_bf16<<<nblk(mlp::NPARAM, 256), 256, 0, s>>>(c->mlp_p, c->mlp_wb);
  CK(cudaGetLastError());
  c->mlp_step = step;
  c->mlp_ready = true;
  return VD_OK;
}

int vd_mlp_get_state(vd_ctx* c, float* params, float* adam_m, float* adam_v, int64_t* step) {
  if (!c) return VD_ERR_ARG;
  if (!c->mlp_ready) return VD_ERR_STATE;
  const size_t bytes = sizeof(float) * mlp::NPARAM;
  cudaStream_t s = c->stream;
  if (params) CK(cudaMemcpyAsync(params, c->mlp_p, bytes, cudaMemcpyDeviceToDevice, s));
  if (adam_m) CK(cudaMemcpyAsync(adam_m, c->mlp_m, bytes, cudaMemcpyDeviceToDevice, s));
  if (adam_v) CK(cudaMemcpyAsync(adam_v, c->mlp_v, bytes, cudaMemcpyDeviceToDevice, s));
  CK(cudaStreamSynchronize(s));
  if (step) *step = c->mlp_step;
  return VD_OK;
}

// ---- model file: magic, nparam, step, params, adam_m, adam_v, FNV-1a of all that ----
namespace {
const char kModelMagic[8] = {'V', 'D', 'M', 'L', 'P', '0', '1', '\0'};

unsigned long long fnv1a(const unsigned char* p, size_t n, unsigned long long h) {
  for (size_t k = 0; k < n; ++k) { h ^= p[k]; h *= 0x100000001b3ull; }
  return h;
}
}  // namespace

int vd_model_save(vd_ctx* c, const char* path) {
  if (!c || !path) return VD_ERR_ARG;
  if (!c->mlp_ready) return VD_ERR_STATE;
  const size_t np = mlp::NPARAM;
  std::vector<unsigned char> buf(8 + 16 + 3 * np * sizeof(float));
  std::memcpy(buf.data(), kModelMagic, 8);
  long long hdr[2] = {(long long)np, c->mlp_step};
  std::memcpy(buf.data() + 8, hdr, 16);
  float* body = reinterpret_cast<float*>(buf.data() + 24);
  cudaStream_t s = c->stream;
  CK(cudaMemcpyAsync(body, c->mlp_p, np * sizeof(float), cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpyAsync(body + np, c->mlp_m, np * sizeof(float), cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpyAsync(body + 2 * np, c->mlp_v, np * sizeof(float), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  unsigned long long h = fnv1a(buf.data(), buf.size(), 0xcbf29ce484222325ull);
  FILE* f = std::fopen(path, "wb");
  if (!f) return VD_ERR_IO;
  bool ok = std::fwrite(buf.data(), 1, buf.size(), f) == buf.size() && std::fwrite(&h, 8, 1, f) == 1;
  ok = (std::fclose(f) == 0) && ok;
  return ok ? VD_OK : VD_ERR_IO;
}

int vd_model_load(vd_ctx* c, const char* path) {
  if (!c || !path) return VD_ERR_ARG;
  const size_t np = mlp::NPARAM;
  std::vector<unsigned char> buf(8 + 16 + 3 * np * sizeof(float));
  unsigned long long h = 0;
  FILE* f = std::fopen(path, "rb");
  if (!f) return VD_ERR_IO;
  bool ok = std::fread(buf.data(), 1, buf.size(), f) == buf.size() && std::fread(&h, 8, 1, f) == 1;
  unsigned char extra;
  ok = ok && std::fread(&extra, 1, 1, f) == 0;  // nothing after the hash
  std::fclose(f);
  if (!ok || std::memcmp(buf.data(), kModelMagic, 8) != 0) return VD_ERR_IO;
  long long hdr[2];
  std::memcpy(hdr, buf.data() + 8, 16);
  if (hdr[0] != (long long)np || hdr[1] < 0) return VD_ERR_IO;
  if (fnv1a(buf.data(), buf.size(), 0xcbf29ce484222325ull) != h) return VD_ERR_IO;
  int rc = mlp_alloc(c);
  if (rc) return rc;
  const float* body = reinterpret_cast<const float*>(buf.data() + 24);
  cudaStream_t s = c->stream;
  CK(cudaMemcpyAsync(c->mlp_p, body, np * sizeof(float), cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(c->mlp_m, body + np, np * sizeof(float), cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(c->mlp_v, body + 2 * np, np * sizeof(float), cudaMemcpyHostToDevice, s));
  mlp::k_to_bf16<<<nblk(mlp::NPARAM, 256), 256, 0, s>>>(c->mlp_p, c->mlp_wb);
  CK(cudaGetLastError());
  CK(cudaStreamSynchronize(s));
  c->mlp_step = hdr[1];
  c->mlp_ready = true;
  return VD_OK;
}

int vd_mlp_features(vd_ctx* c, void* x, uint32_t* labels) {
  if (!c) return VD_ERR_ARG;
  if (!c->computed || !c->sites_fresh || (labels && c->last_status != VD_OK)) return VD_ERR_STATE;
  return c->dtype == VD_F64 ? mlp_features_t<double>(c, x, labels) : mlp_features_t<float>(c, x, labels);
}

int vd_mlp_grad(vd_ctx* c, const void* x, const uint32_t* labels, int64_t rows, float* grads, float* loss) {
  if (!c || !x || !labels || !grads || !loss || rows < 1 || rows > (int64_t)0x7fffffff) return VD_ERR_ARG;
  if (!c->mlp_ready) return VD_ERR_STATE;
  cudaStream_t s = c->stream;
  CK(cudaMemsetAsync(grads, 0, sizeof(float) * mlp::NPARAM, s));
  CK(cudaMemsetAsync(c->mlp_loss, 0, sizeof(float), s));
  mlp::k_mlp_train<<<train_grid(c, rows), 128, sizeof(mlp::TrainSmem), s>>>(
      c->mlp_wb, c->mlp_p, (const mlp::bf16*)x, labels, rows, 0, (int)rows, 1, 0, grads, c->mlp_loss);
  mlp::k_scale<<<1, 32, 0, s>>>(c->mlp_loss, loss, 1, (float)(1.0 / ((double)rows * mlp::NOUT)));
  CK(cudaGetLastError());
  return VD_OK;
}

int vd_mlp_forward(vd_ctx* c, const void* x, int64_t rows, float* logits) {
  if (!c || !x || !logits || rows < 1) return VD_ERR_ARG;
  if (!c->mlp_ready) return VD_ERR_STATE;
  long long blocks = std::min<long long>((long long)c->nsm * MLP_RANK_BLOCKS, ((rows + 15) / 16 + 3) / 4);
  mlp::k_mlp_forward<<<(unsigned)std::max<long long>(1, blocks), 128, sizeof(mlp::RankSmem), c->stream>>>(
      c->mlp_wb, c->mlp_p, (const mlp::bf16*)x, rows, logits);
  CK(cudaGetLastError());
  return VD_OK;
}

int vd_get_candidate_masks(vd_ctx* c, uint32_t* masks) {
  if (!c || !masks) return VD_ERR_ARG;
  if (!c->computed || !c->sites_fresh || !c->knn_fresh || !lists_active(c)) return VD_ERR_STATE;
  CK(cudaMemcpyAsync(masks, c->cmask, sizeof(unsigned) * c->n, cudaMemcpyDeviceToDevice, c->stream));
  return VD_OK;
}

int vd_mlp_train(vd_ctx* c, const void* x, const uint32_t* labels, int64_t rows, int batch, int epochs, float lr,
                 uint64_t seed, float* epoch_loss) {
  if (!c || !x || !labels || rows < 1 || rows > (int64_t)0x7fffffff || batch < 1 || batch > (1 << 22) || epochs < 1 ||
      epochs > MLP_MAX_EPOCHS || !(lr > 0.f))
    return VD_ERR_ARG;
  if (!c->mlp_ready) return VD_ERR_STATE;
  cudaStream_t s = c->stream;
  const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
  CK(cudaMemsetAsync(c->mlp_loss, 0, sizeof(float) * epochs, s));
  const unsigned long long R = (unsigned long long)rows;
  for (int e = 0; e < epochs; ++e) {
    // visiting order of this epoch: t -> (pa t + pc) mod rows with gcd(pa, rows) = 1
    unsigned long long h = host_mix((unsigned long long)seed ^ host_mix(0xD1B54A32D192ED03ull * (e + 1ull)));
    unsigned long long pa = R > 1 ? 1 + h % (R - 1) : 1, pc = R > 1 ? host_mix(h) % R : 0;
    while (gcd_u64(pa, R) != 1) pa = pa % (R - 1) + 1;
    for (long long b0 = 0; b0 < rows; b0 += batch) {
      const int count = (int)std::min<long long>(batch, rows - b0);
      CK(cudaMemsetAsync(c->mlp_g, 0, sizeof(float) * mlp::NPARAM, s));
      mlp::k_mlp_train<<<train_grid(c, count), 128, sizeof(mlp::TrainSmem), s>>>(
          c->mlp_wb, c->mlp_p, (const mlp::bf16*)x, labels, rows, b0, count, (long long)pa, (long long)pc, c->mlp_g,
          c->mlp_loss + e);
      ++c->mlp_step;
      const float c1 = (float)(1.0 - std::pow((double)b1, (double)c->mlp_step));
      const float c2 = (float)(1.0 - std::pow((double)b2, (double)c->mlp_step));
      mlp::k_adam<<<nblk(mlp::NPARAM, 256), 256, 0, s>>>(c->mlp_p, c->mlp_g, c->mlp_m, c->mlp_v, c->mlp_wb, lr, b1,
                                                          b2, eps, c1, c2);
    }
  }
  CK(cudaGetLastError());
  if (epoch_loss) {
    CK(cudaMemcpyAsync(epoch_loss, c->mlp_loss, sizeof(float) * epochs, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    for (int e = 0; e < epochs; ++e) epoch_loss[e] = (float)(epoch_loss[e] / ((double)rows * mlp::NOUT));
  } else {
    CK(cudaStreamSynchronize(s));
  }
  return VD_OK;
}

}  // extern "C"
