/*
 * vd.h -- C ABI of libvd: clipped (2D, 3D) and restricted (surface) Voronoi
 * diagrams computed on the GPU by edge-based clipping driven by point-in-cell
 * tests (Xiao, Cao, Chen, "Efficient Computation of Voronoi Diagrams Using
 * Point-in-Cell Tests").
 *
 * Problem (Sec. 2.1, Eq. 1): sites v_1..v_n and a domain M made of simplices
 * T_1..T_m (triangles in 2D or on a surface, tetrahedra in 3D).  The cell of v_i
 * is Omega_i = { x : |x - v_i| <= |x - v_j| for all j }; the output is, for
 * every site, Omega_i intersected with M: its measure (area or volume), its
 * centroid and the sites whose cells share a face of positive measure with it
 * (the positive face flags of Sec. 2.2).
 *
 * Conventions shared by every entry point:
 *   - All device pointers are CUDA device addresses on the context's device.
 *     Inputs are caller-owned and copied before the call returns or, for the
 *     asynchronous calls, before any later call on the same stream runs.
 *   - Results (vd_result, vd_pieces) point into memory owned by the context.
 *     They stay valid until the next vd_compute / vd_update_sites /
 *     vd_set_domain / vd_destroy on the same context.
 *   - Errors are returned as negative codes (vd_strerror names them); no entry
 *     point throws, aborts or prints.  A failed call leaves the context usable
 *     unless the code is VD_ERR_CUDA.
 *   - Work is enqueued on the context's stream (vd_set_stream; default: the
 *     legacy default stream).
 */
#ifndef VD_H_
#define VD_H_

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct vd_ctx vd_ctx;

enum {
  VD_OK = 0,
  VD_ERR_ARG = -1,        /* bad argument (null pointer, size, mode, dtype) */
  VD_ERR_CUDA = -2,       /* a CUDA runtime call failed */
  VD_ERR_OOM = -3,        /* device allocation failed */
  VD_ERR_CAPACITY = -4,   /* a fixed capacity was exceeded (polytope corners or
                             planes, work queue, pair set); results are invalid */
  VD_ERR_LIMIT = -5,      /* a bounded loop or wait hit its limit; results invalid */
  VD_ERR_DOMAIN = -6,     /* the mesh failed validation (bad index, zero-measure
                             simplex, face shared by more than two simplices) */
  VD_ERR_UNCERTAIN = -7,  /* reserved: a sign could not be certified even in FP64
                             (reported through the stats, results still written) */
  VD_ERR_STATE = -8,      /* call out of order (e.g. vd_compute before vd_set_domain) */
  VD_ERR_DUPLICATE = -9,  /* two sites coincide: their bisector is undefined and Eq. 1 would
                             give both the same cell (found by vd_compute's nearest-site pass) */
  VD_ERR_IO = -10         /* a model file could not be opened, read or written, or is not a
                             model file of this library (wrong magic, size or checksum) */
};

enum { VD_F32 = 0, VD_F64 = 1 };

/* dim / simplex_verts select the mode: (2,3) planar triangles, (3,3) surface
 * triangles in R^3 (restricted diagram), (3,4) tetrahedra (clipped diagram) */
enum { VD_MODE_2D = 2, VD_MODE_SURFACE = 3, VD_MODE_3D = 4 };

/* statistics slots of vd_result.stats (counted only when vd_options.stats = 1,
 * except the ones marked "always") */
enum {
  VD_STAT_PAIRS = 0,          /* (simplex, site) pairs processed (always) */
  VD_STAT_NONEMPTY = 1,       /* pairs with a non-empty piece (always) */
  VD_STAT_NN_QUERIES = 2,     /* nearest-site scans (point-in-cell and search) */
  VD_STAT_CORNER_TESTS = 3,   /* point-in-cell tests on corners */
  VD_STAT_CLIPS = 4,          /* clips performed */
  VD_STAT_LAMBDA_STEPS = 5,   /* start-point steps of the improved search */
  VD_STAT_SEARCH_STEPS = 6,   /* bisector-search steps */
  VD_STAT_FP64 = 7,           /* sign decisions settled in FP64 (always) */
  VD_STAT_UNCERTAIN = 8,      /* decisions not certified in FP64 (always) */
  VD_STAT_TIES = 9,           /* exact ties (value zero), counted as inside (always) */
  VD_STAT_SITES_SCANNED = 10, /* site-distance evaluations in nearest-site scans */
  VD_STAT_LEARNED_HITS = 11,  /* bisectors found by the learned candidate shortcut */
  VD_STAT_FALLBACK = 12,      /* searches that fell back to the certified witness */
  VD_STAT_LAUNCHES = 13,      /* kernels launched by the call (always) */
  VD_STAT_ILLCOND = 14,       /* corners too ill-conditioned for the FP32 filter (always) */
  VD_STAT_ERROR_LINE = 15,    /* source line of the first device-side error (diagnostics) */
  VD_STAT_DIAG = 16,          /* 16..23: first FP64 decision that was not certified or was an
                                 exact tie: simplex, site, the 4 plane sources, tie flag, kind */
  VD_STAT_WHOLE_CELLS = 24,   /* split = 1: sites whose cell was computed whole (always) */
  VD_STAT_BOUNDARY_SITES = 25,/* split = 1: sites whose cell meets the boundary surface (always) */
  VD_STAT_BISECTOR_FACES = 26,/* bisector faces (edges in 2D / on surfaces) of positive measure in
                                 the final pieces.  Sec. 3.3: every clip of Alg. 1
                                 contributes a face, so there it equals VD_STAT_CLIPS */
  VD_STAT_EXCESS_CLIPS = 27,  /* clips whose bisector is not a face of positive measure of the
                                 final piece, summed over the pieces.  Alg. 3 searches on
                                 the virtual edge v_i -> p; when v_i lies outside the simplex the
                                 exit point of Omega_i on it may lie outside the simplex too, so
                                 a clip need not contribute (Sec. 4.1); with v_i inside the
                                 simplex (or the box) every clip does, except a clip by a
                                 certified witness after an FP32 search failed
                                 (VD_STAT_FALLBACK) */
  VD_STAT_LIST_TESTS = 30,    /* point-in-cell tests and queries settled from the 32 nearest
                                 sites of the cell's site, with no grid scan (learned form) */
  VD_STAT_MAPPING = 31,       /* clip-kernel mapping used: mapping | chunk << 8 | list << 16
                                 (list: 64 or 32 sites per learned list) (always) */
  VD_STAT_N = 32
};

/* phases timed with CUDA events on the context stream when vd_options.timing = 1 */
enum { VD_PHASE_GRID = 0, VD_PHASE_DELTA = 1, VD_PHASE_SEED = 2, VD_PHASE_CLIP = 3, VD_PHASE_REDUCE = 4,
       VD_PHASE_N = 8 };

typedef struct {
  int learned;             /* 1: use the candidate lists set by vd_set_candidates */
  int mapping;             /* clip kernel: 0 automatic (autotuned on the first compute and
                              cached until the options or the domain change), 1 one warp per
                              pair, 2 one thread per pair (3D FP32; other modes use 1) */
  int chunk;               /* queue slots claimed per access (0: autotuned with mapping 0, else 1;
                              at most 64) */
  int stats;               /* 1: collect the counters marked above */
  int64_t queue_capacity;  /* pairs (0: automatic, 8 (n + m) + 4096) */
  int max_clips;           /* clips per pair before VD_ERR_LIMIT (0: 256) */
  int max_search;          /* bisector-search steps per clip (0: 256) */
  int max_lambda;          /* start-point steps per clip (0: 64) */
  double wait_limit_s;     /* longest wait of an idle worker on the queue (0: 10 s) */
  int timing;              /* 1: time the phases of vd_compute with CUDA events */
  double grid_density;     /* target sites per grid cell (0: 3.0); read by vd_set_domain */
  int topk;                /* candidates per site used by the learned proposal (0: 24, max 32) */
  int proposal;            /* learned form's ranking of the 32 nearest sites: VD_PROPOSAL_DISTANCE
                              (the topk nearest) or VD_PROPOSAL_MLP (the topk largest logits of
                              the context's network, vd_mlp_*) */
  int split;               /* 3D tetrahedra (FP32), Alg. 5: 1 first computes the restricted
                              diagram on the domain's boundary triangles; a site whose
                              restricted cell there is empty and that lies strictly inside a
                              tetrahedron has its whole Voronoi cell inside the domain and gets
                              one piece, (m, i): the mesh's bounding box clipped by its
                              bisectors (Sec. 4.2).  The pieces of the other sites are the
                              per-tetrahedron pieces, reached from the boundary pieces' incident
                              tetrahedra (and the site's own) through negative flags.  Measures,
                              centroids and neighbours are those of split = 0 (the same cells,
                              summed in fewer pieces); ignored in other modes and by vd_set_box.
                              Clip kernel: one warp per pair. */
  int nearest;             /* learned form (32-NN lists): 64 also stores the 33rd..64th nearest
                              and settles point-in-cell tests and searches out to half their
                              radius from the lists (fewer grid scans, a costlier list pass);
                              32 the 32 only; 0 chosen by the autotuner with mapping 0 (64
                              until tuned). */
  int force_exact;         /* 1: no FP32 filter in the clip -- every side decision of a corner
                              against a clipping plane, and every new corner, goes through the
                              float64 path (the exact sign with its error bound, the corner from
                              its exact planes).  A test of that path (a filter failure forced
                              from the host): the topology is the same as with 0, measures and
                              centroids differ by rounding.  Slower; 0 by default. */
} vd_options;

enum { VD_PROPOSAL_DISTANCE = 0, VD_PROPOSAL_MLP = 1 };

typedef struct {
  int64_t n;               /* sites */
  int64_t nnz;             /* total neighbour entries */
  int64_t n_pieces;        /* non-empty pieces */
  int dtype;               /* VD_F32 / VD_F64: element type of measure and centroid */
  const void* measure;     /* device [n]: area or volume of Omega_i within M */
  const void* centroid;    /* device [n*3]: centroid (v_i for an empty cell) */
  const int64_t* nbr_off;  /* device [n+1]: CSR offsets */
  const int32_t* nbr_idx;  /* device [nnz]: neighbours of each site, ascending */
  int64_t stats[VD_STAT_N];
  int status;              /* VD_OK or the first device-side error code */
  double phase_ms[VD_PHASE_N]; /* per-phase device time (vd_options.timing = 1), else 0 */
} vd_result;

typedef struct {
  int64_t n_pieces;        /* number of (simplex, site) pairs processed */
  const int32_t* simplex;  /* device [n_pieces] */
  const int32_t* site;     /* device [n_pieces] */
  const void* measure;     /* device [n_pieces] (dtype of the context); 0 for empty pieces */
  const void* moment;      /* device [n_pieces*3]: first moment in the frame of the site */
  const int64_t* flag_off; /* device [n_pieces+1] */
  const int32_t* flags;    /* device: face flags of positive measure; j >= 0: bisector with
                              site j; -(b+1): face shared with simplex b; INT32_MIN: mesh
                              boundary (Sec. 2.2) */
} vd_pieces;

/* Create a context for n sites of the given dimension (2 or 3) and dtype.
 * sites: device pointer, n*dim elements of dtype, row-major; copied.
 * Sec. 2.1 (the sites V).  Returns VD_ERR_ARG for n < 1, dim not in {2,3},
 * dtype not in {VD_F32, VD_F64}. */
int vd_create(vd_ctx** out, const void* sites, int64_t n, int dim, int dtype);

/* Power diagram in the plane (the paper's extension to power diagrams by
 * lifting): the power distance of x to site i is |x - v_i|^2 - w_i.  Creates a
 * 3D FP32 context whose sites are the lifted points (x_i, y_i, sqrt(eta - w_i)),
 * eta = max_i w_i (found on the device): for x in the plane z = 0,
 * |x - p_i|^2 = |x - v_i|^2 - w_i + eta, so the restricted diagram of the lifted
 * sites on a planar triangle mesh at z = 0 (vd_set_domain with 3 vertices per
 * simplex) is the power diagram on that mesh.  xy: device float [n*2]; w: device
 * float [n]; copied.  The power weights the diagram realises are exactly
 * -h_i^2 + eta with h_i the float lift, i.e. w_i up to the rounding of h_i.  Cells
 * may be empty (dominated sites): measure 0, centroid = the lifted site.
 * VD_ERR_ARG for a weight that is not finite. */
int vd_create_power2d(vd_ctx** out, const float* xy, const float* w, int64_t n);

/* Power diagram in 3D or on a surface (the paper's extension to power diagrams
 * by lifting, Sec. 6.3): the power distance of x to site i is
 * |x - v_i|^2 - w_i.  Every site is lifted to (v_i, h_i) one dimension up,
 * h_i = sqrt(eta - w_i) with eta = max_i w_i (found on the device); the domain
 * lies at height 0, where |x - (v_i, h_i)|^2 = |x - v_i|^2 - w_i + eta, so the
 * clipped (restricted) Voronoi diagram of the lifted sites is the power
 * diagram.  Alg. 3 runs on the lifted sites: corners are tested against the
 * lifted sites, the virtual edge goes from (v_i, h_i) to the corner, and the
 * bisector planes are the power bisectors |w|^2 + h_j^2 - h_i^2 = 2 w.x
 * (w = v_j - v_i; the float64 sign tests use the same h).  The weights realised
 * are exactly eta - h_i^2 for the float h_i, i.e. w_i up to the rounding of h_i.
 * w: device float [n], copied; NULL returns to the Voronoi diagram.  Power cells
 * may be empty (a dominated site) or not contain their site.  The learned form's
 * nearest lists, the split and the thread-per-pair mapping are not used while
 * weights are set (the plain search, one warp per pair, per-simplex pieces).
 * FP32 contexts with dim = 3 (tetrahedra, surface triangles or vd_set_box);
 * planar diagrams use vd_create_power2d.  VD_ERR_ARG for another context or a
 * weight that is not finite.  Synchronises the context stream. */
int vd_set_weights(vd_ctx* ctx, const float* w);

/* Set the domain M = {T_a} (Sec. 2.1).  verts: device pointer, nv*dim elements of
 * the context dtype; simplices: device pointer, m*simplex_verts int32 vertex
 * indices (3: triangles, 4: tetrahedra).  Copied and validated (indices in
 * range, non-zero measure, faces shared by at most two simplices); builds the
 * simplex adjacency that initialises the negative face flags (Sec. 2.2) and the
 * simplex locator used to seed pairs.  Synchronises the context stream. */
int vd_set_domain(vd_ctx* ctx, const void* verts, int64_t nv, const int32_t* simplices, int64_t m,
                  int simplex_verts);

/* Set the domain to the axis-aligned box [lo, hi] (host pointers, 3 doubles
 * each, rounded to float) for a 3D FP32 context: the convex-domain form of
 * Sec. 4.2, where every site's cell starts as the whole box (8 corners, 6 faces)
 * and is clipped by Alg. 3 -- one piece per site, no tetrahedra and no flood.
 * Results as for the box split into tetrahedra (measure, centroid, neighbours);
 * the pieces are (0, i) per site, box faces flagged INT32_MIN.  Clip kernel: one
 * warp per pair.  VD_ERR_ARG for another dim/dtype or an empty box.
 * Synchronises the context stream. */
int vd_set_box(vd_ctx* ctx, const double* lo, const double* hi);

/* Replace the options (NULL restores the defaults).  Service call: the paper
 * fixes none of these knobs (capacities, limits and the batching / learned
 * choices are this library's).  Drops the autotuned choice and any captured
 * Lloyd graph. */
int vd_set_options(vd_ctx* ctx, const vd_options* opt);

/* Enqueue all later work on this cudaStream_t (NULL: legacy default stream).
 * Service call (the paper has no counterpart). */
int vd_set_stream(vd_ctx* ctx, void* cuda_stream);

/* Replace the site coordinates V (Sec. 2.1; same n and dim; device pointer,
 * n*dim elements of the context dtype, row-major, copied on the context
 * stream).  Also the site update of one Lloyd step (Sec. 6.4). */
int vd_update_sites(vd_ctx* ctx, const void* sites);

/* Host-pointer variant of vd_update_sites (pinned or pageable host memory,
 * n*dim elements; copied on the context stream through a staging buffer
 * owned by the context). */
int vd_update_sites_host(vd_ctx* ctx, const void* sites_host);

/* Compute the clipped / restricted diagram of the current sites (Alg. 3 for
 * every (simplex, site) pair, pairs discovered by the flag propagation of
 * Alg. 4 / Alg. 5, improved search of Sec. 5.1, grid search of Sec. 5.2).
 * Synchronises the stream once at the end to read the status and counts.
 * out may be NULL.  Returns the first device-side error, if any.  Equivalent
 * to vd_compute_async followed by vd_get_status and vd_get_result. */
int vd_compute(vd_ctx* ctx, vd_result* out);

/* Enqueue the work of vd_compute on the context stream and return without
 * waiting for it or reading anything back: no host synchronisation, no
 * allocation, no event record, so the call can be captured into a caller's
 * CUDA graph (stream capture on the context stream) and replayed.  Results
 * land in the context's buffers when the stream reaches the end of the work;
 * vd_get_status then reads the device status word and the counts.  Returns
 * VD_ERR_STATE before vd_set_domain, when the learned form wants a network
 * that is not set, or when mapping = 0 (autotuned) has no cached choice yet:
 * run vd_autotune (or one vd_compute) first, outside any capture. */
int vd_compute_async(vd_ctx* ctx);

/* Wait for the context stream and read back the device status word of the
 * last vd_compute_async (or vd_compute / vd_lloyd) with its counts: *status
 * (host int) receives VD_OK or the first device-side error code.  The call
 * itself returns VD_OK, VD_ERR_STATE when nothing was enqueued, or
 * VD_ERR_CUDA.  After it, vd_get_result, vd_get_pieces and
 * vd_copy_result_host see that computation. */
int vd_get_status(vd_ctx* ctx, int* status);

/* Fill out (as vd_compute does) from the computation that vd_get_status last
 * read back: device pointers owned by the context, counts, stats, status.
 * No synchronisation.  VD_ERR_STATE before any status was read. */
int vd_get_result(vd_ctx* ctx, vd_result* out);

/* Partition of one diagram across ranks (one context per rank, each on its
 * own GPU).  The pieces P_{a,i} are independent (Sec. 4: "no inter-thread
 * synchronisation"), so every rank computes the pieces of the sites it owns:
 * owner (device int32[n], copied) gives the rank of each site and rank is this
 * context's.  Seeding pushes only owned sites' pairs (each rank seeds its own,
 * Alg. 4 / Alg. 5; the split's boundary pass runs whole on every rank); a pair
 * (T, j) that the flood finds for a site j of another rank (a positive flag,
 * Alg. 4) goes once to this rank's outbox instead of its queue.  After
 * vd_compute the caller sends each outbox key to the owner of its site and
 * hands what it receives to vd_resume, until no rank has outgoing pairs; the
 * per-site results of a rank are then final for its sites (measure 0 and no
 * neighbours elsewhere).  owner NULL: one rank owns all sites (the default).
 * Errors: VD_ERR_ARG (rank < 0), VD_ERR_STATE (before vd_set_domain or while a
 * vd_compute_async is pending), VD_ERR_OOM.  vd_lloyd refuses a partitioned
 * context (an iteration needs the exchange of pairs and of the moved sites). */
int vd_set_partition(vd_ctx* ctx, const int32_t* owner, int rank);

/* The pairs for other ranks found by the last vd_compute / vd_resume: *keys
 * (device, owned by the context, valid until the next compute or resume) holds
 * *count keys (simplex << 32) | site, each at most once per computation.
 * *count is 0 without a partition.  VD_ERR_STATE before a computation. */
int vd_get_outbox(vd_ctx* ctx, const uint64_t** keys, int64_t* count);

/* Continue the last computation with pairs received from other ranks: keys
 * (device uint64[count], (simplex << 32) | site, caller-owned, read before the
 * call returns) enter the pair set; the new ones are clipped and flooded like
 * seeds, the outbox restarts with what they lead to, and the per-site
 * reduction (Sec. 2.1) is redone over all pieces.  *added (may be NULL)
 * receives the number of new pairs; out (may be NULL) is filled as by
 * vd_compute.  Synchronises.  Errors: VD_ERR_ARG (a key outside the domain or
 * the sites, also as the device status), VD_ERR_STATE (no successful
 * computation to continue), the device-side codes of vd_compute. */
int vd_resume(vd_ctx* ctx, const uint64_t* keys, int64_t count, int64_t* added, vd_result* out);

/* One Lloyd update (Sec. 6.4) from the last successful computation: every site
 * whose cell has positive measure moves to its centroid (others stay).  In a
 * partitioned context only the rank's own sites move (the others have no
 * pieces here); the caller then assembles the moved sites from their owners
 * and hands them to vd_update_sites.  Synchronises.  VD_ERR_STATE without a
 * successful computation since the last update. */
int vd_lloyd_step(vd_ctx* ctx);

/* Autotune the clip kernel now on the current sites (batching, Sec. 4.3: one
 * persistent launch drains the pair queue): runs vd_compute's work once per
 * candidate -- one warp or one thread per pair (3D FP32 tetrahedra without the
 * split), queue chunk 1, 2, 4, 8 or 16 (or vd_options.chunk alone when set; the
 * thread mapping's chunks beyond 1 only when its chunk 1 beat every warp one) --
 * times the clip phase with CUDA events and caches the fastest for mapping 0.
 * In the learned form with vd_options.nearest = 0 it first compares lists of
 * the 32 and of the 64 nearest (warp per pair, chunk 1) on the time of the
 * list pass, the seeding and the clip, and keeps the faster for the mapping
 * candidates.  mapping, chunk (may be NULL) receive the choice; times_ms (host
 * float[12], may be NULL) the candidates' clip times in the order (warp,1),
 * (warp,2), (warp,4), (warp,8), (warp,16), (thread,1), ..., (thread,16), then
 * the list comparison (32, 64), -1 for those not run.  All
 * candidates compute the same diagram; the result of the last one is left as
 * the current result.  Synchronises the context stream. */
int vd_autotune(vd_ctx* ctx, int* mapping, int* chunk, float* times_ms);

/* Copy the per-site measure [n], centroid [n*3] (context dtype) and, when
 * nbr_off is not NULL, the CSR (nbr_off [n+1] int64, nbr_idx [nnz] int32) of the
 * last vd_compute to host memory.  nbr_idx must hold the nnz of that result.
 * The output of Sec. 2.1 (measure and centroid of Omega_i within M) and the
 * neighbours given by the positive flags of Sec. 2.2.  Synchronises the
 * context stream; VD_ERR_STATE before the first computation. */
int vd_copy_result_host(vd_ctx* ctx, void* measure, void* centroid, int64_t* nbr_off, int32_t* nbr_idx);

/* Lloyd's method (Sec. 6.4, density 1): iters times { compute the diagram;
 * v_i <- centroid_i (sites with empty cells stay) }.  use_graph = 1 captures
 * min(iters, 10) whole iterations in one CUDA graph (cached while that count,
 * the options and the domain stay the same) and replays it, the remaining
 * iters % 10 running as ordinary launches on the same stream; the host reads
 * the status once at the end.  The last iteration's diagram is not recomputed
 * for the final sites. */
int vd_lloyd(vd_ctx* ctx, int iters, int use_graph);

/* Copy the current site coordinates V (Sec. 2.1; after vd_lloyd, the relaxed
 * sites of Sec. 6.4) to a device buffer: n*3 elements of the context dtype
 * (z = 0 in 2D), enqueued on the context stream. */
int vd_get_sites(vd_ctx* ctx, void* sites_out);

/* Per-piece output of the last vd_compute: every processed pair (T_a, v_i)
 * with its piece P_{a,i} = T_a intersected with Omega_i (Sec. 2.1) and the face
 * flags of the piece (Sec. 2.2: j >= 0 for the face on bisector B_ij, -(b+1) for
 * the face shared with simplex b, INT32_MIN for the mesh boundary), as device
 * arrays owned by the context (allocated on first use, valid until the next
 * compute).  Synchronises the context stream; VD_ERR_STATE before the first
 * computation. */
int vd_get_pieces(vd_ctx* ctx, vd_pieces* out);

/* Learned proposal (ranking of likely bisector neighbours; the paper has no
 * counterpart): candidate site indices per site, device int32 [n*k], -1 =
 * unused slot, k <= 32; copied.  They only order the bisector search of
 * Sec. 3.2; every clip is still decided by the exact test, so the output does
 * not change.  k = 0 clears them. */
int vd_set_candidates(vd_ctx* ctx, const int32_t* cand, int k);

/* Piece export into caller-owned device buffers, with no device allocation.
 *
 * The paper has no counterpart: this is a service entry point.  vd_get_pieces
 * allocates its export buffers on first use and its prefix sum uses scratch
 * allocated with the context.  Some callers must not call cudaMalloc at the
 * point where they read the pieces: a host framework whose caching allocator
 * or fixed arena owns all device memory, or a steady-state loop where a
 * cudaMalloc / cudaFree would synchronise the device.  This variant writes
 * into buffers the caller already owns and keeps the prefix-sum scratch in a
 * fixed array inside the library: 40,960 int64 (320 KiB) per device that
 * loads the library, held until the process exits.
 *
 * simplex, site: int32 [pieces_capacity]; flag_off: int64 [pieces_capacity+1];
 * flags: int32 [flags_capacity]; measure (context dtype [pieces_capacity]) and
 * moment ([3*pieces_capacity]) may be NULL.  The number of pieces is
 * vd_result.stats[VD_STAT_PAIRS] of the last vd_compute; *n_pieces and
 * *n_flags receive the sizes written.  Layout and meaning as in vd_pieces.
 * Returns VD_ERR_CAPACITY when the pieces exceed pieces_capacity or the limit
 * of 67,108,863, or the flags exceed flags_capacity (nothing is written past a
 * capacity); VD_ERR_STATE before the first vd_compute.  The first call on a
 * device looks up the scratch array's device address (once per device); make
 * that first call before any stream capture.  Every call on a device shares
 * the same scratch array, which keeps the previous call's contents (the prefix
 * sum overwrites all of it before reading), so calls that overlap on the GPU
 * race: run them on one stream or one after another.  Synchronises the
 * context stream. */
int vd_get_pieces_noalloc(vd_ctx* ctx, int32_t* simplex, int32_t* site, int64_t* flag_off, int32_t* flags,
                          void* measure, void* moment, int64_t pieces_capacity, int64_t flags_capacity,
                          int64_t* n_pieces, int64_t* n_flags);

/* ---------------------------------------------------------------------------
 * Learned proposal network.  The paper has no counterpart: the paper's search
 * (Sec. 3.2, Sec. 5.1) finds every bisector by point-in-cell tests alone.  The
 * learned form orders its candidate tests by a ranking of each site's 32 nearest
 * sites; the exact tests still decide every clip, so the diagram is the same for
 * any ranking, trained or not.
 *
 * Network: input = the offsets (v_k - v_i) / d_1 of the 32 nearest sites v_k of
 * v_i in ascending distance, d_1 = distance of the nearest (96 values, bf16,
 * row-major [slot][xyz]; z = 0 in 2D); layers 96 -> 64 -> 64 -> 32 with ReLU;
 * output = one logit per slot.  Parameters: VD_MLP_NPARAM FP32 values, flat:
 * W1 [96][64], b1 [64], W2 [64][64], b2 [64], W3 [64][32], b3 [32] (weights
 * row-major, input index first).  Products use the bf16-rounded weights and
 * activations with FP32 accumulation; biases and logits are FP32.
 * Loss: mean over rows and 32 slots of the binary cross-entropy of the logit
 * against the label bit (1: the slot's site is a bisector neighbour).
 * Every call runs on the context stream; pointers are device pointers.
 * ------------------------------------------------------------------------- */
enum { VD_MLP_NPARAM = 12448, VD_MLP_NIN = 96, VD_MLP_NOUT = 32 };

/* Initialise the network: weights uniform in +-sqrt(6 / fan_in) from a 64-bit
 * hash of (seed, index), biases 0, Adam moments 0, step 0. */
int vd_mlp_init(vd_ctx* ctx, uint64_t seed);

/* Set the state: params [VD_MLP_NPARAM] (required); adam_m, adam_v (NULL: 0);
 * step = Adam steps taken (for bias correction on resume).  Copied. */
int vd_mlp_set_state(vd_ctx* ctx, const float* params, const float* adam_m, const float* adam_v, int64_t step);

/* Read the state into caller buffers (each may be NULL; step is a host
 * pointer).  VD_ERR_STATE before vd_mlp_init / vd_mlp_set_state.
 * Synchronises the context stream. */
int vd_mlp_get_state(vd_ctx* ctx, float* params, float* adam_m, float* adam_v, int64_t* step);

/* Save the network state (parameters, Adam moments and step: everything a
 * resumed training needs) to a file: the 8 bytes "VDMLP01\0", int64
 * VD_MLP_NPARAM, int64 step, then params, adam_m, adam_v as little-endian
 * FP32 [VD_MLP_NPARAM] each, then the 64-bit FNV-1a hash of the preceding
 * bytes.  VD_ERR_STATE without a network, VD_ERR_IO when the file cannot be
 * written.  Synchronises the context stream. */
int vd_model_save(vd_ctx* ctx, const char* path);

/* Load a file written by vd_model_save into the context's network (as
 * vd_mlp_set_state with all three arrays and the step); the learned form with
 * proposal = VD_PROPOSAL_MLP then ranks with it.  VD_ERR_IO when the file is
 * missing, short, not of this format or fails its hash (the state is then
 * left unchanged).  Synchronises the context stream. */
int vd_model_load(vd_ctx* ctx, const char* path);

/* Training data from the last vd_compute (the sites must not have changed
 * since): x = the network input of every site (bf16 [n*96], may be NULL) and
 * labels = bit s set when slot s of the site's 32-NN list is in its neighbour
 * CSR (uint32 [n], may be NULL).  Builds the 32-NN lists when that compute did
 * not.  VD_ERR_STATE without a current vd_compute. */
int vd_mlp_features(vd_ctx* ctx, void* x, uint32_t* labels);

/* Gradient of the mean loss over `rows` rows (x bf16 [rows*96], labels [rows])
 * at the current parameters, written to grads [VD_MLP_NPARAM] (FP32, device);
 * the mean loss to *loss (device float).  Parameters are not changed. */
int vd_mlp_grad(vd_ctx* ctx, const void* x, const uint32_t* labels, int64_t rows, float* grads, float* loss);

/* Logits [rows*32] (FP32, device) of rows x (bf16 [rows*96]). */
int vd_mlp_forward(vd_ctx* ctx, const void* x, int64_t rows, float* logits);

/* Candidate masks of the last vd_compute of the learned form (uint32 [n],
 * device): bit s set when slot s of the site's 32-NN list is a candidate of the
 * ranking in use.  VD_ERR_STATE when that compute was not of the learned form
 * or the sites changed since. */
int vd_get_candidate_masks(vd_ctx* ctx, uint32_t* masks);

/* Train with Adam (beta1 0.9, beta2 0.999, eps 1e-8, learning rate lr) for
 * `epochs` passes over `rows` rows (at most 2^31 - 1) in batches of `batch`
 * (at most 2^22); each pass visits the
 * rows in the order of an affine permutation drawn from (seed, epoch).  The
 * Adam moments and step continue from the current state.  epoch_loss
 * (host, may be NULL) receives the mean training loss of each epoch.  The
 * gradients are summed with FP32 atomics, so the low bits of the trained
 * weights depend on the summation order.  Synchronises the context stream. */
int vd_mlp_train(vd_ctx* ctx, const void* x, const uint32_t* labels, int64_t rows, int batch, int epochs, float lr,
                 uint64_t seed, float* epoch_loss);

/* Release everything owned by the context (NULL is allowed).  Synchronises
 * the context stream first.  Service call (the paper has no counterpart). */
void vd_destroy(vd_ctx* ctx);

/* Static string naming an error code (service call). */
const char* vd_strerror(int code);

#ifdef __cplusplus
}
#endif

#endif /* VD_H_ */
