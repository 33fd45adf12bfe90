/*
 * vt.h -- C ABI of the GB300 Voronoi tessellation library (libvt.so).
 *
 * The library computes 3D Voronoi cells one cell at a time, the method of the
 * votess paper (Summary): the generators are sorted into a uniform grid, a
 * k-nearest-neighbour search runs per generator, and each cell is obtained by
 * clipping the bounding box with the perpendicular bisector planes of the
 * generator and its neighbours, nearest first, until the "security radius"
 * condition proves that no farther generator can cut it. Cells that fail the
 * condition are re-run on the device with k doubled (where the paper falls
 * back to the CPU); cells that still fail at k_max are finished by clipping
 * with every generator that can still cut them (all generators within twice
 * the cell's radius), also on the device.
 *
 * Conventions (every entry point):
 *  - Every array argument is a DEVICE pointer unless its comment says host.
 *    "Device" means memory device code can use at that address: device or
 *    managed allocations, or pinned host memory (cudaHostAlloc /
 *    cudaHostRegister, mapped at the same address under unified addressing),
 *    so outputs can be written straight into host memory. Every entry point
 *    that launches work checks its buffers first (cudaPointerGetAttributes,
 *    skipped while the stream is being captured) and returns
 *    VT_ERR_INVALID_ARG for any other memory (pageable host memory) without
 *    launching a kernel.
 *    Buffers are owned by the caller; the library never allocates, frees or
 *    keeps a pointer after a call returns.
 *  - Scratch memory is a caller-allocated device workspace of at least
 *    vt_workspace_size() bytes, passed as (ws, ws_bytes). Its contents need not
 *    be initialised and are clobbered.
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *    stream). Stage calls (vt_grid_build, vt_knn, vt_clip_cells, vt_emit) only
 *    enqueue work and return; vt_tessellate synchronises the stream once per
 *    re-queue pass to read a 192-byte status block (documented below).
 *  - Work runs on the calling thread's current CUDA device; every device
 *    buffer and the stream must belong to it (the library never switches
 *    devices: make the buffers' device current first).
 *  - Points are float32 (x, y, z) triples inside the half-open box
 *    [box_lo, box_hi), pairwise distinct.
 *  - Return value: vt_status. On failure vt_last_error() (per host thread)
 *    describes the problem. A CUDA launch error is VT_ERR_CUDA.
 *  - "sorted index" = position of a generator after the grid sort;
 *    "original index" = its row in the caller's input.
 */
#ifndef VT_H
#define VT_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define VT_API __attribute__((visibility("default")))
#else
#define VT_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

/* ------------------------------------------------------------------ */
/* status, parameters, outputs                                         */
/* ------------------------------------------------------------------ */

typedef enum {
    VT_OK = 0,
    VT_ERR_INVALID_ARG = 1,      /* bad argument, or a point that is not finite or not inside the box */
    VT_ERR_CUDA = 2,             /* a CUDA call failed (see vt_last_error) */
    VT_ERR_CAPACITY = 3,         /* an output buffer is too small: vt_cells_out.needed_* hold the sizes */
    VT_ERR_UNVALIDATED = 4,      /* some cells could not be validated (count in vt_stats.unvalidated, ids
                                    from vt_unvalidated_cells; their vol / cen / m2 are NaN) */
    VT_ERR_DUPLICATE_POINTS = 5, /* two generators coincide (a neighbour at distance 0) */
    VT_ERR_TIMEOUT = 6,          /* a bounded device wait gave up */
    VT_ERR_WORKSPACE = 7,        /* ws_bytes smaller than vt_workspace_size() */
    VT_ERR_INTERNAL = 8          /* a bounds check of a debug build (VT_CHECKS) failed */
} vt_status;

enum { VT_FP64 = 0, VT_FP32_RECHECK = 1 };          /* vt_params.precision */
enum { VT_INDEX_ORIGINAL = 0, VT_INDEX_SORTED = 1 }; /* vt_params.index_space */

/* vt_params.emit bitmask */
enum {
    VT_EMIT_NBR = 1,   /* neighbour CSR (nbr_off, nbr) */
    VT_EMIT_VOL = 2,   /* cell volume */
    VT_EMIT_CEN = 4,   /* cell centroid */
    VT_EMIT_M2 = 8,    /* second moment: integral of |x - p_i|^2 over the cell */
    VT_EMIT_GEOM = 16  /* vertices and faces (vtx_off/vtx, face_off/face_nbr/face_vtx_off/face_vtx) */
};

typedef struct vt_params {
    int k0;                 /* initial k of the neighbour lists (default 16) */
    int k_max;              /* largest k of the doubling passes, <= 256 (default 32; the exhaustive
                               pass that follows finishes every remaining cell exactly) */
    float grid_density;     /* target generators per grid cell rho; G = ceil(cbrt(n / rho)) (default 2) */
    int grid_res;           /* G override per axis (0 = derive from grid_density) */
    int threads_per_cell;   /* lanes cooperating on one cell: 8, 16 or 32 (0 = default 32) */
    int precision;          /* VT_FP64 or VT_FP32_RECHECK */
    int emit;               /* VT_EMIT_* bitmask */
    int index_space;        /* VT_INDEX_ORIGINAL (default) or VT_INDEX_SORTED */
    float box_lo[3];        /* domain box [box_lo, box_hi); periodic with VT_FLAG_PERIODIC */
    float box_hi[3];
    int flags;              /* VT_FLAG_* bitmask (default 0) */
} vt_params;

/* vt_params.flags */
enum {
    VT_FLAG_STAGE_TIMES = 1, /* time every kernel group with CUDA events on the call's stream
                               (vt_stats.ms_*); costs one event pair per launch group */
    VT_FLAG_NO_SYNC = 2,     /* fixed schedule: passes k0, 2k0, ... <= k_max, then the exhaustive
                               pass, each launched over the worst-case cell count and reading its
                               true count from device memory. The call never waits on the device,
                               so it can be captured in a CUDA graph; errors and output sizes are
                               read afterwards with vt_read_stats. Outputs that do not fit the
                               caller's capacities are not written (VT_ERR_CAPACITY there). The
                               neighbour-list buffer grows to n * k_max entries. */
    VT_FLAG_PERIODIC = 4,    /* periodic box: every generator also stands at all its images
                               p + t L (L = box_hi - box_lo, t integer). The cell of p_i starts
                               as the cube [p_i - L/2, p_i + L/2] (the bisectors of p_i's own
                               images at +-L_a) and is cut by the images of the other
                               generators. Vertices and centroids are not wrapped: they lie
                               around p_i and may leave the box. A face's neighbour id is the
                               generator whose image it faces, so an id may repeat when two
                               images of one generator are faces, and the cube's own faces
                               (only in sets of a handful of points) carry the cell's own id.
                               Requires |L|^2 <= 4 min_a L_a^2 (images shifted by more than two
                               periods cannot then cut) and fewer than 2^24 points in the call
                               (a batch counts all its sets); otherwise VT_ERR_INVALID_ARG. */
    VT_FLAG_FUSED = 8        /* kNN and clipping in one kernel: no neighbour lists. Every cell
                               starts from the box and walks the grid shells around its generator,
                               clipping the candidates of each batch of grid cells nearest first,
                               until the security radius (no unvisited generator within 2R)
                               concludes it. The n x k list buffer and the saved polyhedra are
                               not allocated (vt_workspace_size is smaller); k0 and k_max are
                               still validated and size only the robust variant's lists. Cells
                               and outputs are those of the list schedules. Combines with
                               VT_FLAG_NO_SYNC and VT_FLAG_PERIODIC. */
};

/* Fills *p with the defaults above, unit box, FP32_RECHECK, emit NBR|VOL|CEN. */
VT_API void vt_params_default(vt_params* p);

/* Outputs of a tessellation. Index space per vt_params.index_space: cell i is
 * original generator i (ORIGINAL) or sorted generator i (SORTED), and
 * neighbour / face ids use the same space. Any pointer whose VT_EMIT bit is
 * off may be NULL. Variable-length arrays are CSR: cell i owns entries
 * [off[i], off[i+1]). Every face list is counter-clockwise seen from outside
 * the cell. Wall faces carry ids -1..-6 (x=lo, x=hi, y=lo, y=hi, z=lo, z=hi).
 * A generator is a neighbour when its face's area exceeds a small fraction of
 * V^(2/3) (1e-12 in the FP64 form, 1e-11 in the FP32 form): faces below it
 * (near-degenerate vertex configurations) stay in the geometry, so a cell's
 * faces are its neighbours, its walls and those tiny faces. Because the
 * threshold follows each cell's own volume, such a face can make a pair a
 * neighbour on one side only. */
typedef struct vt_cells_out {
    double* vol;            /* [n] */
    double* cen;            /* [n*3] */
    double* m2;             /* [n] */
    int64_t* nbr_off;       /* [n+1] */
    int32_t* nbr;           /* [nbr_cap] neighbour ids, ascending per cell */
    int64_t nbr_cap;
    int64_t* vtx_off;       /* [n+1] */
    double* vtx;            /* [vtx_cap*3] vertex coordinates (global frame) */
    int64_t vtx_cap;
    int64_t* face_off;      /* [n+1] faces of cell i */
    int32_t* face_nbr;      /* [face_cap] neighbour id or wall id of each face */
    int64_t* face_vtx_off;  /* [face_cap+1] CSR over face_vtx, global */
    int32_t* face_vtx;      /* [face_vtx_cap] vertex index within the cell's vertex list */
    int64_t face_cap;
    int64_t face_vtx_cap;
    int32_t* perm;          /* [n] optional: sorted index -> original index */
    /* filled by vt_tessellate / vt_emit (host memory, inside this struct) */
    int64_t needed_nbr, needed_vtx, needed_face, needed_face_vtx;
} vt_cells_out;

/* Grid of one point set of a batch, made on the host by vt_batch_plan and
 * copied to device memory by the caller before vt_tessellate_batch. */
typedef struct vt_set_desc {
    int G;                  /* grid cells per axis of this set */
    float lo[3], hi[3];     /* the set's box */
    float scale[3];         /* float32(G) / (hi - lo) */
    double cw[3];           /* cell width */
    double margin;          /* rounding margin of the shell-walk stop rule */
    int64_t cell_base;      /* first global grid cell of this set */
    int64_t pt_begin;       /* first point of this set in the concatenated input */
    int64_t npts;           /* points in this set */
    int32_t periodic;       /* 1: the set's box is periodic (VT_FLAG_PERIODIC) */
    int32_t reserved;
} vt_set_desc;

#define VT_MAX_PASSES 16

typedef struct vt_stats {
    int passes;                          /* clip passes run (1 + doubling passes + exhaustive) */
    int k_of_pass[VT_MAX_PASSES];        /* k of each pass (0 = exhaustive pass) */
    int64_t cells_of_pass[VT_MAX_PASSES];/* cells entering each pass */
    int64_t exhaustive_cells;            /* cells finished by the exhaustive pass */
    int64_t capacity_retries;            /* cells re-run because a polyhedron outgrew its slots */
    int64_t precision_retries;           /* FP32 cells re-run in FP64 after an inconsistency */
    int64_t fp64_rechecks;               /* FP32 sign / radius tests re-decided in FP64 */
    int64_t unvalidated;                 /* cells left without a validated cell */
    int grid_res;                        /* G used */
    int launches;                        /* kernels launched by the call */
    int clip_launches;                   /* clipper launches among them */
    int knn_launches;                    /* kNN launches among them */
    double ms_grid, ms_knn, ms_clip, ms_emit; /* device time per stage (VT_FLAG_STAGE_TIMES), else 0 */
    double ms_clip_pass[VT_MAX_PASSES];  /* clipper device time of each pass (VT_FLAG_STAGE_TIMES) */
    int64_t clip_events[5];              /* diagnostic counts of clip steps that: removed every vertex,
                                            hit the plane cap, hit the vertex cap, found an inconsistent
                                            ring, or placed a vertex by edge interpolation */
    double ms_knn_lists;                 /* the k-nearest-neighbour kernels' part of ms_knn (the rest is
                                            the range lists of the last pass) */
    int64_t knn_candidates;              /* candidates the k-nearest-neighbour kernels examined (one
                                            squared distance each) */
    int64_t knn_queries;                 /* queries they answered */
    int64_t walk_cells;                  /* walks over the grid shells within 2R of a cell in the last
                                            pass (range lists and the exhaustive walk; a cell whose
                                            range list overflows walks twice) */
    int64_t walk_candidates;             /* generators those walks examined. Most cells walking with
                                            about n each means near-degenerate input (coplanar or
                                            collinear generators: every cell reaches the walls), whose
                                            cost grows as n^2 */
} vt_stats;

/* ------------------------------------------------------------------ */
/* sizing                                                              */
/* ------------------------------------------------------------------ */

/* Grid resolution G per axis that vt_tessellate uses for n generators (the
 * uniform grid of the paper's Summary; its size is a reading): p->grid_res
 * when positive, else G = ceil(cbrt(n / p->grid_density)), at most
 * ceil(cbrt(8 n)) + 1 and 1024, at least 1 (n <= 0 gives 1). Returns G, or
 * -1 when p is invalid (the reason in vt_last_error). Host-only. */
VT_API int vt_grid_resolution(const vt_params* p, int64_t n);

/* Bytes of device workspace needed by vt_tessellate (and by any stage call
 * with the same p and n). Writes *bytes; returns VT_ERR_INVALID_ARG for a bad
 * p or n < 0. Host-only; no CUDA call. */
VT_API int vt_workspace_size(const vt_params* p, int64_t n, size_t* bytes);

/* ------------------------------------------------------------------ */
/* stage 1: grid counting sort (paper, Summary)                        */
/* ------------------------------------------------------------------ */

/* Sorts the n points pts[n*3] into a G^3 uniform grid over the box.
 * cell id = (ix*G + iy)*G + iz with ix = min(G-1, floor(fl(fl(x - lo) * s)))
 * and s = float32(G) / (hi - lo) in float32 (every operation rounded
 * separately). The sort is stable: generators in a grid cell keep input order.
 * Outputs: sorted[n*4] = (x, y, z, original index as int32 bits), perm[n]
 * (sorted index -> original index), cell_off[G^3+1] (first sorted index of
 * each grid cell; cell_off[G^3] = n). Checks that every point is finite and
 * inside the box; a violation sets a device flag that vt_tessellate reports
 * as VT_ERR_INVALID_ARG (stage callers read it with vt_read_status). */
VT_API int vt_grid_build(const float* pts, int64_t n, const vt_params* p, int G,
                  float* sorted, int32_t* perm, int32_t* cell_off,
                  void* ws, size_t ws_bytes, void* stream);

/* The grid sort of vt_grid_build for callers that cannot allocate device
 * memory: a host program whose device memory is handed out up front by an
 * arena or pool it does not control (a cudaMalloc there would fail or
 * fragment the pool), or an embedding that must keep its device footprint
 * fixed after start-up. Its scratch is a device array inside this library,
 * 17 MiB on every GPU that loads the library, held until the process exits;
 * inputs and outputs are still the caller's buffers (same layout as
 * vt_grid_build; no workspace). pts, sorted, perm and cell_off must be memory
 * device code can use; any other memory (pageable host) is VT_ERR_INVALID_ARG
 * before anything is launched.
 * Limits: n <= 1,048,576 points and G^3 <= 1,048,576 grid cells; larger
 * requests return VT_ERR_INVALID_ARG without launching anything.
 * Every call looks up the array's device address on the current device (no
 * address is kept between calls, so a reset device is handled). Every call
 * reuses the same array and clears what must start at zero; calls whose work
 * overlaps on a GPU (other streams, other host threads) race on it, so
 * serialise them. Blocking: synchronises `stream` and returns after the sort
 * has finished, so it must not be called while `stream` is being captured
 * (VT_ERR_INVALID_ARG). A point that is not finite or outside the box gives
 * VT_ERR_INVALID_ARG. The paper has no counterpart: this is a deployment
 * variant of the grid-sort stage. */
VT_API int vt_grid_build_static(const float* pts, int64_t n, const vt_params* p, int G,
                                float* sorted, int32_t* perm, int32_t* cell_off, void* stream);

/* ------------------------------------------------------------------ */
/* stage 2: k nearest neighbours (paper, Summary)                      */
/* ------------------------------------------------------------------ */

/* k nearest generators of each query (self excluded), nearest first, by a
 * walk over Chebyshev shells of grid cells around the query's cell.
 * queries[nq]: sorted indices to search for (NULL = all n, in order).
 * nbr[nq*k]: sorted indices of the neighbours; d2[nq*k]: squared distances
 * (double for VT_FP64, float for VT_FP32_RECHECK; may be NULL).
 * Order: (d2, original index) ascending. VT_FP64 computes
 * d2 = ((dx*dx + dy*dy) + dz*dz) in double with dx = double(x_j) - double(x_i)
 * and no fused multiply-add, so lists are exact and reproducible;
 * VT_FP32_RECHECK evaluates the same expression in float32.
 * 1 <= k <= 256. If fewer than k other generators exist, the remaining
 * slots get -1 and +inf.
 * VT_FLAG_PERIODIC: the candidates are the images p_j + t L, t in
 * [-2, 2]^3, of every generator but the query's own; an entry packs the
 * sorted index j (bits 0..23) with the image code (tx+2)*25 + (ty+2)*5 +
 * (tz+2) (bits 24..30); dx = (double(x_j) - double(x_i)) + tx * L_x in
 * double; ties go by (original index, code). A list ends early (-1) when
 * every image closer than |L| is in it (nothing farther can cut a cell). */
VT_API int vt_knn(const float* sorted, const int32_t* cell_off, int G, int64_t n,
           const int32_t* queries, int64_t nq, int k, const vt_params* p,
           int32_t* nbr, void* d2, void* ws, size_t ws_bytes, void* stream);

/* ------------------------------------------------------------------ */
/* stage 3: per-cell bisector clipping (paper, Summary)                */
/* ------------------------------------------------------------------ */

/* Clips the box around each query generator by the bisectors of its k
 * listed neighbours, nearest first, checking the security radius before each
 * clip: the cell is final when 4 R^2 <= d2 of the next listed neighbour
 * (R = largest vertex distance from the generator), or, after all k, when
 * 4 R^2 <= d2 of the k-th; when the list holds every other generator the cell
 * is final by construction. k = 0 selects the exhaustive mode (no list:
 * every generator closer than 2R, found by a grid walk).
 * Writes vol/cen/m2 of finished cells into `out` (at the cell's index in the
 * chosen index space) and the cell's faces and vertices into the workspace
 * for vt_emit. Cells that are not validated are appended to failed[] (sorted
 * indices) and counted in *n_failed (a device int32 the caller zeroes).
 * The workspace must be the one that vt_grid_build / vt_tessellate use. */
VT_API int vt_clip_cells(const float* sorted, const int32_t* cell_off, int G, int64_t n,
                  const int32_t* queries, int64_t nq, const int32_t* nbr, const void* d2, int k,
                  const vt_params* p, vt_cells_out* out, int32_t* failed, int32_t* n_failed,
                  void* ws, size_t ws_bytes, void* stream);

/* Writes the variable-length outputs (neighbour CSR, geometry) of the last
 * vt_tessellate call on this workspace into `out`. Blocking: reads the totals
 * back to fill out->needed_*; returns VT_ERR_CAPACITY when a *_cap is too
 * small (nothing written). */
VT_API int vt_emit(int64_t n, const vt_params* p, vt_cells_out* out, void* ws, size_t ws_bytes, void* stream);

/* ------------------------------------------------------------------ */
/* whole path                                                          */
/* ------------------------------------------------------------------ */

/* Tessellates the n generators pts[n*3] (device) in the box of p: grid sort,
 * kNN with k0, clipping, re-queue with k doubled up to k_max, exhaustive pass
 * for what is left, then the requested outputs. Synchronises `stream` once
 * per pass (a 192-byte device-to-host read of the status block, which holds
 * the failed count) and once at
 * the end. Returns VT_ERR_CAPACITY (with out->needed_* set and vol/cen/m2
 * written) when a variable-length buffer is too small: allocate and call
 * vt_emit. stats may be NULL. n = 0 is valid (nothing to do); n = 1 gives
 * the whole box. */
VT_API int vt_tessellate(const float* pts, int64_t n, const vt_params* p, vt_cells_out* out,
                  vt_stats* stats, void* ws, size_t ws_bytes, void* stream);

/* ------------------------------------------------------------------ */
/* batches of independent point sets                                   */
/* ------------------------------------------------------------------ */

/* Batches (the paper treats one point set at a time; many independent sets
 * of uneven sizes run here as one tessellation over a concatenated input).
 * Every set has its own uniform grid over the box of p and is tessellated on
 * its own: its cells see only its own generators. Each stage runs as one
 * launch over the cells of all sets, so small sets share the GPU with large
 * ones.
 *
 * vt_batch_plan (host, no device work): set_off[n_sets+1] (host) are the
 * point offsets of the sets in the concatenated input (set_off[0] = 0,
 * non-decreasing); grid_res[n_sets] (host, may be NULL) overrides G per set
 * (0 = from p->grid_density and the set's size). Writes plan[n_sets] (host)
 * and *total_cells, the grid cells of all sets together. The caller copies
 * plan and set_off to device memory for vt_tessellate_batch. */
VT_API int vt_batch_plan(const int64_t* set_off, int n_sets, const vt_params* p, const int* grid_res,
                         vt_set_desc* plan, int64_t* total_cells);

/* Workspace bytes of a batch of n_total points whose grids have total_cells
 * cells (from vt_batch_plan). Host-only; VT_ERR_INVALID_ARG for a bad p,
 * n_total < 0, total_cells < 1 or, in a periodic box, n_total >= 2^24. */
VT_API int vt_batch_workspace_size(const vt_params* p, int64_t n_total, int64_t total_cells, size_t* bytes);

/* Tessellates every set of a batch. pts[n_total*3] (device), plan[n_sets] and
 * set_off[n_sets+1] (device copies of vt_batch_plan's plan and offsets).
 * Outputs as vt_tessellate over the concatenated input: cell i is point i of
 * the concatenation (VT_INDEX_ORIGINAL) and neighbour ids are indices into it,
 * so they never leave the cell's own set. With VT_FLAG_NO_SYNC the call only
 * enqueues work (capturable in a CUDA graph; read errors and sizes with
 * vt_read_stats); otherwise it behaves like vt_tessellate. */
VT_API int vt_tessellate_batch(const float* pts, int64_t n_total, const vt_set_desc* plan,
                               const int64_t* set_off, int n_sets, int64_t total_cells, const vt_params* p,
                               vt_cells_out* out, vt_stats* stats, void* ws, size_t ws_bytes, void* stream);

/* ------------------------------------------------------------------ */
/* autotuning of threads per cell, k0, k_max and grid density          */
/* ------------------------------------------------------------------ */

/* The paper sets its launch parameters by hand for one GPU; these calls pick
 * them by timing the whole path (grid, kNN, clipping, re-queue, emit) with
 * CUDA events on the caller's points, one parameter at a time: grid density,
 * k0, the k_max multiple, threads per cell. */

#define VT_TUNE_CLASSES 4
#define VT_TUNE_MAX_TRIED 64

/* Morisita index of each set on its grid: I = G^3 * sum_c n_c (n_c - 1) /
 * (n (n - 1)) over the grid cells c (n_c generators each), about 1 for
 * uniform i.i.d. points, above 1 when clustered, 0 for n < 2. plan = NULL:
 * one set over the grid of p (workspace of vt_workspace_size); else the
 * device plan and set_off of a batch (workspace of vt_batch_workspace_size).
 * index[n_sets] is host memory. Blocking; VT_ERR_INVALID_ARG for points
 * outside the box. */
VT_API int vt_cluster_index(const float* pts, int64_t n_total, const vt_set_desc* plan, const int64_t* set_off,
                            int n_sets, int64_t total_cells, const vt_params* p, double* index, void* ws,
                            size_t ws_bytes, void* stream);

/* Clustering class of a Morisita index: 0 below 2, 1 below 8, 2 below 32, else 3. */
VT_API int vt_cluster_class(double index);

typedef struct vt_tune_space {
    int n_tpc, tpc[4];          /* threads-per-cell candidates (8, 16, 32) */
    int n_k0, k0[8];            /* initial k candidates */
    int n_kmax, kmax_mult[4];   /* k_max = min(256, k0 * mult) candidates */
    int n_rho;                  /* grid-density candidates */
    float rho[8];
    int reps;                   /* timed runs per candidate after one untimed run */
} vt_tune_space;

typedef struct vt_tune_trial {
    int threads_per_cell, k0, k_max, cls;   /* cls: the class whose density was varied */
    float grid_density;
    int status;                             /* VT_OK or the run's error */
    double ms;                              /* minimum over reps, -1 if it failed */
} vt_tune_trial;

typedef struct vt_tune_result {
    vt_params best;                         /* base with the tuned fields */
    float density_of_class[VT_TUNE_CLASSES];/* batches: grid density per clustering class */
    double best_ms;
    int n_tried;                            /* candidates timed (tried[] keeps the first 64) */
    vt_tune_trial tried[VT_TUNE_MAX_TRIED];
} vt_tune_result;

/* Default space: tpc {8,16,32}, k0 {8,12,16,24,32}, mult {1,2,4}, rho {1,2,3,4,6}, reps 3. */
VT_API void vt_tune_space_default(vt_tune_space* s);

/* Workspace bytes for vt_autotune on n points (the widest candidate). */
VT_API int vt_autotune_workspace_size(const vt_params* base, const vt_tune_space* s, int64_t n, size_t* bytes);

/* Tunes one point set pts[n*3] (device) starting from base (whose emit,
 * precision, box and flags every candidate keeps); out holds output buffers
 * for n cells (capacities as for vt_tessellate). res->best is the fastest
 * candidate that completed with VT_OK. Blocking. */
VT_API int vt_autotune(const float* pts, int64_t n, const vt_params* base, const vt_tune_space* s,
                       vt_cells_out* out, vt_tune_result* res, void* ws, size_t ws_bytes, void* stream);

/* Workspace bytes for vt_autotune_batch (the widest candidate). */
VT_API int vt_autotune_batch_workspace_size(const int64_t* set_off, int n_sets, const vt_params* base,
                                            const vt_tune_space* s, size_t* bytes);

/* Tunes a batch: one grid density per clustering class (set_class[n_sets],
 * host, from vt_cluster_class), and k0, k_max, threads per cell for the whole
 * batch. set_off_host / set_off_dev are the offsets on the host and device;
 * plan_dev (device, n_sets descriptors) is overwritten by each candidate's
 * plan. The schedule of base->flags (VT_FLAG_NO_SYNC or not) is the one
 * timed. Blocking. */
VT_API int vt_autotune_batch(const float* pts, const int64_t* set_off_host, const int64_t* set_off_dev, int n_sets,
                             const int* set_class, const vt_params* base, const vt_tune_space* s,
                             vt_set_desc* plan_dev, vt_cells_out* out, vt_tune_result* res, void* ws,
                             size_t ws_bytes, void* stream);

/* ------------------------------------------------------------------ */
/* adjoint of the cell moments (for Lloyd relaxation and cell losses)  */
/* ------------------------------------------------------------------ */

/* Vector-Jacobian product of the cell volumes V_i, centroids c_i and second
 * moments M2_i (integral over C_i of |x - p_i|^2) with respect to the
 * generators: grad[k] = sum_i gV_i dV_i/dp_k + gC_i . dc_i/dp_k + gM_i dM2_i/dp_k.
 * The cells move through their bisector faces (a face between p_i and p_j
 * moves along its normal with speed (x - p_i).dp_i / |p_j - p_i| and
 * (p_j - x).dp_j / |p_j - p_i|; walls are fixed), so the product is a sum of
 * exact face integrals of cubic polynomials plus 2 gM_k V_k (p_k - c_k).
 * In a periodic box p_j is the image of the neighbour the face belongs to,
 * p_j + t L with t read off the face's own plane (t = round of the
 * reflection of p_i across the face, minus p_j, over L); moving p_j moves
 * that image.
 * pts[n*3]: the generators of the tessellation (original order).
 * cells: vol, cen and the geometry (vtx_off, vtx, face_off, face_nbr,
 * face_vtx_off, face_vtx) of a vt_tessellate call on pts with
 * VT_EMIT_VOL|VT_EMIT_CEN|VT_EMIT_GEOM and VT_INDEX_ORIGINAL.
 * gV[n], gC[n*3], gM[n]: upstream gradients, each may be NULL (zero).
 * p: the parameters of the tessellation (NULL: the defaults of
 * vt_params_default with precision VT_FP64). p->precision VT_FP64 integrates
 * the faces in FP64; VT_FP32_RECHECK in float32 in each generator's frame
 * (for cells of the FP32 form, whose vertices carry float32 round-off anyway;
 * the per-generator sums stay FP64). p->box_lo/box_hi and VT_FLAG_PERIODIC
 * give the periods.
 * grad[n*3] (FP64) is overwritten. Deterministic: each generator's gradient
 * is summed by one warp in a fixed order. Asynchronous on `stream`. */
VT_API int vt_moments_adjoint(const float* pts, int64_t n, const vt_cells_out* cells, const double* gV,
                              const double* gC, const double* gM, const vt_params* p, double* grad,
                              void* stream);

/* Lloyd relaxation (not in the paper; Lloyd's centroid update written as a
 * gradient step on the energy sum_i M2_i): out[k] = p_k - grad_k / (2 V_k),
 * which is the centroid c_k when grad is vt_moments_adjoint's gradient of
 * sum_i M2_i (2 V_k (p_k - c_k)). pts[n*3], out[n*3] float32 (out may equal
 * pts), grad[n*3] and vol[n] FP64, all device memory. The step runs in FP64
 * and is rounded once to float32. p->box_lo/box_hi and VT_FLAG_PERIODIC give
 * the box: in a periodic box the new point is moved by whole periods into
 * [lo, hi) (from its float32 value, in FP64, rounded again; a coordinate that
 * rounds onto hi becomes lo); in a walled box a coordinate that rounds onto
 * hi becomes the largest float below hi. A NaN volume (an unvalidated cell)
 * gives a NaN point, which the next tessellation refuses. Asynchronous on
 * `stream`. */
VT_API int vt_lloyd_step(const float* pts, int64_t n, const double* grad, const double* vol, const vt_params* p,
                         float* out, void* stream);

/* ------------------------------------------------------------------ */
/* diagnostics                                                         */
/* ------------------------------------------------------------------ */

/* Reads the device status flags of the workspace (blocking on `stream`):
 * returns VT_OK, VT_ERR_INVALID_ARG (bad point) or VT_ERR_DUPLICATE_POINTS. */
VT_API int vt_read_status(void* ws, size_t ws_bytes, void* stream);

/* Measured fused multiply-add throughput of the current device (blocking on
 * `stream`): precision VT_FP32_RECHECK times float32 FMAs, VT_FP64 float64
 * ones (eight independent chains per thread, eight blocks of 256 threads per
 * SM, CUDA events; about 5 ms each on a GB300). *tflops receives the rate in
 * TFLOP/s counting an FMA as 2 flops: the measured peak of ALU-bound rooflines. */
VT_API int vt_probe_fma(int precision, double* tflops, void* stream);

/* After a VT_FLAG_NO_SYNC call (or any call) on workspace ws (blocking on
 * `stream`): fills the device-counted fields of *stats (fp64_rechecks,
 * capacity_retries, precision_retries, unvalidated, clip_events, knn_candidates,
 * knn_queries, walk_cells, walk_candidates; other fields
 * are left as they are) and out->needed_* (either may be NULL). Returns the
 * call's error: VT_ERR_INVALID_ARG / VT_ERR_DUPLICATE_POINTS for bad input,
 * VT_ERR_CAPACITY when an output did not fit (nothing of that output was
 * written), VT_ERR_UNVALIDATED when cells stayed unvalidated, else VT_OK. */
VT_API int vt_read_stats(void* ws, size_t ws_bytes, vt_stats* stats, vt_cells_out* out, void* stream);

/* The cells the last vt_tessellate / vt_tessellate_batch call on workspace
 * ws left unvalidated (the paper's security radius never proved them final;
 * the call returned VT_ERR_UNVALIDATED). p and n are that call's parameters
 * and point count (n_total for a batch). Blocking on `stream`: *count (host)
 * receives how many there are, and, when ids is not NULL, ids[0..count)
 * (device) their indices in p->index_space, in no particular order;
 * VT_ERR_CAPACITY when count > cap (nothing written). The calls themselves
 * write NaN into vol, cen and m2 of those cells, leave them without
 * neighbours, faces or vertices, and keep every other cell exact. Not
 * capturable (it reads a count). */
VT_API int vt_unvalidated_cells(const vt_params* p, int64_t n, int32_t* ids, int64_t cap, int64_t* count, void* ws,
                                size_t ws_bytes, void* stream);

/* Message of the last failure on this host thread ("" if none). */
VT_API const char* vt_last_error(void);

/* Number of kernels this library has launched in this process. */
VT_API int64_t vt_launch_count(void);

/* Library version string. */
VT_API const char* vt_version(void);

#ifdef __cplusplus
}
#endif
#endif /* VT_H */
