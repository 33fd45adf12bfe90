// vt_internal.cuh -- shared declarations of the CUDA path (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "vt.h"

namespace vt {

// ---------------------------------------------------------------------------
// grid description (host-computed, passed by value to kernels)
// ---------------------------------------------------------------------------
struct GridDesc {
    int G;            // cells per axis
    float lo[3];      // box
    float hi[3];
    float scale[3];   // float32(G) / (hi - lo), rounded once on the host
    double cw[3];     // cell width (hi - lo) / G in double (stop-rule geometry only)
    double margin;    // safety margin of the shell-walk stop rule (coordinates)
    int64_t cell_base;  // first global grid cell of this point set (batches)
    int64_t pt_begin;   // first input point of this point set
    int64_t npts;       // points in this point set
};
static_assert(sizeof(GridDesc) == sizeof(vt_set_desc), "vt_set_desc mirrors GridDesc");

// grid of the point set that sorted point q belongs to
__device__ __forceinline__ const GridDesc& grid_of(const GridDesc& g0, const GridDesc* sets, const int32_t* set_of,
                                                   int q)
{
    return sets ? sets[set_of[q]] : g0;
}

// distance from q (in grid cell (ix, iy, iz)) to the outside of the block of
// shells 0..s, minus the rounding margin; 1e300 when the block reaches every
// wall of the box (no generator lies beyond it)
__device__ __forceinline__ double shell_gap(const GridDesc& g, float4 q, int ix, int iy, int iz, int s)
{
    const int G = g.G;
    const double q0 = q.x, q1 = q.y, q2 = q.z;
    double gap = 1e300;
    if (ix - s > 0) gap = fmin(gap, q0 - ((double)g.lo[0] + (ix - s) * g.cw[0]) - g.margin);
    if (ix + s + 1 < G) gap = fmin(gap, ((double)g.lo[0] + (ix + s + 1) * g.cw[0]) - q0 - g.margin);
    if (iy - s > 0) gap = fmin(gap, q1 - ((double)g.lo[1] + (iy - s) * g.cw[1]) - g.margin);
    if (iy + s + 1 < G) gap = fmin(gap, ((double)g.lo[1] + (iy + s + 1) * g.cw[1]) - q1 - g.margin);
    if (iz - s > 0) gap = fmin(gap, q2 - ((double)g.lo[2] + (iz - s) * g.cw[2]) - g.margin);
    if (iz + s + 1 < G) gap = fmin(gap, ((double)g.lo[2] + (iz + s + 1) * g.cw[2]) - q2 - g.margin);
    return gap;
}

GridDesc make_grid(const vt_params* p, int G);

// grid cell of a point: every operation a separately rounded float32 op
__device__ __forceinline__ int cell_coord(float x, float lo, float scale, int G)
{
    float t = __fmul_rn(__fsub_rn(x, lo), scale);
    int c = (int)floorf(t);
    c = c < 0 ? 0 : c;
    return c > G - 1 ? G - 1 : c;
}

__device__ __forceinline__ int cell_id(int ix, int iy, int iz, int G) { return (ix * G + iy) * G + iz; }

// Segment e of Chebyshev shell s around grid cell (ix, iy, iz): a contiguous
// range [a, b) of the sorted points (empty when outside the grid). Row
// (dx, dy), dx, dy in [-s, s], owns segments 2*row and 2*row + 1: a row on the
// shell's rim (|dx| = s or |dy| = s) contributes the z-range [iz-s, iz+s] as
// its first segment; an inner row contributes the two cells z = iz-s and
// z = iz+s. A shell has 2 (2s+1)^2 segments, s = 0 has the cell itself.
__device__ __forceinline__ void shell_segment(int e, int s, int ix, int iy, int iz, int G,
                                              const int32_t* __restrict__ cell_off, int& a, int& b)
{
    const int W = 2 * s + 1;
    const int row = e >> 1, half = e & 1;
    const int dx = row / W - s, dy = row - (row / W) * W - s;
    const int x = ix + dx, y = iy + dy;
    a = b = 0;
    if (x < 0 || x >= G || y < 0 || y >= G) return;
    const bool rim = dx == -s || dx == s || dy == -s || dy == s;
    const int base = (x * G + y) * G;
    if (rim) {
        if (half) return;
        const int z0 = iz - s < 0 ? 0 : iz - s, z1 = iz + s > G - 1 ? G - 1 : iz + s;
        a = cell_off[base + z0];
        b = cell_off[base + z1 + 1];
    } else {
        const int z = half ? iz + s : iz - s;
        if (z < 0 || z >= G) return;
        a = cell_off[base + z];
        b = cell_off[base + z + 1];
    }
}

// kNN ordering keys. FP64 form: ((dx*dx + dy*dy) + dz*dz) in double with
// dx = double(x_j) - double(x_i), every operation separately rounded (no FMA),
// so lists are exact and reproducible. FP32 form: the same in float32 with FMA.
__device__ __forceinline__ double knn_d2_f64(float4 a, float4 b)
{
    const double dx = __dsub_rn((double)b.x, (double)a.x);
    const double dy = __dsub_rn((double)b.y, (double)a.y);
    const double dz = __dsub_rn((double)b.z, (double)a.z);
    return __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
}
__device__ __forceinline__ float knn_d2_f32(float4 a, float4 b)
{
    const float dx = b.x - a.x, dy = b.y - a.y, dz = b.z - a.z;
    return fmaf(dz, dz, fmaf(dy, dy, dx * dx));
}

// ---------------------------------------------------------------------------
// device status block at the start of every workspace
// ---------------------------------------------------------------------------
struct DevStatus {
    int32_t bad_point;        // 1 + smallest offending input index, 0 if none
    int32_t duplicate;        // nonzero once a neighbour at distance 0 was seen
    int32_t n_fail_next;      // cells that need the next k (failed validation)
    int32_t n_fail_robust;    // cells that need the robust variant (capacity / precision)
    int32_t n_big_cells;      // grid cells too large for the per-thread fix-up sort
    int32_t record_overflow;  // cells whose final polyhedron does not fit an output record
    int32_t cap_overflow;     // an output buffer was too small for the emitted data (device check)
    int32_t n_unval;          // cells left unvalidated (no-sync schedule)
    unsigned long long fp64_rechecks;
    unsigned long long capacity_events;
    unsigned long long precision_events;
    long long totals[4];      // nbr, vtx, face, face_vtx totals written by the emit scan
    unsigned int detail[8];   // clip events: 0 keep-none, 1 plane cap, 2 vertex cap, 3 ring, 4 interpolated
    int32_t list_overflow;    // a device-counted pass had more cells than its list buffers hold
    int32_t pad2;
};
static_assert(sizeof(DevStatus) % 64 == 0, "status block must stay 64-byte sized");

// ---------------------------------------------------------------------------
// per-cell output record (fixed stride, in the workspace)
// ---------------------------------------------------------------------------
constexpr int REC_FACES = 64;      // faces of a final cell
constexpr int REC_VERTS = 128;     // vertices of a final cell
struct RecHeader {
    int32_t nnbr;                  // neighbours kept (area > threshold)
    int32_t nface;                 // faces written (geometry)
    int32_t nvtx;                  // vertices written (geometry)
    int32_t nfv;                   // face-vertex entries (geometry)
};
// layout: RecHeader | int32 nbr[REC_FACES] | (geometry:) int32 face_nbr[REC_FACES] |
//         uint8 face_deg[REC_FACES] | uint8 face_vtx[3*REC_VERTS] | double vtx[REC_VERTS*3]
constexpr size_t REC_NBR_OFF = sizeof(RecHeader);
constexpr size_t REC_FNBR_OFF = REC_NBR_OFF + 4 * REC_FACES;
constexpr size_t REC_FDEG_OFF = REC_FNBR_OFF + 4 * REC_FACES;
constexpr size_t REC_FVTX_OFF = REC_FDEG_OFF + REC_FACES;
constexpr size_t REC_VTX_OFF = (REC_FVTX_OFF + 3 * REC_VERTS + 15) / 16 * 16;
constexpr size_t REC_STRIDE_NBR = REC_FNBR_OFF;                              // 272 B
constexpr size_t REC_STRIDE_GEOM = REC_VTX_OFF + 8 * 3 * REC_VERTS;          // ~4 KB

// fail reasons stored per cell
enum : int8_t { CELL_DONE = 0, CELL_NEED_K = 1, CELL_NEED_ROBUST = 2, CELL_UNVALIDATED = 3 };

// ---------------------------------------------------------------------------
// workspace layout
// ---------------------------------------------------------------------------
struct Layout {
    int G;
    int64_t n, g3;
    int64_t knn_cap;            // entries of the neighbour-list buffer
    size_t rec_stride;
    size_t status, cid, ticket, counts, cell_off, big, scan_tmp, sorted, perm;
    size_t state_stride;
    size_t list_a, list_b, list_r, knn_nbr, knn_d2, rec, cnt, off64, scan_emit, state, set_of, ctr;
    size_t total;
};
// cells < 0: the single-set grid of p; otherwise the total grid cells of a batch
Layout make_layout(const vt_params* p, int64_t n, int64_t cells = -1, bool batch = false);

// ---------------------------------------------------------------------------
// launch helpers shared by the translation units
// ---------------------------------------------------------------------------
int set_error(int code, const char* msg);  // records msg for vt_last_error, returns code
void count_launch(int n = 1);
int64_t launches();

// exclusive scans (grid-wide, multi-kernel); tmp needs scan_tmp_bytes(n)
size_t scan_tmp_bytes(int64_t n);
void exclusive_scan_i32(const int32_t* in, int32_t* out, int64_t n, void* tmp, cudaStream_t s);
void exclusive_scan_i32_to_i64(const int32_t* in, int64_t* out, int64_t n, void* tmp, cudaStream_t s);

// stage launchers (return cudaError_t of the launch)
// batches: sets (device, nsets descriptors), set_off (device, nsets + 1 point
// offsets), g3 = total grid cells of all sets; set_of receives the set of each
// sorted point. A single set passes sets = set_off = set_of = nullptr.
struct BatchArgs {
    const GridDesc* sets;
    const int64_t* set_off;
    int nsets;
    int32_t* set_of;
};
cudaError_t launch_grid_build(const float* pts, int64_t n, const GridDesc& g, float4* sorted, int32_t* perm,
                              int32_t* cell_off, int32_t* cid, int32_t* ticket, int32_t* counts, int32_t* big,
                              void* scan_tmp, DevStatus* st, cudaStream_t s, const BatchArgs* batch = nullptr,
                              int64_t g3 = -1);

// acc[s] = sum over the grid cells of set s of n_c (n_c - 1) (sets = nullptr: one set)
cudaError_t launch_pair_counts(const int32_t* cell_off, int64_t g3, const GridDesc* sets, int nsets,
                               unsigned long long* acc, cudaStream_t s);

// nq_dev: the query count is read from device memory, clamped to nq (more sets
// st->list_overflow)
cudaError_t launch_knn(const float4* sorted, const int32_t* cell_off, const GridDesc& g, int64_t n,
                       const int32_t* queries, int64_t nq, int k, int precision, int32_t* nbr, void* d2,
                       DevStatus* st, cudaStream_t s, const GridDesc* sets = nullptr, const int32_t* set_of = nullptr,
                       const int32_t* nq_dev = nullptr);

struct ClipArgs {
    const float4* sorted;
    const int32_t* cell_off;
    GridDesc g;
    int64_t n;
    const int32_t* queries;   // sorted indices (NULL = 0..nq-1)
    int64_t nq;
    const int32_t* nbr;       // [nq*k] (k > 0)
    const void* d2;           // [nq*k] float or double
    int k;                    // list entries per cell (0 = no list)
    int exhaustive;           // 1: after the list (or the resumed state), walk every generator within 2R
    int emit;
    int index_space;
    double* vol;
    double* cen;
    double* m2;
    uint8_t* rec;             // records base (NULL = none)
    size_t rec_stride;
    int32_t* fail_next;       // appended: cells needing a larger k
    int32_t* fail_robust;     // appended: cells needing the robust variant (or, from
                              // the robust variant itself, cells left unvalidated)
    int32_t* ctr_next;        // device counters of the two lists
    int32_t* ctr_robust;
    const GridDesc* sets;     // per-set grids of a batch (NULL: the single grid g)
    const int32_t* set_of;    // set of each sorted point (batches)
    const int32_t* nq_dev;    // when set, the cell count is read from device memory
    int64_t nq_cap;           // with nq_dev: at most this many cells fit the list buffers (more sets
                              // DevStatus::list_overflow and the rest is not processed)
    int k_prev;               // > 0: resume saved cells; list entries [0, k_prev) are done
    uint8_t* state;           // per-cell saved polyhedra (sorted index * state_stride), or NULL
    size_t state_stride;
    DevStatus* st;
};
// variant: 0 = FP32 regular, 1 = FP64 regular, 2 = FP64 robust (bigger capacity)
cudaError_t launch_clip(const ClipArgs& a, int variant, int threads_per_cell, cudaStream_t s);
size_t clip_state_bytes(int precision);  // per-cell state of the regular variant

struct EmitArgs {
    int64_t n;
    int emit;
    const uint8_t* rec;
    size_t rec_stride;
    int32_t* cnt;             // [4*n] scratch counts
    int64_t* off64;           // [4*(n+1)] scratch offsets
    void* scan_tmp;
    DevStatus* st;
};
cudaError_t launch_emit_count(const EmitArgs& a, cudaStream_t s);  // counts + scans + totals
cudaError_t launch_emit_write(const EmitArgs& a, const vt_cells_out& out, cudaStream_t s);  // device-checked caps
cudaError_t launch_adjoint(const float* pts, int64_t n, const vt_cells_out& c, const double* gV, const double* gC,
                           const double* gM, double* grad, cudaStream_t s);

}  // namespace vt
