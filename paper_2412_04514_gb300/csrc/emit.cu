// emit.cu -- variable-length outputs (votess paper, Features: the neighbours
// of each cell as a jagged array; Summary: cell geometry).
//
// The clipper leaves one fixed-stride record per cell in the workspace. Emit
// counts the entries of every record, turns the counts into CSR offsets with
// grid-wide scans, then a group of 8 threads per cell copies its record into
// the caller's CSR arrays (neighbour ids, vertices, faces, face-vertex lists).
#include "vt_internal.cuh"

namespace vt {

namespace {

__global__ void k_emit_count(const uint8_t* __restrict__ rec, size_t stride, int64_t n, int geom,
                             int32_t* __restrict__ cnt)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const RecHeader h = *reinterpret_cast<const RecHeader*>(rec + (size_t)i * stride);
        cnt[i] = h.nnbr;
        if (geom) {
            cnt[n + i] = h.nvtx;
            cnt[2 * n + i] = h.nface;
            cnt[3 * n + i] = h.nfv;
        }
    }
}

__global__ void k_emit_totals(const int64_t* __restrict__ off, int64_t n, int geom, DevStatus* st)
{
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        for (int a = 0; a < 4; ++a) st->totals[a] = (a == 0 || geom) ? off[a * (n + 1) + n] : 0;
    }
}

// CSR index check of debug builds (see vt_ck)
__device__ __forceinline__ int64_t vt_ck64(int64_t i, int64_t cap, DevStatus* st)
{
    if (VT_CHECKED && (uint64_t)i >= (uint64_t)cap) {
        atomicCAS(&st->check_fail, 0, CK_CSR);
        return 0;
    }
    return i;
}

constexpr int EMIT_LANES = 8;

__global__ void k_emit_write(const uint8_t* __restrict__ rec, size_t stride, int64_t n, int emit, int vtx_f32,
                             const int64_t* __restrict__ off, vt_cells_out out, DevStatus* st)
{
    // EMIT_LANES threads per cell: a cell's arrays are short (16 neighbours,
    // 90 vertex coordinates), so more cells in flight hide more of the
    // dependent record loads than wider groups (measured on 1M cells: emit
    // 1.06 ms with 32 lanes, 0.90 with 16, 0.86 with 8, 0.83 with 4)
    const int lane = threadIdx.x & (EMIT_LANES - 1);
    const int64_t wid = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / EMIT_LANES;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) / EMIT_LANES;
    const int64_t* o_nbr = off;
    const int64_t* o_vtx = off + (n + 1);
    const int64_t* o_face = off + 2 * (n + 1);
    const int64_t* o_fv = off + 3 * (n + 1);
    for (int64_t i = wid; i < n; i += nw) {
        const uint8_t* r = rec + (size_t)i * stride;
        const RecHeader h = *reinterpret_cast<const RecHeader*>(r);
        // capacities are checked here as well, so a run that never synchronises
        // (a captured graph) cannot write past the caller's buffers
        const bool nbr_fits = !(emit & VT_EMIT_NBR) || o_nbr[n] <= out.nbr_cap;
        const bool geo_fits = !(emit & VT_EMIT_GEOM) ||
                              (o_vtx[n] <= out.vtx_cap && o_face[n] <= out.face_cap && o_fv[n] <= out.face_vtx_cap);
        if (!nbr_fits || !geo_fits) {
            if (lane == 0 && i == 0) atomicExch((int*)&st->cap_overflow, 1);
            continue;
        }
        if (emit & VT_EMIT_NBR) {
            const int64_t b = o_nbr[i];
            const int32_t* src = reinterpret_cast<const int32_t*>(r + REC_NBR_OFF);
            for (int t = lane; t < h.nnbr; t += EMIT_LANES) out.nbr[vt_ck64(b + t, out.nbr_cap, st)] = src[t];
            if (lane == 0) {
                out.nbr_off[i] = b;
                if (i == n - 1) out.nbr_off[n] = o_nbr[n];
            }
        }
        if (emit & VT_EMIT_GEOM) {
            const int64_t bv = o_vtx[i], bf = o_face[i], bfv = o_fv[i];
            if (vtx_f32) {  // float offsets from the generator
                const float* v = reinterpret_cast<const float*>(r + REC_VTX_OFF);
                for (int t = lane; t < 3 * h.nvtx; t += EMIT_LANES) {
                    const int a = t % 3;  // (selected, not indexed: h stays in registers)
                    const float pa = a == 0 ? h.p[0] : (a == 1 ? h.p[1] : h.p[2]);
                    out.vtx[vt_ck64(3 * bv + t, 3 * out.vtx_cap, st)] = (double)pa + (double)v[t];
                }
            } else {
                const double* v = reinterpret_cast<const double*>(r + REC_VTX_OFF);
                for (int t = lane; t < 3 * h.nvtx; t += EMIT_LANES)
                    out.vtx[vt_ck64(3 * bv + t, 3 * out.vtx_cap, st)] = v[t];
            }
            const int32_t* fn = reinterpret_cast<const int32_t*>(r + REC_FNBR_OFF);
            const uint8_t* fd = r + REC_FDEG_OFF;
            const uint8_t* fv = r + REC_FVTX_OFF;
            for (int t = lane; t < h.nface; t += EMIT_LANES) out.face_nbr[vt_ck64(bf + t, out.face_cap, st)] = fn[t];
            for (int t = lane; t < h.nfv; t += EMIT_LANES) out.face_vtx[vt_ck64(bfv + t, out.face_vtx_cap, st)] = fv[t];
            // per-face offsets: prefix of the degrees (faces per cell are few)
            if (lane == 0) {
                int64_t p = bfv;
                for (int t = 0; t < h.nface; ++t) {
                    out.face_vtx_off[bf + t] = p;
                    p += fd[t];
                }
                out.vtx_off[i] = bv;
                out.face_off[i] = bf;
                if (i == n - 1) {
                    out.vtx_off[n] = o_vtx[n];
                    out.face_off[n] = o_face[n];
                    out.face_vtx_off[o_face[n]] = o_fv[n];
                }
            }
        }
    }
}

// Cells left unvalidated: NaN into their moments, so that no stale or
// partial value is mistaken for a cell. list[] holds sorted indices; the
// count is *n_dev when set (the no-sync schedule), else n_host, which the
// first thread also stores in the status block for vt_read_stats.
__global__ void k_mark_unvalidated(const int32_t* __restrict__ list, const int32_t* n_dev, int64_t n_host,
                                   const float4* __restrict__ sorted, int index_space, double* vol, double* cen,
                                   double* m2, DevStatus* st)
{
    const int64_t cnt = n_dev ? (int64_t)*n_dev : n_host;
    if (!n_dev && blockIdx.x == 0 && threadIdx.x == 0) st->n_unval = (int32_t)n_host;
    const double nan = __longlong_as_double(0x7ff8000000000000ll);
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < cnt; i += (int64_t)gridDim.x * blockDim.x) {
        const int32_t q = list[i];
        const int64_t o = index_space == VT_INDEX_ORIGINAL ? (int64_t)__float_as_int(sorted[q].w) : (int64_t)q;
        if (vol) vol[o] = nan;
        if (cen) cen[3 * o] = cen[3 * o + 1] = cen[3 * o + 2] = nan;
        if (m2) m2[o] = nan;
    }
}

// ids of the unvalidated cells in the chosen index space (at most cap)
__global__ void k_unvalidated_ids(const int32_t* __restrict__ list, int64_t cnt, const float4* __restrict__ sorted,
                                  int index_space, int32_t* __restrict__ ids)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < cnt; i += (int64_t)gridDim.x * blockDim.x) {
        const int32_t q = list[i];
        ids[i] = index_space == VT_INDEX_ORIGINAL ? __float_as_int(sorted[q].w) : q;
    }
}

}  // namespace

cudaError_t launch_mark_unvalidated(const int32_t* list, const int32_t* n_dev, int64_t n_host, int64_t n_bound,
                                    const float4* sorted, int index_space, double* vol, double* cen, double* m2,
                                    DevStatus* st, cudaStream_t s)
{
    int64_t blocks = (n_bound + 255) / 256;
    if (blocks > 152 * 8) blocks = 152 * 8;
    if (blocks < 1) blocks = 1;
    k_mark_unvalidated<<<(unsigned)blocks, 256, 0, s>>>(list, n_dev, n_host, sorted, index_space, vol, cen, m2, st);
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_unvalidated_ids(const int32_t* list, int64_t cnt, const float4* sorted, int index_space,
                                   int32_t* ids, cudaStream_t s)
{
    if (cnt <= 0) return cudaSuccess;
    int64_t blocks = (cnt + 255) / 256;
    if (blocks > 152 * 8) blocks = 152 * 8;
    k_unvalidated_ids<<<(unsigned)blocks, 256, 0, s>>>(list, cnt, sorted, index_space, ids);
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_emit_count(const EmitArgs& a, cudaStream_t s)
{
    const int geom = (a.emit & VT_EMIT_GEOM) ? 1 : 0;
    if (a.n > 0) {
        int64_t blocks = (a.n + 255) / 256;
        if (blocks > 152 * 64) blocks = 152 * 64;
        k_emit_count<<<(unsigned)blocks, 256, 0, s>>>(a.rec, a.rec_stride, a.n, geom, a.cnt);
        count_launch();
    }
    const int narr = geom ? 4 : 1;
    for (int k = 0; k < narr; ++k) exclusive_scan_i32_to_i64(a.cnt + k * a.n, a.off64 + k * (a.n + 1), a.n, a.scan_tmp, s);
    k_emit_totals<<<1, 32, 0, s>>>(a.off64, a.n, geom, a.st);
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_emit_write(const EmitArgs& a, const vt_cells_out& out, cudaStream_t s)
{
    if (a.n <= 0) return cudaSuccess;
    constexpr int cells_per_block = 256 / EMIT_LANES;
    int64_t blocks = (a.n + cells_per_block - 1) / cells_per_block;
    if (blocks > 152 * 32) blocks = 152 * 32;
    k_emit_write<<<(unsigned)blocks, 256, 0, s>>>(a.rec, a.rec_stride, a.n, a.emit, a.vtx_f32, a.off64, out, a.st);
    count_launch();
    return cudaGetLastError();
}

}  // namespace vt
