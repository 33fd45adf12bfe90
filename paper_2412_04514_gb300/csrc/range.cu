// range.cu -- candidate lists for the last clipping pass.
//
// After the k_max list pass a cell that is not yet validated has clipped by
// its k_max nearest neighbours; it can still be cut only by a generator q
// beyond the list (key above the last list key) with |q - p|^2 < 4 R^2 (the
// security radius, Summary section of the paper) whose bisector reaches the
// cell's bounding box. This kernel gathers exactly those generators for each
// such cell -- one warp per cell walks the grid shells around it, restricted
// to grid cells that meet the ball of radius 2R and are not inside the ball
// the list already covered -- and writes them sorted by the kNN key, so the
// clipper can process them nearest first and stop by the security radius.
// R, the bounding box and the last list key come from the cell's saved
// state. In the FP64 form a cell with more than `cap` candidates walks again,
// keeping only the generators whose bisector comes near one of its saved
// vertices; what still overflows goes to the clipper's own exhaustive walk
// (overflow list).
#include <float.h>
#include <limits.h>

#include "vt_internal.cuh"

namespace vt {

namespace {

constexpr unsigned FULL = 0xffffffffu;
constexpr int RANGE_BLOCK = 256;
constexpr int RANGE_VCAP = 64;  // vertex slots of the regular clipper's saved state

// The cell's far vertices into vb (x, y, z, |v|^2 rows of RANGE_VCAP), sorted
// by |v| descending: a generator at distance d >= sqrt(lkey) cuts only
// vertices with |v| > d / 2 (less the test's tolerance), so only vertices
// beyond sqrt(lkey) / 2 are kept. Returns their count; warp-collective.
template <typename Real>
__device__ __forceinline__ int load_far_vertices_t(const StateHdr* h, const uint8_t* st_pos, Real lkey, int last_orig,
                                                   float R2, float* vb, int lane)
{
    const uint64_t alive = h->alive[0];
    const Real* pos = reinterpret_cast<const Real*>(st_pos);
    const float rmin = 0.5f * sqrtf((float)lkey) * (1.0f - 1e-5f) - 2e-5f * sqrtf(R2);
    const float rmin2 = last_orig >= 0 && rmin > 0.0f ? rmin * rmin : -1.0f;
    float vx[2], vy[2], vz[2], vr[2];
    bool far[2];
#pragma unroll
    for (int h2 = 0; h2 < 2; ++h2) {
        const int v = lane + 32 * h2;
        far[h2] = false;
        vx[h2] = vy[h2] = vz[h2] = vr[h2] = 0.0f;
        if ((alive >> v) & 1ull) {
            vx[h2] = (float)pos[v];
            vy[h2] = (float)pos[RANGE_VCAP + v];
            vz[h2] = (float)pos[2 * RANGE_VCAP + v];
            vr[h2] = vx[h2] * vx[h2] + vy[h2] * vy[h2] + vz[h2] * vz[h2];
            far[h2] = vr[h2] > rmin2;
        }
    }
    const unsigned f0 = __ballot_sync(FULL, far[0]), f1 = __ballot_sync(FULL, far[1]);
#pragma unroll
    for (int h2 = 0; h2 < 2; ++h2) {
        int rank = 0;  // by |v|^2 descending, ties by slot
        for (int w = 0; w < 2; ++w) {
            for (unsigned m = w ? f1 : f0; m; m &= m - 1u) {
                const int src = __ffs(m) - 1;
                const float r = __shfl_sync(FULL, w ? vr[1] : vr[0], src);
                rank += (r > vr[h2] || (r == vr[h2] && src + 32 * w < lane + 32 * h2)) ? 1 : 0;
            }
        }
        if (far[h2]) {
            vb[rank] = vx[h2];
            vb[RANGE_VCAP + rank] = vy[h2];
            vb[2 * RANGE_VCAP + rank] = vz[h2];
            vb[3 * RANGE_VCAP + rank] = vr[h2];
        }
    }
    __syncwarp();
    return __popc(f0) + __popc(f1);
}

// true when the bisector of n (|n|^2 = d2) comes within 1e-5 |n| R of a far vertex
__device__ __forceinline__ bool reaches_far(const float* vb, int nv, float nx, float ny, float nz, float d2, float R2)
{
    const float lim = 0.5f * d2 - 1e-5f * sqrtf(d2 * R2) - 1e-30f;
    const float vmin = 0.5f * sqrtf(d2) * (1.0f - 1e-5f) - 2e-5f * sqrtf(R2);
    const float vmin2 = vmin > 0.0f ? vmin * vmin : -1.0f;
    for (int v = 0; v < nv && vb[3 * RANGE_VCAP + v] > vmin2; ++v)
        if (nx * vb[v] + ny * vb[RANGE_VCAP + v] + nz * vb[2 * RANGE_VCAP + v] > lim) return true;
    return false;
}

// resident blocks per SM: 6 for the FP32 kernel (40 registers; with the work
// queue measured 0.06 ms faster per 1M-cell step than 5 and 0.18 ms faster
// than 4; its periodic form 4, which spills more), 3 for the FP64 one (at
// most 80 registers)
#ifndef VT_RANGE_MINB_F32
#define VT_RANGE_MINB_F32 6
#endif
#ifndef VT_RANGE_MINB_F64
#define VT_RANGE_MINB_F64 3
#endif
template <typename Real, bool PER>
__global__ void __launch_bounds__(RANGE_BLOCK, (sizeof(Real) == 4 ? (PER ? 4 : VT_RANGE_MINB_F32) : VT_RANGE_MINB_F64))
    k_range(const float4* __restrict__ sorted,
                                                       const int32_t* __restrict__ cell_off0,
                                                       const __grid_constant__ GridDesc g0,
                                                       const GridDesc* __restrict__ sets,
                                                       const int32_t* __restrict__ set_of,
                                                       const int32_t* __restrict__ queries, int64_t nq_host,
                                                       const int32_t* __restrict__ nq_dev, int64_t nq_off,
                                                       const uint8_t* __restrict__ state, size_t state_stride,
                                                       size_t pos_off, int cap, int32_t* __restrict__ rnbr, Real* __restrict__ rd2,
                                                       int32_t* __restrict__ rlen, int32_t* __restrict__ over_list,
                                                       int32_t* __restrict__ over_ctr, DevStatus* st,
                                                       int32_t* __restrict__ queue)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    Real* bk = reinterpret_cast<Real*>(smem_raw) + warp * RANGE_CAP;
    int32_t* bo = reinterpret_cast<int32_t*>(smem_raw + sizeof(Real) * RANGE_CAP * (RANGE_BLOCK / 32)) +
                  warp * RANGE_CAP;
    int32_t* bj = bo + RANGE_CAP * (RANGE_BLOCK / 32);
    float* vb = reinterpret_cast<float*>(smem_raw + (sizeof(Real) + 2 * sizeof(int32_t)) * RANGE_CAP * (RANGE_BLOCK / 32)) +
                warp * 4 * RANGE_VCAP;
    int64_t nq = nq_host;
    if (nq_dev) {  // device-counted: list entries [nq_off, nq_off + nq_host)
        const int64_t want = (int64_t)*nq_dev - nq_off;
        nq = want < 0 ? 0 : (want < nq_host ? want : nq_host);
    }
    // walks and the generators they examined, added once per warp
    unsigned walk_cells = 0, walk_cands = 0;
    // cells come from a launch-wide counter, one per warp at a time
    auto next_cell = [&]() {
        int v = 0;
        if (lane == 0) v = atomicAdd(queue, 1);
        return (int64_t)__shfl_sync(FULL, v, 0);
    };
    for (int64_t c = next_cell(); c < nq; c = next_cell()) {
        const int q = queries[c];
        const float4 pq = sorted[q];
        const GridDesc& g = grid_of(g0, sets, set_of, q);
        const int G = g.G;
        const int32_t* cell_off = cell_off0 + g.cell_base;
        const StateHdr* h = reinterpret_cast<const StateHdr*>(state + (size_t)q * state_stride);
        const float R2 = (float)h->R2;
        const Real lkey = (Real)h->last_d2;  // exact: the key was stored from a Real
        const int last_orig = h->last_orig;
        const float lo3[3] = {h->bb_lo[0], h->bb_lo[1], h->bb_lo[2]};
        const float hi3[3] = {h->bb_hi[0], h->bb_hi[1], h->bb_hi[2]};
        const float r4 = 4.0f * R2 * (1.0f + 1e-4f);
        const float r_out2 = 4.0f * R2 * (1.0f + 2e-4f);
        const float r_in2 = last_orig >= 0 ? (float)lkey * (1.0f - 1e-4f) : -1.0f;
        const int ix = cell_coord(pq.x, g.lo[0], g.scale[0], G);
        const int iy = cell_coord(pq.y, g.lo[1], g.scale[1], G);
        const int iz = cell_coord(pq.z, g.lo[2], g.scale[2], G);
        int count = 0;
        bool over = false;
        int nv = 0;  // far vertices in vb (second attempt)
        ++walk_cells;
        // first attempt: radius and bounding-box tests. In the FP64 form a cell
        // whose candidates overflow the list (a sparse cell next to a clump)
        // walks again with the exact test against its saved vertices, which
        // keeps only the generators whose bisector can reach a vertex: cheaper
        // there than the FP64 clipper's own walk (measured); the FP32 clipper's
        // walk is cheaper than a second attempt (measured: the range lists 1.1 ms
        // slower per 1M-cell step, the clipping 0.8 ms faster; the vertex test
        // from the first attempt on, 1.55 ms slower and 1.2 ms faster)
        constexpr int attempts = sizeof(Real) == 8 ? 2 : 1;
        for (int attempt = 0; attempt < attempts; ++attempt) {
        if (attempt == 1) {
            if (!over) break;
            over = false;
            count = 0;
            nv = load_far_vertices_t<Real>(h, state + (size_t)q * state_stride + pos_off, lkey, last_orig, R2, vb,
                                           lane);
        }
        constexpr bool per = PER;
        for (int s = 0; !over; ++s) {
            const bool wrap = per && (ix - s < 0 || iy - s < 0 || iz - s < 0 || ix + s >= G || iy + s >= G || iz + s >= G);
            const int M = wrap ? seg_per_row(g, s) : 2;
            const int nseg = M * (2 * s + 1) * (2 * s + 1);
            for (int e0 = 0; e0 < nseg && !over; e0 += 32) {
                int sa = 0, sb = 0, sc = IMG_NONE;
                if (e0 + lane < nseg) {
                    if (wrap)
                        shell_segment_ball_p(e0 + lane, s, M, ix, iy, iz, g, cell_off, pq, r_out2, r_in2, sa, sb, sc);
                    else
                        shell_segment_ball(e0 + lane, s, ix, iy, iz, g, cell_off, pq, r_out2, r_in2, sa, sb);
                }
                const int len = sb - sa;
                int incl = len;
#pragma unroll
                for (int d = 1; d < 32; d <<= 1) {
                    const int u = __shfl_up_sync(FULL, incl, d);
                    if (lane >= d) incl += u;
                }
                const int total = __shfl_sync(FULL, incl, 31);
                const int start = incl - len;
                walk_cands += (unsigned)total;
                for (int c0 = 0; c0 < total && !over; c0 += 32) {
                    const int i = c0 + lane;
                    int seg = 0;
#pragma unroll
                    for (int step = 16; step >= 1; step >>= 1)
                        if (__shfl_sync(FULL, incl, (seg + step - 1) & 31) <= i) seg += step;
                    const int aj = __shfl_sync(FULL, sa, seg & 31), sj = __shfl_sync(FULL, start, seg & 31);
                    const int code = per ? __shfl_sync(FULL, sc, seg & 31) : IMG_NONE;
                    const int j0 = aj + (i - sj);
                    const int jj = per ? img_pack(j0, code) : j0;
                    bool keep = false;
                    Real key = (Real)0;
                    int ko = 0;
                    if (i < total && j0 != q) {
                        const float4 pc = sorted[j0];
                        const float3 o = img_off_t<PER>(pq, pc, code, g);
                        const float ex = o.x, ey = o.y, ez = o.z;
                        const float d2 = fmaf(ez, ez, fmaf(ey, ey, ex * ex));
                        const float hb = fmaxf(ex * lo3[0], ex * hi3[0]) + fmaxf(ey * lo3[1], ey * hi3[1]) +
                                         fmaxf(ez * lo3[2], ez * hi3[2]);
                        keep = r4 > d2 && hb > 0.5f * d2 * (1.0f - 1e-4f) - 1e-6f * sqrtf(d2 * R2) - 1e-30f;
                        if (keep && attempt == 1) keep = reaches_far(vb, nv, ex, ey, ez, d2, R2);
                        if (keep) {
                            key = sizeof(Real) == 8 ? (Real)img_key64(pq, sorted, jj, g) : (Real)d2;
                            ko = img_tie_t<PER>(pc, code);
                            if (last_orig >= 0 && (key < lkey || (key == lkey && ko <= last_orig)))
                                keep = false;  // the list already held it
                        }
                    }
                    const unsigned m = __ballot_sync(FULL, keep);
                    const int pos = count + __popc(m & ((1u << lane) - 1u));
                    if (keep && pos < cap) {
                        bk[pos] = key;
                        bo[pos] = ko;
                        bj[pos] = jj;
                    }
                    count += __popc(m);
                    over = count > cap;
                }
            }
            if (over) break;
            if (per) {  // R <= |L| / 2: the walk ends within |L|
                const float gap = shell_gap_p(g, pq, ix, iy, iz, s);
                if (gap > 0.0f && 4.0f * R2 * (1.0f + 2e-5f) <= gap * gap) break;
                continue;
            }
            const bool covers = ix - s <= 0 && iy - s <= 0 && iz - s <= 0 && ix + s >= G - 1 && iy + s >= G - 1 &&
                                iz + s >= G - 1;
            if (covers) break;
            const float gap = shell_gap(g, pq, ix, iy, iz, s);
            if (gap > 0.0f && 4.0f * R2 * (1.0f + 2e-5f) <= gap * gap) break;
        }
        }
        if (over) {
            if (lane == 0) {
                rlen[c] = -1;
                over_list[atomicAdd(over_ctr, 1)] = q;
            }
            __syncwarp();
            continue;
        }
        __syncwarp();
        // rank sort by (key, original index): keys are distinct
        for (int e = lane; e < count; e += 32) {
            const Real ke = bk[e];
            const int oe = bo[e];
            int rank = 0;
            for (int f = 0; f < count; ++f) rank += (bk[f] < ke || (bk[f] == ke && bo[f] < oe)) ? 1 : 0;
            rnbr[c * (int64_t)cap + rank] = bj[e];
            rd2[c * (int64_t)cap + rank] = ke;
        }
        if (lane == 0) rlen[c] = count;
        __syncwarp();
    }
    if (lane == 0 && walk_cells) {
        atomicAdd(&st->walk_cells, (unsigned long long)walk_cells);
        atomicAdd(&st->walk_cands, (unsigned long long)walk_cands);
    }
}

}  // namespace

size_t range_smem_bytes(int precision)
{
    const size_t key = precision == VT_FP64 ? sizeof(double) : sizeof(float);
    // the far vertices of the second attempt: FP64 form only
    const size_t far = precision == VT_FP64 ? 4 * sizeof(float) * RANGE_VCAP : 0;
    return ((key + 2 * sizeof(int32_t)) * RANGE_CAP + far) * (RANGE_BLOCK / 32);
}

template <typename Real>
cudaError_t launch_range_t(const RangeArgs& a, cudaStream_t s)
{
    const size_t smem = range_smem_bytes(a.precision);
    auto kern = a.g.periodic ? k_range<Real, true> : k_range<Real, false>;
    // as many blocks as are resident at once (their warps take cells from the counter)
    int dev = 0, sms = 0, per_sm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, RANGE_BLOCK, smem);
    if (e == cudaSuccess) e = cudaMemsetAsync(a.queue, 0, sizeof(int32_t), s);
    if (e != cudaSuccess) return e;
    int64_t blocks = (a.nq + RANGE_BLOCK / 32 - 1) / (RANGE_BLOCK / 32);
    const int64_t resident = (int64_t)sms * (per_sm > 0 ? per_sm : 1);
    if (blocks > resident) blocks = resident;
    kern<<<(unsigned)blocks, RANGE_BLOCK, smem, s>>>(a.sorted, a.cell_off, a.g, a.sets, a.set_of, a.queries, a.nq,
                                                     a.nq_dev, a.nq_off, a.state, a.state_stride, a.pos_off, RANGE_CAP,
                                                     a.rnbr, (Real*)a.rd2, a.rlen, a.over_list, a.over_ctr, a.st,
                                                     a.queue);
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_range(const RangeArgs& a, cudaStream_t s)
{
    if (a.nq <= 0) return cudaSuccess;
    return a.precision == VT_FP64 ? launch_range_t<double>(a, s) : launch_range_t<float>(a, s);
}

}  // namespace vt
