// grid.cu -- stage 1: stable counting sort of the generators into a uniform
// grid (votess paper, Summary: the input points are sorted into a grid).
//
//   k_grid_count   : cell id per point + atomic histogram (the atomic's return
//                    value is a provisional rank inside the cell)
//   scan           : exclusive prefix sum of the counts -> cell offsets
//   k_grid_scatter : sorted[off[cid] + rank] = (x, y, z, original index bits)
//   k_grid_fix     : restores input order inside each grid cell (the atomic
//                    ranks are arbitrary): small cells by one thread,
//   k_grid_fix_big : large cells by a block-wide bitonic sort in place
//   k_grid_perm    : perm[sorted index] = original index
#include <limits.h>

#include "vt_internal.cuh"

namespace vt {

namespace {

constexpr int SMALL_CELL = 32;

// set of input point i: the last s with set_off[s] <= i (binary search)
__device__ __forceinline__ int set_of_point(const int64_t* __restrict__ set_off, int nsets, int64_t i)
{
    int lo = 0, hi = nsets - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (set_off[mid] <= i) lo = mid; else hi = mid - 1;
    }
    return lo;
}

__global__ void k_grid_count(const float* __restrict__ pts, int64_t n, GridDesc g0, const GridDesc* __restrict__ sets,
                             const int64_t* __restrict__ set_off, int nsets, int32_t* __restrict__ cid,
                             int32_t* __restrict__ ticket, int32_t* __restrict__ counts, DevStatus* st)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const GridDesc& g = sets ? sets[set_of_point(set_off, nsets, i)] : g0;
        float x = pts[3 * i], y = pts[3 * i + 1], z = pts[3 * i + 2];
        bool ok = (x >= g.lo[0]) & (x < g.hi[0]) & (y >= g.lo[1]) & (y < g.hi[1]) & (z >= g.lo[2]) & (z < g.hi[2]);
        if (!ok) {  // NaN fails every comparison
            atomicCAS((int*)&st->bad_point, 0, (int)(i + 1));
            x = g.lo[0]; y = g.lo[1]; z = g.lo[2];
        }
        int c = (int)g.cell_base + cell_id(cell_coord(x, g.lo[0], g.scale[0], g.G),
                                           cell_coord(y, g.lo[1], g.scale[1], g.G),
                                           cell_coord(z, g.lo[2], g.scale[2], g.G), g.G);
        cid[i] = c;
        ticket[i] = atomicAdd(&counts[c], 1);
    }
}

__global__ void k_grid_scatter(const float* __restrict__ pts, int64_t n, const int32_t* __restrict__ cid,
                               const int32_t* __restrict__ ticket, const int32_t* __restrict__ cell_off,
                               float4* __restrict__ sorted)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        int pos = cell_off[cid[i]] + ticket[i];
        sorted[pos] = make_float4(pts[3 * i], pts[3 * i + 1], pts[3 * i + 2], __int_as_float((int)i));
    }
}

// one thread per grid cell: insertion sort by original index for small cells,
// hand large ones to k_grid_fix_big
__global__ void k_grid_fix(float4* __restrict__ sorted, const int32_t* __restrict__ cell_off, int64_t g3,
                           int32_t* __restrict__ big, DevStatus* st)
{
    for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < g3; c += (int64_t)gridDim.x * blockDim.x) {
        int a = cell_off[c], m = cell_off[c + 1] - a;
        if (m <= 1) continue;
        if (m > SMALL_CELL) {
            int slot = atomicAdd(&st->n_big_cells, 1);
            big[slot] = (int)c;
            continue;
        }
        float4 buf[SMALL_CELL];
        for (int i = 0; i < m; ++i) buf[i] = sorted[a + i];
        for (int i = 1; i < m; ++i) {
            float4 v = buf[i];
            int key = __float_as_int(v.w);
            int j = i - 1;
            while (j >= 0 && __float_as_int(buf[j].w) > key) {
                buf[j + 1] = buf[j];
                --j;
            }
            buf[j + 1] = v;
        }
        for (int i = 0; i < m; ++i) sorted[a + i] = buf[i];
    }
}

// keys a block sorts in shared memory (48 KB); larger cells sort in place
constexpr int FIX_SMEM_KEYS = 12288;

// one block per large grid cell: bitonic sort of sorted[a, a+m) by original
// index. Every comparator orders ascending (first step of each merge compares
// mirrored pairs). A cell of up to FIX_SMEM_KEYS points sorts its keys (the
// original indices) in shared memory, padded to a power of two with INT_MAX,
// and rebuilds its entries from the input points; a larger cell runs the same
// network in place in global memory, padding virtually (a comparator touching
// the padding is a no-op).
__global__ void __launch_bounds__(512) k_grid_fix_big(const float* __restrict__ pts, float4* __restrict__ sorted,
                                                      const int32_t* __restrict__ cell_off,
                                                      const int32_t* __restrict__ big, const DevStatus* st)
{
    __shared__ int32_t key[FIX_SMEM_KEYS];
    const int nbig = st->n_big_cells;
    for (int b = blockIdx.x; b < nbig; b += gridDim.x) {
        const int c = big[b];
        const int a = cell_off[c], m = cell_off[c + 1] - a;
        float4* s = sorted + a;
        int P = 1;
        while (P < m) P <<= 1;
        if (P <= FIX_SMEM_KEYS) {
            for (int t = threadIdx.x; t < P; t += blockDim.x) key[t] = t < m ? __float_as_int(s[t].w) : INT_MAX;
            __syncthreads();
            for (int size = 2; size <= P; size <<= 1) {
                const int half = size >> 1;
                for (int t = threadIdx.x; t < P / 2; t += blockDim.x) {  // mirrored step
                    const int blk = t / half, off = t % half;
                    const int i = blk * size + off, j = blk * size + size - 1 - off;
                    const int u = key[i], v = key[j];
                    if (u > v) { key[i] = v; key[j] = u; }
                }
                __syncthreads();
                for (int h = half >> 1; h >= 1; h >>= 1) {  // half-cleaners
                    for (int t = threadIdx.x; t < P / 2; t += blockDim.x) {
                        const int blk = t / h, off = t % h;
                        const int i = blk * 2 * h + off, j = i + h;
                        const int u = key[i], v = key[j];
                        if (u > v) { key[i] = v; key[j] = u; }
                    }
                    __syncthreads();
                }
            }
            for (int t = threadIdx.x; t < m; t += blockDim.x) {
                const int64_t o = key[t];
                s[t] = make_float4(pts[3 * o], pts[3 * o + 1], pts[3 * o + 2], __int_as_float((int)o));
            }
            __syncthreads();  // the next cell reuses key[]
            continue;
        }
        for (int size = 2; size <= P; size <<= 1) {
            const int half = size >> 1;
            for (int t = threadIdx.x; t < P / 2; t += blockDim.x) {  // mirrored step
                int blk = t / half, off = t % half;
                int i = blk * size + off, j = blk * size + size - 1 - off;
                if (j < m) {
                    float4 u = s[i], v = s[j];
                    if (__float_as_int(u.w) > __float_as_int(v.w)) { s[i] = v; s[j] = u; }
                }
            }
            __syncthreads();
            for (int h = half >> 1; h >= 1; h >>= 1) {  // half-cleaners
                for (int t = threadIdx.x; t < P / 2; t += blockDim.x) {
                    int blk = t / h, off = t % h;
                    int i = blk * 2 * h + off, j = i + h;
                    if (j < m) {
                        float4 u = s[i], v = s[j];
                        if (__float_as_int(u.w) > __float_as_int(v.w)) { s[i] = v; s[j] = u; }
                    }
                }
                __syncthreads();
            }
        }
        __syncthreads();
    }
}

__global__ void k_grid_perm(const float4* __restrict__ sorted, int64_t n, int32_t* __restrict__ perm,
                            const int64_t* __restrict__ set_off, int nsets, int32_t* __restrict__ set_of)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int o = __float_as_int(sorted[i].w);
        perm[i] = o;
        if (set_of) set_of[i] = set_of_point(set_off, nsets, o);
    }
}

unsigned blocks_for(int64_t n, int threads)
{
    int64_t b = (n + threads - 1) / threads;
    if (b < 1) b = 1;
    if (b > 152 * 64) b = 152 * 64;  // grid-stride beyond 64 waves of the 152 SMs
    return (unsigned)b;
}

// sum over grid cells of n_c (n_c - 1), per set (exact 64-bit integer sums);
// the set of global cell c is the last s with cell_base <= c
__global__ void k_pair_counts(const int32_t* __restrict__ cell_off, int64_t g3, const GridDesc* __restrict__ sets,
                              int nsets, unsigned long long* __restrict__ acc)
{
    for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < g3; c += (int64_t)gridDim.x * blockDim.x) {
        const long long m = (long long)cell_off[c + 1] - cell_off[c];
        if (m < 2) continue;
        int s = 0;
        if (sets) {
            int lo = 0, hi = nsets - 1;
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (sets[mid].cell_base <= c) lo = mid; else hi = mid - 1;
            }
            s = lo;
        }
        atomicAdd(&acc[s], (unsigned long long)(m * (m - 1)));
    }
}

}  // namespace

cudaError_t launch_pair_counts(const int32_t* cell_off, int64_t g3, const GridDesc* sets, int nsets,
                               unsigned long long* acc, cudaStream_t s)
{
    cudaError_t e = cudaMemsetAsync(acc, 0, sizeof(unsigned long long) * (nsets > 0 ? nsets : 1), s);
    if (e != cudaSuccess) return e;
    k_pair_counts<<<blocks_for(g3, 256), 256, 0, s>>>(cell_off, g3, sets, nsets, acc);
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_grid_build(const float* pts, int64_t n, const GridDesc& g, float4* sorted, int32_t* perm,
                              int32_t* cell_off, int32_t* cid, int32_t* ticket, int32_t* counts, int32_t* big,
                              void* scan_tmp, DevStatus* st, cudaStream_t s, const BatchArgs* batch, int64_t g3)
{
    if (g3 < 0) g3 = (int64_t)g.G * g.G * g.G;
    const GridDesc* sets = batch ? batch->sets : nullptr;
    const int64_t* set_off = batch ? batch->set_off : nullptr;
    const int nsets = batch ? batch->nsets : 1;
    int32_t* set_of = batch ? batch->set_of : nullptr;
    cudaError_t e = cudaMemsetAsync(counts, 0, (size_t)g3 * sizeof(int32_t), s);
    if (e != cudaSuccess) return e;
    if (n > 0) {
        k_grid_count<<<blocks_for(n, 256), 256, 0, s>>>(pts, n, g, sets, set_off, nsets, cid, ticket, counts, st);
        count_launch();
    }
    exclusive_scan_i32(counts, cell_off, g3, scan_tmp, s);
    if (n == 0) return cudaGetLastError();
    k_grid_scatter<<<blocks_for(n, 256), 256, 0, s>>>(pts, n, cid, ticket, cell_off, sorted);
    k_grid_fix<<<blocks_for(g3, 128), 128, 0, s>>>(sorted, cell_off, g3, big, st);
    k_grid_fix_big<<<152 * 2, 512, 0, s>>>(pts, sorted, cell_off, big, st);
    k_grid_perm<<<blocks_for(n, 256), 256, 0, s>>>(sorted, n, perm, set_off, nsets, set_of);
    count_launch(4);
    return cudaGetLastError();
}

}  // namespace vt
