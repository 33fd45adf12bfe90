// knn.cu -- stage 2: k nearest neighbours per generator (votess paper,
// Summary: a k-nearest-neighbour search over the grid-sorted points).
//
// One warp per query. The warp walks Chebyshev shells s = 0, 1, 2, ... of
// grid cells around the query's cell. Cells (x, y, z..z') with consecutive z
// are consecutive in the sorted array, so each (x, y) row of a shell is one
// contiguous, coalesced float4 range; the 32 lanes take 32 candidates at a
// time. The k best candidates so far live in a sorted list spread over the
// warp's registers (entry e = r*32 + lane, KPL registers per lane); a
// qualifying candidate is inserted with one ballot per register row and one
// shuffle-shift. In the one-row float32 lists (k <= 32) qualifying candidates
// first collect in a per-warp buffer of 32 in shared memory, which joins the
// list by one bitonic sort and merge when it is full or the shell ends (a few
// by single insertion). After each shell the walk stops once the list is full and the
// k-th distance is no larger than the distance from the query to the outside
// of the scanned block (minus a rounding margin), or the block covers the grid.
#include <float.h>
#include <limits.h>

#include "vt_internal.cuh"

namespace vt {

namespace {

constexpr unsigned FULL = 0xffffffffu;

// batches with at least this many qualifying candidates are merged into the
// list by bitonic networks; smaller ones are inserted one at a time
#ifndef VT_KNN_MERGE_MIN
#define VT_KNN_MERGE_MIN 12
#endif
// one-row float32 lists: qualifying candidates wait in a per-warp buffer of 32
// and join the list by one sort-and-merge when it fills or the shell ends
// (buffers of at most this many are inserted one at a time instead)
// (measured on the 1M mixed cloud: 12 against 6; merging at 16 buffered
// entries instead of 32, or inserting batches of 2 or 4 at once, was slower)
#ifndef VT_KNN_FLUSH_SINGLE
#define VT_KNN_FLUSH_SINGLE 12
#endif
constexpr int KNN_BLOCK = 256;

template <typename Real>
struct Dist;

template <>
struct Dist<double> {
    // the exact key of the FP64 form: ((dx*dx + dy*dy) + dz*dz), no contraction
    static __device__ __forceinline__ double d2(float4 a, float4 b) { return knn_d2_f64(a, b); }
    static __device__ __forceinline__ double inf() { return __longlong_as_double(0x7ff0000000000000ll); }
};

template <>
struct Dist<float> {
    static __device__ __forceinline__ float d2(float4 a, float4 b) { return knn_d2_f32(a, b); }
    static __device__ __forceinline__ float inf() { return __int_as_float(0x7f800000); }
};

template <typename Real>
__device__ __forceinline__ bool key_less(Real da, int oa, Real db, int ob)
{
    return da < db || (da == db && oa < ob);
}

template <typename Real, int KPL>
struct WarpList {
    Real d[KPL];
    int o[KPL];  // original index (tie-break key)
    int j[KPL];  // sorted index (payload)

    __device__ void init()
    {
#pragma unroll
        for (int r = 0; r < KPL; ++r) { d[r] = Dist<Real>::inf(); o[r] = INT_MAX; j[r] = -1; }
    }

    // inserts (cd, co, cj) if it ranks among the first k; warp-uniform call
    __device__ void insert(Real cd, int co, int cj, int k, int lane)
    {
        int p = 0;
#pragma unroll
        for (int r = 0; r < KPL; ++r) p += __popc(__ballot_sync(FULL, key_less(d[r], o[r], cd, co)));
        if (p >= k) return;
        Real nd[KPL];
        int no[KPL], nj[KPL];
#pragma unroll
        for (int r = 0; r < KPL; ++r) {
            Real ud = __shfl_up_sync(FULL, d[r], 1);
            int uo = __shfl_up_sync(FULL, o[r], 1);
            int uj = __shfl_up_sync(FULL, j[r], 1);
            Real wd = ud;
            int wo = uo, wj = uj;
            if (r > 0) {
                wd = __shfl_sync(FULL, d[r - 1], 31);
                wo = __shfl_sync(FULL, o[r - 1], 31);
                wj = __shfl_sync(FULL, j[r - 1], 31);
            }
            Real pd = lane == 0 ? wd : ud;
            int po = lane == 0 ? wo : uo, pj = lane == 0 ? wj : uj;
            int e = r * 32 + lane;
            nd[r] = e > p ? pd : (e == p ? cd : d[r]);
            no[r] = e > p ? po : (e == p ? co : o[r]);
            nj[r] = e > p ? pj : (e == p ? cj : j[r]);
        }
#pragma unroll
        for (int r = 0; r < KPL; ++r) { d[r] = nd[r]; o[r] = no[r]; j[r] = nj[r]; }
    }

    // key of entry e (warp-uniform e)
    __device__ void entry(int e, Real& kd, int& ko) const
    {
        Real dd = d[0];
        int oo = o[0];
#pragma unroll
        for (int r = 1; r < KPL; ++r)
            if (r == e / 32) { dd = d[r]; oo = o[r]; }
        kd = __shfl_sync(FULL, dd, e % 32);
        ko = __shfl_sync(FULL, oo, e % 32);
    }
};

// One compare-exchange stage of a warp-wide bitonic network over (key,
// original index, payload), one element per lane: partner lane ^ j; the lane
// keeps the smaller of the pair when it is the lower lane of an ascending
// block (or the upper lane of a descending one).
__device__ __forceinline__ void bitonic_step(float& d, int& o, int& jv, int j, bool asc, int lane)
{
    const float pd = __shfl_xor_sync(FULL, d, j);
    const int po = __shfl_xor_sync(FULL, o, j);
    const int pj = __shfl_xor_sync(FULL, jv, j);
    const bool lower = (lane & j) == 0;
    const bool partner_less = pd < d || (pd == d && po < o);
    const bool take = (lower == asc) ? partner_less : (!partner_less && !(pd == d && po == o));
    if (take) { d = pd; o = po; jv = pj; }
}

// sorts 32 elements ascending (one per lane)
__device__ __forceinline__ void bitonic_sort32(float& d, int& o, int& jv, int lane)
{
#pragma unroll
    for (int k = 2; k <= 32; k <<= 1)
#pragma unroll
        for (int j = k >> 1; j > 0; j >>= 1) bitonic_step(d, o, jv, j, (lane & k) == 0 || k == 32, lane);
}

// merges a sorted batch into the sorted list (both ascending, one element per
// lane), keeping the 32 smallest: the element-wise minimum of the list and
// the reversed batch is bitonic, and one merge network sorts it
__device__ __forceinline__ void merge32(float& ld, int& lo, int& lj, float bd, int bo, int bj, int lane)
{
    const float rd = __shfl_sync(FULL, bd, 31 - lane);
    const int ro = __shfl_sync(FULL, bo, 31 - lane), rj = __shfl_sync(FULL, bj, 31 - lane);
    if (rd < ld || (rd == ld && ro < lo)) { ld = rd; lo = ro; lj = rj; }
#pragma unroll
    for (int j = 16; j > 0; j >>= 1) bitonic_step(ld, lo, lj, j, true, lane);
}

// Moves the warp's buffered candidates (nb of them, in bd/bo/bj) into the
// one-row list: a few by single insertion, more by one bitonic sort and merge.
// Updates count and, once the list holds k entries, the k-th key (kd, ko).
template <int KPL>
__device__ __forceinline__ void flush_buffer(WarpList<float, KPL>& L, const float* bd, const int* bo, const int* bj,
                                             int nb, int k, int& count, float& kd, int& ko, int lane)
{
    if (nb <= VT_KNN_FLUSH_SINGLE) {
        for (int i = 0; i < nb; ++i) {
            // a buffered candidate may have been overtaken by earlier ones
            if (count == k && !key_less(bd[i], bo[i], kd, ko)) continue;
            L.insert(bd[i], bo[i], bj[i], k, lane);
            if (count < k) ++count;
            if (count == k) L.entry(k - 1, kd, ko);
        }
        return;
    }
    float d = lane < nb ? bd[lane] : __int_as_float(0x7f800000);
    int o = lane < nb ? bo[lane] : INT_MAX, j = lane < nb ? bj[lane] : -1;
    bitonic_sort32(d, o, j, lane);
    merge32(L.d[0], L.o[0], L.j[0], d, o, j, lane);
    count = count + nb < k ? count + nb : k;
    if (count == k) L.entry(k - 1, kd, ko);
}

// The FP64 form's list: entries keep the float32 key f (relative error below
// 3e-7 of the exact distance) and the exact FP64 key d, computed only when
// two float32 keys are too close to order (within 2e-6) or at the end (d is
// NaN until then). Orders are the FP64 keys' (with ties by original index),
// so the list equals one built from FP64 keys throughout, with far fewer
// FP64 operations (the part's FP64 rate is 1/64 of float32).
template <int KPL>
struct WarpList64 {
    float f[KPL];
    double d[KPL];
    int o[KPL];
    int j[KPL];

    __device__ void init()
    {
#pragma unroll
        for (int r = 0; r < KPL; ++r) {
            f[r] = __int_as_float(0x7f800000);
            d[r] = __longlong_as_double(0x7ff0000000000000ll);
            o[r] = INT_MAX;
            j[r] = -1;
        }
    }

    // inserts the candidate (float key cf, original index co, sorted index cj)
    // if it ranks among the first k; warp-uniform call
    __device__ void insert(float cf, int co, int cj, float4 pq, const float4* __restrict__ sorted, const GridDesc& g,
                           int k, int lane)
    {
        const double nanv = __longlong_as_double(0x7ff8000000000000ll);
        double cd = nanv;  // the candidate's exact key, when needed
        int p = 0;
#pragma unroll
        for (int r = 0; r < KPL; ++r) {
            bool less = f[r] < cf * (1.0f - 2e-6f);
            const bool amb = !less && f[r] <= cf * (1.0f + 2e-6f) && o[r] != INT_MAX;
            if (__any_sync(FULL, amb)) {
                if (isnan(cd)) cd = img_key64(pq, sorted, cj, g);  // uniform
                if (amb) {
                    if (isnan(d[r])) d[r] = img_key64(pq, sorted, j[r], g);
                    less = d[r] < cd || (d[r] == cd && o[r] < co);
                }
            }
            p += __popc(__ballot_sync(FULL, less));
        }
        if (p >= k) return;
        float nf[KPL];
        double nd[KPL];
        int no[KPL], nj[KPL];
#pragma unroll
        for (int r = 0; r < KPL; ++r) {
            float uf = __shfl_up_sync(FULL, f[r], 1);
            double ud = __shfl_up_sync(FULL, d[r], 1);
            int uo = __shfl_up_sync(FULL, o[r], 1);
            int uj = __shfl_up_sync(FULL, j[r], 1);
            if (r > 0) {
                const float wf = __shfl_sync(FULL, f[r - 1], 31);
                const double wd = __shfl_sync(FULL, d[r - 1], 31);
                const int wo = __shfl_sync(FULL, o[r - 1], 31), wj = __shfl_sync(FULL, j[r - 1], 31);
                if (lane == 0) { uf = wf; ud = wd; uo = wo; uj = wj; }
            }
            const int e = r * 32 + lane;
            nf[r] = e > p ? uf : (e == p ? cf : f[r]);
            nd[r] = e > p ? ud : (e == p ? cd : d[r]);
            no[r] = e > p ? uo : (e == p ? co : o[r]);
            nj[r] = e > p ? uj : (e == p ? cj : j[r]);
        }
#pragma unroll
        for (int r = 0; r < KPL; ++r) { f[r] = nf[r]; d[r] = nd[r]; o[r] = no[r]; j[r] = nj[r]; }
    }

    // float key of entry e (warp-uniform e)
    __device__ float key(int e) const
    {
        float ff = f[0];
#pragma unroll
        for (int r = 1; r < KPL; ++r)
            if (r == e / 32) ff = f[r];
        return __shfl_sync(FULL, ff, e % 32);
    }

    // every entry's exact key
    __device__ void finish(float4 pq, const float4* __restrict__ sorted, const GridDesc& g)
    {
#pragma unroll
        for (int r = 0; r < KPL; ++r)
            if (isnan(d[r]) && j[r] >= 0) d[r] = img_key64(pq, sorted, j[r], g);
    }
};

// resident blocks per SM the one-row lists are compiled for: 5 blocks of 256
// threads (48 registers) hide more of the walk's load latency than 4 or 3
// (measured on the 1M mixed cloud with the work queue: kNN stage 6.17 ms at 5,
// 6.19 at 4, 6.91 at 3)
#ifndef VT_KNN_MINB
#define VT_KNN_MINB 5
#endif
template <typename Real, int KPL, bool PER>
__global__ void __launch_bounds__(KNN_BLOCK, (KPL == 1 ? VT_KNN_MINB : 1)) k_knn(const float4* __restrict__ sorted, const int32_t* __restrict__ cell_off0,
                                             const __grid_constant__ GridDesc g0, const GridDesc* __restrict__ sets,
                                             const int32_t* __restrict__ set_of, const int32_t* __restrict__ queries,
                                             int64_t nq_host, const int32_t* __restrict__ nq_dev,
                                             int64_t nq_off, int k,
                                             int32_t* __restrict__ nbr, Real* __restrict__ d2out, DevStatus* st,
                                             int32_t* __restrict__ queue)
{
    const int lane = threadIdx.x & 31;
    // candidate buffer of the warp (one-row float32 lists)
    __shared__ float s_bd[KNN_BLOCK / 32][32];
    __shared__ int s_bo[KNN_BLOCK / 32][32], s_bj[KNN_BLOCK / 32][32];
    float* bufd = s_bd[threadIdx.x >> 5];
    int* bufo = s_bo[threadIdx.x >> 5];
    int* bufj = s_bj[threadIdx.x >> 5];
    constexpr bool BUF = sizeof(Real) == 4 && KPL == 1;
    int64_t nq = nq_host;
    if (nq_dev) {  // device-counted: this launch takes entries [nq_off, nq_off + nq_host) of the list
        const int64_t want = (int64_t)*nq_dev - nq_off;
        nq = want < 0 ? 0 : (want < nq_host ? want : nq_host);
    }
    // statistics: candidates examined (the query itself included) and
    // queries answered, added once per warp
    unsigned long long evals = 0, answered = 0;
    // queries come from a launch-wide counter, one per warp at a time (their
    // costs differ by orders of magnitude between clumps and voids)
    auto next_query = [&]() {
        int v = 0;
        if (lane == 0) v = atomicAdd(queue, 1);
        return (int64_t)__shfl_sync(FULL, v, 0);
    };
    for (int64_t c = next_query(); c < nq; c = next_query()) {
        ++answered;
        const int q = queries ? queries[c] : (int)c;
        const float4 pq = sorted[q];
        const GridDesc& g = grid_of(g0, sets, set_of, q);
        const int G = g.G;
        const int32_t* cell_off = cell_off0 + g.cell_base;
        const int ix = cell_coord(pq.x, g.lo[0], g.scale[0], G);
        const int iy = cell_coord(pq.y, g.lo[1], g.scale[1], G);
        const int iz = cell_coord(pq.z, g.lo[2], g.scale[2], G);
        constexpr bool F64 = sizeof(Real) == 8;
        WarpList<float, KPL> L;    // FP32 form
        WarpList64<KPL> L64;       // FP64 form
        if (F64) L64.init(); else L.init();
        int count = 0;
        int nb = 0;  // buffered candidates
        float kd = __int_as_float(0x7f800000);  // float key of the k-th entry once the list is full
        int ko = INT_MAX;
        bool dup = false;
        // periodic box: candidates are the images of the other generators; no
        // image farther than |L| can cut a cell, so the walk ends there
        constexpr bool per = PER;
        const float lim2 = per ? period_norm2(g) * (1.0f + 1e-4f) : 0.0f;

        for (int s = 0;; ++s) {
            // the shell's segments, 32 at a time: lanes load segment bounds in
            // parallel, then the segments' candidates are spread over all lanes
            // a periodic shell that stays inside the grid is walked like a walled one
            const bool wrap = per && (ix - s < 0 || iy - s < 0 || iz - s < 0 || ix + s >= G || iy + s >= G || iz + s >= G);
            const int M = wrap ? seg_per_row_outer(g, s) : 2;
            const int nseg = M * (2 * s + 1) * (2 * s + 1);
            for (int e0 = 0; e0 < nseg; e0 += 32) {
                // once the list is full, only grid cells that reach into the
                // ball of the current k-th distance can hold a better candidate
                int sa = 0, sb = 0, sc = IMG_NONE;
                if (e0 + lane < nseg) {
                    if (wrap)
                        shell_segment_outer_p(e0 + lane, s, M, ix, iy, iz, g, cell_off, pq,
                                              count == k ? fminf(kd * (1.0f + 1e-5f), lim2) : lim2, sa, sb, sc);
                    else if (count == k)
                        shell_segment_ball(e0 + lane, s, ix, iy, iz, g, cell_off, pq, kd * (1.0f + 1e-5f), -1.0f, sa,
                                           sb);
                    else
                        shell_segment(e0 + lane, s, ix, iy, iz, G, cell_off, sa, sb);
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
                evals += (unsigned)total;
                for (int c0 = 0; c0 < total; c0 += 32) {
                    const int i = c0 + lane;
                    int seg = 0;  // number of segments ending at or before i
#pragma unroll
                    for (int step = 16; step >= 1; step >>= 1)
                        if (__shfl_sync(FULL, incl, (seg + step - 1) & 31) <= i) seg += step;
                    const int aj = __shfl_sync(FULL, sa, seg & 31), sj = __shfl_sync(FULL, start, seg & 31);
                    const int code = per ? __shfl_sync(FULL, sc, seg & 31) : IMG_NONE;
                    const int j0 = aj + (i - sj);
                    const bool valid = i < total && j0 != q;  // (all of the query's own images)
                    const int jj = per ? img_pack(j0, code) : j0;
                    float cd = __int_as_float(0x7f800000);
                    int co = INT_MAX;
                    bool cand = false;
                    if (valid) {
                        const float4 pc = sorted[j0];
                        if (per) {
                            co = img_tie(pc, code, g);
                            if (code == IMG_NONE && pc.x == pq.x && pc.y == pq.y && pc.z == pq.z) dup = true;
                            cd = key_f32(img_off(pq, pc, code, g));
                        } else {
                            co = __float_as_int(pc.w);
                            if (pc.x == pq.x && pc.y == pq.y && pc.z == pq.z) dup = true;
                            cd = knn_d2_f32(pq, pc);
                        }
                        // FP64 form: the float key only rules out candidates clearly
                        // beyond the k-th entry; insert() orders the close ones exactly
                        cand = count < k || (F64 ? cd <= kd * (1.0f + 2e-6f) : key_less(cd, co, kd, ko));
                    }
                    unsigned m = __ballot_sync(FULL, cand);
                    if (BUF) {
                        // into the buffer; a full buffer is merged and the rest
                        // of the batch re-tested against the new k-th key
                        int add = __popc(m);
                        int rank = __popc(m & ((1u << lane) - 1u));
                        while (add > 0) {
                            const int room = 32 - nb;
                            if (cand && rank < room) {
                                bufd[nb + rank] = cd;
                                bufo[nb + rank] = co;
                                bufj[nb + rank] = jj;
                            }
                            if (add < room) {
                                nb += add;
                                break;
                            }
                            __syncwarp();
                            flush_buffer<KPL>(L, bufd, bufo, bufj, 32, k, count, kd, ko, lane);
                            nb = 0;
                            __syncwarp();
                            cand = cand && rank >= room && (count < k || key_less(cd, co, kd, ko));
                            m = __ballot_sync(FULL, cand);
                            add = __popc(m);
                            rank = __popc(m & ((1u << lane) - 1u));
                        }
                        m = 0;
                    }
                    if (!BUF && !F64 && KPL == 1 && __popc(m) >= VT_KNN_MERGE_MIN) {
                        // many candidates at once (the list filling up): sort the
                        // batch and merge it into the list with bitonic networks
                        float bd = cand ? cd : __int_as_float(0x7f800000);
                        int bo = cand ? co : INT_MAX, bj = cand ? jj : -1;
                        bitonic_sort32(bd, bo, bj, lane);
                        merge32(L.d[0], L.o[0], L.j[0], bd, bo, bj, lane);
                        count = count + __popc(m) < k ? count + __popc(m) : k;
                        if (count == k) L.entry(k - 1, kd, ko);
                        m = 0;
                    }
                    while (m) {
                        const int src = __ffs(m) - 1;
                        m &= m - 1;
                        const float bd = __shfl_sync(FULL, cd, src);
                        const int bo = __shfl_sync(FULL, co, src);
                        const int bj = __shfl_sync(FULL, jj, src);
                        if (F64) {
                            L64.insert(bd, bo, bj, pq, sorted, g, k, lane);
                            if (count < k) ++count;
                            if (count == k) kd = L64.key(k - 1);
                        } else {
                            L.insert(bd, bo, bj, k, lane);
                            if (count < k) ++count;
                            if (count == k) L.entry(k - 1, kd, ko);
                        }
                    }
                }
            }
            if (BUF && nb > 0) {  // the shell's candidates join the list before the stop test
                __syncwarp();
                flush_buffer<KPL>(L, bufd, bufo, bufj, nb, k, count, kd, ko, lane);
                nb = 0;
                __syncwarp();
            }
            // stop rule
            if (per) {
                const float gap = shell_gap_p(g, pq, ix, iy, iz, s);
                if (count == k && gap > 0.0f && kd * (1.0f + 2e-6f) <= gap * gap * (1.0f - 1e-5f)) break;
                if (gap > 0.0f && gap * gap >= lim2) break;  // every image that can cut is listed
                continue;
            }
            const bool covers = ix - s <= 0 && iy - s <= 0 && iz - s <= 0 && ix + s >= G - 1 && iy + s >= G - 1 &&
                                iz + s >= G - 1;
            if (covers) break;
            if (count == k) {
                const float gap = shell_gap(g, pq, ix, iy, iz, s);
                if (gap > 0.0f && kd * (1.0f + 2e-6f) <= gap * gap * (1.0f - 1e-5f)) break;
            }
        }
        if (__any_sync(FULL, dup) && lane == 0) atomicExch((int*)&st->duplicate, 1);
        if (F64) L64.finish(pq, sorted, g);
#pragma unroll
        for (int r = 0; r < KPL; ++r) {
            const int e = r * 32 + lane;
            if (e < k) {
                nbr[c * k + e] = F64 ? L64.j[r] : L.j[r];
                if (d2out) d2out[c * k + e] = F64 ? (Real)L64.d[r] : (Real)L.d[r];
            }
        }
    }
    if (lane == 0 && answered) {
        atomicAdd(&st->knn_evals, evals);
        atomicAdd(&st->knn_queries, answered);
    }
}

template <typename Real>
cudaError_t launch_knn_t(const float4* sorted, const int32_t* cell_off, const GridDesc& g, const GridDesc* sets,
                         const int32_t* set_of, const int32_t* queries, int64_t nq, const int32_t* nq_dev,
                         int64_t nq_off, int k,
                         int32_t* nbr, Real* d2, DevStatus* st, cudaStream_t s, int32_t* queue)
{
    if (nq <= 0) return cudaSuccess;
    // the periodic walk is its own instantiation (the non-periodic kernels keep their registers)
    auto kern = k <= 32 ? (g.periodic ? k_knn<Real, 1, true> : k_knn<Real, 1, false>)
              : k <= 64 ? (g.periodic ? k_knn<Real, 2, true> : k_knn<Real, 2, false>)
              : k <= 128 ? (g.periodic ? k_knn<Real, 4, true> : k_knn<Real, 4, false>)
                         : (g.periodic ? k_knn<Real, 8, true> : k_knn<Real, 8, false>);
    // as many blocks as are resident at once (their warps take queries from the counter)
    int dev = 0, sms = 0, per_sm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, KNN_BLOCK, 0);
    if (e == cudaSuccess) e = cudaMemsetAsync(queue, 0, sizeof(int32_t), s);
    if (e != cudaSuccess) return e;
    int64_t blocks = (nq + KNN_BLOCK / 32 - 1) / (KNN_BLOCK / 32);
    const int64_t resident = (int64_t)sms * (per_sm > 0 ? per_sm : 1);
    if (blocks > resident) blocks = resident;
    dim3 grid((unsigned)blocks), block(KNN_BLOCK);
    kern<<<grid, block, 0, s>>>(sorted, cell_off, g, sets, set_of, queries, nq, nq_dev, nq_off, k, nbr, d2, st, queue);
    count_launch();
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_knn(const float4* sorted, const int32_t* cell_off, const GridDesc& g, int64_t n,
                       const int32_t* queries, int64_t nq, int k, int precision, int32_t* nbr, void* d2,
                       DevStatus* st, cudaStream_t s, const GridDesc* sets, const int32_t* set_of,
                       const int32_t* nq_dev, int64_t nq_off, int32_t* queue)
{
    (void)n;
    if (k < 1 || k > 256 || !queue) return cudaErrorInvalidValue;
    if (precision == VT_FP64)
        return launch_knn_t<double>(sorted, cell_off, g, sets, set_of, queries, nq, nq_dev, nq_off, k, nbr, (double*)d2, st,
                                    s, queue);
    return launch_knn_t<float>(sorted, cell_off, g, sets, set_of, queries, nq, nq_dev, nq_off, k, nbr, (float*)d2, st,
                               s, queue);
}

}  // namespace vt
