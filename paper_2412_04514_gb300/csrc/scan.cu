// scan.cu -- grid-wide exclusive prefix sums (cell offsets of the grid sort,
// CSR offsets of the outputs). Three phases per level: block scan with block
// totals, recursive scan of the totals, add-back. out has n+1 entries:
// out[n] receives the grand total.
#include "vt_internal.cuh"

namespace vt {

namespace {

constexpr int SCAN_THREADS = 256;
constexpr int SCAN_ITEMS = 4;
constexpr int SCAN_TILE = SCAN_THREADS * SCAN_ITEMS;  // 1024 elements per block

template <typename TO>
__device__ __forceinline__ TO warp_inclusive(TO v, int lane)
{
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        TO u = __shfl_up_sync(0xffffffffu, v, d);
        if (lane >= d) v += u;
    }
    return v;
}

// Exclusive scan of one 1024-element tile per block. in and out may alias.
// Writes the tile total to tile_sum[blockIdx.x] (if non-null) and, for a
// single-tile scan, the grand total to out[n].
template <typename TI, typename TO>
__global__ void __launch_bounds__(SCAN_THREADS) k_scan_tile(const TI* in, TO* out, TO* tile_sum, int64_t n)
{
    __shared__ TO warp_tot[SCAN_THREADS / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t base = (int64_t)blockIdx.x * SCAN_TILE + (int64_t)threadIdx.x * SCAN_ITEMS;
    TO v[SCAN_ITEMS];
    TO tsum = 0;
#pragma unroll
    for (int i = 0; i < SCAN_ITEMS; ++i) {
        int64_t idx = base + i;
        v[i] = idx < n ? (TO)in[idx] : (TO)0;
        tsum += v[i];
    }
    TO incl = warp_inclusive<TO>(tsum, lane);
    if (lane == 31) warp_tot[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        TO w = lane < SCAN_THREADS / 32 ? warp_tot[lane] : (TO)0;
        TO wi = warp_inclusive<TO>(w, lane);
        if (lane < SCAN_THREADS / 32) warp_tot[lane] = wi - w;
    }
    __syncthreads();
    TO run = incl - tsum + warp_tot[warp];
#pragma unroll
    for (int i = 0; i < SCAN_ITEMS; ++i) {
        int64_t idx = base + i;
        if (idx < n) out[idx] = run;
        run += v[i];
    }
    if (threadIdx.x == SCAN_THREADS - 1) {
        if (tile_sum) tile_sum[blockIdx.x] = run;
        if (gridDim.x == 1) out[n] = run;
    }
}

template <typename TO>
__global__ void k_scan_add(TO* out, const TO* tile_off, int64_t n)
{
    const int64_t base = (int64_t)blockIdx.x * SCAN_TILE;
    const TO add = tile_off[blockIdx.x];
    for (int i = threadIdx.x; i < SCAN_TILE; i += blockDim.x) {
        int64_t idx = base + i;
        if (idx < n) out[idx] += add;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) out[n] = tile_off[gridDim.x];
}

int64_t tiles(int64_t n) { return (n + SCAN_TILE - 1) / SCAN_TILE; }

template <typename TI, typename TO>
void scan_rec(const TI* in, TO* out, int64_t n, int64_t* tmp, cudaStream_t s)
{
    int64_t nb = tiles(n);
    if (nb <= 1) {
        k_scan_tile<TI, TO><<<1, SCAN_THREADS, 0, s>>>(in, out, (TO*)nullptr, n);
        count_launch();
        return;
    }
    // tile totals in tmp[0..nb], scanned in place (tmp[nb] = grand total)
    int64_t* sums = tmp;
    k_scan_tile<TI, TO><<<(unsigned)nb, SCAN_THREADS, 0, s>>>(in, out, (TO*)sums, n);
    count_launch();
    scan_rec<int64_t, int64_t>(sums, sums, nb, tmp + nb + 1, s);
    k_scan_add<TO><<<(unsigned)nb, SCAN_THREADS, 0, s>>>(out, (const TO*)sums, n);
    count_launch();
}

// the int32 -> int32 path keeps 64-bit tile totals
template <>
void scan_rec<int32_t, int32_t>(const int32_t* in, int32_t* out, int64_t n, int64_t* tmp, cudaStream_t s)
{
    int64_t nb = tiles(n);
    if (nb <= 1) {
        k_scan_tile<int32_t, int32_t><<<1, SCAN_THREADS, 0, s>>>(in, out, (int32_t*)nullptr, n);
        count_launch();
        return;
    }
    int32_t* sums = (int32_t*)tmp;
    k_scan_tile<int32_t, int32_t><<<(unsigned)nb, SCAN_THREADS, 0, s>>>(in, out, sums, n);
    count_launch();
    int64_t* next = tmp + (nb + 2) / 2 + 1;
    scan_rec<int32_t, int32_t>(sums, sums, nb, next, s);
    k_scan_add<int32_t><<<(unsigned)nb, SCAN_THREADS, 0, s>>>(out, sums, n);
    count_launch();
}

}  // namespace

size_t scan_tmp_bytes(int64_t n)
{
    size_t total = 0;
    int64_t m = n;
    while (true) {
        int64_t nb = tiles(m);
        if (nb <= 1) break;
        total += (size_t)(nb + 2) * sizeof(int64_t);
        m = nb;
    }
    return total + 64;
}

void exclusive_scan_i32(const int32_t* in, int32_t* out, int64_t n, void* tmp, cudaStream_t s)
{
    scan_rec<int32_t, int32_t>(in, out, n, (int64_t*)tmp, s);
}

void exclusive_scan_i32_to_i64(const int32_t* in, int64_t* out, int64_t n, void* tmp, cudaStream_t s)
{
    scan_rec<int32_t, int64_t>(in, out, n, (int64_t*)tmp, s);
}

}  // namespace vt
