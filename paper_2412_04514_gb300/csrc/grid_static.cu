// grid_static.cu -- vt_grid_build_static: the grid counting sort of
// vt_grid_build with its scratch memory in a fixed array that this library
// owns in device memory, for callers that cannot allocate device memory.
//
// The scratch is a file-scope __device__ array of STATIC_SCRATCH_BYTES. Every
// GPU that loads the library holds it until the process exits. Host code may
// not use the array's name as a device pointer (it names a host-side shadow),
// so every call resolves the real address with cudaGetSymbolAddress on the
// current device. Nothing is cached: after cudaDeviceReset, or when the
// primary context is torn down and made again, the module is loaded anew and
// the array may sit at another address. The lookup costs microseconds, next
// to a blocking sort.
#include <cstdio>

#include "vt_internal.cuh"

namespace vt {

namespace {

constexpr int64_t STATIC_MAX_POINTS = int64_t(1) << 20;  // generators per call
constexpr int64_t STATIC_MAX_CELLS = int64_t(1) << 20;   // grid cells G^3 per call
size_t al256(size_t x) { return (x + 255) & ~size_t(255); }

// scratch layout (offsets in bytes), sized for the limits above
constexpr size_t OFF_STATUS = 0;
constexpr size_t OFF_CID = 256;
constexpr size_t OFF_TICKET = OFF_CID + sizeof(int32_t) * STATIC_MAX_POINTS;
constexpr size_t OFF_COUNTS = OFF_TICKET + sizeof(int32_t) * STATIC_MAX_POINTS;
constexpr size_t OFF_BIG = OFF_COUNTS + sizeof(int32_t) * (STATIC_MAX_CELLS + 64);
constexpr size_t OFF_SCAN = OFF_BIG + sizeof(int32_t) * (STATIC_MAX_CELLS + 64);
constexpr size_t SCAN_BYTES = 64 * 1024;  // >= scan_tmp_bytes(2^20) (two levels of tile totals)
constexpr size_t STATIC_SCRATCH_BYTES = OFF_SCAN + SCAN_BYTES;

static __device__ __align__(256) unsigned char g_grid_scratch[STATIC_SCRATCH_BYTES];

// device address of g_grid_scratch in the current device's context
cudaError_t scratch_address(unsigned char** out)
{
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_grid_scratch);
    if (e != cudaSuccess) return e;
    *out = static_cast<unsigned char*>(p);
    return cudaSuccess;
}

}  // namespace

}  // namespace vt

using namespace vt;

extern "C" VT_API int vt_grid_build_static(const float* pts, int64_t n, const vt_params* p, int G, float* sorted,
                                           int32_t* perm, int32_t* cell_off, void* stream)
{
    const int g_want = vt_grid_resolution(p, n);
    if (g_want < 1) return set_error(VT_ERR_INVALID_ARG, "invalid vt_params");
    if (n < 0) return set_error(VT_ERR_INVALID_ARG, "n must be >= 0");
    if (G != g_want) return set_error(VT_ERR_INVALID_ARG, "G does not match vt_grid_resolution");
    const int64_t g3 = (int64_t)G * G * G;
    if (n > STATIC_MAX_POINTS || g3 > STATIC_MAX_CELLS) {
        char msg[200];
        snprintf(msg, sizeof(msg),
                 "vt_grid_build_static is limited to %lld points and %lld grid cells (got n = %lld, G^3 = %lld)",
                 (long long)STATIC_MAX_POINTS, (long long)STATIC_MAX_CELLS, (long long)n, (long long)g3);
        return set_error(VT_ERR_INVALID_ARG, msg);
    }
    if (scan_tmp_bytes(n > g3 ? n : g3) > SCAN_BYTES) return set_error(VT_ERR_INVALID_ARG, "scan scratch too small");
    if ((n > 0 && (!pts || !sorted || !perm)) || !cell_off) return set_error(VT_ERR_INVALID_ARG, "NULL buffer");
    // the call waits for its own result, which a stream capture forbids
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing((cudaStream_t)stream, &cs) != cudaSuccess) (void)cudaGetLastError();
    if (cs != cudaStreamCaptureStatusNone)
        return set_error(VT_ERR_INVALID_ARG, "vt_grid_build_static synchronises its stream and cannot be captured");
    {
        // a kernel is never launched on memory it cannot reach (pageable host
        // memory): that is an argument error, not a fault
        const void* ptrs[] = {pts, sorted, perm, cell_off};
        const char* names[] = {"pts", "sorted", "perm", "cell_off"};
        const int r = check_device_buffers(stream, ptrs, names, 4);
        if (r) return r;
    }
    unsigned char* base = nullptr;
    cudaError_t e = scratch_address(&base);
    if (e != cudaSuccess) return set_error(VT_ERR_CUDA, cudaGetErrorString(e));
    cudaStream_t s = (cudaStream_t)stream;
    DevStatus* st = reinterpret_cast<DevStatus*>(base + OFF_STATUS);
    // the previous call's contents remain: clear the status block (the
    // histogram is cleared inside the launch sequence)
    e = cudaMemsetAsync(st, 0, sizeof(DevStatus), s);
    if (e == cudaSuccess)
        e = launch_grid_build(pts, n, make_grid(p, G), reinterpret_cast<float4*>(sorted), perm, cell_off,
                              reinterpret_cast<int32_t*>(base + OFF_CID), reinterpret_cast<int32_t*>(base + OFF_TICKET),
                              reinterpret_cast<int32_t*>(base + OFF_COUNTS), reinterpret_cast<int32_t*>(base + OFF_BIG),
                              base + OFF_SCAN, st, s);
    DevStatus h;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h, st, sizeof(DevStatus), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return set_error(VT_ERR_CUDA, cudaGetErrorString(e));
    if (h.bad_point) return set_error(VT_ERR_INVALID_ARG, "a point is not finite or not inside [box_lo, box_hi)");
    return VT_OK;
}
