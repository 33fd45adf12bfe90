// probe.cu -- fused multiply-add throughput of the device in float32 and
// float64: the measured counterpart of the unit-count peak that ALU-bound
// rooflines divide by. Every thread runs eight independent FMA chains (enough
// to cover the FMA latency with the resident warps), eight blocks of 256
// threads per SM; the chains' sum is written only under a condition that never
// holds, so the compiler keeps them and no result is stored.
#include "vt_internal.cuh"

namespace vt {

namespace {

template <typename Real>
__global__ void __launch_bounds__(256) k_fma(Real seed, int iters, Real* out)
{
    Real a[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) a[i] = seed + (Real)(threadIdx.x + i);
    const Real m = (Real)0.999, c = (Real)1e-3;  // contracting: the chains stay finite
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int i = 0; i < 8; ++i) a[i] = fma(a[i], m, c);
    }
    Real s = 0;
#pragma unroll
    for (int i = 0; i < 8; ++i) s += a[i];
    if (s == (Real)-12345) out[0] = s;
}

template <typename Real>
int probe(int iters, double* tflops, cudaStream_t s)
{
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return set_error(VT_ERR_CUDA, "device query failed");
    const unsigned blocks = (unsigned)sms * 8u;
    cudaEvent_t a, b;
    if (cudaEventCreate(&a) != cudaSuccess) return set_error(VT_ERR_CUDA, "event creation failed");
    if (cudaEventCreate(&b) != cudaSuccess) {
        cudaEventDestroy(a);
        return set_error(VT_ERR_CUDA, "event creation failed");
    }
    k_fma<Real><<<blocks, 256, 0, s>>>((Real)1, iters / 8, nullptr);  // warm-up
    cudaEventRecord(a, s);
    k_fma<Real><<<blocks, 256, 0, s>>>((Real)1, iters, nullptr);
    cudaEventRecord(b, s);
    count_launch(2);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaEventSynchronize(b);
    float ms = 0.0f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, a, b);
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    if (e != cudaSuccess) return set_error(VT_ERR_CUDA, cudaGetErrorString(e));
    const double flops = 2.0 * 8.0 * (double)iters * 256.0 * (double)blocks;
    *tflops = flops / (ms * 1e-3) / 1e12;
    return VT_OK;
}

}  // namespace

}  // namespace vt

extern "C" VT_API int vt_probe_fma(int precision, double* tflops, void* stream)
{
    if (!tflops) return vt::set_error(VT_ERR_INVALID_ARG, "tflops is NULL");
    if (precision == VT_FP64) return vt::probe<double>(1 << 11, tflops, (cudaStream_t)stream);
    if (precision == VT_FP32_RECHECK) return vt::probe<float>(1 << 16, tflops, (cudaStream_t)stream);
    return vt::set_error(VT_ERR_INVALID_ARG, "precision must be VT_FP64 or VT_FP32_RECHECK");
}
