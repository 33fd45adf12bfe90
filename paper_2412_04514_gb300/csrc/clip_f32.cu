// clip_f32.cu -- FP32 clipper instantiations (8, 16, 32 lanes per cell).
#include "clip_impl.cuh"

namespace vt {

cudaError_t launch_clip_f32(const ClipArgs& a, int t, cudaStream_t s)
{
    if (t == 32) return launch_variant<float, 32, 2, 64, false>(a, s);
    if (t == 16) return launch_variant<float, 16, 4, 64, false>(a, s);
    return launch_variant<float, 8, 8, 64, false>(a, s);
}

}  // namespace vt

#ifdef VT_PROFILE
// diagnostic builds: read (and optionally clear) the FP32 clip kernels' counters
extern "C" VT_API int vt_debug_clip_profile(unsigned long long* out32, int reset)
{
    if (cudaMemcpyFromSymbol(out32, vt::g_vt_prof, sizeof(unsigned long long) * 32) != cudaSuccess) return 1;
    if (reset) {
        static const unsigned long long zero[32] = {};
        if (cudaMemcpyToSymbol(vt::g_vt_prof, zero, sizeof(zero)) != cudaSuccess) return 1;
    }
    return 0;
}
#endif
