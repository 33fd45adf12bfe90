// clip_f64.cu -- plain FP64 clipper instantiations (8, 16, 32 lanes per cell).
#include "clip_impl.cuh"

namespace vt {

cudaError_t launch_clip_f64(const ClipArgs& a, int t, cudaStream_t s)
{
    if (t == 32) return launch_variant<double, 32, 2, 64, false>(a, s);
    if (t == 16) return launch_variant<double, 16, 4, 64, false>(a, s);
    return launch_variant<double, 8, 8, 64, false>(a, s);
}

}  // namespace vt
