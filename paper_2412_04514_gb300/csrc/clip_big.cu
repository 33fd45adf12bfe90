// clip_big.cu -- FP32 clipper with the robust variant's capacity (a warp per
// cell, 128 vertex slots, 128 planes): the FP32 form's first fallback for
// cells that outgrow the regular 64 slots, before the FP64 robust variant.
#include "clip_impl.cuh"

namespace vt {

cudaError_t launch_clip_big(const ClipArgs& a, cudaStream_t s)
{
    return launch_variant<float, 32, 4, 128, true>(a, s);
}

}  // namespace vt
