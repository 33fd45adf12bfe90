// clip_robust.cu -- robust FP64 clipper (a warp per cell, 128 vertex slots,
// 128 planes) for cells that outgrow the regular capacity or whose FP32
// topology became inconsistent; plus the variant dispatch.
#include "clip_impl.cuh"

namespace vt {

cudaError_t launch_clip_f32(const ClipArgs& a, int t, cudaStream_t s);
cudaError_t launch_clip_f64(const ClipArgs& a, int t, cudaStream_t s);
cudaError_t launch_clip_big(const ClipArgs& a, cudaStream_t s);

size_t clip_state_pos_offset(int precision)
{
    return precision == VT_FP64 ? StateLayout<double, 64, 64>::POS : StateLayout<float, 64, 64>::POS;
}

size_t clip_state_bytes(int precision)
{
    // the regular variants all hold 64 vertex slots and 64 planes
    return precision == VT_FP64 ? state_bytes<double, 8, 8, 64>() : state_bytes<float, 8, 8, 64>();
}

cudaError_t launch_clip(const ClipArgs& a, int variant, int threads_per_cell, cudaStream_t s)
{
    if (a.nq <= 0) return cudaSuccess;
    const int t = threads_per_cell == 0 ? 32 : threads_per_cell;
    if (variant == 2) return launch_variant<double, 32, 4, 128, true>(a, s);
    if (variant == 3) return launch_clip_big(a, s);
    if (variant == 0) return launch_clip_f32(a, t, s);
    return launch_clip_f64(a, t, s);
}

}  // namespace vt
