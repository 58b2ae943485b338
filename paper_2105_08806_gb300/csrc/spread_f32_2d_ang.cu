// Spreading kernels for d = 2 with an angular factor b(cos theta) in the collision kernel
// (Eq. collision_form): FP32 point generation and split 64-bit fixed-point shared-memory accumulation.
#include "spread_impl.cuh"

namespace pgb {

cudaError_t launch_spread_f32_d2_ang(const SpreadArgs &a, int w, int blocks, int threads, size_t smem,
                                      cudaStream_t s)
{
    return spread_detail::WidthDispatch<true, 2, kMinWidth, kMaxWidthF32, true>::run(a, w, blocks, threads, smem, s);
}

}  // namespace pgb
