// Spreading kernels for d = 3, VHS kernels: FP32 point generation and split 64-bit fixed-point shared-memory accumulation.
// Angular kernels B(|g|, cos theta) use the instantiations of spread_f32_3d_ang.cu.
#include "spread_impl.cuh"

namespace pgb {

cudaError_t launch_spread_f32_d3(const SpreadArgs &a, int w, int blocks, int threads, size_t smem,
                                  cudaStream_t s)
{
    if (a.nang_even) return launch_spread_f32_d3_ang(a, w, blocks, threads, smem, s);
    return spread_detail::WidthDispatch<true, 3, kMinWidth, kMaxWidthF32, false>::run(a, w, blocks, threads, smem, s);
}

}  // namespace pgb
