// Spreading kernels for d = 2: FP32 point generation and int32 fixed-point shared-memory accumulation.
#include "spread_impl.cuh"

namespace pgb {

cudaError_t launch_spread_f32_d2(const SpreadArgs &a, int w, int blocks, int threads, size_t smem,
                                  cudaStream_t s)
{
    return spread_detail::WidthDispatch<true, 2, kMinWidth, kMaxWidthF32>::run(a, w, blocks, threads, smem, s);
}

}  // namespace pgb
