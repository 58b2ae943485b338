// FP32 spreading kernels (point generation and shared-memory accumulation in FP32).
#include "spread_impl.cuh"

namespace pgb {

cudaError_t launch_spread_f32(const SpreadArgs &a, int w, int blocks, int threads, size_t smem,
                              cudaStream_t s)
{
    using namespace spread_detail;
    if (a.d == 2) return WidthDispatch<float, 2, kMinWidth, kMaxWidthF32>::run(a, w, blocks, threads, smem, s);
    return WidthDispatch<float, 3, kMinWidth, kMaxWidthF32>::run(a, w, blocks, threads, smem, s);
}

}  // namespace pgb
