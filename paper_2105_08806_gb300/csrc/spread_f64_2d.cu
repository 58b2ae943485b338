// Spreading kernels for d = 2: FP64 point generation and int64 fixed-point shared-memory accumulation.
#include "spread_impl.cuh"

namespace pgb {

cudaError_t launch_spread_f64_d2(const SpreadArgs &a, int w, int blocks, int threads, size_t smem,
                                  cudaStream_t s)
{
    return spread_detail::WidthDispatch<false, 2, kMinWidth, kMaxWidthF64>::run(a, w, blocks, threads, smem, s);
}

}  // namespace pgb
