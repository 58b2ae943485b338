// Spreading kernels for d = 3, VHS kernels: FP64 point generation and FP64 shared-memory partial sums.
// Angular kernels B(|g|, cos theta) use the instantiations of spread_f64_3d_ang.cu.
#include "spread_impl.cuh"

namespace pgb {

cudaError_t launch_spread_f64_d3(const SpreadArgs &a, int w, int blocks, int threads, size_t smem,
                                  cudaStream_t s)
{
    if (a.nang_even) return launch_spread_f64_d3_ang(a, w, blocks, threads, smem, s);
    return spread_detail::WidthDispatch<false, 3, kMinWidth, kMaxWidthF64, false>::run(a, w, blocks, threads, smem, s);
}

}  // namespace pgb
