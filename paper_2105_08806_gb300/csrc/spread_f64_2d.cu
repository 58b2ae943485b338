// Spreading kernels for d = 2, VHS kernels: FP64 point generation and FP64 shared-memory partial sums.
// Angular kernels B(|g|, cos theta) use the instantiations of spread_f64_2d_ang.cu.
#include "spread_impl.cuh"

namespace pgb {

cudaError_t launch_spread_f64_d2(const SpreadArgs &a, int w, int blocks, int threads, size_t smem,
                                  cudaStream_t s)
{
    if (a.nang_even) return launch_spread_f64_d2_ang(a, w, blocks, threads, smem, s);
    return spread_detail::WidthDispatch<false, 2, kMinWidth, kMaxWidthF64, false>::run(a, w, blocks, threads, smem, s);
}

}  // namespace pgb
