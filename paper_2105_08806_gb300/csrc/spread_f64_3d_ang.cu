// Spreading kernels for d = 3 with an angular factor b(cos theta) in the collision kernel
// (Eq. collision_form): FP64 point generation and FP64 shared-memory partial sums.
#include "spread_impl.cuh"

namespace pgb {

cudaError_t launch_spread_f64_d3_ang(const SpreadArgs &a, int w, int blocks, int threads, size_t smem,
                                      cudaStream_t s)
{
    return spread_detail::WidthDispatch<false, 3, kMinWidth, kMaxWidthF64, true>::run(a, w, blocks, threads, smem, s);
}

}  // namespace pgb
