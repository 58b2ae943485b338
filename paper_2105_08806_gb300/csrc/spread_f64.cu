// FP64 spreading kernels (point generation and shared-memory accumulation in FP64).
#include "spread_impl.cuh"

namespace pgb {

cudaError_t launch_spread_f64(const SpreadArgs &a, int w, int blocks, int threads, size_t smem,
                              cudaStream_t s)
{
    using namespace spread_detail;
    if (a.d == 2) return WidthDispatch<double, 2, kMinWidth, kMaxWidthF64>::run(a, w, blocks, threads, smem, s);
    return WidthDispatch<double, 3, kMinWidth, kMaxWidthF64>::run(a, w, blocks, threads, smem, s);
}

}  // namespace pgb
