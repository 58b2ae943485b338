// Projection f -> f~ for callers that cannot allocate device memory.
//
// Some host applications hand all device memory to their own pool or arena and do not
// let libraries call cudaMalloc after start-up; others (thin language bindings, embedded
// solvers) can only pass pointers they already own.  Such callers cannot create a
// pg_boltz plan, because a plan allocates its tables and workspace.  This file gives them
// one entry point that allocates nothing: the projection of sampled values of f onto the
// trial space, with every intermediate (the projection matrix and the two partial
// contractions) placed in one library-owned static device array.
//
// The array is a file-scope __device__ variable: every GPU that loads the library holds
// it until the process exits, and every call shares it.  Host code cannot use the
// variable's name as a device address, so every call looks the address up with
// cudaGetSymbolAddress, with the caller's device current.  The lookup allocates nothing, and
// doing it on every call (instead of caching one address per device) keeps the address right
// after a device reset or when the caller switches contexts.  On the first call in a context
// the lookup may load the library's device code (lazy module loading).
#include <cuda_runtime.h>

#include <cmath>

#include "pg_boltz.h"
#include "pgb_internal.cuh"

#define PG_API extern "C" __attribute__((visibility("default")))

namespace {

constexpr size_t kScratchDoubles = PG_BOLTZ_NOALLOC_SCRATCH_BYTES / sizeof(double);
static __device__ __align__(256) double g_noalloc_scratch[kScratchDoubles];

int fail(int code, const char *msg) { return pgb::record_error(code, msg); }

// P[k][q] = (pi/Mp) mu(xi_q)^-4 T_k(xi_q) / sqrt(c_k), xi_q = -cos(phi_q),
// phi_q = (2q+1) pi / (2 Mp): Chebyshev-Gauss quadrature of Eq. MultiD_spectral_coef along one
// axis, with mu^-4 = S^2 / sin(phi)^(2(1+r)) (Eq. 1D_mu_function).
__global__ void k_projection_matrix(int N, int Mp, double S, int r, double *P)
{
    const double pi = 3.14159265358979323846;
    const int total = (N + 1) * Mp;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < total; e += gridDim.x * blockDim.x) {
        const int k = e / Mp, q = e % Mp;
        const double phi = (2.0 * q + 1.0) * pi / (2.0 * Mp);
        const double sn = sin(phi);
        double sp = 1.0;
        for (int i = 0; i < 2 * (1 + r); ++i) sp *= sn;
        const double ck = sqrt(k == 0 ? pi : 0.5 * pi);
        P[e] = (pi / Mp) * (S * S / sp) * cos(k * (pi - phi)) / ck;
    }
}

}  // namespace

PG_API int pg_boltz_project_noalloc(int d, int N, double S, int map_log, int Mp, const double *fvals_dev,
                                    double *ftilde_dev, void *cuda_stream)
{
    pgb::record_error(PG_OK, "");
    if (d != 2 && d != 3) return fail(PG_ERR_ARG, "d must be 2 or 3");
    if (N < 2 || Mp < 1) return fail(PG_ERR_ARG, "need N >= 2 and Mp >= 1");
    if (!(S > 0.0) || !std::isfinite(S)) return fail(PG_ERR_ARG, "S must be positive");
    if (map_log != 0 && map_log != 1) return fail(PG_ERR_ARG, "map_log must be 0 or 1");
    if (!fvals_dev || !ftilde_dev) return fail(PG_ERR_ARG, "NULL device pointer");
    // scratch layout: P ((N+1) x Mp), then the two partial contractions of the passes
    const double n1 = N + 1.0;
    const double need_t1 = n1 * std::pow((double)Mp, d - 1);
    const double need_t2 = (d == 3) ? n1 * n1 * Mp : 0.0;
    const double need = n1 * Mp + need_t1 + need_t2;
    if (need > (double)kScratchDoubles)
        return fail(PG_ERR_ARG, "pg_boltz_project_noalloc: (N+1)*Mp + (N+1)*Mp^(d-1) [+ (N+1)^2*Mp in 3D] "
                                "doubles exceed the static scratch of PG_BOLTZ_NOALLOC_SCRATCH_BYTES");
    void *ptr = nullptr;
    if (cudaGetSymbolAddress(&ptr, g_noalloc_scratch) != cudaSuccess || !ptr) {
        cudaGetLastError();
        return fail(PG_ERR_CUDA, "cudaGetSymbolAddress of the static scratch failed (no usable current device?)");
    }
    double *base = static_cast<double *>(ptr);
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    double *P = base;
    double *t1 = P + (size_t)(N + 1) * Mp;
    double *t2 = t1 + (size_t)need_t1;
    k_projection_matrix<<<64, 256, 0, s>>>(N, Mp, S, map_log ? 0 : 1, P);
    if (cudaGetLastError() != cudaSuccess) return fail(PG_ERR_CUDA, "projection matrix launch failed");
    // every scratch element a pass reads was written earlier in the same call: nothing to clear
    pgb::Dims3 dims;
    dims.e[0] = (d == 2) ? 1 : Mp;
    dims.e[1] = Mp;
    dims.e[2] = Mp;
    const double *cur = fvals_dev;
    double *bufs[2] = {t1, t2};
    int which = 0;
    for (int ax = 3 - d; ax < 3; ++ax) {
        double *dst = (ax == 2) ? ftilde_dev : bufs[which];
        if (pgb::launch_axis_pass(cur, dims, ax, P, N + 1, dst, s) != cudaSuccess)
            return fail(PG_ERR_CUDA, "projection pass launch failed");
        dims.e[ax] = N + 1;
        cur = dst;
        which ^= 1;
    }
    return PG_OK;
}
