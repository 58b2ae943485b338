// Measured peaks for the spreading kernels' rooflines (no counterpart in the paper): 32-bit integer
// atomic adds to shared memory at random addresses, as the spreading kernels issue them, and the
// FP32 / FP64 fused multiply-add and conflict-free shared-atomic rates of the whole GPU.  Also the
// FP32 grid coordinates of the spreading kernels for given velocities, for testing them.
#include <cuda_runtime.h>

#include <algorithm>

#include "pg_boltz.h"
#include "pgb_internal.cuh"
#include "spread_impl.cuh"

#define PG_API extern "C" __attribute__((visibility("default")))

namespace {

constexpr int kCells = 16900;  // a 130 x 130 folded grid, the 2D N = 64 tile
constexpr int kIters = 4096;

__global__ void __launch_bounds__(1024) k_shared_atomic_rate(unsigned *sink)
{
    extern __shared__ unsigned tile[];
    for (int c = threadIdx.x; c < kCells; c += blockDim.x) tile[c] = 0u;
    __syncthreads();
    unsigned h = threadIdx.x * 2654435761u + blockIdx.x * 97u + 1u;
    for (int it = 0; it < kIters; ++it) {
        h = h * 1664525u + 1013904223u;
        atomicAdd(tile + (h >> 8) % kCells, 1u);
    }
    __syncthreads();
    unsigned s = 0u;
    for (int c = threadIdx.x; c < kCells; c += blockDim.x) s += tile[c];
    if (s == 0xffffffffu) sink[0] = s;  // keeps the work observable
}

constexpr int kPipeIters = 2048;
constexpr int kChains = 8;  // independent FMA chains per thread (covers the pipe latency)

// kChains independent FMA chains of kPipeIters steps each per thread
template <typename T>
__global__ void __launch_bounds__(1024) k_fma_rate(T seed, T *sink)
{
    T acc[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) acc[c] = seed + T(threadIdx.x + c);
    const T m = T(0.999999), a = T(1e-7);
    for (int it = 0; it < kPipeIters; ++it) {
#pragma unroll
        for (int c = 0; c < kChains; ++c) acc[c] = fma(acc[c], m, a);
    }
    T s = T(0);
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += acc[c];
    if (s == T(-1)) sink[0] = s;  // keeps the work observable
}

// Conflict-free shared atomics: lane l of every warp adds to bank l (a different word per warp).
__global__ void __launch_bounds__(1024) k_shared_atomic_free(unsigned *sink)
{
    extern __shared__ unsigned tile[];
    for (int c = threadIdx.x; c < kCells; c += blockDim.x) tile[c] = 0u;
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    unsigned *w = tile + (warp * 32 + lane) % kCells;
    for (int it = 0; it < kIters; ++it) atomicAdd(w, 1u);
    __syncthreads();
    unsigned s = 0u;
    for (int c = threadIdx.x; c < kCells; c += blockDim.x) s += tile[c];
    if (s == 0xffffffffu) sink[0] = s;
}

__global__ void k_grid_coords(const float *v, long long n, pgb::TypedConsts<float> K, int alg, double *cell,
                              double *frac, double *m2)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        float X, F;
        pgb::spread_detail::grid_coord_f32(K, v[i], alg != 0, X, F);
        const float w = pgb::spread_detail::axis_m2_f32(K, v[i], alg != 0);
        cell[i] = (double)X;
        frac[i] = (double)F;
        m2[i] = (double)w;
    }
}

// Time `launch` (already warmed up once) on stream s; returns ms or -1.
template <typename L>
float time_launch(L launch, cudaStream_t s, cudaEvent_t a, cudaEvent_t b)
{
    launch();
    cudaEventRecord(a, s);
    launch();
    cudaEventRecord(b, s);
    float ms = -1.0f;
    if (cudaEventSynchronize(b) != cudaSuccess || cudaEventElapsedTime(&ms, a, b) != cudaSuccess) return -1.0f;
    return ms;
}

}  // namespace

PG_API int pg_boltz_probe_pipes(void *cuda_stream, double *rates_out)
{
    if (!rates_out) return pgb::record_error(PG_ERR_ARG, "rates_out is NULL");
    pgb::record_error(PG_OK, "");
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    int dev = 0;
    cudaDeviceProp prop;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaGetDeviceProperties(&prop, dev) != cudaSuccess) {
        cudaGetLastError();
        return pgb::record_error(PG_ERR_CUDA, "no CUDA device");
    }
    const int threads = 1024, blocks = prop.multiProcessorCount * 2;
    const size_t smem = kCells * sizeof(unsigned);
    void *sink = nullptr;
    cudaEvent_t a = nullptr, b = nullptr;
    int rc = PG_OK;
    if (cudaFuncSetAttribute(k_shared_atomic_free, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess ||
        cudaMalloc(&sink, 64) != cudaSuccess || cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&b) != cudaSuccess) {
        rc = pgb::record_error(PG_ERR_CUDA, "probe setup failed");
    } else {
        const double fmas = (double)blocks * threads * kChains * kPipeIters;
        const float t32 = time_launch([&] { k_fma_rate<float><<<blocks, threads, 0, s>>>(1.0f, (float *)sink); }, s, a, b);
        // FP64: GB300's FP64 pipe is narrow; a tenth of the blocks keeps the probe short
        const int b64 = std::max(prop.multiProcessorCount, blocks / 10);
        const float t64 = time_launch([&] { k_fma_rate<double><<<b64, threads, 0, s>>>(1.0, (double *)sink); }, s, a, b);
        const float tat = time_launch([&] { k_shared_atomic_free<<<blocks, threads, smem, s>>>((unsigned *)sink); }, s, a, b);
        if (t32 <= 0.0f || t64 <= 0.0f || tat <= 0.0f) {
            rc = pgb::record_error(PG_ERR_CUDA, "probe launch failed");
        } else {
            rates_out[0] = fmas / (t32 * 1e-3);
            rates_out[1] = fmas * b64 / blocks / (t64 * 1e-3);
            rates_out[2] = (double)blocks * threads * kIters / (tat * 1e-3);
        }
    }
    cudaGetLastError();
    if (a) cudaEventDestroy(a);
    if (b) cudaEventDestroy(b);
    if (sink) cudaFree(sink);
    return rc;
}

PG_API int pg_boltz_grid_coords_f32(const float *v_dev, long long n, double S, int map_log, int n_grid,
                                    double *cell_dev, double *frac_dev, double *m2_dev, void *cuda_stream)
{
    pgb::record_error(PG_OK, "");
    if (n < 0 || (n > 0 && (!v_dev || !cell_dev || !frac_dev || !m2_dev))) return pgb::record_error(PG_ERR_ARG, "bad arrays");
    if (!(S > 0.0) || n_grid < 2 || (n_grid & 1) || (map_log != 0 && map_log != 1))
        return pgb::record_error(PG_ERR_ARG, "need S > 0, an even n_grid >= 2 and map_log in {0, 1}");
    if (n == 0) return PG_OK;
    pgb::SpreadArgs a{};
    a.S = S;
    a.n = n_grid;
    a.grid_scale = n_grid / (2.0 * 3.14159265358979323846);
    a.Wsig = 1.0;
    a.angmax = 1.0;
    a.wmax_frac = 1.0;
    pgb::fill_spread_consts(a);
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    k_grid_coords<<<256, 256, 0, s>>>(v_dev, n, a.cf, map_log ? 0 : 1, cell_dev, frac_dev, m2_dev);
    if (cudaGetLastError() != cudaSuccess) return pgb::record_error(PG_ERR_CUDA, "grid coordinate launch failed");
    return PG_OK;
}

PG_API int pg_boltz_probe_shared_atomics(void *cuda_stream, double *rate_out)
{
    if (!rate_out) return pgb::record_error(PG_ERR_ARG, "rate_out is NULL");
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    int dev = 0;
    cudaDeviceProp prop;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaGetDeviceProperties(&prop, dev) != cudaSuccess) {
        cudaGetLastError();
        return pgb::record_error(PG_ERR_CUDA, "no CUDA device");
    }
    const size_t smem = kCells * sizeof(unsigned);
    const int threads = 1024;
    const int blocks = prop.multiProcessorCount * 2;  // two 1024-thread blocks fill an SM's 2048 threads
    unsigned *sink = nullptr;
    cudaEvent_t a = nullptr, b = nullptr;
    int rc = PG_OK;
    if (cudaFuncSetAttribute(k_shared_atomic_rate, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess ||
        cudaMalloc(&sink, 64) != cudaSuccess || cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&b) != cudaSuccess) {
        rc = pgb::record_error(PG_ERR_CUDA, "probe setup failed");
    } else {
        k_shared_atomic_rate<<<blocks, threads, smem, s>>>(sink);  // warm-up
        cudaEventRecord(a, s);
        k_shared_atomic_rate<<<blocks, threads, smem, s>>>(sink);
        cudaEventRecord(b, s);
        float ms = 0.0f;
        if (cudaEventSynchronize(b) != cudaSuccess || cudaEventElapsedTime(&ms, a, b) != cudaSuccess || ms <= 0.0f)
            rc = pgb::record_error(PG_ERR_CUDA, "probe launch failed");
        else
            *rate_out = (double)blocks * threads * kIters / (ms * 1e-3);
    }
    cudaGetLastError();
    if (a) cudaEventDestroy(a);
    if (b) cudaEventDestroy(b);
    if (sink) cudaFree(sink);
    return rc;
}
