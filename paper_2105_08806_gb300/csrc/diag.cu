// Throughput probe of the unit that bounds spreading: 32-bit integer atomic adds to shared
// memory at random addresses, from every SM, as the spreading kernels issue them.
#include <cuda_runtime.h>

#include "pg_boltz.h"
#include "pgb_internal.cuh"

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

}  // namespace

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
