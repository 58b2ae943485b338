// Spreading kernel templates shared by the FP32 and FP64 translation units.
#pragma once
// Fused post-collision point generation + exponential-of-semicircle spreading
// onto the folded cosine grid (Section 4.2, Eq. num_fast_k and Eq. nufft).
//
// One thread owns one node pair (i, j) and walks the M sphere points sigma_m:
//   v'     = (v_i + v_j)/2 + |v_i - v_j| sigma_m / 2
//   z_l    = arccos(xi(v'_l))                     angle of the l-th mapped coordinate
//   q      = a_i a_j B(|v_i - v_j|) w_m prod_l mu(xi(v'_l))^-2
// and adds q prod_l psi(x_{g_l} - z_l) to the w^d cells of the folded grid
// around z.  The gain coefficient is the cosine sum sum_p q_p prod_l cos(k_l z_pl);
// cos is even and 2 pi periodic, so the periodic grid of n cells can be folded
// onto its n/2 + 1 cells g = 0..n/2 (cell u and cell n - u carry the same cosine):
// every unfolded support index u is added at fold(u) = min(u mod n, n - u mod n).
//
// Stable forms of the angle and the weight from the map formulas of Section 2.1:
//   r = 1 (algebraic):   cos z = v/sqrt(S^2+v^2), sin z = S/sqrt(S^2+v^2)
//                        -> z = atan2(S, v),      mu^-2 = (S^2 + v^2)/S
//   r = 0 (logarithmic): cos z = tanh(v/S), sin z = sech(v/S)
//                        -> z = atan2(1, sinh(v/S)), mu^-2 = S cosh(v/S)
//
// Each block accumulates in a private shared-memory copy of a slab of the
// folded grid (all of it when it fits) with shared-memory atomics, then adds
// the slab to the FP64 global grid.  Points whose axis-0 support misses the
// block's slab are skipped after their first coordinate is formed.
#include <cuda_runtime.h>

#include "pgb_internal.cuh"

namespace pgb {
namespace spread_detail {

template <typename T>
struct Fn;

template <>
struct Fn<float> {
    static __device__ __forceinline__ float sqrt_(float x) { return sqrtf(x); }
    static __device__ __forceinline__ float exp_(float x) { return __expf(x); }
    static __device__ __forceinline__ float atan2_(float y, float x) { return atan2f(y, x); }
    static __device__ __forceinline__ float sinh_(float x) { return sinhf(x); }
    static __device__ __forceinline__ float cosh_(float x) { return coshf(x); }
    static __device__ __forceinline__ float pow_(float x, float y) { return powf(x, y); }
    static __device__ __forceinline__ float floor_(float x) { return floorf(x); }
};

template <>
struct Fn<double> {
    static __device__ __forceinline__ double sqrt_(double x) { return sqrt(x); }
    static __device__ __forceinline__ double exp_(double x) { return exp(x); }
    static __device__ __forceinline__ double atan2_(double y, double x) { return atan2(y, x); }
    static __device__ __forceinline__ double sinh_(double x) { return sinh(x); }
    static __device__ __forceinline__ double cosh_(double x) { return cosh(x); }
    static __device__ __forceinline__ double pow_(double x, double y) { return pow(x, y); }
    static __device__ __forceinline__ double floor_(double x) { return floor(x); }
};

// Fold an unfolded periodic index u onto 0..n/2.
__device__ __forceinline__ int fold_index(int u, int n)
{
    int g = u % n;
    if (g < 0) g += n;
    return (g > (n >> 1)) ? n - g : g;
}

// The w kernel weights psi(x_u - z) of one axis, u = s..s+w-1, in units where
// one grid cell is 1 and x = z n / (2 pi): psi = exp(beta (sqrt(1 - t^2) - 1)),
// t = (u - x) * 2 / w.  Fold indices go to idx[].
template <typename T, int W>
__device__ __forceinline__ void axis_weights(T x, T beta, int n, T *wt, int *idx)
{
    const int s = (int)Fn<T>::floor_(x - T(0.5 * W)) + 1;
    const T inv_hw = T(2.0 / W);
#pragma unroll
    for (int a = 0; a < W; ++a) {
        const T t = (T(s + a) - x) * inv_hw;
        const T one_m = T(1) - t * t;
        wt[a] = one_m > T(0) ? Fn<T>::exp_(beta * (Fn<T>::sqrt_(one_m) - T(1))) : T(0);
        idx[a] = fold_index(s + a, n);
    }
}

template <typename T, int D, int W>
__global__ void __launch_bounds__(256) k_spread(const SpreadArgs p)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *tile = reinterpret_cast<T *>(smem_raw);

    const int nf = p.nf;
    const int n = p.n;
    const int plane = (D == 3) ? nf * nf : nf;  // cells in one axis-0 row
    const int slab = blockIdx.x % p.nslab;
    const int row_lo = slab * p.rows_per_slab;
    const int row_hi = min(row_lo + p.rows_per_slab, nf);
    const int nrows = row_hi - row_lo;
    if (nrows <= 0) return;  // uniform over the block: an empty trailing slab does nothing
    const int ncell = nrows * plane;
    for (int c = threadIdx.x; c < ncell; c += blockDim.x) tile[c] = T(0);
    __syncthreads();

    const T *vnode = static_cast<const T *>(p.vnode);
    const T *acoef = static_cast<const T *>(p.a);
    const T *sig = static_cast<const T *>(p.sig);
    const T *wsig = static_cast<const T *>(p.wsig);
    const T S = T(p.S);
    const T SS = S * S;
    const T invS = T(1) / S;
    const T gs = T(p.grid_scale);
    const T beta = T(p.beta);
    const T Bc = T(p.Bconst);
    const T gam = T(p.gamma);
    const int N = p.N;
    const int nnode = p.nnode;
    const int M = p.M;
    const bool alg = (p.r == 1);

    const long long groups = gridDim.x / p.nslab;
    const long long stride = groups * blockDim.x;
    for (long long pr = (long long)(blockIdx.x / p.nslab) * blockDim.x + threadIdx.x; pr < p.npairs;
         pr += stride) {
        const int i = (int)(pr / nnode);
        const int j = (int)(pr - (long long)i * nnode);
        T vi[D], vj[D], cen[D];
        int ii = i, jj = j;
#pragma unroll
        for (int l = D - 1; l >= 0; --l) {
            vi[l] = vnode[ii % N];
            ii /= N;
            vj[l] = vnode[jj % N];
            jj /= N;
        }
        T g2 = T(0);
#pragma unroll
        for (int l = 0; l < D; ++l) {
            const T dl = vi[l] - vj[l];
            g2 += dl * dl;
            cen[l] = T(0.5) * (vi[l] + vj[l]);
        }
        const T g = Fn<T>::sqrt_(g2);
        T B;
        switch (p.fast_gamma) {
        case 0: B = Bc; break;
        case 1: B = Bc * g; break;
        case 2: B = Bc * Fn<T>::sqrt_(g); break;
        default: B = Bc * Fn<T>::pow_(g, gam); break;
        }
        const T base = acoef[i] * acoef[j] * B;
        if (base == T(0)) continue;
        const T rad = T(0.5) * g;

        for (int m = 0; m < M; ++m) {
            T q = base * wsig[m];
            T x[D];
#pragma unroll
            for (int l = 0; l < D; ++l) {
                const T vp = cen[l] + rad * sig[m * D + l];
                T z, m2;
                if (alg) {
                    z = Fn<T>::atan2_(S, vp);
                    m2 = (SS + vp * vp) * invS;
                } else {
                    const T u = vp * invS;
                    z = Fn<T>::atan2_(T(1), Fn<T>::sinh_(u));
                    m2 = S * Fn<T>::cosh_(u);
                }
                q *= m2;
                x[l] = z * gs;
            }
            T w0[W];
            int r0[W];
            axis_weights<T, W>(x[0], beta, n, w0, r0);
            bool hit = false;
#pragma unroll
            for (int a = 0; a < W; ++a) {
                r0[a] -= row_lo;
                hit |= ((unsigned)r0[a] < (unsigned)nrows);
                w0[a] *= q;
            }
            if (!hit) continue;
            T w1[W];
            int c1[W];
            axis_weights<T, W>(x[1], beta, n, w1, c1);
            if (D == 2) {
#pragma unroll
                for (int a = 0; a < W; ++a) {
                    if ((unsigned)r0[a] >= (unsigned)nrows) continue;
                    T *row = tile + r0[a] * plane;
#pragma unroll
                    for (int b = 0; b < W; ++b) atomicAdd(row + c1[b], w0[a] * w1[b]);
                }
            } else {
                T w2[W];
                int c2[W];
                axis_weights<T, W>(x[D - 1], beta, n, w2, c2);
#pragma unroll
                for (int b = 0; b < W; ++b) c1[b] *= nf;
                for (int a = 0; a < W; ++a) {
                    if ((unsigned)r0[a] >= (unsigned)nrows) continue;
                    T *row = tile + r0[a] * plane;
#pragma unroll
                    for (int b = 0; b < W; ++b) {
                        const T wab = w0[a] * w1[b];
                        T *line = row + c1[b];
#pragma unroll
                        for (int c = 0; c < W; ++c) atomicAdd(line + c2[c], wab * w2[c]);
                    }
                }
            }
        }
    }
    __syncthreads();
    double *gdst = p.grid + (size_t)row_lo * plane;
    for (int c = threadIdx.x; c < ncell; c += blockDim.x) {
        const T v = tile[c];
        if (v != T(0)) atomicAdd(gdst + c, (double)v);
    }
}

template <typename T, int D, int W>
cudaError_t launch_one(const SpreadArgs &a, int blocks, int threads, size_t smem, cudaStream_t s)
{
    auto kern = k_spread<T, D, W>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    kern<<<blocks, threads, smem, s>>>(a);
    return cudaGetLastError();
}

template <typename T, int D, int W, int WMAX>
struct WidthDispatch {
    static cudaError_t run(const SpreadArgs &a, int w, int blocks, int threads, size_t smem,
                           cudaStream_t s)
    {
        if (w == W) return launch_one<T, D, W>(a, blocks, threads, smem, s);
        return WidthDispatch<T, D, W + 1, WMAX>::run(a, w, blocks, threads, smem, s);
    }
};

template <typename T, int D, int WMAX>
struct WidthDispatch<T, D, WMAX, WMAX> {
    static cudaError_t run(const SpreadArgs &a, int w, int blocks, int threads, size_t smem,
                           cudaStream_t s)
    {
        if (w == WMAX) return launch_one<T, D, WMAX>(a, blocks, threads, smem, s);
        return cudaErrorInvalidValue;
    }
};

}  // namespace spread_detail
}  // namespace pgb
