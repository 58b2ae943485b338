// Batched evaluation of many independent collision operators (one velocity distribution
// per spatial cell of an inhomogeneous solver), each with its own N, M, S and gamma, in
// three launches replayed as a CUDA graph:
//   1. k_batch_prep   (one block per cell): reconstruction of f_N at the interior CGL nodes,
//      loss weights h_i (Eq. Qminus) and the strength bound B_c of the cell;
//   2. k_batch_spread (persistent, one or more blocks per SM): work items (cell, range of
//      node pairs) are taken from a global counter; a block keeps the folded grid of its
//      current cell in shared memory and adds it to the cell's global fixed-point grid when
//      it moves to another cell;
//   3. k_batch_final  (one block per cell): cosine transform + deconvolution of the cell's
//      grid, forward Chebyshev transform of the loss, Q = Q+ - Q-.
// The per-point arithmetic is the same as the single-plan path (spread_impl.cuh).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <new>
#include <tuple>
#include <vector>

#include "host.cuh"
#include "spread_impl.cuh"

#define PG_API extern "C" __attribute__((visibility("default")))

using namespace pgbh;

namespace pgb {

struct CellDesc {
    int N, M, nf, n, nnode, fast_gamma;
    double S, gamma, Wsig;
    long long pairs;     // unordered node pairs, nnode (nnode + 1) / 2
    long long f_off;     // packed modes (f~ and Q)
    long long a_off;     // packed node values (a, h)
    long long grid_off;  // packed folded grids
    long long s_off;     // packed scratch: four buffers of s_len doubles
    long long s_len;
    int node_off;        // node tables (v, scale_a, inv_mu2)
    int R_off;           // R (N x (N+1)) and E ((N+1) x N)
    int D_off;           // D ((N+1) x nf)
    int sig_off;         // sphere points (M x d) and weights (M)
    int chunk;           // node pairs per work item
    int item0;           // first work item of the cell
    double corr;         // FP32 plans: exact / FP32 constant factors of the strengths (1 for FP64)
};

struct BatchArgs {
    int d, r, ncell, nitems, w;
    double Bconst, beta, screen_eps;
    const CellDesc *cells;
    const int *item_cell;
    int *counter;
    const double *f;
    double *Q;
    double *a64;
    float *a32;
    double *h;
    double *Bcell;
    double *Tcell;  // per-cell screening threshold (0: spread every pair)
    unsigned long long *grid;
    int *carry;          // FP32: per-block carry counters, blocks x carry_stride
    int carry_stride;    // cells of the largest cell tile
    int queue_off;       // FP32: byte offset of the warps' point queues in dynamic shared memory
    double *scratch;
    const double *v64;
    const float *v32;
    const float *v32lo;  // v - (double)v32 (FP32 nodes' rounding)
    const double *scale_a;
    const double *inv_mu2;
    const double *R;
    const double *E;
    const double *D;
    const double *sig64;
    const float *sig32;
    const double *wsig64;
    const float *wsig32;
    const double *kpoly;  // FP64: the kernel's polynomial coefficients (SpreadArgs::kpoly)
};

namespace {

constexpr int kPrepThreads = 256;

__device__ __forceinline__ Dims3 dims3(int d, int a, int b, int c)
{
    Dims3 x;
    x.e[0] = (d == 2) ? 1 : a;
    x.e[1] = b;
    x.e[2] = c;
    return x;
}

// out = A contracted with `in` along axis ax, by the whole block.
__device__ void block_pass(const double *in, Dims3 id, int ax, const double *A, int m, double *out)
{
    Dims3 od = id;
    od.e[ax] = m;
    const int total = od.e[0] * od.e[1] * od.e[2];
    const int len = id.e[ax];
    const int sax = (ax == 2) ? 1 : (ax == 1 ? id.e[2] : id.e[1] * id.e[2]);
    for (int o = threadIdx.x; o < total; o += blockDim.x) {
        int oc[3];
        oc[2] = o % od.e[2];
        const int t = o / od.e[2];
        oc[1] = t % od.e[1];
        oc[0] = t / od.e[1];
        const int k = oc[ax];
        oc[ax] = 0;
        const int base = (oc[0] * id.e[1] + oc[1]) * id.e[2] + oc[2];
        double acc = 0.0;
        for (int s = 0; s < len; ++s) acc = fma(A[k * len + s], in[base + s * sax], acc);
        out[o] = acc;
    }
}

__device__ void block_pass_fixed(const unsigned long long *in, Dims3 id, int ax, const double *A, int m,
                                 double unit, double *out)
{
    Dims3 od = id;
    od.e[ax] = m;
    const int total = od.e[0] * od.e[1] * od.e[2];
    const int len = id.e[ax];
    const int sax = (ax == 2) ? 1 : (ax == 1 ? id.e[2] : id.e[1] * id.e[2]);
    for (int o = threadIdx.x; o < total; o += blockDim.x) {
        int oc[3];
        oc[2] = o % od.e[2];
        const int t = o / od.e[2];
        oc[1] = t % od.e[1];
        oc[0] = t / od.e[1];
        const int k = oc[ax];
        oc[ax] = 0;
        const int base = (oc[0] * id.e[1] + oc[1]) * id.e[2] + oc[2];
        double acc = 0.0;
        for (int s = 0; s < len; ++s) acc = fma(A[k * len + s], (double)(long long)in[base + s * sax], acc);
        out[o] = acc * unit;
    }
}

__device__ double block_reduce_sum(double v, double *warp_part)
{
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
    if ((threadIdx.x & 31) == 0) warp_part[threadIdx.x >> 5] = v;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x == 0)
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += warp_part[w];  // fixed order
    __syncthreads();
    return s;
}

// One block per cell: a_i, h_i and the strength bound B_c (same formulas as k_recon_last,
// k_loss and k_bound_reduce of the single-plan path).  PT is the arithmetic of the pair
// distances and |v_i - v_j|^gamma (float for FP32 plans; sums are FP64 either way).
template <typename PT, int D>
__global__ void __launch_bounds__(kPrepThreads) k_batch_prep(const __grid_constant__ BatchArgs b)
{
    __shared__ double warp_part[kPrepThreads / 32];
    __shared__ unsigned s_hist[kScreenBins];
    const bool screen = b.screen_eps > 0.0;
    for (int k = threadIdx.x; k < kScreenBins; k += blockDim.x) s_hist[k] = 0u;
    const int c = blockIdx.x;
    const CellDesc cd = b.cells[c];
    constexpr int d = D;
    const int N = cd.N, nnode = cd.nnode;
    double *s1 = b.scratch + cd.s_off, *s2 = s1 + cd.s_len;
    const double *R = b.R + cd.R_off;
    // 1. reconstruction: leading passes, then the last axis with a_i = W_i mu_i^2 P_i
    Dims3 dims = dims3(d, N + 1, N + 1, N + 1);
    const double *cur = b.f + cd.f_off;
    double *bufs[2] = {s1, s2};
    int which = 0;
    for (int ax = 3 - d; ax < 2; ++ax) {
        block_pass(cur, dims, ax, R, N, bufs[which]);
        __syncthreads();
        dims.e[ax] = N;
        cur = bufs[which];
        which ^= 1;
    }
    const double *sa = b.scale_a + cd.node_off;
    double *a = b.a64 + cd.a_off;
    float *af = b.a32 + cd.a_off;
    for (int o = threadIdx.x; o < nnode; o += blockDim.x) {
        const int o2 = o % N, t = o / N, o1 = t % dims.e[1], o0 = t / dims.e[1];
        const double *src = cur + (o0 * dims.e[1] + o1) * (N + 1);
        double acc = 0.0;
        for (int s = 0; s <= N; ++s) acc = fma(R[o2 * (N + 1) + s], src[s], acc);
        double scl = sa[o1] * sa[o2];
        if (d == 3) scl *= sa[o0];
        a[o] = acc * scl;
        af[o] = (float)(acc * scl);
    }
    __syncthreads();
    // 2. loss sums and the strength bound
    const PT *vn = nullptr;
    const float *vlo = nullptr;  // FP32 nodes' rounding, added back to the node differences
    if constexpr (sizeof(PT) == 4) {
        vn = b.v32 + cd.node_off;
        vlo = b.v32lo + cd.node_off;
    } else {
        vn = b.v64 + cd.node_off;
    }
    const double *im = b.inv_mu2 + cd.node_off;
    const double Bw = b.Bconst * cd.Wsig;
    const PT S = PT(cd.S), invS = PT(1) / S, gam = PT(cd.gamma);
    double bsum = 0.0;
    for (int i = threadIdx.x; i < nnode; i += blockDim.x) {
        int idx[D], t = i;
#pragma unroll
        for (int l = d - 1; l >= 0; --l) {
            idx[l] = t % N;
            t /= N;
        }
        PT vi[D], vil[D];
#pragma unroll
        for (int l = 0; l < d; ++l) {
            vi[l] = vn[idx[l]];
            vil[l] = vlo ? PT(vlo[idx[l]]) : PT(0);
        }
        double L = 0.0, U = 0.0;
        float Ls = 0.0f, Lc = 0.0f;  // FP32 plans: the loss terms' sum as Ls + Lc (two-sum)
        int jl[D];                   // axis indices of node j (C order), advanced with carries
#pragma unroll
        for (int l = 0; l < d; ++l) jl[l] = 0;
        for (int j0 = 0; j0 < nnode; j0 += 64) {
            PT Up = PT(0);  // bound: partial sums of 64 terms, then FP64
            const int j1 = min(j0 + 64, nnode);
            for (int j = j0; j < j1; ++j) {
                PT g2 = PT(0), mu = PT(1);
                PT vj[D];
#pragma unroll
                for (int l = 0; l < d; ++l) {
                    const int nj = jl[l];
                    vj[l] = vn[nj];
                    PT dl = vi[l] - vj[l];
                    if (vlo) dl += vil[l] - PT(vlo[nj]);
                    g2 += dl * dl;
                }
#pragma unroll
                for (int l = d - 1; l >= 0; --l) {  // next node
                    if (++jl[l] < N) break;
                    jl[l] = 0;
                }
                const PT g = sqrt(g2);
                PT B;
                switch (cd.fast_gamma) {
                case 0: B = PT(1); break;
                case 1: B = g; break;
                case 2: B = sqrt(g); break;
                default: B = (g2 > PT(0)) ? pow(g, gam) : PT(0); break;
                }
                PT aj;
                if constexpr (sizeof(PT) == 4) {  // as the single-plan loss kernel
                    aj = af[j];
                    const float pt = B * aj;
                    const float pe = fmaf(B, aj, -pt);
                    const float tt = Ls + pt;
                    const float bv = tt - Ls;
                    Lc += ((Ls - (tt - bv)) + (pt - bv)) + pe;
                    Ls = tt;
                } else {
                    aj = PT(a[j]);
                    L = fma(double(B), a[j], L);
                }
#pragma unroll
                for (int l = 0; l < d; ++l) {
                    const PT R_ = fabs(PT(0.5) * (vi[l] + vj[l])) + PT(0.5) * g;
                    mu *= (b.r == 1) ? (S * S + R_ * R_) * invS : S * cosh(R_ * invS);
                }
                const PT pb = fabs(aj) * B * mu;
                Up += pb;
                if (screen && pb > PT(0)) atomicAdd(&s_hist[screen_bin(fabs(a[i]) * Bw * (double)pb)], 1u);
            }
            U += (double)Up;
        }
        L += (double)Ls + (double)Lc;
        double scl = 1.0;
        for (int l = 0; l < d; ++l) scl *= im[idx[l]];
        b.h[cd.a_off + i] = a[i] * Bw * L * scl;
        bsum += fabs(a[i]) * Bw * U;
    }
    const double tot = block_reduce_sum(bsum, warp_part);
    if (threadIdx.x == 0) {
        const double Bv = tot * (1.0 + 1e-5);  // margin for the FP32 partial sums
        b.Bcell[c] = Bv;
        // screening threshold of the cell: same rule as k_bound_reduce of the single-plan path
        double t = 0.0;
        if (screen && Bv > 0.0) {
            double cum = 0.0;
            int k = 0;
            for (; k < kScreenBins - 1; ++k) {
                const double add = (double)s_hist[k] * ldexp(1.0, k + 1 - kScreenOffset);
                if (cum + add > b.screen_eps * Bv) break;
                cum += add;
            }
            t = ldexp(1.0, k - kScreenOffset);
        }
        b.Tcell[c] = t;
    }
}

// Spreading arguments of one cell for the shared per-point code.
__device__ __forceinline__ void cell_args(const BatchArgs &b, const CellDesc &cd, bool f32, SpreadArgs &sa)
{
    sa.d = b.d;
    sa.N = cd.N;
    sa.M = cd.M;
    sa.r = b.r;
    sa.nnode = cd.nnode;
    sa.npairs = cd.pairs;
    sa.n = cd.n;
    sa.nf = cd.nf;
    sa.rows_per_slab = cd.nf;
    sa.nslab = 1;
    sa.fast_gamma = cd.fast_gamma;
    sa.S = cd.S;
    sa.gamma = cd.gamma;
    sa.Bconst = b.Bconst;
    sa.beta = b.beta;
    sa.grid_scale = cd.n / (2.0 * 3.14159265358979323846);
    sa.vnode = f32 ? (const void *)(b.v32 + cd.node_off) : (const void *)(b.v64 + cd.node_off);
    sa.vnode_lo = f32 ? b.v32lo + cd.node_off : nullptr;
    sa.a = f32 ? (const void *)(b.a32 + cd.a_off) : (const void *)(b.a64 + cd.a_off);
    sa.sig = f32 ? (const void *)(b.sig32 + cd.sig_off * b.d) : (const void *)(b.sig64 + cd.sig_off * b.d);
    sa.wsig = f32 ? (const void *)(b.wsig32 + cd.sig_off) : (const void *)(b.wsig64 + cd.sig_off);
    sa.Wsig = cd.Wsig;
    sa.wmax_frac = 1.0 / cd.M;  // the sphere sets have equal weights
    sa.bound = nullptr;
    sa.tau = nullptr;  // the batched kernel reads Tcell directly
    sa.grid = b.grid + cd.grid_off;
    sa.simple_fold = (b.w <= cd.n / 2) ? 1 : 0;
    sa.nang_even = 0;  // batched cells use VHS kernels
    sa.angmax = 1.0;
    sa.cpad = tile_col_pad(b.w);
    sa.ncol = cd.nf + 2 * sa.cpad;
    sa.kpoly = b.kpoly;
    sa.queued = 0;
    fill_spread_consts(sa);
}

template <typename T, int D>
constexpr int max_threads_of() { return sizeof(T) == 4 ? kBatchThreadsF32 : max_threads_f64(D); }

// Add a cell's block tile to the cell's global grid (padding columns folded onto their cells).
template <bool F32, int D>
__device__ __forceinline__ void batch_flush(const int *lo, const int *carry, const spread_detail::WideTile &wt,
                                            int ncell, int nf, int ncol, int cpad, int n, unsigned long long *grid,
                                            int shift)
{
    for (int e = threadIdx.x; e < ncell; e += blockDim.x) {
        const int gc = spread_detail::tile_to_grid_cell(e, D, nf, ncol, cpad, n, 0);
        if constexpr (F32) {
            const long long v = (long long)carry[e] * 4294967296LL + lo[e];
            if (v) atomicAdd(grid + gc, (unsigned long long)(v * (1ll << shift)));
        } else {
            const long long v = wt.value(e);  // grid units
            if (v) atomicAdd(grid + gc, (unsigned long long)v);
        }
    }
}

template <typename T, int D, int W>
__global__ void __launch_bounds__(max_threads_of<T, D>(), 1) k_batch_spread(const __grid_constant__ BatchArgs b)
{
    using namespace spread_detail;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ int s_item;
    __shared__ CellDesc s_cd;
    constexpr bool F32 = (sizeof(T) == 4);
    int cur = -1, ncell = 0, plane = 0, Eg = 0, shift = 0;
    T sc = T(0), tau = T(0), floor_q = T(0);
    // the current cell's spreading arguments live in shared memory: kept in registers they cost
    // 30-odd registers per thread (fewer resident warps, or spills under a 1024-thread bound)
    __shared__ SpreadArgs s_sa;
    SpreadArgs &sa = s_sa;
    if constexpr (!F32) load_kernel_poly(b.kpoly);  // the same kernel polynomial for every cell
    int *lo = reinterpret_cast<int *>(smem_raw);
    int *carry = F32 ? b.carry + (size_t)blockIdx.x * b.carry_stride : nullptr;
    // FP64: fraction, low and high words of the largest cell tile (carry_stride cells)
    unsigned *words = reinterpret_cast<unsigned *>(smem_raw);
    const WideTile wt{words, words + b.carry_stride, reinterpret_cast<int *>(words + 2 * b.carry_stride)};
    // add the current cell's tile to its grid (padding columns folded onto their cells)
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
    for (;;) {
        if (threadIdx.x == 0) s_item = atomicAdd(b.counter, 1);
        __syncthreads();
        const int item = s_item;
        if (item >= b.nitems) break;  // uniform over the block
        const int cell = b.item_cell[item];
        if (cell != cur) {
            if (cur >= 0)  // the previous cell's tile
                batch_flush<F32, D>(lo, carry, wt, ncell, s_cd.nf, sa.ncol, sa.cpad, s_cd.n, sa.grid, shift);
            __syncthreads();
            if (threadIdx.x == 0) s_cd = b.cells[cell];
            __syncthreads();
            cur = cell;
            if (threadIdx.x == 0) cell_args(b, s_cd, F32, sa);
            __syncthreads();
            plane = (D == 3) ? s_cd.nf * sa.ncol : sa.ncol;
            ncell = plane * s_cd.nf;
            const double Bc = b.Bcell[cell];
            Eg = global_exponent(Bc);
            const int Et = F32 ? min(Eg - tile_bits(D), 120) : Eg;
            shift = Eg - Et;
            sc = T(ldexp(1.0, Et));  // strengths in tile units (FP64: grid units, Et = Eg)
            tau = T(b.Tcell[cell]);
            // negligible points: FP32 points below 0.1 tile unit add exactly zero; FP64 pairs whose
            // summed bounds stay below 2^-64 B are skipped
            floor_q = F32 ? T(spread_detail::kNegligibleF32)
                          : T(ldexp(Bc, Eg - 64) * sa.cd.wmax / (double)s_cd.pairs);
            for (int e = threadIdx.x; e < ncell; e += blockDim.x) {
                if constexpr (F32) {
                    lo[e] = 0;
                    carry[e] = 0;
                } else {
                    wt.fr[e] = 0u;
                    wt.lo[e] = 0u;
                    wt.hi[e] = 0;
                }
            }
            __syncthreads();
        }
        // the item's node pairs; lanes of a warp take pairs nwarp apart
        const long long p0 = (long long)(item - s_cd.item0) * s_cd.chunk;
        const long long p1 = min(p0 + (long long)s_cd.chunk, s_cd.pairs);
        const long long first = p0 + (long long)lane * nwarp + warp;
        if constexpr (F32) {
            // the warp's queue compacts the points that add something (FP32 points below 0.1 tile
            // unit add exactly zero), so that every lane spreads a real point
            float *buf = reinterpret_cast<float *>(smem_raw + b.queue_off) + warp * 32 * spread_queue_values(D, true);
            spread_pairs_queued<T, D, W, SplitTile, false, false>(sa, first, p1, blockDim.x, sc, tau, floor_q,
                                                                   SplitTile{lo, carry}, 0, s_cd.nf, plane, buf);
        } else
            spread_pairs<T, D, W, WideTile, false>(sa, first, p1, blockDim.x, sc, tau, floor_q, wt, 0,
                                                      s_cd.nf, plane);
        __syncthreads();
    }
    if (cur >= 0) batch_flush<F32, D>(lo, carry, wt, ncell, s_cd.nf, sa.ncol, sa.cpad, s_cd.n, sa.grid, shift);
}

// One block per cell: Q = D(grid) - E(h) along every axis (Section 4.2).
__global__ void __launch_bounds__(kPrepThreads) k_batch_final(const __grid_constant__ BatchArgs b)
{
    const int c = blockIdx.x;
    const CellDesc cd = b.cells[c];
    const int d = b.d, N = cd.N, nf = cd.nf;
    double *s1 = b.scratch + cd.s_off, *s2 = s1 + cd.s_len, *s3 = s2 + cd.s_len, *s4 = s3 + cd.s_len;
    const double *Dm = b.D + cd.D_off;
    const double *E = b.E + cd.R_off;
    const double unit = ldexp(cd.corr, -global_exponent(b.Bcell[c]));
    Dims3 gd = dims3(d, nf, nf, nf);
    const int ax0 = 3 - d;
    block_pass_fixed(b.grid + cd.grid_off, gd, ax0, Dm, N + 1, unit, s1);
    __syncthreads();
    gd.e[ax0] = N + 1;
    const double *gcur = s1;
    if (d == 3) {
        block_pass(s1, gd, 1, Dm, N + 1, s2);
        __syncthreads();
        gd.e[1] = N + 1;
        gcur = s2;
    }
    Dims3 hd = dims3(d, N, N, N);
    const double *hcur = b.h + cd.a_off;
    double *hb[2] = {s3, s4};
    int which = 0;
    for (int ax = 3 - d; ax < 2; ++ax) {
        block_pass(hcur, hd, ax, E, N + 1, hb[which]);
        __syncthreads();
        hd.e[ax] = N + 1;
        hcur = hb[which];
        which ^= 1;
    }
    const int total = gd.e[0] * gd.e[1] * (N + 1);
    double *Q = b.Q + cd.f_off;
    for (int o = threadIdx.x; o < total; o += blockDim.x) {
        const int o2 = o % (N + 1), row = o / (N + 1);
        const double *gs = gcur + row * nf;
        const double *hs = hcur + row * N;
        double qp = 0.0, qm = 0.0;
        for (int s = 0; s < nf; ++s) qp = fma(Dm[o2 * nf + s], gs[s], qp);
        for (int s = 0; s < N; ++s) qm = fma(E[o2 * N + s], hs[s], qm);
        Q[o] = qp - qm;
    }
}

template <typename T, int D, int W>
cudaError_t set_spread_attr(size_t smem)
{
    return cudaFuncSetAttribute(k_batch_spread<T, D, W>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
}

template <typename T, int D, int W, int WMAX>
struct BatchDispatch {
    static cudaError_t attr(int w, size_t smem)
    {
        if (w == W) return set_spread_attr<T, D, W>(smem);
        return BatchDispatch<T, D, W + 1, WMAX>::attr(w, smem);
    }
    static cudaError_t launch(int w, const BatchArgs &b, int blocks, int threads, size_t smem, cudaStream_t s)
    {
        if (w == W) {
            k_batch_spread<T, D, W><<<blocks, threads, smem, s>>>(b);
            return cudaGetLastError();
        }
        return BatchDispatch<T, D, W + 1, WMAX>::launch(w, b, blocks, threads, smem, s);
    }
    static cudaError_t occupancy(int w, int threads, size_t smem, int *nblocks)
    {
        if (w == W) return cudaOccupancyMaxActiveBlocksPerMultiprocessor(nblocks, k_batch_spread<T, D, W>, threads, smem);
        return BatchDispatch<T, D, W + 1, WMAX>::occupancy(w, threads, smem, nblocks);
    }
};
template <typename T, int D, int WMAX>
struct BatchDispatch<T, D, WMAX, WMAX> {
    static cudaError_t attr(int w, size_t smem)
    {
        return (w == WMAX) ? set_spread_attr<T, D, WMAX>(smem) : cudaErrorInvalidValue;
    }
    static cudaError_t launch(int w, const BatchArgs &b, int blocks, int threads, size_t smem, cudaStream_t s)
    {
        if (w != WMAX) return cudaErrorInvalidValue;
        k_batch_spread<T, D, WMAX><<<blocks, threads, smem, s>>>(b);
        return cudaGetLastError();
    }
    static cudaError_t occupancy(int w, int threads, size_t smem, int *nblocks)
    {
        if (w != WMAX) return cudaErrorInvalidValue;
        return cudaOccupancyMaxActiveBlocksPerMultiprocessor(nblocks, k_batch_spread<T, D, WMAX>, threads, smem);
    }
};

// The batched spreading kernels cover the widths the FP32 path uses (w <= 10) in FP32 and
// the FP64 widths up to 16.
cudaError_t batch_spread_attr(bool f32, int d, int w, size_t smem)
{
    if (f32) return d == 2 ? BatchDispatch<float, 2, kMinWidth, kMaxWidthF32>::attr(w, smem)
                           : BatchDispatch<float, 3, kMinWidth, kMaxWidthF32>::attr(w, smem);
    return d == 2 ? BatchDispatch<double, 2, kMinWidth, kMaxWidthF64>::attr(w, smem)
                  : BatchDispatch<double, 3, kMinWidth, kMaxWidthF64>::attr(w, smem);
}

// Resident blocks per SM of the batched spreading kernel for a launch shape.
cudaError_t batch_spread_occupancy(bool f32, int d, int w, int threads, size_t smem, int *nblocks)
{
    if (f32) return d == 2 ? BatchDispatch<float, 2, kMinWidth, kMaxWidthF32>::occupancy(w, threads, smem, nblocks)
                           : BatchDispatch<float, 3, kMinWidth, kMaxWidthF32>::occupancy(w, threads, smem, nblocks);
    return d == 2 ? BatchDispatch<double, 2, kMinWidth, kMaxWidthF64>::occupancy(w, threads, smem, nblocks)
                  : BatchDispatch<double, 3, kMinWidth, kMaxWidthF64>::occupancy(w, threads, smem, nblocks);
}

cudaError_t batch_spread_launch(bool f32, int d, int w, const BatchArgs &b, int blocks, int threads, size_t smem,
                                cudaStream_t s)
{
    if (f32) return d == 2 ? BatchDispatch<float, 2, kMinWidth, kMaxWidthF32>::launch(w, b, blocks, threads, smem, s)
                           : BatchDispatch<float, 3, kMinWidth, kMaxWidthF32>::launch(w, b, blocks, threads, smem, s);
    return d == 2 ? BatchDispatch<double, 2, kMinWidth, kMaxWidthF64>::launch(w, b, blocks, threads, smem, s)
                  : BatchDispatch<double, 3, kMinWidth, kMaxWidthF64>::launch(w, b, blocks, threads, smem, s);
}

}  // namespace
}  // namespace pgb

// ============================================================================ host

struct BatchState {
    int d = 2, ncell = 0, r = 1, prec = PG_PREC_FP32, w = 0;
    double tol = 1e-6, sigma = 2.0, beta = 0.0;
    std::vector<long long> offsets;  // ncell + 1 packed mode offsets
    long long points = 0, pairs = 0, grid_cells = 0;
    int nitems = 0;
    int spread_blocks = 0, spread_threads = 0;
    size_t spread_smem = 0;
    size_t tile_smem = 0;    // dynamic shared memory of the largest cell tile (16-byte multiple)
    size_t static_smem = 0;  // the spreading kernel's static shared memory
    std::vector<pgb::CellDesc> cells;  // host copy of the cell descriptors (work items change)
    pgb::CellDesc *d_cells = nullptr;
    int *d_items = nullptr;   // cell of each work item
    int item_capacity = 0;    // work items d_items holds (the smallest item size's count)
    long long item_points = 0;  // points per work item
    int carry_blocks = 0;  // blocks the FP32 carry-counter array was sized for
    pgb::BatchArgs args{};
    bool use_graph = true;
    cudaStream_t cap_stream = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    const double *g_f = nullptr;
    double *g_Q = nullptr;
    cudaEvent_t ev[2] = {nullptr, nullptr};
    bool timing = false, timed = false;
};

void pg_free_batch(BatchState *b)
{
    if (!b) return;
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    if (b->cap_stream) cudaStreamDestroy(b->cap_stream);
    for (cudaEvent_t e : b->ev)
        if (e) cudaEventDestroy(e);
    delete b;
}

namespace {

constexpr long long kItemPoints = 1 << 17;     // points per work item (default)
constexpr long long kItemPointsMin = 1 << 15;  // the autotuner's work-item sizes: 2^15 .. 2^19
constexpr long long kItemPointsMax = 1 << 19;

// Split every cell's node pairs into work items of about item_points points (at least 64 pairs):
// sets each cell's chunk and first item; item_cell (optional) receives the cell of every item.
// Returns the number of items.
long long split_items(std::vector<pgb::CellDesc> &cells, long long item_points, std::vector<int> *item_cell)
{
    long long n = 0;
    if (item_cell) item_cell->clear();
    for (size_t c = 0; c < cells.size(); ++c) {
        pgb::CellDesc &cd = cells[c];
        cd.chunk = (int)std::max<long long>(64, item_points / cd.M);
        cd.item0 = (int)n;
        const long long nitem = (cd.pairs + cd.chunk - 1) / cd.chunk;
        if (item_cell) item_cell->insert(item_cell->end(), (size_t)nitem, (int)c);
        n += nitem;
    }
    return n;
}

// Dynamic shared memory of a spreading launch with `threads` threads: the largest cell's tile,
// then (FP32) one point queue per warp.
size_t batch_smem(const BatchState &B, int threads)
{
    return B.tile_smem + (B.prec == PG_PREC_FP32 ? pgb::spread_queue_bytes(threads, B.d, true) : 0);
}

int enqueue_batch(pg_boltz_plan_t *p, cudaStream_t s, const double *f, double *Q)
{
    BatchState &B = *p->batch;
    pgb::BatchArgs a = B.args;
    a.f = f;
    a.Q = Q;
    int rc;
    // the work counter and the grids share one allocation: [counter | 256-byte gap | grids]
    if ((rc = cuda_check(cudaMemsetAsync(a.counter, 0, 256 + (size_t)B.grid_cells * 8, s), "memset grids")))
        return rc;
    const bool f32 = (B.prec == PG_PREC_FP32);
    if (f32 && B.d == 2) pgb::k_batch_prep<float, 2><<<B.ncell, pgb::kPrepThreads, 0, s>>>(a);
    else if (f32) pgb::k_batch_prep<float, 3><<<B.ncell, pgb::kPrepThreads, 0, s>>>(a);
    else if (B.d == 2) pgb::k_batch_prep<double, 2><<<B.ncell, pgb::kPrepThreads, 0, s>>>(a);
    else pgb::k_batch_prep<double, 3><<<B.ncell, pgb::kPrepThreads, 0, s>>>(a);
    if ((rc = cuda_check(cudaGetLastError(), "batched prep"))) return rc;
    if ((rc = cuda_check(pgb::batch_spread_launch(f32, B.d, B.w, a, B.spread_blocks, B.spread_threads, B.spread_smem, s),
                         "batched spread")))
        return rc;
    pgb::k_batch_final<<<B.ncell, pgb::kPrepThreads, 0, s>>>(a);
    return cuda_check(cudaGetLastError(), "batched final");
}

}  // namespace

PG_API pg_boltz_plan_t *pg_boltz_plan_batched_ex(const pg_boltz_opts_t *opts, int ncell, const int *Ns, const int *Ms,
                                                 const double *Ss, const double *gammas)
{
    if (!opts || !Ns || !Ms || !Ss || !gammas || ncell < 1) {
        set_error(PG_ERR_ARG, "batched plan: NULL array or ncell < 1");
        return nullptr;
    }
    const pg_boltz_opts_t &o = *opts;
    if (o.d != 2 && o.d != 3) {
        set_error(PG_ERR_ARG, "d must be 2 or 3 (got %d)", o.d);
        return nullptr;
    }
    if (!(o.tol >= 1e-15 && o.tol <= 1e-2)) {
        set_error(PG_ERR_ARG, "tol must be in [1e-15, 1e-2] (got %g)", o.tol);
        return nullptr;
    }
    if (o.upsampfac != 0.0 && !(o.upsampfac >= 1.5 && o.upsampfac <= 4.0)) {
        set_error(PG_ERR_ARG, "upsampfac must be in [1.5, 4] (got %g)", o.upsampfac);
        return nullptr;
    }
    if (o.angular_terms != 0) {
        set_error(PG_ERR_ARG, "batched plans support VHS kernels only (angular_terms must be 0)");
        return nullptr;
    }
    for (int c = 0; c < ncell; ++c) {
        if (Ns[c] < 2 || Ns[c] > (o.d == 2 ? 200 : 40) || Ms[c] < 2 || Ms[c] % 2 || !(Ss[c] > 0.0) ||
            !(gammas[c] >= 0.0 && gammas[c] <= 1.0)) {
            set_error(PG_ERR_ARG, "cell %d: need 2 <= N <= %d, even M >= 2, S > 0, 0 <= gamma <= 1", c,
                      o.d == 2 ? 200 : 40);
            return nullptr;
        }
    }
    pg_boltz_plan_t *p = new (std::nothrow) pg_boltz_plan_t();
    BatchState *B = p ? new (std::nothrow) BatchState() : nullptr;
    if (!p || !B) {
        delete p;
        set_error(PG_ERR_NOMEM, "host allocation failed");
        return nullptr;
    }
    p->batch = B;
    if (cudaGetDevice(&p->device) != cudaSuccess) {
        cudaGetLastError();
        set_error(PG_ERR_CUDA, "no CUDA device available");
        free_plan(p);
        return nullptr;
    }
    const int d = o.d;
    B->d = d;
    B->ncell = ncell;
    B->r = o.map_log ? 0 : 1;
    B->tol = o.tol;
    B->prec = (o.precision == PG_PREC_AUTO) ? (o.tol < 1e-8 ? PG_PREC_FP64 : PG_PREC_FP32) : o.precision;
    B->sigma = (o.upsampfac > 0.0) ? o.upsampfac : 2.0;
    B->w = width_for(o.tol, B->sigma);
    const bool f32 = (B->prec == PG_PREC_FP32);
    const int wmax = f32 ? pgb::kMaxWidthF32 : pgb::kMaxWidthF64;
    if (B->w > wmax) {
        if (f32) B->w = wmax;
        else {
            set_error(PG_ERR_ARG, "tol %g needs kernel width %d > %d", o.tol, B->w, wmax);
            free_plan(p);
            return nullptr;
        }
    }
    B->beta = kernel_beta(B->w, B->sigma);
    const int sphere = (d == 3) ? (o.sphere == PG_SPHERE_AUTO ? PG_SPHERE_ANTIPODAL : o.sphere) : PG_SPHERE_AUTO;

    // ---- tables, shared between cells with equal parameters
    std::vector<double> v64, scale_a, inv_mu2, R, E, D, sig64, wsig64;
    std::map<std::pair<int, double>, int> node_key;
    std::map<int, std::pair<int, int>> mat_key;  // N -> (R_off, D_off)
    std::map<int, int> sig_key;
    std::vector<pgb::CellDesc> cells(ncell);
    std::vector<int> item_cell;
    long long f_off = 0, a_off = 0, grid_off = 0, s_off = 0;
    int max_cells_tile = 0;
    B->offsets.assign(ncell + 1, 0);
    for (int c = 0; c < ncell; ++c) {
        pgb::CellDesc &cd = cells[c];
        const int N = Ns[c], M = Ms[c];
        cd.N = N;
        cd.M = M;
        cd.n = grid_size(N, B->sigma);
        cd.nf = cd.n / 2 + 1;
        cd.nnode = (d == 2) ? N * N : N * N * N;
        cd.fast_gamma = (gammas[c] == 0.0) ? 0 : (gammas[c] == 1.0) ? 1 : (gammas[c] == 0.5) ? 2 : 3;
        cd.S = Ss[c];
        cd.gamma = gammas[c];
        cd.pairs = pgb::unordered_pairs(cd.nnode);
        auto nk = std::make_pair(N, Ss[c]);
        if (!node_key.count(nk)) {
            NodeTables nt = node_tables(N, Ss[c], B->r);
            node_key[nk] = (int)v64.size();
            v64.insert(v64.end(), nt.v.begin(), nt.v.end());
            scale_a.insert(scale_a.end(), nt.scale_a.begin(), nt.scale_a.end());
            inv_mu2.insert(inv_mu2.end(), nt.inv_mu2.begin(), nt.inv_mu2.end());
        }
        cd.node_off = node_key[nk];
        if (!mat_key.count(N)) {
            NodeTables nt = node_tables(N, 1.0, B->r);  // R and E do not depend on S
            std::vector<double> Dm = transform_matrix(N, cd.n, B->w, B->beta);
            mat_key[N] = std::make_pair((int)R.size(), (int)D.size());
            R.insert(R.end(), nt.R.begin(), nt.R.end());
            E.insert(E.end(), nt.E.begin(), nt.E.end());
            D.insert(D.end(), Dm.begin(), Dm.end());
        }
        cd.R_off = mat_key[N].first;
        cd.D_off = mat_key[N].second;
        if (!sig_key.count(M)) {
            std::vector<double> sp, sw;
            sphere_points(d, M, sphere, sp, sw);
            sig_key[M] = (int)wsig64.size();
            sig64.insert(sig64.end(), sp.begin(), sp.end());
            wsig64.insert(wsig64.end(), sw.begin(), sw.end());
        }
        cd.sig_off = sig_key[M];
        cd.Wsig = 0.0;
        for (int m = 0; m < M; ++m) cd.Wsig += wsig64[cd.sig_off + m];
        cd.corr = (B->prec == PG_PREC_FP32)
                      ? pgb::fp32_strength_correction(1.0 / (d == 2 ? 2.0 * kPi : 4.0 * kPi), wsig64[cd.sig_off], Ss[c], d)
                      : 1.0;
        const long long modes = (long long)ipow(N + 1, d);
        cd.f_off = f_off;
        B->offsets[c] = f_off;
        f_off += modes;
        cd.a_off = a_off;
        a_off += cd.nnode;
        const long long cells_tile = (long long)ipow(cd.nf, d);
        cd.grid_off = grid_off;
        grid_off += cells_tile;
        // block tile: the last axis padded with unfolded columns (see spread_impl.cuh)
        const long long tile_cells = (long long)ipow(cd.nf, d - 1) * (cd.nf + 2 * pgb::tile_col_pad(B->w));
        max_cells_tile = std::max<int>(max_cells_tile, (int)tile_cells);
        cd.s_len = std::max<long long>(modes, (long long)(N + 1) * (long long)ipow(cd.nf, d - 1));
        cd.s_off = s_off;
        s_off += 4 * cd.s_len;
        B->points += cd.pairs * M;
        B->pairs += cd.pairs;
    }
    B->offsets[ncell] = f_off;
    // work items: room for the autotuner's smallest item size, the default size to start with
    const long long capacity = split_items(cells, kItemPointsMin, nullptr);
    if (capacity > (1ll << 30)) {
        set_error(PG_ERR_ARG, "batched plan: too many work items (%lld)", capacity);
        free_plan(p);
        return nullptr;
    }
    B->item_capacity = (int)capacity;
    B->item_points = kItemPoints;
    split_items(cells, kItemPoints, &item_cell);
    B->nitems = (int)item_cell.size();
    B->grid_cells = grid_off;
    std::vector<float> v32(v64.begin(), v64.end()), sig32(sig64.begin(), sig64.end()), wsig32(wsig64.begin(), wsig64.end());
    std::vector<float> v32lo(v64.size());
    for (size_t k = 0; k < v64.size(); ++k) v32lo[k] = (float)(v64[k] - (double)v32[k]);

    pgb::BatchArgs &a = B->args;
    a.d = d;
    a.r = B->r;
    a.ncell = ncell;
    a.nitems = B->nitems;
    a.w = B->w;
    a.Bconst = 1.0 / (d == 2 ? 2.0 * kPi : 4.0 * kPi);
    a.beta = B->beta;
    a.screen_eps = o.screen ? 0.05 * o.tol : 0.0;
    pgb::CellDesc *d_cells = nullptr;
    int *d_items = nullptr;
    double *d_v64 = nullptr, *d_sa = nullptr, *d_im = nullptr, *d_R = nullptr, *d_E = nullptr, *d_D = nullptr,
           *d_s64 = nullptr, *d_w64 = nullptr, *d_kp = nullptr;
    float *d_v32 = nullptr, *d_v32lo = nullptr, *d_s32 = nullptr, *d_w32 = nullptr;
    void *counter_grid = nullptr;
    std::vector<double> kpoly(pgb::kPolyCoefF64, 0.0);
    kernel_poly(B->w, B->beta, kpoly.data());
    // each failing call has recorded its error for pg_boltz_last_error
    std::vector<int> items_room(item_cell);  // the item array has room for the smallest item size
    items_room.resize((size_t)B->item_capacity, 0);
    if (upload(p, &d_cells, cells) || upload(p, &d_kp, kpoly) || upload(p, &d_items, items_room) ||
        upload(p, &d_v64, v64) || upload(p, &d_v32, v32) || upload(p, &d_v32lo, v32lo) || upload(p, &d_sa, scale_a) ||
        upload(p, &d_im, inv_mu2) ||
        upload(p, &d_R, R) || upload(p, &d_E, E) || upload(p, &d_D, D) || upload(p, &d_s64, sig64) ||
        upload(p, &d_s32, sig32) || upload(p, &d_w64, wsig64) || upload(p, &d_w32, wsig32) ||
        dev_alloc(p, (void **)&a.a64, a_off * 8) || dev_alloc(p, (void **)&a.a32, a_off * 4) ||
        dev_alloc(p, (void **)&a.h, a_off * 8) || dev_alloc(p, (void **)&a.Bcell, (size_t)ncell * 8) ||
        dev_alloc(p, (void **)&a.Tcell, (size_t)ncell * 8) || dev_alloc(p, &counter_grid, 256 + (size_t)grid_off * 8) ||
        dev_alloc(p, (void **)&a.scratch, (size_t)s_off * 8)) {
        free_plan(p);
        return nullptr;
    }
    a.cells = d_cells;
    a.item_cell = d_items;
    B->cells = cells;
    B->d_cells = d_cells;
    B->d_items = d_items;
    a.counter = static_cast<int *>(counter_grid);
    a.grid = reinterpret_cast<unsigned long long *>(static_cast<char *>(counter_grid) + 256);
    a.v64 = d_v64;
    a.v32 = d_v32;
    a.v32lo = d_v32lo;
    a.scale_a = d_sa;
    a.inv_mu2 = d_im;
    a.R = d_R;
    a.E = d_E;
    a.D = d_D;
    a.sig64 = d_s64;
    a.sig32 = d_s32;
    a.wsig64 = d_w64;
    a.wsig32 = d_w32;
    a.kpoly = d_kp;

    // ---- persistent spreading launch shape
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, p->device) != cudaSuccess) {
        set_error(PG_ERR_CUDA, "cudaGetDeviceProperties failed");
        free_plan(p);
        return nullptr;
    }
    // FP32: one 32-bit word per cell; FP64: three
    B->tile_smem = pgb::tile_bytes((size_t)max_cells_tile, f32);
    a.queue_off = (int)B->tile_smem;
    // the kernel's static shared memory: the current cell's descriptor and spreading arguments,
    // FP64: the kernel polynomial
    B->static_smem =
        sizeof(pgb::CellDesc) + sizeof(pgb::SpreadArgs) + 64 + (f32 ? 0 : sizeof(double) * pgb::kPolyCoefF64);
    const size_t per_block_extra = B->static_smem + 1024 + prop.reservedSharedMemPerBlock;
    if (batch_smem(*B, 128) + B->static_smem > prop.sharedMemPerBlockOptin) {
        set_error(PG_ERR_ARG, "largest cell's folded grid (%d cells) does not fit shared memory", max_cells_tile);
        free_plan(p);
        return nullptr;
    }
    const int max_threads = f32 ? pgb::kBatchThreadsF32 : pgb::max_threads_f64(B->d);
    int per_sm = (int)(prop.sharedMemPerMultiprocessor / (batch_smem(*B, 128) + per_block_extra));
    per_sm = std::max(per_sm, 1);
    if (o.spread_blocks_per_sm > 0) per_sm = std::min(per_sm, o.spread_blocks_per_sm);
    B->spread_threads = (o.spread_threads > 0) ? o.spread_threads
                                                : std::max(128, std::min(max_threads, (1024 / per_sm) / 32 * 32));
    if (B->spread_threads % 32 || B->spread_threads > max_threads) {
        set_error(PG_ERR_ARG, "spread_threads must be a multiple of 32 and <= %d", max_threads);
        free_plan(p);
        return nullptr;
    }
    B->spread_smem = batch_smem(*B, B->spread_threads);
    if (B->spread_smem + B->static_smem > prop.sharedMemPerBlockOptin) {
        set_error(PG_ERR_ARG, "largest cell's folded grid (%d cells) and the queues of %d threads do not fit "
                  "shared memory", max_cells_tile, B->spread_threads);
        free_plan(p);
        return nullptr;
    }
    per_sm = std::min(per_sm, std::max(1, prop.maxThreadsPerMultiProcessor / B->spread_threads));
    per_sm = std::min(per_sm, std::max(1, (int)(prop.sharedMemPerMultiprocessor / (B->spread_smem + per_block_extra))));
    B->spread_blocks = prop.multiProcessorCount * per_sm;
    a.carry = nullptr;
    a.carry_stride = max_cells_tile;
    B->carry_blocks = B->spread_blocks;
    if (f32 && dev_alloc(p, (void **)&a.carry, (size_t)B->spread_blocks * max_cells_tile * sizeof(int))) {
        free_plan(p);
        return nullptr;
    }
    // the attribute covers every launch shape the autotuner may try
    const size_t smem_attr = std::min(batch_smem(*B, max_threads), prop.sharedMemPerBlockOptin - B->static_smem);
    if (cuda_check(pgb::batch_spread_attr(f32, d, B->w, smem_attr), "batched spread attribute")) {
        free_plan(p);
        return nullptr;
    }
    pg_boltz_info_t &in = p->info;
    in.d = d;
    in.N = Ns[0];
    in.M = Ms[0];
    in.r = B->r;
    in.precision = B->prec;
    in.sphere = sphere;
    in.tol = o.tol;
    in.upsampfac = B->sigma;
    in.kernel_width = B->w;
    in.kernel_beta = B->beta;
    in.slabs = 1;
    in.spread_blocks = B->spread_blocks;
    in.spread_threads = B->spread_threads;
    in.spread_smem_bytes = B->spread_smem;
    in.points = B->points;
    in.pairs = B->pairs;
    in.launches_per_collide = 4;
    in.kernels_per_collide = 3;
    in.device_bytes = p->device_bytes;
    p->d = d;
    p->prec = B->prec;
    return p;
}

PG_API pg_boltz_plan_t *pg_boltz_plan_batched(int d, int ncell, const int *N, const int *M, const double *S,
                                              const double *kernel_gamma, double tol)
{
    pg_boltz_opts_t o;
    std::memset(&o, 0, sizeof(o));
    o.d = d;
    o.tol = tol;
    return pg_boltz_plan_batched_ex(&o, ncell, N, M, S, kernel_gamma);
}

PG_API int pg_boltz_batched_offsets(const pg_boltz_plan_t *p, long long *offsets_host)
{
    if (!p || !p->batch || !offsets_host) return set_error(PG_ERR_ARG, "not a batched plan, or NULL output");
    std::memcpy(offsets_host, p->batch->offsets.data(), sizeof(long long) * p->batch->offsets.size());
    return PG_OK;
}

PG_API int pg_boltz_collide_batched(pg_boltz_plan_t *p, const double *f_dev, double *Q_dev)
{
    if (!p) return set_error(PG_ERR_ARG, "plan is NULL");
    if (!p->batch) return set_error(PG_ERR_STATE, "pg_boltz_collide_batched needs a batched plan");
    if (!f_dev || !Q_dev) return set_error(PG_ERR_ARG, "f or Q is NULL");
    BatchState &B = *p->batch;
    const long long modes = B.offsets.back();
    const char *fb = reinterpret_cast<const char *>(f_dev);
    const char *qb = reinterpret_cast<const char *>(Q_dev);
    if (fb < qb + modes * 8 && qb < fb + modes * 8) return set_error(PG_ERR_ARG, "f and Q overlap");
    DeviceGuard guard(p->device);
    if (!guard.ok) return set_error(PG_ERR_CUDA, "cannot select the plan's device");
    int rc;
    if (B.timing) cudaEventRecord(B.ev[0], p->stream);
    if (!B.use_graph) {
        if ((rc = enqueue_batch(p, p->stream, f_dev, Q_dev))) return rc;
    } else {
        if (!B.exec || B.g_f != f_dev || B.g_Q != Q_dev) {
            // capture the launch sequence once per (f, Q) pair, then replay it
            if (B.exec) {
                cudaGraphExecDestroy(B.exec);
                B.exec = nullptr;
            }
            if (B.graph) {
                cudaGraphDestroy(B.graph);
                B.graph = nullptr;
            }
            if (!B.cap_stream && (rc = cuda_check(cudaStreamCreateWithFlags(&B.cap_stream, cudaStreamNonBlocking),
                                                  "capture stream")))
                return rc;
            if ((rc = cuda_check(cudaStreamBeginCapture(B.cap_stream, cudaStreamCaptureModeThreadLocal), "begin capture")))
                return rc;
            rc = enqueue_batch(p, B.cap_stream, f_dev, Q_dev);
            cudaGraph_t g = nullptr;
            cudaError_t e = cudaStreamEndCapture(B.cap_stream, &g);
            if (rc) {
                if (g) cudaGraphDestroy(g);
                return rc;
            }
            if ((rc = cuda_check(e, "end capture"))) return rc;
            B.graph = g;
            if ((rc = cuda_check(cudaGraphInstantiate(&B.exec, B.graph, 0), "graph instantiate"))) return rc;
            B.g_f = f_dev;
            B.g_Q = Q_dev;
        }
        if ((rc = cuda_check(cudaGraphLaunch(B.exec, p->stream), "graph launch"))) return rc;
    }
    if (B.timing) {
        cudaEventRecord(B.ev[1], p->stream);
        B.timed = true;
    }
    p->have_q = false;
    return PG_OK;
}

PG_API int pg_boltz_batched_use_graph(pg_boltz_plan_t *p, int enable)
{
    if (!p || !p->batch) return set_error(PG_ERR_ARG, "not a batched plan");
    p->batch->use_graph = enable != 0;
    return PG_OK;
}

// Time a set of launch shapes of the persistent spreading kernel on the caller's data and keep the
// fastest: threads per block in {128, 256, 512, 1024} (within the kernel's bound) and every
// blocks-per-SM count the kernel's occupancy allows, up to the blocks the carry counters were
// sized for.  Each shape: one launch sequence to warm up, then the best of `trials` timed ones.
namespace {

// Re-split the cells into work items of about item_points points and upload the new item table
// (synchronises the plan's stream: the host tables are temporaries).
int apply_item_points(pg_boltz_plan_t *p, long long item_points)
{
    BatchState &B = *p->batch;
    std::vector<int> item_cell;
    const long long n = split_items(B.cells, item_points, &item_cell);
    if (n > B.item_capacity) return set_error(PG_ERR_STATE, "work items exceed the plan's item table");
    int rc;
    if ((rc = cuda_check(cudaMemcpyAsync(B.d_cells, B.cells.data(), B.cells.size() * sizeof(pgb::CellDesc),
                                         cudaMemcpyHostToDevice, p->stream), "upload cells")) ||
        (rc = cuda_check(cudaMemcpyAsync(B.d_items, item_cell.data(), (size_t)n * sizeof(int),
                                         cudaMemcpyHostToDevice, p->stream), "upload work items")) ||
        (rc = cuda_check(cudaStreamSynchronize(p->stream), "stream sync")))
        return rc;
    B.nitems = (int)n;
    B.args.nitems = (int)n;
    B.item_points = item_points;
    return PG_OK;
}

}  // namespace

PG_API int pg_boltz_batched_autotune(pg_boltz_plan_t *p, const double *f_dev, double *Q_dev, int trials,
                                     int *threads_out, int *blocks_out, long long *item_points_out, double *ms_out)
{
    if (!p) return set_error(PG_ERR_ARG, "plan is NULL");
    if (!p->batch) return set_error(PG_ERR_STATE, "pg_boltz_batched_autotune needs a batched plan");
    if (!f_dev || !Q_dev) return set_error(PG_ERR_ARG, "f or Q is NULL");
    if (trials < 1 || trials > 100) return set_error(PG_ERR_ARG, "trials must be in [1, 100]");
    BatchState &B = *p->batch;
    const long long modes = B.offsets.back();
    const char *fb = reinterpret_cast<const char *>(f_dev);
    const char *qb = reinterpret_cast<const char *>(Q_dev);
    if (fb < qb + modes * 8 && qb < fb + modes * 8) return set_error(PG_ERR_ARG, "f and Q overlap");
    DeviceGuard guard(p->device);
    if (!guard.ok) return set_error(PG_ERR_CUDA, "cannot select the plan's device");
    cudaDeviceProp prop;
    int rc = cuda_check(cudaGetDeviceProperties(&prop, p->device), "cudaGetDeviceProperties");
    if (rc) return rc;
    const bool f32 = (B.prec == PG_PREC_FP32);
    const int max_threads = f32 ? pgb::kBatchThreadsF32 : pgb::max_threads_f64(B.d);
    const int best0_threads = B.spread_threads, best0_blocks = B.spread_blocks;
    const long long best0_items = B.item_points;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if ((rc = cuda_check(cudaEventCreate(&e0), "event")) || (rc = cuda_check(cudaEventCreate(&e1), "event"))) {
        if (e0) cudaEventDestroy(e0);
        return rc;
    }
    // best of `trials` timed runs of the current configuration after one warm-up
    auto time_config = [&](double &ms_best) -> int {
        ms_best = 1e300;
        int r = PG_OK;
        for (int t = 0; t <= trials && r == PG_OK; ++t) {
            if ((r = cuda_check(cudaEventRecord(e0, p->stream), "event record"))) break;
            if ((r = enqueue_batch(p, p->stream, f_dev, Q_dev))) break;
            if ((r = cuda_check(cudaEventRecord(e1, p->stream), "event record"))) break;
            if ((r = cuda_check(cudaEventSynchronize(e1), "event sync"))) break;
            float ms = 0.0f;
            if ((r = cuda_check(cudaEventElapsedTime(&ms, e0, e1), "elapsed"))) break;
            if (t > 0) ms_best = std::min(ms_best, (double)ms);  // t = 0 warms up
        }
        return r;
    };
    // 1. launch shapes at the current work-item size
    int best_threads = best0_threads, best_blocks = best0_blocks;
    double best_ms = 1e300;
    for (int threads = 128; threads <= max_threads && rc == PG_OK; threads *= 2) {
        int occ = 0;
        const size_t smem = batch_smem(B, threads);
        if (smem + B.static_smem > prop.sharedMemPerBlockOptin) continue;
        if (pgb::batch_spread_occupancy(f32, B.d, B.w, threads, smem, &occ) != cudaSuccess || occ < 1) continue;
        for (int per_sm = 1; per_sm <= occ && rc == PG_OK; ++per_sm) {
            const int blocks = prop.multiProcessorCount * per_sm;
            if (f32 && blocks > B.carry_blocks) break;  // no carry counters for more blocks
            B.spread_threads = threads;
            B.spread_blocks = blocks;
            B.spread_smem = smem;
            double ms_best = 1e300;
            rc = time_config(ms_best);
            if (rc == PG_OK && ms_best < best_ms) {
                best_ms = ms_best;
                best_threads = threads;
                best_blocks = blocks;
            }
        }
    }
    // 2. work-item sizes at the best shape
    long long best_items = B.item_points;
    if (rc == PG_OK) {
        B.spread_threads = best_threads;
        B.spread_blocks = best_blocks;
        B.spread_smem = batch_smem(B, best_threads);
        for (long long ip = kItemPointsMin; ip <= kItemPointsMax && rc == PG_OK; ip *= 2) {
            if (ip == best_items) continue;  // timed in step 1
            double ms_best = 1e300;
            if ((rc = apply_item_points(p, ip)) || (rc = time_config(ms_best))) break;
            if (ms_best < best_ms) {
                best_ms = ms_best;
                best_items = ip;
            }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    B.spread_threads = (rc == PG_OK) ? best_threads : best0_threads;
    B.spread_blocks = (rc == PG_OK) ? best_blocks : best0_blocks;
    B.spread_smem = batch_smem(B, B.spread_threads);
    const int rc_items = apply_item_points(p, (rc == PG_OK) ? best_items : best0_items);
    // the captured graph holds the old launch shape and item count: capture again on the next call
    if (B.exec) {
        cudaGraphExecDestroy(B.exec);
        B.exec = nullptr;
    }
    if (B.graph) {
        cudaGraphDestroy(B.graph);
        B.graph = nullptr;
    }
    if (rc) return rc;
    if (rc_items) return rc_items;
    p->info.spread_threads = B.spread_threads;
    p->info.spread_blocks = B.spread_blocks;
    p->info.spread_smem_bytes = B.spread_smem;
    if (threads_out) *threads_out = B.spread_threads;
    if (blocks_out) *blocks_out = B.spread_blocks;
    if (item_points_out) *item_points_out = B.item_points;
    if (ms_out) *ms_out = best_ms;
    return PG_OK;
}

// Timing of batched plans (called by pg_boltz_set_timing / pg_boltz_stage_times): events around
// the whole call (prep, spreading and finalisation), reported as the spreading stage.
int pg_batched_timing(pg_boltz_plan_t *p, int enable)
{
    BatchState &B = *p->batch;
    if (enable && !B.ev[0]) {
        int rc;
        if ((rc = cuda_check(cudaEventCreate(&B.ev[0]), "cudaEventCreate")) ||
            (rc = cuda_check(cudaEventCreate(&B.ev[1]), "cudaEventCreate")))
            return rc;
    }
    B.timing = enable != 0;
    B.timed = false;
    return PG_OK;
}

int pg_batched_elapsed(pg_boltz_plan_t *p, double *ms_out)
{
    BatchState &B = *p->batch;
    if (!B.timed) return set_error(PG_ERR_STATE, "no timed batched collide since timing was enabled");
    int rc = cuda_check(cudaEventSynchronize(B.ev[1]), "cudaEventSynchronize");
    if (rc) return rc;
    float ms = 0.0f;
    if ((rc = cuda_check(cudaEventElapsedTime(&ms, B.ev[0], B.ev[1]), "cudaEventElapsedTime"))) return rc;
    ms_out[0] = 0.0;
    ms_out[1] = 0.0;
    ms_out[2] = ms;
    ms_out[3] = 0.0;
    return PG_OK;
}
