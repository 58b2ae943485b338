// Spreading kernel templates shared by the FP32 and FP64 translation units.
//
// Fused post-collision point generation + exponential-of-semicircle spreading onto
// the folded cosine grid (Section 4.2, Eq. num_fast_k and Eq. nufft).
//
// One thread owns one node pair (i, j) and walks the M sphere points sigma_m:
//   v'     = (v_i + v_j)/2 + |v_i - v_j| sigma_m / 2
//   z_l    = arccos(xi(v'_l))                     angle of the l-th mapped coordinate
//   q      = a_i a_j B(|v_i - v_j|) w_m prod_l mu(xi(v'_l))^-2
// and adds q prod_l psi(x_{g_l} - z_l) to the w^d cells of the folded grid around z.
// The gain coefficient is the cosine sum sum_p q_p prod_l cos(k_l z_pl); cos is even
// and 2 pi periodic, so the periodic grid of n cells folds onto its n/2 + 1 cells
// g = 0..n/2: every unfolded support index u is added at fold(u) = min(u mod n, n - u mod n).
//
// Stable forms of the angle and the weight from the map formulas of Section 2.1:
//   r = 1 (algebraic):   cos z = v/sqrt(S^2+v^2), sin z = S/sqrt(S^2+v^2)
//                        -> z = atan2(S, v),      mu^-2 = (S^2 + v^2)/S
//   r = 0 (logarithmic): cos z = tanh(v/S), sin z = sech(v/S)
//                        -> z = 2 atan(e^(-v/S)), mu^-2 = S cosh(v/S)
//                           (FP64: from e = e^-|v/S| <= 1, z = 2 atan(e) or pi - 2 atan(e))
// Kernel values: FP32 from ex2.approx / rsqrt.approx of the definition; FP64 from per-tap
// polynomials fitted on the host (kernel_weights_f64).
//
// Accumulation:
//  - the global folded grid holds int64 values in units of 2^-Eg, where B >= sum_p |q_p|
//    (an upper bound written by the loss kernel) and B 2^Eg <= 2^61: no cell can overflow,
//    and block partial sums add exactly and in any order;
//  - FP64 kernel: each block adds into a private FP64 copy of its slab of the grid in shared
//    memory; at the end each cell's partial sum is rounded to the grid unit (relative error
//    2^-61 B) and added to the global grid.
//  - FP32 kernel: the private copy holds one signed 32-bit fixed-point word per cell in units of
//    2^-Et, Et = Eg - kTileBits, plus per-cell carry counters in a per-block global array
//    (SplitTile): a contribution goes to its word with one native 32-bit shared atomic, and only
//    an addition that wraps the word's signed range (seen from the returned old value) adds +-1
//    to the cell's carry counter (units of 2^32).  (Floating-point shared atomics are
//    compare-and-swap loops and their rounding limits FP32 accuracy; 64-bit integer shared
//    atomics are several times slower than 32-bit ones.)  At the end each block adds
//    word + carry 2^32 (scaled by 2^kTileBits) to the global grid.  Each contribution is rounded
//    once, to the tile unit; all later additions are exact.
#pragma once

#include <climits>
#include <cuda_runtime.h>

#include "pgb_internal.cuh"

namespace pgb {
namespace spread_detail {

template <typename T>
struct Fn;

template <>
struct Fn<float> {
    static __device__ __forceinline__ float sqrt_(float x) { return sqrtf(x); }
    static __device__ __forceinline__ float atan2_(float y, float x) { return atan2f(y, x); }
    static __device__ __forceinline__ float cosh_(float x) { return coshf(x); }
    static __device__ __forceinline__ float pow_(float x, float y) { return powf(x, y); }
    static __device__ __forceinline__ float floor_(float x) { return floorf(x); }
};

template <>
struct Fn<double> {
    static __device__ __forceinline__ double sqrt_(double x) { return sqrt(x); }
    static __device__ __forceinline__ double atan2_(double y, double x) { return atan2(y, x); }
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

// Unfolded index u -> folded cell; `simple` when u is known to lie in [-n/2, n].
__device__ __forceinline__ int fold_cell(int u, int n, bool simple)
{
    if (simple) {  // u in [-n/2, n]: fold(u) = min(|u|, n - |u|)
        u = abs(u);
        return min(u, n - u);
    }
    return fold_index(u, n);
}

// The w kernel weights psi(x_u - z) of one axis, u = s..s+w-1, in units where one grid cell
// is 1 and x = z n / (2 pi): psi = exp(beta (sqrt(1 - t^2) - 1)), t = (u - x) 2/w.  Returns
// the first unfolded index s.
template <int W>
__device__ __forceinline__ int kernel_weights_f32(const SpreadArgs &p, float x, float *wt);

// FP64: psi of tap a is a polynomial (kernel_poly_terms(w) terms) in the point's offset
// y = 2 (s - x) + w - 1 in (-1, 1] (t = (y + 1 + 2a - w)/w), fitted on the host.  Taps a and
// w-1-a mirror each other (t_{w-1-a}(-y) = -t_a(y) and psi is even), so one even part E_a(y^2)
// and one odd part y O_a(y^2) give both: about w + 2 FMAs per tap pair instead of an exp and a
// sqrt per tap.
// The coefficients sit in shared memory (s_kpoly, filled by load_kernel_poly at the start of each
// FP64 spreading kernel) and are read through an offset the compiler cannot see to be zero: read
// in place they cost one shared load each, whereas hoisted out of the point loops they would
// hold ~4 registers per tap and coefficient (spills at w >= 15).
__shared__ double s_kpoly[kPolyCoefF64];

__device__ __forceinline__ void load_kernel_poly(const double *kpoly)
{
    for (int k = threadIdx.x; k < kPolyCoefF64; k += blockDim.x) s_kpoly[k] = kpoly[k];
}

template <int W>
__device__ __forceinline__ int kernel_weights_f64(double x, double *wt)
{
    constexpr int P = kernel_poly_terms(W), NE = (P + 1) / 2, NO = P / 2;
    int zero;
    asm volatile("mov.b32 %0, 0;" : "=r"(zero));
    const double *cb = s_kpoly + zero;
    const int s = (int)floor(x - 0.5 * W) + 1;
    const double y = fma(2.0, double(s) - x, double(W - 1));
    const double u = y * y;
#pragma unroll
    for (int a = 0; a < (W + 1) / 2; ++a) {
        const double *c = cb + a * P;
        double e = c[NE - 1];
#pragma unroll
        for (int k = NE - 2; k >= 0; --k) e = fma(e, u, c[k]);
        if (2 * a + 1 == W) {  // middle tap of an odd width: even in y
            wt[a] = e;
        } else {
            double o = c[NE + NO - 1];
#pragma unroll
            for (int k = NO - 2; k >= 0; --k) o = fma(o, u, c[NE + k]);
            wt[a] = fma(y, o, e);
            wt[W - 1 - a] = fma(-y, o, e);
        }
    }
    return s;
}

template <typename T, int W>
__device__ __forceinline__ int kernel_weights(const SpreadArgs &p, T x, T *wt)
{
    if constexpr (sizeof(T) == 4) return kernel_weights_f32<W>(p, x, wt);
    else return kernel_weights_f64<W>(x, wt);
}

// The weights and the folded cells fold(s + a) of one axis.
template <typename T, int W>
__device__ __forceinline__ void axis_weights(const SpreadArgs &p, T x, T *wt, int *idx)
{
    const int s = kernel_weights<T, W>(p, x, wt);
    const bool simple = p.simple_fold != 0;
#pragma unroll
    for (int a = 0; a < W; ++a) idx[a] = fold_cell(s + a, p.n, simple);
}

__device__ __forceinline__ float ex2_approx(float x)
{
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float rsqrt_approx(float x)
{
    float y;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__device__ __forceinline__ float rcp_approx(float x)
{
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// atan(t) for t >= 0: t P(t^2) on [0, 1] and pi/2 - atan(1/t) above.  P is a degree-8
// polynomial in t^2 fitted to atan(t)/t on [0, 1] by iteratively reweighted least squares
// (towards the minimax error of t P(t^2)); its error is below 1e-7 when evaluated in FP32.
__device__ __forceinline__ float atan_pos_f32(float t)
{
    const bool inv = t > 1.0f;
    const float u = inv ? rcp_approx(t) : t;
    const float x = u * u;
    float p = 0.002455897797786189f;
    p = fmaf(p, x, -0.014397678937342222f);
    p = fmaf(p, x, 0.03977441675320232f);
    p = fmaf(p, x, -0.07234180246738538f);
    p = fmaf(p, x, 0.10498555283788273f);
    p = fmaf(p, x, -0.1416109770841035f);
    p = fmaf(p, x, 0.19985882274088168f);
    p = fmaf(p, x, -0.33332594819936656f);
    p = fmaf(p, x, 0.9999998857035092f);
    const float r = u * p;
    return inv ? 1.5707963267948966f - r : r;
}

// FP32 angle z = arccos(xi(v)) and weight mu(xi(v))^-2 of one mapped coordinate (Section 2.1):
//   r = 1: z = pi/2 - atan(v/S),          mu^-2 = (S^2 + v^2)/S
//   r = 0: z = 2 atan(exp(-v/S)),         mu^-2 = S (exp(v/S) + exp(-v/S))/2
__device__ __forceinline__ void angle_weight_f32(float v, float S, float invS, bool alg, float &z, float &m2)
{
    if (alg) {
        const float w = v * invS;
        const float at = atan_pos_f32(fabsf(w));
        z = 1.5707963267948966f - copysignf(at, w);
        m2 = fmaf(v, v, S * S) * invS;
    } else {
        const float e = ex2_approx(-v * invS * 1.4426950408889634f);  // exp(-v/S)
        z = 2.0f * atan_pos_f32(e);
        m2 = 0.5f * S * (rcp_approx(e) + e);
    }
}

// FP32 weights: t_a = (s - x) 2/w + a 2/w, psi = 2^(beta log2(e) (sqrt(1 - t^2) - 1)), with the
// square root as (1 - t^2) rsqrt(1 - t^2); both approximations are good to a few 1e-7.
template <int W>
__device__ __forceinline__ int kernel_weights_f32(const SpreadArgs &p, float x, float *wt)
{
    const int s = (int)floorf(x - 0.5f * W) + 1;
    const float h2 = 2.0f / W;
    const float t0 = ((float)s - x) * h2;
    const float bl = (float)(p.beta * 1.4426950408889634);
#pragma unroll
    for (int a = 0; a < W; ++a) {
        const float t = t0 + (float)a * h2;
        const float om = fmaf(-t, t, 1.0f);
        const float e = fmaf(bl, om * rsqrt_approx(om), -bl);
        wt[a] = om > 0.0f ? ex2_approx(e) : 0.0f;
    }
    return s;
}

template <typename T, int D>
struct PairData {
    T cen[D];  // (v_i + v_j)/2
    T rad;     // |v_i - v_j|/2
    T base;    // a_i a_j B(|v_i - v_j|)
    T mult;    // 2 for i != j (the pair stands for (i, j) and (j, i)), 1 for i == j
    T dir[D];  // (v_i - v_j)/|v_i - v_j| (0 for i == j): cos theta = dir . sigma_m
};

// Unordered node pairs.  Swapping i and j keeps the centre (v_i + v_j)/2, the radius
// |v_i - v_j|/2 and the strength a_i a_j B(|v_i - v_j|) w_m, so (i, j) and (j, i) add the same
// M points with the same weights: each unordered pair is spread once with twice the strength.
// Numbering: pair pr = t nnode + i is (i, (i + t) mod nnode), offsets t = 0..floor(nnode/2);
// t = 0 is the diagonal (multiplicity 1) and, for even nnode, the row t = nnode/2 stops at
// i = nnode/2 - 1 (its other half repeats the same pairs): unordered_pairs(nnode) in all.

// Load pair pr; false when its strength is zero.  ANG: also the unit direction (angular kernels).
template <typename T, int D, bool ANG = false>
__device__ __forceinline__ bool load_pair(const SpreadArgs &p, long long pr, PairData<T, D> &P)
{
    const int nnode = p.nnode, N = p.N;
    const int t = (int)(pr / nnode);
    const int i = (int)(pr - (long long)t * nnode);
    int j = i + t;
    if (j >= nnode) j -= nnode;
    P.mult = t ? T(2) : T(1);
    const T *vnode = static_cast<const T *>(p.vnode);
    const T *acoef = static_cast<const T *>(p.a);
    const T aij = acoef[i] * acoef[j];
    if (aij == T(0)) return false;
    int ii = i, jj = j;
    T g2 = T(0);
#pragma unroll
    for (int l = D - 1; l >= 0; --l) {
        const T vi = vnode[ii % N], vj = vnode[jj % N];
        ii /= N;
        jj /= N;
        const T dl = vi - vj;
        g2 += dl * dl;
        P.cen[l] = T(0.5) * (vi + vj);
        if constexpr (ANG) P.dir[l] = dl;
    }
    const T g = Fn<T>::sqrt_(g2);
    if constexpr (ANG) {
        const T ginv = g > T(0) ? T(1) / g : T(0);
#pragma unroll
        for (int l = 0; l < D; ++l) P.dir[l] *= ginv;
    }
    T B;
    switch (p.fast_gamma) {
    case 0: B = T(p.Bconst); break;
    case 1: B = T(p.Bconst) * g; break;
    case 2: B = T(p.Bconst) * Fn<T>::sqrt_(g); break;
    default: B = T(p.Bconst) * Fn<T>::pow_(g, T(p.gamma)); break;
    }
    P.base = aij * B;
    P.rad = T(0.5) * g;
    return P.base != T(0);
}

// U >= sum_m |q_m|: |base| W_sigma prod_l mu^-2(|c_l| + rad), since |v'_l| <= |c_l| + rad and
// mu^-2 grows with |v|.
template <typename T, int D>
__device__ __forceinline__ T pair_bound(const SpreadArgs &p, const PairData<T, D> &P)
{
    const T S = T(p.S), invS = T(1) / S;
    T U = fabs(P.base) * T(p.Wsig * p.angmax);
#pragma unroll
    for (int l = 0; l < D; ++l) {
        const T R = fabs(P.cen[l]) + P.rad;
        U *= (p.r == 1) ? (S * S + R * R) * invS : S * Fn<T>::cosh_(R * invS);
    }
    return U;
}

// Global folded-grid cell of tile cell c (tile layout: see spread_point) in a tile whose first row is row_lo.
__device__ __forceinline__ int tile_to_grid_cell(int c, int D, int nf, int ncol, int cpad, int n, int row_lo)
{
    const int u = c % ncol - cpad;
    const int rest = c / ncol;  // row (2D) or row nf + j (3D), relative to row_lo
    return (row_lo * (D == 3 ? nf : 1) + rest) * nf + fold_index(u, n);
}

// Shared-memory accumulators of the block tile.
//
// FP32 path: one signed 32-bit fixed-point word per cell in shared memory, in units 2^-Et of the
// tile (Et = Eg - kTileBits), plus a per-block carry array of the same layout in global memory.
// A contribution v in [-2^31, 2^31) goes to its word with one native 32-bit atomic; when that
// addition overflows the signed range (visible from the returned old value o and the result r:
// (o ^ r) & (v ^ r) < 0) the wrapped +-1 x 2^32 tile units go to the cell's carry counter.
// Atomic additions on a word are serialised, so every wrap is that of exactly one addition and
// word + 2^32 carry is the exact sum in any order.  Contributions of 2^31 units or more split
// into a word part and a multiple of 2^32 added to the carry directly.  A block's partial sum in
// one cell stays below B 2^Et = 2^(61 - kTileBits), so carries are rare (about B 2^Et / 2^32
// in a whole evaluation) and a counter stays below 2^(29 - kTileBits) in magnitude.
constexpr int kTileBits = 14;

struct SplitTile {
    int *lo;       // tile words (shared memory)
    int *carry;    // this block's carry counters (global memory, same layout)
    int sgn = 1;   // sign of the current point's contributions (spread_point, with_sign)
    // The tile for the contributions of one point of strength q: every kernel weight is >= 0, so
    // they all have the sign of q, and a word wraps only in the direction of its addend's sign,
    // so the counter moves by the point's sign (one value per point, not one per contribution).
    __device__ __forceinline__ SplitTile with_sign(float q) const { return SplitTile{lo, carry, q < 0.0f ? -1 : 1}; }
    // v of sign d (or zero)
    __device__ __forceinline__ void add32(int c, int v, int d) const
    {
        const int o = atomicAdd(lo + c, v);
        const int r = (int)((unsigned)o + (unsigned)v);
        if (((o ^ r) & (v ^ r)) < 0) atomicAdd(carry + c, d);
    }
    __device__ __forceinline__ void add64(int c, long long x) const
    {
        const int xl = (int)(unsigned)(unsigned long long)x;  // low word, signed
        const long long xh = (x - xl) >> 32;                   // exact: x - xl is a multiple of 2^32
        add32(c, xl, xl < 0 ? -1 : 1);
        if (xh) atomicAdd(carry + c, (int)xh);
    }
    // x of sign sgn.  Zero contributions are added too: a branch around them costs more than the
    // atomic.
    __device__ __forceinline__ void add(int c, float x) const
    {
        if (fabsf(x) < 2147483648.0f) add32(c, __float2int_rn(x), sgn);
        else add64(c, __float2ll_rn(x));
    }
    // |x| < 2^31 known in advance
    __device__ __forceinline__ void add_small(int c, float x) const { add32(c, __float2int_rn(x), sgn); }
    // the contribution a b
    __device__ __forceinline__ void add_product(int c, float a, float b) const { add(c, a * b); }
    __device__ __forceinline__ void add_product_small(int c, float a, float b) const { add_small(c, a * b); }
    // the cell's sum in tile units
    __device__ __forceinline__ long long value(int c) const { return (long long)carry[c] * 4294967296LL + lo[c]; }
};
struct DoubleTile {  // FP64 path: FP64 partial sums
    double *v;
    __device__ __forceinline__ DoubleTile with_sign(double) const { return *this; }
    // v[c] += a b (the library's shared-memory FP64 atomic add; a hand-written compare-and-swap
    // loop around one fused multiply-add measured 2-8x slower).  No test for a zero product: the
    // polynomial kernel weights are not zero at the support's ends as the exact kernel's are,
    // and a zero-strength point is skipped whole (spread_point).
    __device__ __forceinline__ void add_product(int c, double a, double b) const { atomicAdd(v + c, a * b); }
    __device__ __forceinline__ void add_product_small(int c, double a, double b) const { add_product(c, a, b); }
};

// Point m of pair P: grid coordinates x (one grid cell = 1, x = z n / (2 pi)) and strength q in
// tile units (qbase = a_i a_j B x multiplicity x tile scale).
template <typename T, int D, bool ANG = false>
__device__ __forceinline__ void make_point(const SpreadArgs &p, const PairData<T, D> &P, T qbase, int m, T *x, T &q)
{
    const T *sig = static_cast<const T *>(p.sig);
    const T *wsig = static_cast<const T *>(p.wsig);
    const T S = T(p.S), SS = S * S, invS = T(1) / S;
    const T gs = T(p.grid_scale);
    const bool alg = (p.r == 1);
    q = qbase * wsig[m];
    if constexpr (ANG) {  // even part of b(cos theta), Horner in cos^2 theta
        T c = T(0);
#pragma unroll
        for (int l = 0; l < D; ++l) c += P.dir[l] * sig[m * D + l];
        const T c2 = c * c;
        T be = T(p.ang_even[p.nang_even - 1]);
        for (int k = p.nang_even - 2; k >= 0; --k) be = be * c2 + T(p.ang_even[k]);
        q *= be;
    }
#pragma unroll
    for (int l = 0; l < D; ++l) {
        const T vp = P.cen[l] + P.rad * sig[m * D + l];
        T z, m2;
        if constexpr (sizeof(T) == 4) {
            angle_weight_f32(vp, S, invS, alg, z, m2);
        } else if (alg) {
            z = Fn<T>::atan2_(S, vp);
            m2 = (SS + vp * vp) * invS;
        } else {
            // z = 2 atan(e^-u) and mu^-2 = S cosh u with e = e^-|u| <= 1 (one exp and one atan
            // instead of sinh, cosh and atan2): for u < 0, 2 atan(e^|u|) = pi - 2 atan(e^-|u|)
            const double u = vp * invS;
            const double e = exp(-fabs(u));
            const double at2 = 2.0 * atan(e);
            z = u >= 0.0 ? at2 : 3.14159265358979323846 - at2;
            m2 = 0.5 * S * (e + 1.0 / e);
        }
        q *= m2;
        x[l] = z * gs;
    }
}

// Tile layout.  A block tile holds rows row_lo..row_lo+nrows-1 of axis 0 of the folded grid, and
// along the last axis it keeps the UNFOLDED columns u = -cpad..nf-1+cpad at u + cpad (ncol =
// nf + 2 cpad cells): the w columns of a point are then consecutive, with no folding and no
// per-contribution index arithmetic.  The padding columns are folded onto their cells when the
// tile is added to the global grid (tile_to_grid_cell).  2D cell (row, u): row ncol + u + cpad;
// 3D cell (row, j, u): (row nf + j) ncol + u + cpad.

// Add the w^d contributions of one point to the block tile.  SMALL: every contribution is known
// to lie in (-2^31, 2^31) tile units, so the tile's cheaper add_small applies.  SLAB: the tile
// holds a slab of the grid's rows and rows outside it are skipped; otherwise it holds every row
// (row_lo = 0, nrows = n/2 + 1).
template <typename T, int D, int W, typename Tile, bool SMALL, bool SLAB>
__device__ __forceinline__ void spread_point(const SpreadArgs &p, const T *x, T q, const Tile &tile_all, int row_lo,
                                             int nrows, int plane)
{
    if constexpr (sizeof(T) == 8) {
        if (q == T(0)) return;  // FP64 tiles add every product (DoubleTile)
    }
    const Tile tile = tile_all.with_sign(q);
    T w0[W];
    int r0[W];
    axis_weights<T, W>(p, x[0], w0, r0);
    bool hit = !SLAB;
#pragma unroll
    for (int a = 0; a < W; ++a) {
        if constexpr (SLAB) {
            r0[a] -= row_lo;
            hit |= ((unsigned)r0[a] < (unsigned)nrows);
        }
        w0[a] *= q;
    }
    if (!hit) return;
    T wl[W];  // last axis: consecutive padded columns cb..cb+w-1 (clamped: x lies in [0, n/2])
    const int cb = min(max(kernel_weights<T, W>(p, x[D - 1], wl) + p.cpad, 0), p.ncol - W);
    if (D == 2) {
#pragma unroll
        for (int a = 0; a < W; ++a) {
            if (SLAB && (unsigned)r0[a] >= (unsigned)nrows) continue;
            const int row = r0[a] * plane + cb;
#pragma unroll
            for (int c = 0; c < W; ++c) {
                if constexpr (SMALL) tile.add_product_small(row + c, w0[a], wl[c]);
                else tile.add_product(row + c, w0[a], wl[c]);
            }
        }
    } else {
        T w1[W];
        int c1[W];
        axis_weights<T, W>(p, x[1], w1, c1);
#pragma unroll
        for (int b = 0; b < W; ++b) c1[b] = c1[b] * p.ncol + cb;
        for (int a = 0; a < W; ++a) {
            if (SLAB && (unsigned)r0[a] >= (unsigned)nrows) continue;
            const int row = r0[a] * plane;
#pragma unroll
            for (int b = 0; b < W; ++b) {
                const T wab = w0[a] * w1[b];
                const int line = row + c1[b];
#pragma unroll
                for (int c = 0; c < W; ++c) {
                    if constexpr (SMALL) tile.add_product_small(line + c, wab, wl[c]);
                    else tile.add_product(line + c, wab, wl[c]);
                }
            }
        }
    }
}


// The M points of one pair, into a tile that holds every row of the grid.
template <typename T, int D, int W, typename Tile, bool SMALL, bool ANG>
__device__ __forceinline__ void spread_points(const SpreadArgs &p, const PairData<T, D> &P, T sc, const Tile &tile,
                                              int row_lo, int nrows, int plane)
{
    const T qbase = P.base * sc;
    for (int m = 0; m < p.M; ++m) {
        T x[D], q;
        make_point<T, D, ANG>(p, P, qbase, m, x, q);
        spread_point<T, D, W, Tile, SMALL, false>(p, x, q, tile, row_lo, nrows, plane);
    }
}

// Spread the M points of one pair into the block tile; `sc` converts to tile units.  Pairs
// whose largest single contribution is bounded below 2^30 tile units in magnitude (pair bound
// x max_m w_m / sum_m w_m, kernel weights <= 1) take the SMALL path.
template <typename T, int D, int W, typename Tile, bool ANG = false>
__device__ __forceinline__ void spread_pair(const SpreadArgs &p, const PairData<T, D> &P, T sc, const Tile &tile,
                                            int row_lo, int nrows, int plane)
{
    if constexpr (sizeof(T) == 4) {
        if (pair_bound<T, D>(p, P) * sc * T(p.wmax_frac) < T(1073741824.0f)) {
            spread_points<T, D, W, Tile, true, ANG>(p, P, sc, tile, row_lo, nrows, plane);
            return;
        }
    }
    spread_points<T, D, W, Tile, false, ANG>(p, P, sc, tile, row_lo, nrows, plane);
}

// ---- slabbed grids: warp point queues
//
// When the folded grid is split into slabs along axis 0, a point adds to a block's slab only
// if one of its w axis-0 rows lies there, and with a few slabs most points of a warp miss it:
// spreading them where they are generated would leave most lanes idle while the others add.
// Instead each warp appends the points that hit its slab to a queue of 32 entries in shared
// memory (D coordinates and the strength, slot-major) and spreads a full queue with all 32
// lanes, one point per lane.

// Whether any of the w axis-0 rows of a point at grid coordinate x0 lies in the slab (the
// rows of axis_weights).
template <typename T, int W>
__device__ __forceinline__ bool rows_hit(const SpreadArgs &p, T x0, int row_lo, int nrows)
{
    const int s = (int)Fn<T>::floor_(x0 - T(0.5 * W)) + 1;
    const bool simple = p.simple_fold != 0;
    bool hit = false;
#pragma unroll
    for (int a = 0; a < W; ++a) hit |= (unsigned)(fold_cell(s + a, p.n, simple) - row_lo) < (unsigned)nrows;
    return hit;
}

template <typename T, int D>
__device__ __forceinline__ void queue_put(T *buf, int slot, const T *x, T q)
{
#pragma unroll
    for (int l = 0; l < D; ++l) buf[l * 32 + slot] = x[l];
    buf[D * 32 + slot] = q;
}

// Spread queue slot `lane` (when valid) with the whole warp; the FP32 fast add applies when
// every queued strength is below 2^30 tile units (kernel weights are <= 1).
template <typename T, int D, int W, typename Tile>
__device__ __forceinline__ void queue_spread(const SpreadArgs &p, const T *buf, int lane, bool valid,
                                             const Tile &tile, int row_lo, int nrows, int plane)
{
    T x[D], q = T(0);
    if (valid) {
#pragma unroll
        for (int l = 0; l < D; ++l) x[l] = buf[l * 32 + lane];
        q = buf[D * 32 + lane];
    }
    if constexpr (sizeof(T) == 4) {
        const bool small = __all_sync(0xffffffffu, fabsf(q) < 1073741824.0f);
        if (!valid) return;
        if (small) spread_point<T, D, W, Tile, true, true>(p, x, q, tile, row_lo, nrows, plane);
        else spread_point<T, D, W, Tile, false, true>(p, x, q, tile, row_lo, nrows, plane);
    } else {
        if (valid) spread_point<T, D, W, Tile, false, true>(p, x, q, tile, row_lo, nrows, plane);
    }
}

// The pairs pr = first, first + nthr, ... of one thread, spread into one slab through the
// warp's queue `buf` ((D + 1) x 32 values).  Every loop condition is uniform over the warp.
template <typename T, int D, int W, typename Tile, bool ANG>
__device__ __forceinline__ void spread_pairs_queued(const SpreadArgs &p, long long first, long long nthr, T sc, T tau,
                                                    const Tile &tile, int row_lo, int nrows, int plane, T *buf)
{
    const unsigned full = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const unsigned lt = (1u << lane) - 1u;
    int count = 0;  // queued points, the same in every lane
    for (long long pr = first; __any_sync(full, pr < p.npairs); pr += nthr) {
        PairData<T, D> P;
        bool ok = pr < p.npairs && load_pair<T, D, ANG>(p, pr, P);
        if (ok && tau > T(0) && pair_bound<T, D>(p, P) < tau) ok = false;
        if (!__any_sync(full, ok)) continue;
        const T qbase = ok ? P.base * P.mult * sc : T(0);
        for (int m = 0; m < p.M; ++m) {
            T x[D], q = T(0);
            bool hit = false;
            if (ok) {
                make_point<T, D, ANG>(p, P, qbase, m, x, q);
                hit = rows_hit<T, W>(p, x[0], row_lo, nrows);
            }
            const unsigned mask = __ballot_sync(full, hit);
            const int n = __popc(mask), rank = __popc(mask & lt), room = 32 - count;
            if (hit && rank < room) queue_put<T, D>(buf, count + rank, x, q);
            if (n >= room) {  // full: spread 32 points, then queue the rest
                __syncwarp();
                queue_spread<T, D, W, Tile>(p, buf, lane, true, tile, row_lo, nrows, plane);
                __syncwarp();
                if (hit && rank >= room) queue_put<T, D>(buf, rank - room, x, q);
                count = n - room;
            } else {
                count += n;
            }
        }
    }
    __syncwarp();
    queue_spread<T, D, W, Tile>(p, buf, lane, lane < count, tile, row_lo, nrows, plane);
}

struct SlabGeom {
    int row_lo, nrows, plane, ncell;
};

__device__ __forceinline__ SlabGeom slab_geometry(const SpreadArgs &p, int D)
{
    SlabGeom g;
    g.plane = (D == 3) ? p.nf * p.ncol : p.ncol;
    const int slab = blockIdx.x % p.nslab;
    g.row_lo = slab * p.rows_per_slab;
    const int row_hi = min(g.row_lo + p.rows_per_slab, p.nf);
    g.nrows = row_hi - g.row_lo;
    g.ncell = g.nrows * g.plane;
    return g;
}

// Pair numbering: the threads of one slab cover the pairs with stride `nthr`, thread r of the
// slab (r = 32 warp + lane) starting at (r A) mod nthr with A = 1000003, a prime above any
// thread count (at most SMs x 2048), so the starts are a permutation of 0..nthr-1.  Lanes of a
// warp then take pairs A apart modulo nthr: unrelated (t, i), whose 32 points rarely hit the
// same grid cells.  Neighbouring pairs produce neighbouring points and would serialise the
// shared-memory atomics; a plain lane stride of nwarps keeps the lanes on one node column
// whenever nwarps and N share a power of two.
__device__ __forceinline__ void pair_schedule(const SpreadArgs &p, long long &first, long long &nthr)
{
    const long long groups = gridDim.x / p.nslab;
    nthr = groups * blockDim.x;
    const long long r = (long long)(blockIdx.x / p.nslab) * blockDim.x + threadIdx.x;
    first = (r * 1000003LL) % nthr;
}

template <int D, int W, bool ANG>
__global__ void __launch_bounds__(kMaxThreadsF32) k_spread_f32(const __grid_constant__ SpreadArgs p)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const SlabGeom G = slab_geometry(p, D);
    if (G.nrows <= 0) return;  // uniform over the block: an empty trailing slab does nothing
    int *words = reinterpret_cast<int *>(smem_raw);
    int *carry = p.carry + (size_t)blockIdx.x * p.tile_cells;
    for (int c = threadIdx.x; c < G.ncell; c += blockDim.x) {
        words[c] = 0;
        carry[c] = 0;
    }
    __syncthreads();
    const double Bnd = *p.bound;
    const int Eg = global_exponent(Bnd);
    // Tile unit 2^-Et with Et = Eg - kTileBits (2^-47 B or finer); kept inside the float range for
    // tiny inputs (a coarser unit there).
    const int Et = min(Eg - kTileBits, 120);
    const int shift = Eg - Et;
    const SplitTile tile{words, carry};
    const float sc = (float)ldexp(1.0, Et);
    const float tau = (float)*p.tau;
    long long first, nthr;
    pair_schedule(p, first, nthr);
    if (p.nslab > 1) {
        float *buf = reinterpret_cast<float *>(smem_raw + (size_t)p.rows_per_slab * G.plane * 4) +
                     (threadIdx.x >> 5) * 32 * (D + 1);
        spread_pairs_queued<float, D, W, SplitTile, ANG>(p, first, nthr, sc, tau, tile, G.row_lo, G.nrows, G.plane,
                                                          buf);
    } else {
        for (long long pr = first; pr < p.npairs; pr += nthr) {
            PairData<float, D> P;
            if (!load_pair<float, D, ANG>(p, pr, P)) continue;
            if (tau > 0.0f && pair_bound<float, D>(p, P) < tau) continue;
            P.base *= P.mult;
            spread_pair<float, D, W, SplitTile, ANG>(p, P, sc, tile, G.row_lo, G.nrows, G.plane);
        }
    }
    __syncthreads();
    for (int c = threadIdx.x; c < G.ncell; c += blockDim.x) {
        const long long v = tile.value(c);
        // |v 2^shift| <= B 2^Eg <= 2^61
        if (v)
            atomicAdd(p.grid + tile_to_grid_cell(c, D, p.nf, p.ncol, p.cpad, p.n, G.row_lo),
                      (unsigned long long)(v * (1ll << shift)));
    }
}

template <int D, int W, bool ANG>
__global__ void __launch_bounds__(kMaxThreadsF64) k_spread_f64(const __grid_constant__ SpreadArgs p)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const SlabGeom G = slab_geometry(p, D);
    if (G.nrows <= 0) return;  // uniform over the block
    DoubleTile tile{reinterpret_cast<double *>(smem_raw)};
    for (int c = threadIdx.x; c < G.ncell; c += blockDim.x) tile.v[c] = 0.0;
    load_kernel_poly(p.kpoly);
    __syncthreads();
    const double Bnd = *p.bound;
    const int Eg = global_exponent(Bnd);
    const double tau = *p.tau;
    long long first, nthr;
    pair_schedule(p, first, nthr);
    if (p.nslab > 1) {
        double *buf = reinterpret_cast<double *>(smem_raw + (size_t)p.rows_per_slab * G.plane * 8) +
                      (threadIdx.x >> 5) * 32 * (D + 1);
        spread_pairs_queued<double, D, W, DoubleTile, ANG>(p, first, nthr, 1.0, tau, tile, G.row_lo, G.nrows,
                                                            G.plane, buf);
    } else {
        for (long long pr = first; pr < p.npairs; pr += nthr) {
            PairData<double, D> P;
            if (!load_pair<double, D, ANG>(p, pr, P)) continue;
            if (tau > 0.0 && pair_bound<double, D>(p, P) < tau) continue;
            P.base *= P.mult;
            spread_pair<double, D, W, DoubleTile, ANG>(p, P, 1.0, tile, G.row_lo, G.nrows, G.plane);
        }
    }
    __syncthreads();
    // block partial sums -> the grid's fixed-point unit (|v| 2^Eg <= 2^61); the rounding of a
    // partial sum is 2^-61 B at most
    const double sc = ldexp(1.0, Eg);
    for (int c = threadIdx.x; c < G.ncell; c += blockDim.x) {
        const long long v = __double2ll_rn(tile.v[c] * sc);
        if (v)
            atomicAdd(p.grid + tile_to_grid_cell(c, D, p.nf, p.ncol, p.cpad, p.n, G.row_lo), (unsigned long long)v);
    }
}

template <int D, int W, bool ANG>
cudaError_t launch_f32(const SpreadArgs &a, int blocks, int threads, size_t smem, cudaStream_t s)
{
    auto kern = k_spread_f32<D, W, ANG>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    kern<<<blocks, threads, smem, s>>>(a);
    return cudaGetLastError();
}

template <int D, int W, bool ANG>
cudaError_t launch_f64(const SpreadArgs &a, int blocks, int threads, size_t smem, cudaStream_t s)
{
    auto kern = k_spread_f64<D, W, ANG>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    kern<<<blocks, threads, smem, s>>>(a);
    return cudaGetLastError();
}

// Compile-time dispatch on the kernel width w in [W, WMAX].  ANG: the angular-kernel variant
// (instantiated in its own translation units).
template <bool F32, int D, int W, int WMAX, bool ANG>
struct WidthDispatch {
    static cudaError_t run(const SpreadArgs &a, int w, int blocks, int threads, size_t smem, cudaStream_t s)
    {
        if (w == W) {
            if constexpr (F32) return launch_f32<D, W, ANG>(a, blocks, threads, smem, s);
            else return launch_f64<D, W, ANG>(a, blocks, threads, smem, s);
        }
        if constexpr (W < WMAX) return WidthDispatch<F32, D, W + 1, WMAX, ANG>::run(a, w, blocks, threads, smem, s);
        return cudaErrorInvalidValue;
    }
};

}  // namespace spread_detail
}  // namespace pgb
