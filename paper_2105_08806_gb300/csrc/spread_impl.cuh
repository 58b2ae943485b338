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
//  - FP64 kernel: each block adds into a private copy of its slab of the grid in shared memory
//    that holds each cell as a 96-bit integer, 32 bits finer than the grid unit, in three 32-bit
//    words (WideTile: native 32-bit atomics, the next word's only when a carry or a high part
//    needs it).  The kernel weights are FP64; per point, a row factor R = round(q psi_a 2^(Eg+s))
//    with a per-point scale s that keeps R below 2^62 (3D: then round(R psi_b) in integers) is
//    formed once per row, and each contribution is round(R psi_c) from a 61-bit fixed-point psi_c
//    by four 32 x 32-bit integer products, so no FP64 operation runs per cell (the FP64 pipe of
//    this GPU runs at about 1/70 of the FP32 rate) and each contribution keeps about 2^-61 of its
//    size plus 2^-32 grid units.  At the end each cell rounds to the grid unit once per block.
//  - FP32 kernel: the private copy holds one signed 32-bit word per cell in units of 2^-Et,
//    Et = Eg - tile_bits(d), plus per-cell carry counters in a per-block global array (SplitTile):
//    the cell's value is word + 2^32 carry.  A contribution goes to its word with one native 32-bit
//    shared atomic, and only an addition that overflows the word's signed range (seen from the
//    returned old value) moves the cell's carry counter; the wraps of a run of w cells are
//    collected in a register mask and their carries added after the run.  (Floating-point shared atomics are
//    compare-and-swap loops and their rounding limits FP32 accuracy; 64-bit integer shared atomics
//    are several times slower than 32-bit ones.)  Points below 2^29 tile units -- nearly all of
//    them -- form their contributions in integers: the row factor 4 q psi_a (psi_b) and the column
//    factor 2^30 psi_c are rounded once per row and column, and a contribution is the rounded high
//    word of their 64-bit product (one integer multiply-add).  At the end each block adds
//    word + 2^32 carry (scaled by 2^tile_bits(d)) to the global grid.  Each contribution is rounded
//    to the tile unit (at most about one unit); all later additions are exact.
//
// Negligible pairs: in the FP32 kernels a pair whose strength bound keeps every one of its points
// below 0.1 tile unit adds exactly zero (every contribution rounds to zero), so it is skipped, and
// so are such points one by one; the FP64 kernels skip pairs whose summed bounds stay below
// 2^-64 B (2^-3 grid units in all).  Each lane searches ahead for its
// next pair that is not negligible, so that the lanes of a warp spread real pairs together (with
// the node sets of the workloads here, 25-75% of all pairs lie in the tails of f and are skipped).
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

// Kernel weights psi(x_u - z) of one axis, u = s..s+w-1, in units where one grid cell is 1 and
// x = z n / (2 pi): psi = exp(beta (sqrt(1 - t^2) - 1)), t = (u - x) 2/w.

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

// FP64 weights and the folded cells fold(s + a) of one axis.
template <int W>
__device__ __forceinline__ void axis_weights_f64(const SpreadArgs &p, double x, double *wt, int *idx)
{
    const int s = kernel_weights_f64<W>(x, wt);
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

// atan(u) - u for |u| <= 1 as u^3 R(u^2): R is a degree-9 polynomial in u^2 fitted by
// fit_atan_f32.py (iteratively reweighted least squares towards the minimax error of atan; the
// fit's error is 1.7e-10, and evaluated in FP32 the correction carries at most 3e-8).  The
// leading term u stays exact, so atan(u) is carried as the two terms u + correction.
__device__ __forceinline__ float atan_correction_f32(float u)
{
    const float s = u * u;
    float r = 0.000990882766560405f;
    r = fmaf(r, s, -0.0066840073563619829f);
    r = fmaf(r, s, 0.021143804646584562f);
    r = fmaf(r, s, -0.042978293426904776f);
    r = fmaf(r, s, 0.066138929468158386f);
    r = fmaf(r, s, -0.087516064688656053f);
    r = fmaf(r, s, 0.1104117269740377f);
    r = fmaf(r, s, -0.14276990716236754f);
    r = fmaf(r, s, 0.19999428419267529f);
    r = fmaf(r, s, -0.33333319184448684f);
    return u * s * r;
}

// The factor mu^-2 of one mapped coordinate v in a point's strength (Section 2.1), FP32:
// (S^2 + v^2)/S (algebraic map) or S cosh(v/S) = S (e^-|v/S| + e^|v/S|)/2 (logarithmic map).
__device__ __forceinline__ float axis_m2_f32(const TypedConsts<float> &K, float v, bool alg)
{
    if (alg) return fmaf(v, v, K.SS) * K.invS;
    const float w = fmaf(v, K.invS, v * K.invS_lo);
    const float e = exp2f(-fabsf(w) * 1.4426950408889634f);
    return 0.5f * K.S * (__frcp_rn(e) + e);
}

// FP32 grid coordinate x = z n/(2 pi) of the angle z = arccos(xi(v)) of one mapped coordinate, as an
// integer cell X (an integer-valued float) and a fraction F in [0, 1) (Section 2.1).  With w = v/S:
//   r = 1: |w| <= 1: x = n/4 - gs atan(w);  w > 1: x = gs atan(S/v);  w < -1: x = n/2 + gs atan(S/v)
//          (z = pi/2 - atan(w) = atan(1/w) or pi + atan(1/w))
//   r = 0: x = 2 gs atan(e) (v >= 0) or n/2 - 2 gs atan(e) (v < 0), e = exp(-|v|/S)
// with gs = n/(2 pi), i.e. x = base - sg c atan(u) with |u| <= 1 and base in {0, n/4, n/2}.  The
// offsets are exact, c = gs (or 2 gs) is a two-term constant, atan(u) = u + correction is
// renormalised into two terms (Fast2Sum) and multiplied by c with its exact FMA residual, and
// base - sg c atan(u) is summed exactly (Fast2Sum), so the fraction F is accurate to about 1e-7
// of a cell: a grid coordinate rounded to FP32 as a whole (about 1e-6 of a cell at x ~ 100)
// shifts points that share a coordinate -- and many do, on a tensor grid of nodes -- coherently.
__device__ __forceinline__ void grid_coord_f32(const TypedConsts<float> &K, float v, bool alg, float &X, float &F)
{
    float base, sg, u, ch = K.gs, cl = K.gs_lo;
    if (alg) {
        const float w = fmaf(v, K.invS, v * K.invS_lo);  // v/S
        if (fabsf(w) <= 1.0f) {
            base = K.xq;
            sg = 1.0f;
            u = w;
        } else {  // u = S/v: the approximate reciprocal and one Newton step
            const float rv = rcp_approx(v);
            const float u0 = K.S * rv;
            u = fmaf(rv, fmaf(-v, u0, K.S), u0);
            base = v > 0.0f ? 0.0f : 2.0f * K.xq;
            sg = -1.0f;
        }
    } else {
        const float w = fmaf(v, K.invS, v * K.invS_lo);
        const float e = exp2f(-fabsf(w) * 1.4426950408889634f);  // exp(-|v|/S)
        u = e;
        base = v >= 0.0f ? 0.0f : 2.0f * K.xq;
        sg = v >= 0.0f ? -1.0f : 1.0f;
        ch = 2.0f * K.gs;
        cl = 2.0f * K.gs_lo;
    }
    const float corr = atan_correction_f32(u);
    const float ah = u + corr;                            // atan(u) = ah + al
    const float al = (u - ah) + corr;                     // exact (Fast2Sum: |u| >= |corr|)
    const float p1 = ch * ah;
    const float e1 = fmaf(ch, ah, -p1);                   // exact: p1 + e1 = ch ah
    const float pl = e1 + fmaf(ch, al, cl * ah);          // the rest of c atan(u): a few ulp of p1
    const float hi = base - sg * p1;
    const float err = (base - hi) - sg * p1;              // exact (|base| >= |p1| or base = 0)
    const float lo = err - sg * pl;
    X = floorf(hi);
    F = (hi - X) + lo;                                    // |lo| is far below one cell
    if (F < 0.0f) {
        F += 1.0f;
        X -= 1.0f;
        if (F >= 1.0f) {  // -F below half an ulp of 1: the point sits on the cell boundary
            F = 0.0f;
            X += 1.0f;
        }
    } else if (F >= 1.0f) {
        F -= 1.0f;
        X += 1.0f;
    }
}

// FP32 kernel value psi(t) 2^lsc = 2^(bl (sqrt(1 - t^2) - 1) + lsc) for |t| < 1 and 0 outside, with
// bl = beta log2(e) and bias = lsc - bl; the square root as (1 - t^2) rsqrt(1 - t^2).  Both
// approximations are good to a few 1e-7.
__device__ __forceinline__ float es_f32(float t, float bl, float bias)
{
    const float om = fmaf(-t, t, 1.0f);
    const float e = fmaf(bl, om * rsqrt_approx(om), bias);
    return om > 0.0f ? ex2_approx(e) : 0.0f;
}

// First tap s = X + c0 of a point at X + F for kernel width W (s = floor(x - W/2) + 1) and the tap
// offset t0 = (s - x) 2/W; tap a has t = t0 + a 2/W.
template <int W>
__device__ __forceinline__ int first_tap_f32(float X, float F, float &t0)
{
    int c0;
    if constexpr (W % 2 == 0) c0 = 1 - W / 2;
    else c0 = (F >= 0.5f ? 1 : 0) - (W - 1) / 2;
    t0 = ((float)c0 - F) * (2.0f / W);
    return (int)X + c0;
}

// FP32 weights psi(t_a) of one axis and the folded cells fold(s + a).
template <int W>
__device__ __forceinline__ void axis_weights_f32(const SpreadArgs &p, float X, float F, float *wt, int *idx)
{
    float t0;
    const int s = first_tap_f32<W>(X, F, t0);
    const float h2 = 2.0f / W;
    const float bl = p.cf.bl;
    const bool simple = p.simple_fold != 0;
#pragma unroll
    for (int a = 0; a < W; ++a) {
        wt[a] = es_f32(fmaf((float)a, h2, t0), bl, -bl);
        idx[a] = fold_cell(s + a, p.n, simple);
    }
}

// Row shear of the pair numbering (load_pair); t K stays below 2^32 for every node count a plan
// accepts (t <= nnode/2 <= 2^21).
constexpr unsigned kPairShear = 1597u;

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
// Numbering: pair pr = t nnode + u is (i, (i + t) mod nnode) with i = (u + t K) mod nnode, offsets
// t = 0..floor(nnode/2); t = 0 is the diagonal (multiplicity 1) and, for even nnode, the row
// t = nnode/2 stops at u = nnode/2 - 1 (its other half repeats the same pairs) and is not sheared:
// unordered_pairs(nnode) in all.  The shear by K = kPairShear per row is a bijection of each row; it
// makes a lane that strides through the pairs by a multiple of nnode (the single-plan launches
// stride by SMs x threads, often a multiple of N^d) visit every node i instead of one, so the
// lanes of a warp meet the negligible pairs of the tails of f at the same rate.

// A position in the pair numbering, advanced by a fixed stride without divisions: pr = t nnode + u
// and the sheared first node i = (u + t K) mod nnode.  A stride of dt nnode + du moves i by
// di = (du + dt K) mod nnode, and by K mod nnode more when u wraps.
struct PairCursor {
    long long pr;
    int t, u, i;
};
struct PairStep {
    long long d;
    int dt, du, di, dk;
};

__device__ __forceinline__ PairCursor pair_cursor(const SpreadArgs &p, long long pr)
{
    PairCursor c;
    c.pr = pr;
    c.t = (int)(pr / p.nnode);
    c.u = (int)(pr - (long long)c.t * p.nnode);
    c.i = (int)(((long long)c.u + (long long)c.t * kPairShear) % p.nnode);
    return c;
}

__device__ __forceinline__ PairStep pair_step(const SpreadArgs &p, long long stride)
{
    PairStep s;
    s.d = stride;
    s.dt = (int)(stride / p.nnode);
    s.du = (int)(stride - (long long)s.dt * p.nnode);
    s.di = (int)(((long long)s.du + (long long)s.dt * kPairShear) % p.nnode);
    s.dk = (int)(kPairShear % p.nnode);
    return s;
}

__device__ __forceinline__ void pair_advance(const SpreadArgs &p, PairCursor &c, const PairStep &s)
{
    const int nnode = p.nnode;
    c.pr += s.d;
    c.t += s.dt;
    c.u += s.du;
    c.i += s.di;
    if (c.i >= nnode) c.i -= nnode;
    if (c.u >= nnode) {
        c.u -= nnode;
        c.t += 1;
        c.i += s.dk;
        if (c.i >= nnode) c.i -= nnode;
    }
}

// Axis indices of node k (C order, axis D-1 fastest) from float quotients: (k + 1/2)/N lies at
// least 1/(2N) from an integer and its FP32 value within 2^-23 (k + 1/2)/N < 1/(4N) of it for
// k < 2^21 (every node count a plan allows), so the truncation is the exact quotient.
template <int D>
__device__ __forceinline__ void node_axes(int k, int N, float invN, int (&ax)[D])
{
#pragma unroll
    for (int l = D - 1; l > 0; --l) {
        const int q = __float2int_rz(((float)k + 0.5f) * invN);
        ax[l] = k - q * N;
        k = q;
    }
    ax[0] = k;
}

// Load the pair at cursor c; false when its strength is zero.  ANG: also the unit direction
// (angular kernels).
template <typename T, int D, bool ANG = false>
__device__ __forceinline__ bool load_pair(const SpreadArgs &p, const PairCursor &c, PairData<T, D> &P)
{
    const int nnode = p.nnode, N = p.N;
    const int t = c.t;
    const int i = (2 * t != nnode) ? c.i : c.u;  // the half row t = nnode/2 is not sheared
    int j = i + t;
    if (j >= nnode) j -= nnode;
    P.mult = t ? T(2) : T(1);
    const T *vnode = static_cast<const T *>(p.vnode);
    const T *acoef = static_cast<const T *>(p.a);
    const T aij = acoef[i] * acoef[j];
    if (aij == T(0)) return false;
    const float invN = 1.0f / (float)N;
    int ai[D], aj[D];
    node_axes<D>(i, N, invN, ai);
    node_axes<D>(j, N, invN, aj);
    T g2 = T(0);
#pragma unroll
    for (int l = D - 1; l >= 0; --l) {
        const int ni = ai[l], nj = aj[l];
        const T vi = vnode[ni], vj = vnode[nj];
        T dl = vi - vj, sl = vi + vj;
        if constexpr (sizeof(T) == 4) {  // FP32 nodes carry their rounding in a second term
            const float li = p.vnode_lo[ni], lj = p.vnode_lo[nj];
            dl += li - lj;
            sl += li + lj;
        }
        g2 += dl * dl;
        P.cen[l] = T(0.5) * sl;
        if constexpr (ANG) P.dir[l] = dl;
    }
    const T g = Fn<T>::sqrt_(g2);
    if constexpr (ANG) {
        const T ginv = g > T(0) ? T(1) / g : T(0);
#pragma unroll
        for (int l = 0; l < D; ++l) P.dir[l] *= ginv;
    }
    const TypedConsts<T> &K = kconst<T>(p);
    T B;
    switch (p.fast_gamma) {
    case 0: B = K.Bconst; break;
    case 1: B = K.Bconst * g; break;
    case 2: B = K.Bconst * Fn<T>::sqrt_(g); break;
    default: B = K.Bconst * Fn<T>::pow_(g, K.gamma); break;
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
    const TypedConsts<T> &K = kconst<T>(p);
    T U = fabs(P.base) * K.Wang;
#pragma unroll
    for (int l = 0; l < D; ++l) {
        const T R = fabs(P.cen[l]) + P.rad;
        U *= (p.r == 1) ? (K.SS + R * R) * K.invS : K.S * Fn<T>::cosh_(R * K.invS);
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
// tile (Et = Eg - tile_bits(d)), plus a per-block carry array of the same layout in global memory.
// A contribution v in [-2^31, 2^31) goes to its word with one native 32-bit atomic; when that
// addition overflows the signed range (visible from the returned old value o and the result r:
// (o ^ r) & (v ^ r) < 0) the wrapped +-1 x 2^32 tile units go to the cell's carry counter; the
// direction is the addend's sign, which is that of the point's strength (every kernel weight is
// >= 0), so it is one value per point.  Atomic additions on a word are serialised, so every wrap
// is that of exactly one addition and word + 2^32 carry is the exact sum in any order.
// Contributions of 2^31 units or more split into a word part and a multiple of 2^32 added to the
// carry directly.  A block's partial sum in one cell stays below B 2^Et = 2^(61 - bits), so
// carries are rare (about B 2^Et / 2^32 in a whole evaluation) and a counter stays below
// 2^(29 - bits) in magnitude (bits = tile_bits(d)).

struct SplitTile {
    int *lo;     // tile words (shared memory)
    int *carry;  // this block's carry counters (global memory, same layout)
    // v of sign d (or zero)
    __device__ __forceinline__ void add_int(int c, int v, int d) const
    {
        const int o = atomicAdd(lo + c, v);
        const int r = (int)((unsigned)o + (unsigned)v);
        if (((o ^ r) & (v ^ r)) < 0) atomicAdd(carry + c, d);
    }
    // The same addition for a run of consecutive cells: the wrap of this addition is shifted
    // into `mask` (one funnel shift) and the carries of the run are added afterwards, in
    // add_carries, where the mask is rarely non-zero.
    __device__ __forceinline__ unsigned add_int_run(int c, int v, unsigned mask) const
    {
        const int o = atomicAdd(lo + c, v);
        const int r = (int)((unsigned)o + (unsigned)v);
        return __funnelshift_l((unsigned)((o ^ r) & (v ^ r)), mask, 1);
    }
    // carries of a run of n additions to cells c0 .. c0+n-1 (bit n-1-k of mask: cell c0 + k)
    __device__ __forceinline__ void add_carries(int c0, int n, unsigned mask, int d) const
    {
        while (mask) {
            const int b = __ffs(mask) - 1;
            atomicAdd(carry + c0 + (n - 1 - b), d);
            mask &= mask - 1;
        }
    }
    __device__ __forceinline__ void add64(int c, long long x) const
    {
        const int xl = (int)(unsigned)(unsigned long long)x;  // low word, signed
        const long long xh = (x - xl) >> 32;                   // exact: x - xl is a multiple of 2^32
        add_int(c, xl, xl < 0 ? -1 : 1);
        if (xh) atomicAdd(carry + c, (int)xh);
    }
    // any x (zero contributions are added too: a branch around them costs more than the atomic)
    __device__ __forceinline__ void add(int c, float x) const
    {
        if (fabsf(x) < 2147483648.0f) add_int(c, __float2int_rn(x), x < 0.0f ? -1 : 1);
        else add64(c, __float2ll_rn(x));
    }
    // the cell's sum in tile units
    __device__ __forceinline__ long long value(int c) const { return (long long)carry[c] * 4294967296LL + lo[c]; }
};
// FP64 path: one 96-bit two's-complement fixed-point value per cell in units 2^-(Eg+32), 32 bits
// finer than the global grid (B 2^Eg < 2^61), held as a fraction word, a low and a high 32-bit
// word in shared memory.  A contribution I + F 2^-32 (I an int64 in grid units, 0 <= F < 2^32)
// adds F to the fraction word and I plus the carry out of that addition to the low word, each with
// one native 32-bit atomic whose returned old value shows its carry; the high part of I plus the
// low word's carry goes to the high word by a third atomic when not zero (for positive
// contributions below 2^32 grid units, only on a carry).  The sum is exact in any order, and a
// partial sum stays below 2^63 grid units.  Shared-memory FP64 atomic adds, the other choice, run
// several times slower on this hardware (they spend the FP64 pipe).
struct WideTile {
    unsigned *fr;  // fraction words (shared memory)
    unsigned *lo;  // low words
    int *hi;       // high words
    __device__ __forceinline__ void add(int c, long long I, unsigned F) const
    {
        const unsigned of = atomicAdd(fr + c, F);
        const long long J = I + ((of + F < of) ? 1 : 0);
        const unsigned jl = (unsigned)(unsigned long long)J;
        const unsigned o = atomicAdd(lo + c, jl);
        const int vh = (int)(J >> 32) + ((o + jl < o) ? 1 : 0);
        if (vh) atomicAdd(hi + c, vh);
    }
    // the cell's sum rounded to the grid unit
    __device__ __forceinline__ long long value(int c) const
    {
        const long long i = (long long)(((unsigned long long)(unsigned)hi[c] << 32) | lo[c]);
        return i + (fr[c] >= 0x80000000u ? 1 : 0);
    }
};

// Fixed-point kernel weight for the FP64 path: round(w 2^61) = h 2^31 + l with 0 <= l < 2^31
// (w <= 1 up to the polynomial's rounding, so |h| <= 2^30 + 1).
struct FixW {
    int h, l;
};
__device__ __forceinline__ FixW fix_weight(double w)
{
    const long long t = __double2ll_rn(w * 2305843009213693952.0);  // 2^61
    return FixW{(int)(t >> 31), (int)(t & 0x7fffffffll)};
}

// round(R w) for |R| < 2^62 and a fixed-point weight w: with R = Rh 2^31 + Rl (0 <= Rl < 2^31),
// R w 2^61 = 2^62 Rh h + 2^31 (Rh l + Rl h) + Rl l, from four 32 x 32-bit integer products; the
// last one enters truncated to 2^-30 units (error below 2^-30), the result rounds half up.
// Every intermediate stays below 2^63 in magnitude.
__device__ __forceinline__ long long fix_mul(long long R, FixW w)
{
    const int Rh = (int)(R >> 31);
    const int Rl = (int)(R & 0x7fffffffll);
    const long long X = (long long)Rh * w.l + (long long)Rl * w.h + (((long long)Rl * w.l) >> 31);
    return 2 * ((long long)Rh * w.h) + ((X + (1ll << 29)) >> 30);
}

// A point's contributions in the FP64 path: each tap value v (units 2^-(Eg+s) for the point's
// scale s) becomes I + F 2^-32 grid units with I = floor(v 2^-s), F the next 32 bits (truncated,
// below 2^-32 grid units).
struct TapShift {
    int sI;    // min(s, 63): |v| < 2^62, so v >> 63 is the sign
    int sF;    // |s - 32|
    bool up;   // s < 32: F = v << (32 - s); otherwise F = v >> (s - 32)
};
__device__ __forceinline__ TapShift tap_shift(int s)
{
    return TapShift{min(s, 63), s < 32 ? 32 - s : s - 32, s < 32};
}
__device__ __forceinline__ void tap_split(long long v, const TapShift &t, long long &I, unsigned &F)
{
    I = v >> t.sI;
    F = (unsigned)(unsigned long long)(t.up ? (v << t.sF) : (v >> t.sF));
}

// One post-collision point: FP32 points carry each grid coordinate (one grid cell = 1,
// x = z n / (2 pi)) as an integer cell X (an integer-valued float) and a fraction F in [0, 1)
// (grid_coord_f32); FP64 points carry x itself.  q is the strength in tile units.
template <typename T, int D>
struct Point;
template <int D>
struct Point<float, D> {
    float X[D], F[D], q;
};
template <int D>
struct Point<double, D> {
    double x[D], q;
};

// Strength of point m of pair P before the map factors: qbase w_m, times the even part of
// b(cos theta) for angular kernels (Horner in cos^2 theta).
template <typename T, int D, bool ANG>
__device__ __forceinline__ T point_base(const SpreadArgs &p, const PairData<T, D> &P, T qbase, int m)
{
    const T *sig = static_cast<const T *>(p.sig);
    const T *wsig = static_cast<const T *>(p.wsig);
    T q = qbase * wsig[m];
    if constexpr (ANG) {
        const TypedConsts<T> &K = kconst<T>(p);
        T c = T(0);
#pragma unroll
        for (int l = 0; l < D; ++l) c += P.dir[l] * sig[m * D + l];
        const T c2 = c * c;
        T be = K.ang_even[p.nang_even - 1];
        for (int k = p.nang_even - 2; k >= 0; --k) be = be * c2 + K.ang_even[k];
        q *= be;
    }
    return q;
}

// FP32: the post-collision velocity v' = (v_i + v_j)/2 + |v_i - v_j| sigma_m / 2 of point m of
// pair P and its strength q (qbase = a_i a_j B x multiplicity x tile scale), without the grid
// coordinates.
template <int D, bool ANG>
__device__ __forceinline__ float point_velocity_f32(const SpreadArgs &p, const PairData<float, D> &P, float qbase,
                                                    int m, float (&vp)[D])
{
    const float *sig = static_cast<const float *>(p.sig);
    const TypedConsts<float> &K = kconst<float>(p);
    const bool alg = (p.r == 1);
    float q = point_base<float, D, ANG>(p, P, qbase, m);
#pragma unroll
    for (int l = 0; l < D; ++l) {
        vp[l] = fmaf(P.rad, sig[m * D + l], P.cen[l]);
        q *= axis_m2_f32(K, vp[l], alg);
    }
    return q;
}

// Point m of pair P (qbase = a_i a_j B x multiplicity x tile scale).
template <typename T, int D, bool ANG = false>
__device__ __forceinline__ void make_point(const SpreadArgs &p, const PairData<T, D> &P, T qbase, int m,
                                           Point<T, D> &pt)
{
    const TypedConsts<T> &K = kconst<T>(p);
    const bool alg = (p.r == 1);
    if constexpr (sizeof(T) == 4) {
        float vp[D];
        pt.q = point_velocity_f32<D, ANG>(p, P, qbase, m, vp);
#pragma unroll
        for (int l = 0; l < D; ++l) grid_coord_f32(K, vp[l], alg, pt.X[l], pt.F[l]);
    } else {
        const double *sig = static_cast<const double *>(p.sig);
        double q = point_base<double, D, ANG>(p, P, qbase, m);
#pragma unroll
        for (int l = 0; l < D; ++l) {
            const double vp = P.cen[l] + P.rad * sig[m * D + l];
            double z, m2;
            if (alg) {
                z = Fn<T>::atan2_(K.S, vp);
                m2 = (K.SS + vp * vp) * K.invS;
            } else {
                // z = 2 atan(e^-u) and mu^-2 = S cosh u with e = e^-|u| <= 1 (one exp and one atan
                // instead of sinh, cosh and atan2): for u < 0, 2 atan(e^|u|) = pi - 2 atan(e^-|u|)
                const double u = vp * K.invS;
                const double e = exp(-fabs(u));
                const double at2 = 2.0 * atan(e);
                z = u >= 0.0 ? at2 : 3.14159265358979323846 - at2;
                m2 = 0.5 * K.S * (e + 1.0 / e);
            }
            pt.x[l] = z * K.gs;
            q *= m2;
        }
        pt.q = q;
    }
}

// Tile layout.  A block tile holds rows row_lo..row_lo+nrows-1 of axis 0 of the folded grid, and
// along the last axis it keeps the UNFOLDED columns u = -cpad..nf-1+cpad at u + cpad (ncol =
// nf + 2 cpad cells): the w columns of a point are then consecutive, with no folding and no
// per-contribution index arithmetic.  The padding columns are folded onto their cells when the
// tile is added to the global grid (tile_to_grid_cell).  2D cell (row, u): row ncol + u + cpad;
// 3D cell (row, j, u): (row nf + j) ncol + u + cpad.

// ---- FP32 points
//
// Kinds of FP32 point: kInt -- |q| < 2^29 tile units (integer products); kLarge -- any q.
constexpr int kInt = 0, kLarge = 1;
// Points below this many tile units take the integer products; points below kNegligibleF32 add
// exactly zero (4 q psi rounds to 0 for every row) and are skipped, and so are pairs whose points
// all stay below it.
constexpr float kIntLimitF32 = 536870912.0f;  // 2^29
constexpr float kNegligibleF32 = 0.1f;

// round(a b / 2^32) for |a| < 2^31, 0 <= b <= 2^30: the high word of one 64-bit multiply-add
__device__ __forceinline__ int mulhi_rn(int a, int b)
{
    return (int)(((long long)a * (long long)b + 0x80000000LL) >> 32);
}

// Add the w^d contributions q psi_a psi_b psi_c of one FP32 point to the block tile.  kInt: the
// column factors 2^30 psi_c and, per row, 4 q psi_a (psi_b) are rounded to integers, and a
// contribution is mulhi_rn of the two (at most about one tile unit of rounding).  kLarge: the
// product is formed in FP32 and rounded to the tile unit.  SLAB: the tile holds a slab of the grid's
// rows and rows outside it are skipped; otherwise it holds every row (row_lo = 0, nrows = n/2 + 1).
// 3D points loop over their axis-0 rows (computing that row's kernel value in the loop) so that
// the unrolled code stays small.
template <int D, int W, int KIND, bool SLAB>
__device__ __forceinline__ void spread_point_f32(const SpreadArgs &p, const Point<float, D> &pt,
                                                 const SplitTile &tile, int row_lo, int nrows, int plane)
{
    const float q = pt.q;
    if (fabsf(q) < kNegligibleF32) return;  // every contribution rounds to zero
    const float bl = p.cf.bl;
    const float h2 = 2.0f / W;
    const bool simple = p.simple_fold != 0;
    float t00, tl0;
    const int s0 = first_tap_f32<W>(pt.X[0], pt.F[0], t00);          // first row
    const int sl = first_tap_f32<W>(pt.X[D - 1], pt.F[D - 1], tl0);  // first column (unfolded)
    const int cb = min(max(sl + p.cpad, 0), p.ncol - W);            // clamped: x lies in [0, n/2]
    float w1[W];
    int c1[W];
    if constexpr (D == 3) {
        axis_weights_f32<W>(p, pt.X[1], pt.F[1], w1, c1);
#pragma unroll
        for (int b = 0; b < W; ++b) c1[b] = c1[b] * p.ncol + cb;
    }
    if constexpr (KIND == kInt) {
        const int sg = q < 0.0f ? -1 : 1;  // the sign of every contribution (or zero)
        const float q4 = 4.0f * q;
        const float bias30 = 30.0f - bl;
        int wi[W];
#pragma unroll
        for (int c = 0; c < W; ++c) wi[c] = __float2int_rn(es_f32(fmaf((float)c, h2, tl0), bl, bias30));
        if constexpr (D == 2) {
#pragma unroll
            for (int a = 0; a < W; ++a) {
                int r = fold_cell(s0 + a, p.n, simple);
                if constexpr (SLAB) {
                    r -= row_lo;
                    if ((unsigned)r >= (unsigned)nrows) continue;
                }
                const int rq = __float2int_rn(q4 * es_f32(fmaf((float)a, h2, t00), bl, -bl));
                const int row = r * plane + cb;
                unsigned wraps = 0u;
#pragma unroll
                for (int c = 0; c < W; ++c) wraps = tile.add_int_run(row + c, mulhi_rn(rq, wi[c]), wraps);
                if (wraps) tile.add_carries(row, W, wraps, sg);
            }
        } else {
#pragma unroll 1
            for (int a = 0; a < W; ++a) {
                int r = fold_cell(s0 + a, p.n, simple);
                if constexpr (SLAB) {
                    r -= row_lo;
                    if ((unsigned)r >= (unsigned)nrows) continue;
                }
                const float qa = q4 * es_f32(fmaf((float)a, h2, t00), bl, -bl);
                const int row = r * plane;
#pragma unroll
                for (int b = 0; b < W; ++b) {
                    const int rq = __float2int_rn(qa * w1[b]);
                    const int line = row + c1[b];
                    unsigned wraps = 0u;
#pragma unroll
                    for (int c = 0; c < W; ++c) wraps = tile.add_int_run(line + c, mulhi_rn(rq, wi[c]), wraps);
                    if (wraps) tile.add_carries(line, W, wraps, sg);
                }
            }
        }
    } else {
        float wl[W];
#pragma unroll
        for (int c = 0; c < W; ++c) wl[c] = es_f32(fmaf((float)c, h2, tl0), bl, -bl);
        if constexpr (D == 2) {
#pragma unroll
            for (int a = 0; a < W; ++a) {
                int r = fold_cell(s0 + a, p.n, simple);
                if constexpr (SLAB) {
                    r -= row_lo;
                    if ((unsigned)r >= (unsigned)nrows) continue;
                }
                const float qa = q * es_f32(fmaf((float)a, h2, t00), bl, -bl);
                const int row = r * plane + cb;
#pragma unroll
                for (int c = 0; c < W; ++c) tile.add(row + c, qa * wl[c]);
            }
        } else {
#pragma unroll 1
            for (int a = 0; a < W; ++a) {
                int r = fold_cell(s0 + a, p.n, simple);
                if constexpr (SLAB) {
                    r -= row_lo;
                    if ((unsigned)r >= (unsigned)nrows) continue;
                }
                const float qa = q * es_f32(fmaf((float)a, h2, t00), bl, -bl);
                const int row = r * plane;
#pragma unroll
                for (int b = 0; b < W; ++b) {
                    const float qab = qa * w1[b];
                    const int line = row + c1[b];
#pragma unroll
                    for (int c = 0; c < W; ++c) tile.add(line + c, qab * wl[c]);
                }
            }
        }
    }
}

// ---- FP64 points

// Add the w^d contributions of one FP64 point (q in grid units 2^-Eg) to the block tile.  SLAB:
// the tile holds a slab of the grid's rows and rows outside it are skipped; otherwise it holds
// every row (row_lo = 0, nrows = n/2 + 1).  The kernel weights are FP64.  The point works in units
// 2^-(Eg+s) with s = 60 - ilogb|q| (at most 94), so that |q| 2^s < 2^61: each row takes the
// integer R = round(q psi_a 2^s) (3D: then round(R psi_b) in integers) and each cell
// round(R psi_c) from a 61-bit fixed-point psi_c (fix_mul) -- one FP64 product and conversion
// per row instead of per cell, and about 2^-61 relative rounding -- which goes to the tile as
// grid units and 32 fraction bits (tap_split).
template <int D, int W, bool SLAB>
__device__ __forceinline__ void spread_point_f64(const SpreadArgs &p, const Point<double, D> &pt,
                                                 const WideTile &tile, int row_lo, int nrows, int plane)
{
    const double q = pt.q;
    if (q == 0.0) return;
    double w0[W];
    int r0[W];
    axis_weights_f64<W>(p, pt.x[0], w0, r0);
    bool hit = !SLAB;
#pragma unroll
    for (int a = 0; a < W; ++a) {
        if constexpr (SLAB) {
            r0[a] -= row_lo;
            hit |= ((unsigned)r0[a] < (unsigned)nrows);
        }
    }
    if (!hit) return;
    const int s = max(0, min(60 - ilogb(q), 94));
    const double qs = ldexp(q, s);
    const TapShift ts = tap_shift(s);
    double wl[W];  // last axis: consecutive padded columns cb..cb+w-1 (clamped: x lies in [0, n/2])
    const int cb = min(max(kernel_weights_f64<W>(pt.x[D - 1], wl) + p.cpad, 0), p.ncol - W);
    FixW fl[W];
#pragma unroll
    for (int c = 0; c < W; ++c) fl[c] = fix_weight(wl[c]);
    if constexpr (D == 2) {
#pragma unroll 1
        for (int a = 0; a < W; ++a) {
            if (SLAB && (unsigned)r0[a] >= (unsigned)nrows) continue;
            const long long R = __double2ll_rn(qs * w0[a]);
            const int row = r0[a] * plane + cb;
#pragma unroll
            for (int c = 0; c < W; ++c) {
                long long I;
                unsigned F;
                tap_split(fix_mul(R, fl[c]), ts, I, F);
                tile.add(row + c, I, F);
            }
        }
    } else {
        double w1[W];
        int c1[W];
        axis_weights_f64<W>(p, pt.x[1], w1, c1);
        FixW f1[W];
#pragma unroll
        for (int b = 0; b < W; ++b) {
            f1[b] = fix_weight(w1[b]);
            c1[b] = c1[b] * p.ncol + cb;
        }
#pragma unroll 1
        for (int a = 0; a < W; ++a) {
            if (SLAB && (unsigned)r0[a] >= (unsigned)nrows) continue;
            const long long Ra = __double2ll_rn(qs * w0[a]);
            const int row = r0[a] * plane;
#pragma unroll 1
            for (int b = 0; b < W; ++b) {
                const long long R = fix_mul(Ra, f1[b]);
                const int line = row + c1[b];
#pragma unroll
                for (int c = 0; c < W; ++c) {
                    long long I;
                    unsigned F;
                    tap_split(fix_mul(R, fl[c]), ts, I, F);
                    tile.add(line + c, I, F);
                }
            }
        }
    }
}

// One point into a tile (every lane of the warp calls it, lanes without a pair with q = 0).  FP32:
// integer products for points below 2^29 tile units, chosen per lane (a point's contributions must
// not depend on its warp-mates: bitwise reproducibility across launch shapes; points of 2^29 tile
// units or more are rare); a lane whose point is below kNegligibleF32 idles.
template <typename T, int D, int W, typename Tile, bool SLAB>
__device__ __forceinline__ void spread_point_body(const SpreadArgs &p, const Point<T, D> &pt, const Tile &tile,
                                                  int row_lo, int nrows, int plane)
{
    if constexpr (sizeof(T) == 4) {
        if (fabsf(pt.q) < kIntLimitF32) spread_point_f32<D, W, kInt, SLAB>(p, pt, tile, row_lo, nrows, plane);
        else spread_point_f32<D, W, kLarge, SLAB>(p, pt, tile, row_lo, nrows, plane);
    } else {
        spread_point_f64<D, W, SLAB>(p, pt, tile, row_lo, nrows, plane);
    }
}

template <typename T, int D, int W, typename Tile, bool SLAB>
__device__ __noinline__ void spread_point_outlined(const SpreadArgs &p, const Point<T, D> &pt, const Tile &tile,
                                                   int row_lo, int nrows, int plane)
{
    spread_point_body<T, D, W, Tile, SLAB>(p, pt, tile, row_lo, nrows, plane);
}

// 3D points (w^3 taps, two integer kinds) are spread by one out-of-line copy per kernel: inlined
// at each call site the kernel outgrew the instruction cache (stalls on instruction fetch; 13%
// longer on the 3D bi-Maxwellian, 70% on 3D BKW once the one-slab queue added a third site).
// 2D points (w^2 taps) stay inline, where the call's register saves cost 5%.
template <typename T, int D, int W, typename Tile, bool SLAB>
__device__ __forceinline__ void spread_point_any(const SpreadArgs &p, const Point<T, D> &pt, const Tile &tile,
                                                 int row_lo, int nrows, int plane)
{
    if constexpr (D == 3) spread_point_outlined<T, D, W, Tile, SLAB>(p, pt, tile, row_lo, nrows, plane);
    else spread_point_body<T, D, W, Tile, SLAB>(p, pt, tile, row_lo, nrows, plane);
}

// Advance the cursor c (in steps of st, below `end`) to this lane's next pair that is not negligible:
// a loaded pair with non-zero strength, a strength bound not below the screening threshold tau
// (0: no screening), and a bound Ut >= floor_q on every point's |q| in tile units.  On success
// P.base is multiplied by the pair's multiplicity; false when no pair is left.
template <typename T, int D, bool ANG>
__device__ __forceinline__ bool next_pair(const SpreadArgs &p, PairCursor &c, long long end, const PairStep &st, T sc,
                                          T tau, T floor_q, PairData<T, D> &P)
{
    for (; c.pr < end; pair_advance(p, c, st)) {
        if (!load_pair<T, D, ANG>(p, c, P)) continue;
        const T U = pair_bound<T, D>(p, P);
        if (tau > T(0) && U < tau) continue;
        if (U * P.mult * sc * kconst<T>(p).wmax < floor_q) continue;
        P.base *= P.mult;
        return true;
    }
    return false;
}

// A pair of zero strength at the origin: its points add nothing (lanes whose pairs have run out).
template <typename T, int D>
__device__ __forceinline__ void zero_pair(PairData<T, D> &P)
{
#pragma unroll
    for (int l = 0; l < D; ++l) {
        P.cen[l] = T(0);
        P.dir[l] = T(0);
    }
    P.rad = T(0);
    P.base = T(0);
    P.mult = T(0);
}

// The pairs pr = first, first + stride, ... below end of one lane, spread into a tile that holds
// every row.  Every lane of the warp runs every point step (the loop conditions are uniform).
template <typename T, int D, int W, typename Tile, bool ANG>
__device__ __forceinline__ void spread_pairs(const SpreadArgs &p, long long first, long long end, long long stride,
                                             T sc, T tau, T floor_q, const Tile &tile, int row_lo, int nrows, int plane)
{
    PairCursor c = pair_cursor(p, first);
    const PairStep st = pair_step(p, stride);
    for (;;) {
        PairData<T, D> P;
        const bool ok = next_pair<T, D, ANG>(p, c, end, st, sc, tau, floor_q, P);
        if (!__any_sync(0xffffffffu, ok)) break;
        if (!ok) zero_pair<T, D>(P);
        const T qbase = P.base * sc;
        for (int m = 0; m < p.M; ++m) {
            Point<T, D> pt;
            make_point<T, D, ANG>(p, P, qbase, m, pt);
            spread_point_any<T, D, W, Tile, false>(p, pt, tile, row_lo, nrows, plane);
        }
        if (ok) pair_advance(p, c, st);
    }
}

// ---- slabbed grids: warp point queues
//
// When the folded grid is split into slabs along axis 0, a point adds to a block's slab only
// if one of its w axis-0 rows lies there, and with a few slabs most points of a warp miss it:
// spreading them where they are generated would leave most lanes idle while the others add.
// Instead each warp appends the points that hit its slab to a queue of 32 entries in shared
// memory (slot-major) and spreads a full queue with all 32 lanes, one point per lane.

// Whether any of the w axis-0 rows of a point whose first tap is s lies in the slab.
template <int W>
__device__ __forceinline__ bool rows_hit_from(const SpreadArgs &p, int s, int row_lo, int nrows)
{
    const bool simple = p.simple_fold != 0;
    bool hit = false;
#pragma unroll
    for (int a = 0; a < W; ++a) hit |= (unsigned)(fold_cell(s + a, p.n, simple) - row_lo) < (unsigned)nrows;
    return hit;
}

// Whether any of the w axis-0 rows of a point lies in the slab (the rows of the point's spreading).
template <typename T, int D, int W>
__device__ __forceinline__ bool rows_hit(const SpreadArgs &p, const Point<T, D> &pt, int row_lo, int nrows)
{
    int s;
    if constexpr (sizeof(T) == 4) {
        float t0;
        s = first_tap_f32<W>(pt.X[0], pt.F[0], t0);
    } else {
        s = (int)floor(pt.x[0] - 0.5 * W) + 1;
    }
    return rows_hit_from<W>(p, s, row_lo, nrows);
}

// What a warp queue holds for one point.  LATE (FP32): the post-collision velocity v'[D] and the
// strength q, so that the grid coordinates are formed after the queue and only for the points that
// go there -- in a slabbed grid (SLAB) with the axis-0 coordinate X0 + F0 formed before, for the
// slab test; otherwise (FP64) the point itself, x[D] and q.
// Slot layout: value k of slot j at buf[32 k + j].
template <typename T, int D, bool LATE, bool SLAB>
struct QEntry {
    Point<T, D> pt;
    __device__ __forceinline__ T q() const { return pt.q; }
    __device__ __forceinline__ void put(T *buf, int slot) const
    {
#pragma unroll
        for (int l = 0; l < D; ++l) {
            if constexpr (sizeof(T) == 4) {
                buf[l * 32 + slot] = pt.X[l];
                buf[(D + l) * 32 + slot] = pt.F[l];
            } else {
                buf[l * 32 + slot] = pt.x[l];
            }
        }
        buf[(sizeof(T) == 4 ? 2 * D : D) * 32 + slot] = pt.q;
    }
    __device__ __forceinline__ void get(const T *buf, int slot)
    {
#pragma unroll
        for (int l = 0; l < D; ++l) {
            if constexpr (sizeof(T) == 4) {
                pt.X[l] = buf[l * 32 + slot];
                pt.F[l] = buf[(D + l) * 32 + slot];
            } else {
                pt.x[l] = buf[l * 32 + slot];
            }
        }
        pt.q = buf[(sizeof(T) == 4 ? 2 * D : D) * 32 + slot];
    }
    template <bool ANG>
    __device__ __forceinline__ void make(const SpreadArgs &p, const PairData<T, D> &P, T qbase, int m)
    {
        make_point<T, D, ANG>(p, P, qbase, m, pt);
    }
    template <int W>
    __device__ __forceinline__ bool in_slab(const SpreadArgs &p, int row_lo, int nrows)
    {
        return rows_hit<T, D, W>(p, pt, row_lo, nrows);
    }
    __device__ __forceinline__ void point(const SpreadArgs &, Point<T, D> &out) const { out = pt; }
};
template <int D, bool SLAB>
struct QEntry<float, D, true, SLAB> {
    float v[D], qv, X0, F0;
    __device__ __forceinline__ float q() const { return qv; }
    __device__ __forceinline__ void put(float *buf, int slot) const
    {
#pragma unroll
        for (int l = 0; l < D; ++l) buf[l * 32 + slot] = v[l];
        buf[D * 32 + slot] = qv;
        if constexpr (SLAB) {
            buf[(D + 1) * 32 + slot] = X0;
            buf[(D + 2) * 32 + slot] = F0;
        }
    }
    __device__ __forceinline__ void get(const float *buf, int slot)
    {
#pragma unroll
        for (int l = 0; l < D; ++l) v[l] = buf[l * 32 + slot];
        qv = buf[D * 32 + slot];
        if constexpr (SLAB) {
            X0 = buf[(D + 1) * 32 + slot];
            F0 = buf[(D + 2) * 32 + slot];
        }
    }
    template <bool ANG>
    __device__ __forceinline__ void make(const SpreadArgs &p, const PairData<float, D> &P, float qbase, int m)
    {
        qv = point_velocity_f32<D, ANG>(p, P, qbase, m, v);
    }
    // slabs: the axis-0 coordinate, then whether one of the point's rows lies in the slab
    template <int W>
    __device__ __forceinline__ bool in_slab(const SpreadArgs &p, int row_lo, int nrows)
    {
        grid_coord_f32(kconst<float>(p), v[0], p.r == 1, X0, F0);
        float t0;
        return rows_hit_from<W>(p, first_tap_f32<W>(X0, F0, t0), row_lo, nrows);
    }
    // the same point make_point forms (same velocity, strength and coordinates)
    __device__ __forceinline__ void point(const SpreadArgs &p, Point<float, D> &out) const
    {
        const TypedConsts<float> &K = kconst<float>(p);
        const bool alg = (p.r == 1);
#pragma unroll
        for (int l = 0; l < D; ++l) {
            if (SLAB && l == 0) {
                out.X[0] = X0;
                out.F[0] = F0;
            } else {
                grid_coord_f32(K, v[l], alg, out.X[l], out.F[l]);
            }
        }
        out.q = qv;
    }
};

// Spread queue slot `lane` (when valid) with the whole warp.
template <typename T, int D, int W, typename Tile, bool SLAB, bool LATE>
__device__ __forceinline__ void queue_spread(const SpreadArgs &p, const T *buf, int lane, bool valid,
                                             const Tile &tile, int row_lo, int nrows, int plane)
{
    if (!valid) return;
    QEntry<T, D, LATE, SLAB> e;
    e.get(buf, lane);
    Point<T, D> pt;
    e.point(p, pt);
    spread_point_any<T, D, W, Tile, SLAB>(p, pt, tile, row_lo, nrows, plane);
}

// The pairs pr = first, first + nthr, ... below end of one thread, spread through the warp's
// queue `buf` (spread_queue_values(d, fp32) x 32 values) into one slab (SLAB) or a tile that
// holds every row.  Points below floor_q (they add exactly zero) are not queued, so that every
// lane spreads a real point; FP32 points queue their velocity and strength and form their grid
// coordinates after the queue (QEntry; with slabs, all but axis 0's).  Every loop condition is
// uniform over the warp.
template <typename T, int D, int W, typename Tile, bool ANG, bool SLAB = true>
__device__ __forceinline__ void spread_pairs_queued(const SpreadArgs &p, long long first, long long end,
                                                    long long nthr, T sc, T tau, T floor_q, const Tile &tile,
                                                    int row_lo, int nrows, int plane, T *buf)
{
    constexpr bool LATE = (sizeof(T) == 4);
    const unsigned full = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const unsigned lt = (1u << lane) - 1u;
    int count = 0;  // queued points, the same in every lane
    PairCursor c = pair_cursor(p, first);
    const PairStep st = pair_step(p, nthr);
    for (;;) {
        PairData<T, D> P;
        const bool ok = next_pair<T, D, ANG>(p, c, end, st, sc, tau, floor_q, P);
        if (!__any_sync(full, ok)) break;
        const T qbase = ok ? P.base * sc : T(0);
        for (int m = 0; m < p.M; ++m) {
            QEntry<T, D, LATE, SLAB> e;
            bool hit = false;
            if (ok) {
                e.template make<ANG>(p, P, qbase, m);
                // points below floor_q add exactly zero and are not queued
                hit = fabs(e.q()) >= floor_q;
                if constexpr (SLAB) hit = hit && e.template in_slab<W>(p, row_lo, nrows);
            }
            const unsigned mask = __ballot_sync(full, hit);
            const int n = __popc(mask), rank = __popc(mask & lt), room = 32 - count;
            if (hit && rank < room) e.put(buf, count + rank);
            if (n >= room) {  // full: spread 32 points, then queue the rest
                __syncwarp();
                queue_spread<T, D, W, Tile, SLAB, LATE>(p, buf, lane, true, tile, row_lo, nrows, plane);
                __syncwarp();
                if (hit && rank >= room) e.put(buf, rank - room);
                count = n - room;
            } else {
                count += n;
            }
        }
        if (ok) pair_advance(p, c, st);
    }
    __syncwarp();
    queue_spread<T, D, W, Tile, SLAB, LATE>(p, buf, lane, lane < count, tile, row_lo, nrows, plane);
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
    // Tile unit 2^-Et with Et = Eg - tile_bits(D) (2^-47 B or finer in 2D, 2^-53 B in 3D); kept
    // inside the float range for tiny inputs (a coarser unit there).
    const int Et = min(Eg - tile_bits(D), 120);
    const int shift = Eg - Et;
    const SplitTile tile{words, carry};
    const float sc = (float)ldexp(1.0, Et);
    const float tau = (float)*p.tau;
    long long first, nthr;
    pair_schedule(p, first, nthr);
    if (p.nslab > 1) {
        float *buf = reinterpret_cast<float *>(smem_raw + tile_bytes((size_t)p.rows_per_slab * G.plane, true)) +
                     (threadIdx.x >> 5) * 32 * spread_queue_values(D, true);
        spread_pairs_queued<float, D, W, SplitTile, ANG>(p, first, p.npairs, nthr, sc, tau, kNegligibleF32, tile,
                                                          G.row_lo, G.nrows, G.plane, buf);
    } else if (p.queued) {  // one slab: the queues only compact the points that add something
        float *buf = reinterpret_cast<float *>(smem_raw + tile_bytes(G.ncell, true)) +
                     (threadIdx.x >> 5) * 32 * spread_queue_values(D, true);
        spread_pairs_queued<float, D, W, SplitTile, ANG, false>(p, first, p.npairs, nthr, sc, tau, kNegligibleF32,
                                                                 tile, 0, G.nrows, G.plane, buf);
    } else {
        spread_pairs<float, D, W, SplitTile, ANG>(p, first, p.npairs, nthr, sc, tau, kNegligibleF32, tile, G.row_lo,
                                                   G.nrows, G.plane);
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
__global__ void __launch_bounds__(max_threads_f64(D), 1) k_spread_f64(const __grid_constant__ SpreadArgs p)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const SlabGeom G = slab_geometry(p, D);
    if (G.nrows <= 0) return;  // uniform over the block
    // fraction, low and high words of rows_per_slab x plane cells each
    const size_t tile_cells = (size_t)p.rows_per_slab * G.plane;
    unsigned *words = reinterpret_cast<unsigned *>(smem_raw);
    const WideTile tile{words, words + tile_cells, reinterpret_cast<int *>(words + 2 * tile_cells)};
    for (int c = threadIdx.x; c < G.ncell; c += blockDim.x) {
        tile.fr[c] = 0u;
        tile.lo[c] = 0u;
        tile.hi[c] = 0;
    }
    load_kernel_poly(p.kpoly);
    __syncthreads();
    const double Bnd = *p.bound;
    const int Eg = global_exponent(Bnd);
    const double tau = *p.tau;
    const double sc = ldexp(1.0, Eg);  // strengths in grid units
    // pairs whose summed strength bounds stay below 2^-64 B are skipped (per-point bound below
    // floor_q, and at most npairs pairs): 2^-3 grid units at most in all
    const double floor_q = ldexp(Bnd, Eg - 64) * p.cd.wmax / (double)p.npairs;
    long long first, nthr;
    pair_schedule(p, first, nthr);
    if (p.nslab > 1) {
        double *buf = reinterpret_cast<double *>(smem_raw + tile_bytes(tile_cells, false)) +
                      (threadIdx.x >> 5) * 32 * spread_queue_values(D, false);
        spread_pairs_queued<double, D, W, WideTile, ANG>(p, first, p.npairs, nthr, sc, tau, floor_q, tile, G.row_lo,
                                                          G.nrows, G.plane, buf);
    } else {
        spread_pairs<double, D, W, WideTile, ANG>(p, first, p.npairs, nthr, sc, tau, floor_q, tile, G.row_lo,
                                                   G.nrows, G.plane);
    }
    __syncthreads();
    for (int c = threadIdx.x; c < G.ncell; c += blockDim.x) {
        const long long v = tile.value(c);
        if (v) atomicAdd(p.grid + tile_to_grid_cell(c, D, p.nf, p.ncol, p.cpad, p.n, G.row_lo), (unsigned long long)v);
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
