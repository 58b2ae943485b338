// Internal declarations of the sm_103a collision-operator library (not part of the ABI).
#pragma once

#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>

#include "pg_boltz.h"

namespace pgb {

// Everything the spreading kernel reads, passed by value.  The nodes, weights and
// coefficients are in the kernel's arithmetic type T (float or double).
// Angular factor of the collision kernel B(|g|, cos theta) = Bconst |g|^gamma b(cos theta)
// (Eq. collision_form), b(c) = sum_{p < n} c_p c^p; n = 0 is the VHS kernel (b = 1).
constexpr int kMaxAngular = 8;
// Coefficients of the FP64 spreading kernel's piecewise polynomial form (kernel_poly on the host):
// ceil(w/2) taps of kernel_poly_terms(w) each, for widths up to 16.  Degree w interpolates each tap
// to about the kernel's own truncation error exp(-beta) at the default oversampling 2 for w >= 7;
// narrower kernels take two more terms, which keeps oversampling up to 4 within a few times it.
__host__ __device__ constexpr int kernel_poly_terms(int w) { return w < 12 ? w + 3 : w + 1; }
constexpr int kPolyCoefF64 = 8 * 17;
struct Angular {
    int n;
    double c[kMaxAngular];
};

// Loop-invariant constants of the spreading kernels in their arithmetic type, filled once on the
// host (or by the batched kernel's cell switch) so the point loops convert nothing from double.
template <typename T>
struct TypedConsts {
    T S, invS, SS;      // map scale, 1/S, S^2
    T gs;               // grid_scale
    T Bconst, gamma;    // kernel constant and exponent
    T Wang;             // Wsig * angmax (pair bound factor)
    T wmax;             // wmax_frac
    T bl;               // beta log2(e): ES kernel values as powers of two
    T ang_even[kMaxAngular / 2];
    // FP32 point coordinates without systematic offsets or scale errors: a grid coordinate is
    // x = xq -+ atan(v/S) gs (r = 1) or 2 atan(exp(-v/S)) gs (r = 0) with xq = n/4 exact and the
    // products by 1/S and gs carried in two terms (hi + lo); zero in TypedConsts<double>
    T invS_lo, gs_lo, xq;
};

struct SpreadArgs {
    int d, N, M, r;
    int nnode;            // N^d interior nodes
    long long npairs;     // unordered node pairs, unordered_pairs(nnode)
    int n, nf;            // periodic grid size, folded cells per axis (n/2 + 1)
    int rows_per_slab;    // folded-grid rows (axis 0) held in shared memory by one block
    int nslab;            // number of slabs covering axis 0
    int fast_gamma;       // 0: gamma = 0, 1: gamma = 1, 2: gamma = 1/2, 3: general pow
    double S, gamma, Bconst;
    double beta;          // exponential-of-semicircle shape
    double grid_scale;    // n / (2 pi): angle -> grid coordinate
    const void *vnode;    // N node velocities (same on every axis)
    const float *vnode_lo;  // FP32 plans: v - (double)vnode, so that hi + lo carries the node exactly
                            // to about 2^-48 (nullptr for FP64 plans)
    const void *a;        // nnode values a_i = W_i g_i
    const void *sig;      // M x d sphere points
    const void *wsig;     // M sphere weights
    double Wsig;          // sum_m w_m
    double wmax_frac;     // max_m w_m / sum_m w_m: one point's share of a pair's strength bound
    const double *bound;  // device scalar B >= sum_p |q_p| (written by the loss kernel)
    const double *tau;    // device scalar: node pairs whose strength bound is below it are skipped (0: none)
    unsigned long long *grid;  // nf^d folded grid, int64 fixed point in units of 2^-Eg
    int simple_fold;      // 1 when w <= n/2: unfolded indices lie in [-n/2, n] (no modulo needed)
    int cpad;             // unfolded padding columns on each side of the last axis in block tiles
    int ncol;             // nf + 2 cpad: tile cells along the last axis
    int tile_cells;       // cells of one block tile (rows_per_slab rows)
    int *carry;           // FP32: per-block carry counters, blocks x tile_cells (global memory)
    int queued;           // FP32 one-slab grids: 1 when the warps' point queues follow the tile in
                          // shared memory (spread_queue_bytes of the launch's threads)
    // angular kernel: a spread pair stands for both orders, whose cos theta differ in sign, so
    // the gain needs the even part b_e(c) = (b(c) + b(-c))/2 = sum_k ang_even[k] c^(2k) only
    int nang_even;        // terms of ang_even; 0: VHS kernel (no angular factor)
    double ang_even[kMaxAngular / 2];
    double angmax;        // sum_k |ang_even[k]| >= |b_e(c)| on [-1, 1] (1 for VHS)
    // FP64 kernel weights: tap a (< ceil(w/2)) of a point at offset y in [-1, 1] within its cell is
    // E_a(y^2) + y O_a(y^2), and tap w-1-a is E_a(y^2) - y O_a(y^2); with P = kernel_poly_terms(w),
    // kpoly[a P + k] (device, kPolyCoefF64 doubles) holds the (P+1)/2 coefficients of E_a, then
    // the P/2 of O_a, lowest power first
    const double *kpoly;
    TypedConsts<float> cf;   // the double fields above as float (FP32 kernels)
    TypedConsts<double> cd;  // ... and as double (FP64 kernels)
};

// Fill a.cf and a.cd from the double fields (call after setting S, grid_scale, Bconst, gamma,
// Wsig, angmax, wmax_frac, beta and ang_even).
template <typename T>
__host__ __device__ inline void fill_typed_consts(const SpreadArgs &a, TypedConsts<T> &c)
{
    c.S = T(a.S);
    c.invS = T(1.0 / a.S);
    c.SS = T(a.S * a.S);
    c.gs = T(a.grid_scale);
    c.Bconst = T(a.Bconst);
    c.gamma = T(a.gamma);
    c.Wang = T(a.Wsig * a.angmax);
    c.wmax = T(a.wmax_frac);
    c.bl = T(a.beta * 1.4426950408889634);
    for (int k = 0; k < kMaxAngular / 2; ++k) c.ang_even[k] = T(k < a.nang_even ? a.ang_even[k] : 0.0);
    c.invS_lo = T(1.0 / a.S - double(c.invS));
    c.gs_lo = T(a.grid_scale - double(c.gs));
    c.xq = T(0.25 * a.n);
}
__host__ __device__ inline void fill_spread_consts(SpreadArgs &a)
{
    fill_typed_consts<float>(a, a.cf);
    fill_typed_consts<double>(a, a.cd);
}
template <typename T>
__device__ __forceinline__ const TypedConsts<T> &kconst(const SpreadArgs &a)
{
    if constexpr (sizeof(T) == 4) return a.cf;
    else return a.cd;
}

// Node pairs the spreading kernels walk: each unordered pair {i, j} once (the two orders add the
// same points with the same strength), nnode (nnode + 1) / 2 in all.
__host__ __device__ inline long long unordered_pairs(long long nnode) { return nnode * (nnode + 1) / 2; }

// Values per queued point of the slabbed spreading kernels: FP32 points keep each coordinate as
// a cell and a fraction (2d + 1 floats with the strength), FP64 points d + 1 doubles.
__host__ __device__ inline int spread_queue_values(int d, bool f32) { return f32 ? 2 * d + 1 : d + 1; }
// Shared memory of the warp point queues of a slabbed spreading block of `threads` threads:
// 32 points per warp.
__host__ __device__ inline size_t spread_queue_bytes(int threads, int d, bool f32)
{
    return (size_t)(threads / 32) * 32 * spread_queue_values(d, f32) * (f32 ? 4 : 8);
}
// Shared memory of a block tile of `cells` cells, rounded up to 16 bytes (the queues follow it):
// FP32 tiles hold one 32-bit word per cell, FP64 tiles three (fraction, low and high words).
__host__ __device__ inline size_t tile_bytes(size_t cells, bool f32)
{
    return (cells * (f32 ? 4 : 12) + 15) / 16 * 16;
}

// Padding columns of the block tiles' last axis for kernel width w: the unfolded support of a point
// at grid coordinate x in [0, n/2] spans floor(x - w/2) + 1 .. floor(x + w/2), i.e. at most w/2
// columns beyond either end; w/2 + 1 leave a margin for rounding of x.
__host__ __device__ inline int tile_col_pad(int w) { return w / 2 + 1; }

// FP32 block tiles count in units 2^-(Eg - tile_bits(d)), about 2^-47 B (2D) or 2^-53 B (3D) for the
// strength bound B: each contribution is rounded to the tile unit once, and with w^3 contributions
// per point and the deconvolution's growth along three axes, 3D needs the finer unit for the FP32
// path's accuracy (with 2^-47 B the rounding was 3e-6 of the gain norm on the 3D gamma = 1/2
// workload, with 2^-53 B 4e-7); a coarser unit makes more node pairs negligible (skipped exactly)
// and more points fit the integer products, which is faster.
__host__ __device__ constexpr int tile_bits(int d) { return d == 3 ? 8 : 14; }

// Exponent Eg of the grid's fixed-point unit 2^-Eg: the largest E with B 2^E < 2^61 for the
// bound B >= sum_p |q_p| (0 when B is zero or not finite).
__host__ __device__ inline int global_exponent(double B)
{
    if (!(B > 0.0) || !(B < 1.0e300)) return 0;
    return 60 - ilogb(B);
}

// Screening of negligible node pairs: the loss kernel counts the pair bounds per binary
// exponent (kScreenBins bins, bin k holds bounds in [2^(k - kScreenOffset), 2^(k+1 - kScreenOffset)),
// the first and last bins also everything below / above).
constexpr int kScreenBins = 256;
constexpr int kScreenOffset = 200;
// Launch the spreading kernel for (precision, d, w); returns cudaSuccess or the launch error.
// One translation unit per (precision, d) keeps the parallel build short.
cudaError_t launch_spread_f32_d2(const SpreadArgs &a, int w, int blocks, int threads, size_t smem, cudaStream_t s);
cudaError_t launch_spread_f32_d3(const SpreadArgs &a, int w, int blocks, int threads, size_t smem, cudaStream_t s);
cudaError_t launch_spread_f64_d2(const SpreadArgs &a, int w, int blocks, int threads, size_t smem, cudaStream_t s);
cudaError_t launch_spread_f64_d3(const SpreadArgs &a, int w, int blocks, int threads, size_t smem, cudaStream_t s);
// The same with the angular factor of the collision kernel (a.nang_even > 0; called by the above).
cudaError_t launch_spread_f32_d2_ang(const SpreadArgs &a, int w, int blocks, int threads, size_t smem, cudaStream_t s);
cudaError_t launch_spread_f32_d3_ang(const SpreadArgs &a, int w, int blocks, int threads, size_t smem, cudaStream_t s);
cudaError_t launch_spread_f64_d2_ang(const SpreadArgs &a, int w, int blocks, int threads, size_t smem, cudaStream_t s);
cudaError_t launch_spread_f64_d3_ang(const SpreadArgs &a, int w, int blocks, int threads, size_t smem, cudaStream_t s);
// Highest kernel width with a compiled spreading kernel for each type.
constexpr int kMaxWidthF32 = 10;
constexpr int kMaxWidthF64 = 16;
static_assert(kPolyCoefF64 >= ((kMaxWidthF64 + 1) / 2) * kernel_poly_terms(kMaxWidthF64) &&
                  kPolyCoefF64 >= 6 * kernel_poly_terms(11),
              "kernel polynomial storage");
constexpr int kMinWidth = 2;
// Largest spreading block for each type (the kernels' launch bounds).
constexpr int kMaxThreadsF32 = 1024;
// FP64: 2D kernels use up to 255 registers per thread, 3D kernels fit 128 (their per-point
// spreading is out of line), so 3D blocks hold twice the threads (integer shared atomics whose
// returned values feed the next step want many resident warps).
__host__ __device__ constexpr int max_threads_f64(int d) { return d == 3 ? 512 : 256; }
// Largest block of the batched FP32 spreading kernel.
constexpr int kBatchThreadsF32 = 1024;

// Three-axis shape of a C-order array; 2D arrays use e0 = 1.
struct Dims3 {
    int e[3];
};

// out = A contracted with `in` along axis `ax` (A is m x in.e[ax], row-major).
cudaError_t launch_axis_pass(const double *in, Dims3 in_dims, int ax, const double *A, int m,
                             double *out, cudaStream_t s);
// Last reconstruction pass along axis 2, then a_i = acc * prod_l scale[i_l];
// writes a (FP64) and, if af != nullptr, a float copy.
cudaError_t launch_recon_last(const double *in, Dims3 in_dims, const double *A, int m,
                              const double *scale, int d, double *a, float *af, cudaStream_t s);
// Loss: h_i = a_i * Lsum_i * prod_l inv_mu2[i_l], Lsum_i = Bw * sum_j a_j B(|v_i - v_j|) A_ij,
// A_ij = (1/Wsig) sum_m w_m b(cos theta_ijm) for an angular kernel (ang.n > 0; the sum over the
// sphere set then runs per pair), 1 otherwise (Bw = Bconst Wsig);
// also ub_i = |a_i| Bw angmax sum_j |a_j| B_ij prod_l mu^-2(|c_l| + rad), an upper bound of the
// spreading strengths of the pairs (i, .).  FP32 pair terms (node differences with the nodes'
// rounding vnode32_lo added back, summed in FP64) carry a relative error near 1e-7 that differs
// from pair to pair; the bound gets a 1e-5 margin in k_bound_reduce.
// vnode32 != nullptr selects FP32 pair terms (the FP32 path).
// hist != nullptr: also count every pair bound |a_i| Bw |a_j| B_ij prod mu^-2 into the screening histogram.
cudaError_t launch_loss(const double *a, const float *a32, const double *vnode, const float *vnode32,
                        const float *vnode32_lo, int N,
                        int d, int M,
                        const double *sig, const double *wsig, const float *sig32, const float *wsig32,
                        const Angular &ang, double angmax, double Wsig, double gamma,
                        int fast_gamma, double Bw, const double *inv_mu2, double S, int r,
                        double *h, double *ub, unsigned long long *hist, cudaStream_t s);
// Screening bin of a pair bound u > 0.
__host__ __device__ inline int screen_bin(double u)
{
    int e = ilogb(u) + kScreenOffset;
    return e < 0 ? 0 : (e >= kScreenBins ? kScreenBins - 1 : e);
}
// B = sum_i ub_i (fixed summation order), written to *B.  When hist != nullptr also the screening
// threshold *tau = 2^(k - kScreenOffset) for the largest k with
//   sum_{bins j < k} count_j 2^(j+1 - kScreenOffset) <= eps * B
// (an upper bound of the total strength of the pairs below tau), else *tau = 0.
cudaError_t launch_bound_reduce(const double *ub, int n, const unsigned long long *hist, double eps, double *B,
                                double *tau, cudaStream_t s);
// First transform pass reading the int64 fixed-point grid (units 2^-Eg, Eg from *B), times scale.
cudaError_t launch_axis_pass_fixed(const unsigned long long *in, Dims3 in_dims, int ax, const double *A,
                                   int m, const double *B, double scale, double *out, cudaStream_t s);
// Exact / FP32 value of the constant factors of an FP32 point strength: Bconst (the kernel's
// constant), the common sphere weight w and 1/S per axis enter every strength as rounded FP32
// constants, a common relative error that the transform of the FP32 grid divides out in FP64.
inline double fp32_strength_correction(double Bconst, double w, double S, int d)
{
    double c = (Bconst / (double)(float)Bconst) * (w / (double)(float)w);
    for (int l = 0; l < d; ++l) c *= (1.0 / S) / (double)(float)(1.0 / S);
    return c;
}
// Final pass along axis 2: Qp = D . G, Qm = E . H, Q = Qp - Qm (also copied to Qcopy).
cudaError_t launch_final(const double *G, Dims3 g_dims, const double *D, const double *H,
                         Dims3 h_dims, const double *E, int m, double *Q, double *Qplus,
                         double *Qcopy, cudaStream_t s);
// RK stage argument y = x + c k, and the RK4 update f += dt/6 (k1 + 2k2 + 2k3 + k4).
cudaError_t launch_axpy(const double *x, const double *k, double c, double *y, long long n, cudaStream_t s);
cudaError_t launch_rk4_update(double *f, const double *k1, const double *k2, const double *k3, const double *k4,
                              double dt, long long n, cudaStream_t s);
// Discrete weak-form functionals and scales for phi in {1, v_l, |v|^2}, added into out[2(d+2)].
cudaError_t launch_weak_moments(const double *a, const double *vnode, int N, int d, int M, const double *sig,
                                const double *wsig, const Angular &ang, double gamma, int fast_gamma, double Bconst,
                                double *out, cudaStream_t s);
// Diagnostics: mass/energy functionals of Q and Qplus and their L2 norms into out[6].
cudaError_t launch_moments(const double *Q, const double *Qplus, int d, int N, double S,
                           double *out, cudaStream_t s);

// Set the thread-local text returned by pg_boltz_last_error; returns code.
int record_error(int code, const char *msg);

}  // namespace pgb
