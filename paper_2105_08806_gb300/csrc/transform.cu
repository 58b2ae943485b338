// Small FP64 kernels around the spreading step:
//  - separable axis passes (reconstruction of f_N at the nodes, Section 4.2; the
//    cosine transform of the folded grid with the deconvolution folded into its
//    matrix, Eq. nufft; the forward Chebyshev transform of the loss, Eq. Qminus;
//    the projection of Eq. MultiD_spectral_coef),
//  - the loss sum over node pairs (Eq. Qminus, inner integral),
//  - the final pass that forms Q = Q+ - Q- (Section 4.2),
//  - mass / energy diagnostics from the identities of Section 3.3.
// All arrays are C-order three-axis arrays (2D arrays carry a leading axis of 1).
#include <cuda_runtime.h>

#include "pgb_internal.cuh"

namespace pgb {
namespace {

constexpr int kThreads = 256;

__device__ __forceinline__ long long stride_of(const Dims3 &d, int ax)
{
    return ax == 2 ? 1LL : (ax == 1 ? (long long)d.e[2] : (long long)d.e[1] * d.e[2]);
}

// The separable passes and the final combine split each output's dot product over kSplit lanes
// of a warp (lane g takes terms g, g + kSplit, ...) and add the partial sums by a butterfly of
// shuffles, in a fixed order: the outputs are few (thousands) and their dot products long
// (n/2 + 1 terms), so one thread per output left most SMs idle behind a serial chain of FMAs.
constexpr int kSplit = 8;

__device__ __forceinline__ double split_sum(double v)
{
#pragma unroll
    for (int off = kSplit / 2; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    return v;
}

__global__ void k_axis_pass(const double *__restrict__ in, Dims3 id, int ax,
                            const double *__restrict__ A, int m, double *__restrict__ out)
{
    Dims3 od = id;
    od.e[ax] = m;
    const long long total = (long long)od.e[0] * od.e[1] * od.e[2];
    const long long tlanes = total * kSplit;
    const int len = id.e[ax];
    const long long sax = stride_of(id, ax);
    const int lane = threadIdx.x & 31;
    // every lane of a warp runs the same iterations (the shuffles need the whole warp)
    for (long long tt = blockIdx.x * (long long)blockDim.x + threadIdx.x; tt - lane < tlanes;
         tt += (long long)gridDim.x * blockDim.x) {
        const long long o = tt / kSplit;
        const int g = (int)(tt % kSplit);
        double acc = 0.0;
        if (tt < tlanes) {
            int oc[3];
            oc[2] = (int)(o % od.e[2]);
            const long long t = o / od.e[2];
            oc[1] = (int)(t % od.e[1]);
            oc[0] = (int)(t / od.e[1]);
            const int k = oc[ax];
            oc[ax] = 0;
            const long long base = ((long long)oc[0] * id.e[1] + oc[1]) * id.e[2] + oc[2];
            const double *arow = A + (long long)k * len;
            for (int s = g; s < len; s += kSplit) acc = fma(arow[s], in[base + s * sax], acc);
        }
        acc = split_sum(acc);
        if (tt < tlanes && g == 0) out[o] = acc;
    }
}

__global__ void k_recon_last(const double *__restrict__ in, Dims3 id, const double *__restrict__ A,
                             int m, const double *__restrict__ scale, int d, double *__restrict__ a,
                             float *__restrict__ af)
{
    const long long total = (long long)id.e[0] * id.e[1] * m;
    const int len = id.e[2];
    for (long long o = blockIdx.x * (long long)blockDim.x + threadIdx.x; o < total;
         o += (long long)gridDim.x * blockDim.x) {
        const int o2 = (int)(o % m);
        const long long t = o / m;
        const int o1 = (int)(t % id.e[1]);
        const int o0 = (int)(t / id.e[1]);
        const double *src = in + ((long long)o0 * id.e[1] + o1) * len;
        const double *arow = A + (long long)o2 * len;
        double acc = 0.0;
        for (int s = 0; s < len; ++s) acc = fma(arow[s], src[s], acc);
        double sc = scale[o1] * scale[o2];
        if (d == 3) sc *= scale[o0];
        acc *= sc;
        a[o] = acc;
        if (af) af[o] = (float)acc;
    }
}

template <int BLOCK>
__device__ double block_sum(double v)
{
    __shared__ double warp_part[BLOCK / 32];
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
    if ((threadIdx.x & 31) == 0) warp_part[threadIdx.x >> 5] = v;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x < 32) {
        s = (threadIdx.x < BLOCK / 32) ? warp_part[threadIdx.x] : 0.0;
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) s += __shfl_down_sync(0xffffffffu, s, off);
    }
    __syncthreads();
    return s;  // valid in thread 0
}

constexpr int kLossThreads = 128;

// One block per outer node i:
//   Lsum_i = Bw sum_j a_j |v_i - v_j|^gamma,   h_i = a_i Lsum_i / mu_i^2      (Eq. Qminus)
//   ub_i   = |a_i| Bw sum_j |a_j| |v_i - v_j|^gamma prod_l mu^-2(|c_l| + rad)
// where c = (v_i + v_j)/2, rad = |v_i - v_j|/2: every post-collision point of the pair lies
// in the box |v'_l| <= |c_l| + rad and mu^-2 grows with |v|, so ub_i bounds the spreading
// strengths sum_{j,m} |q_ijm| (times Bconst, which Bw carries).  PT is the arithmetic of the
// pair terms: FP64, or FP32 for the FP32 path (node differences with the nodes' FP32 rounding
// added back); the loss sums are FP64 in the FP64 path and float pairs (two-sum, about 2^-44
// relative) over the FP32 coefficients in the FP32 path, the bound's 64-term partial sums FP32.
// b(cos theta) summed over the sphere set for the pair direction dvec = v_i - v_j (|dvec| = g):
// (1/Wsig) sum_m w_m b(dvec . sigma_m / g), cos theta = 0 when g = 0 (Eq. collision_form).
template <typename PT>
__device__ __forceinline__ PT angular_mean(const Angular &ang, const PT *dvec, PT g, int d, int M,
                                           const PT *__restrict__ sig, const PT *__restrict__ wsig, PT inv_wsig)
{
    const PT ginv = g > PT(0) ? PT(1) / g : PT(0);
    PT acc = PT(0);
    for (int m = 0; m < M; ++m) {
        PT c = PT(0);
        for (int l = 0; l < d; ++l) c += dvec[l] * sig[m * d + l];
        c *= ginv;
        PT b = PT(ang.c[ang.n - 1]);
        for (int t = ang.n - 2; t >= 0; --t) b = b * c + PT(ang.c[t]);
        acc += wsig[m] * b;
    }
    return acc * inv_wsig;
}

template <typename PT, int D>
__global__ void __launch_bounds__(kLossThreads) k_loss(const double *__restrict__ a,
                                                        const float *__restrict__ a32,
                                                        const PT *__restrict__ vnode,
                                                        const float *__restrict__ vnode_lo, int N, int M,
                                                        const PT *__restrict__ sig, const PT *__restrict__ wsig,
                                                        const Angular ang, double angmax, double Wsig,
                                                        double gamma, int fast_gamma, double Bw,
                                                        const double *__restrict__ inv_mu2, double S, int r,
                                                        double *__restrict__ h, double *__restrict__ ub,
                                                        unsigned long long *__restrict__ hist)
{
    __shared__ unsigned s_hist[kScreenBins];
    if (hist)
        for (int k = threadIdx.x; k < kScreenBins; k += blockDim.x) s_hist[k] = 0u;
    __syncthreads();
    constexpr int d = D;
    const int nnode = (d == 2) ? N * N : N * N * N;
    const int i = blockIdx.x;
    int idx[3] = {0, 0, 0};
    {
        int t = i;
        for (int l = d - 1; l >= 0; --l) {
            idx[l] = t % N;
            t /= N;
        }
    }
    PT vi[3], vil[3] = {PT(0), PT(0), PT(0)};
    for (int l = 0; l < 3; ++l) vi[l] = (l < d) ? vnode[idx[l]] : PT(0);
    if (vnode_lo)
        for (int l = 0; l < d; ++l) vil[l] = PT(vnode_lo[idx[l]]);
    const PT Sp = PT(S), invS = PT(1) / Sp, gam = PT(gamma);
    const double ai_w = fabs(a[i]) * Bw * angmax;  // pair bound = ai_w * |a_j| B_ij prod mu^-2
    const PT inv_wsig = PT(1.0 / Wsig);
    double acc = 0.0, bnd = 0.0;
    float as = 0.0f, ac = 0.0f;  // FP32 plans: the pair terms' sum as as + ac
    // every thread takes nodes j = threadIdx.x + k blockDim.x, whose axis indices (C order, base N
    // digits) advance by the step's digits with carries; the bound's FP32 partial sums run over 64
    // terms at most
    int jl[D], sl[D];
    {
        int t = threadIdx.x, u = blockDim.x;
#pragma unroll
        for (int l = D - 1; l >= 0; --l) {
            jl[l] = t % N;
            t /= N;
            sl[l] = u % N;
            u /= N;
        }
    }
    PT bp = PT(0);
    int nb = 0;
    for (int j = threadIdx.x; j < nnode; j += blockDim.x) {
        {
            PT g2 = PT(0), vj[3] = {PT(0), PT(0), PT(0)}, dv[3] = {PT(0), PT(0), PT(0)};
#pragma unroll
            for (int l = 0; l < d; ++l) {
                const int nj = jl[l];
                vj[l] = vnode[nj];
                dv[l] = vi[l] - vj[l];
                if (vnode_lo) dv[l] += vil[l] - PT(vnode_lo[nj]);  // FP32 nodes: their rounding, too
                g2 += dv[l] * dv[l];
            }
            const PT g = sqrt(g2);
            PT B;
            switch (fast_gamma) {
            case 0: B = PT(1); break;
            case 1: B = g; break;
            case 2: B = sqrt(g); break;
            default: B = (g2 > PT(0)) ? pow(g, gam) : PT(0); break;
            }
            PT aj;
            if (ang.n) {  // the pair term in PT, its sum in FP64
                aj = PT(a[j]);
                acc = fma(double(B * angular_mean<PT>(ang, dv, g, d, M, sig, wsig, inv_wsig)), a[j], acc);
            } else if constexpr (sizeof(PT) == 4) {
                // FP32: the FP32 coefficient the spreading uses, and the product's exact value
                // (FMA residual) summed as an unevaluated pair of floats (two-sum): no FP64
                // operation per pair, about 2^-44 relative
                aj = a32[j];
                const float pt = B * aj;
                const float pe = fmaf(B, aj, -pt);
                const float t = as + pt;
                const float bv = t - as;
                ac += ((as - (t - bv)) + (pt - bv)) + pe;
                as = t;
            } else {
                aj = PT(a[j]);
                acc = fma(double(B), a[j], acc);
            }
            if (aj != PT(0) && B != PT(0)) {
                PT mu = PT(1);
#pragma unroll
                for (int l = 0; l < d; ++l) {
                    const PT R = fabs(PT(0.5) * (vi[l] + vj[l])) + PT(0.5) * g;
                    mu *= (r == 1) ? (Sp * Sp + R * R) * invS : Sp * cosh(R * invS);
                }
                const PT u = fabs(aj) * B * mu;
                bp += u;
                if (hist) atomicAdd(&s_hist[screen_bin(ai_w * (double)u)], 1u);
            }
        }
        if (++nb == 64) {
            bnd += (double)bp;
            bp = PT(0);
            nb = 0;
        }
        int carry = 0;
#pragma unroll
        for (int l = D - 1; l >= 0; --l) {
            jl[l] += sl[l] + carry;
            carry = jl[l] >= N;
            if (carry) jl[l] -= N;
        }
    }
    bnd += (double)bp;
    acc += (double)as + (double)ac;
    const double tot = block_sum<kLossThreads>(acc);
    const double tb = block_sum<kLossThreads>(bnd);
    if (threadIdx.x == 0) {
        double sc = 1.0;
        for (int l = 0; l < d; ++l) sc *= inv_mu2[idx[l]];
        h[i] = a[i] * Bw * tot * sc;
        ub[i] = fabs(a[i]) * Bw * angmax * tb;
    }
    if (hist) {
        __syncthreads();
        for (int k = threadIdx.x; k < kScreenBins; k += blockDim.x)
            if (s_hist[k]) atomicAdd(hist + k, (unsigned long long)s_hist[k]);
    }
}

constexpr int kReduceThreads = 1024;

// B = (1 + 1e-5) sum_i ub_i in a fixed order (deterministic); the factor covers FP32 rounding
// of the pair terms and of the strengths in the FP32 spreading kernel.
__global__ void __launch_bounds__(kReduceThreads) k_bound_reduce(const double *__restrict__ ub, int n,
                                                                  const unsigned long long *__restrict__ hist,
                                                                  double eps, double *__restrict__ B,
                                                                  double *__restrict__ tau)
{
    double s = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) s += ub[i];
    const double tot = block_sum<kReduceThreads>(s);
    if (threadIdx.x == 0) {
        const double Bv = tot * (1.0 + 1e-5);
        *B = Bv;
        double t = 0.0;
        if (hist && Bv > 0.0) {
            double cum = 0.0;
            int k = 0;
            for (; k < kScreenBins - 1; ++k) {
                const double add = (double)hist[k] * ldexp(1.0, k + 1 - kScreenOffset);
                if (cum + add > eps * Bv) break;
                cum += add;
            }
            t = ldexp(1.0, k - kScreenOffset);
        }
        *tau = t;
    }
}

// First transform pass over the int64 fixed-point grid: out = (A . in) 2^-Eg.
__global__ void k_axis_pass_fixed(const unsigned long long *__restrict__ in, Dims3 id, int ax,
                                  const double *__restrict__ A, int m, const double *__restrict__ Bp,
                                  double scale, double *__restrict__ out)
{
    Dims3 od = id;
    od.e[ax] = m;
    const long long total = (long long)od.e[0] * od.e[1] * od.e[2];
    const long long tlanes = total * kSplit;
    const int len = id.e[ax];
    const long long sax = stride_of(id, ax);
    const double unit = ldexp(scale, -global_exponent(*Bp));
    const int lane = threadIdx.x & 31;
    for (long long tt = blockIdx.x * (long long)blockDim.x + threadIdx.x; tt - lane < tlanes;
         tt += (long long)gridDim.x * blockDim.x) {
        const long long o = tt / kSplit;
        const int g = (int)(tt % kSplit);
        double acc = 0.0;
        if (tt < tlanes) {
            int oc[3];
            oc[2] = (int)(o % od.e[2]);
            const long long t = o / od.e[2];
            oc[1] = (int)(t % od.e[1]);
            oc[0] = (int)(t / od.e[1]);
            const int k = oc[ax];
            oc[ax] = 0;
            const long long base = ((long long)oc[0] * id.e[1] + oc[1]) * id.e[2] + oc[2];
            const double *arow = A + (long long)k * len;
            for (int s = g; s < len; s += kSplit) acc = fma(arow[s], (double)(long long)in[base + s * sax], acc);
        }
        acc = split_sum(acc);
        if (tt < tlanes && g == 0) out[o] = acc * unit;
    }
}

__global__ void k_final(const double *__restrict__ G, Dims3 gd, const double *__restrict__ D,
                        const double *__restrict__ H, Dims3 hd, const double *__restrict__ E, int m,
                        double *__restrict__ Q, double *__restrict__ Qplus, double *__restrict__ Qcopy)
{
    const long long total = (long long)gd.e[0] * gd.e[1] * m;
    const long long tlanes = total * kSplit;
    const int lg = gd.e[2];
    const int lh = hd.e[2];
    const int lane = threadIdx.x & 31;
    for (long long tt = blockIdx.x * (long long)blockDim.x + threadIdx.x; tt - lane < tlanes;
         tt += (long long)gridDim.x * blockDim.x) {
        const long long o = tt / kSplit;
        const int g = (int)(tt % kSplit);
        double qp = 0.0, qm = 0.0;
        if (tt < tlanes) {
            const int o2 = (int)(o % m);
            const long long row = o / m;
            const double *gsrc = G + row * lg;
            const double *hsrc = H + row * lh;
            const double *drow = D + (long long)o2 * lg;
            const double *erow = E + (long long)o2 * lh;
            for (int s = g; s < lg; s += kSplit) qp = fma(drow[s], gsrc[s], qp);
            for (int s = g; s < lh; s += kSplit) qm = fma(erow[s], hsrc[s], qm);
        }
        qp = split_sum(qp);
        qm = split_sum(qm);
        if (tt < tlanes && g == 0) {
            Qplus[o] = qp;
            Q[o] = qp - qm;
            Qcopy[o] = qp - qm;
        }
    }
}

// 1 = a0 That_0 + a2 That_2 and v^2 = b0 That_0 + b2 That_2 per axis (Section 3.3 proof,
// algebraic map): a0 = sqrt(c0)/(2S), a2 = -sqrt(c2)/(2S), b0 = sqrt(c0) S/2, b2 = sqrt(c2) S/2.
__global__ void k_moments(const double *__restrict__ Q, const double *__restrict__ Qp, int d, int N,
                          double S, double *__restrict__ out)
{
    const int nm = (d == 2) ? (N + 1) * (N + 1) : (N + 1) * (N + 1) * (N + 1);
    double q2 = 0.0, p2 = 0.0;
    for (int k = threadIdx.x; k < nm; k += blockDim.x) {
        q2 += Q[k] * Q[k];
        p2 += Qp[k] * Qp[k];
    }
    const double sq2 = block_sum<kThreads>(q2);
    const double sp2 = block_sum<kThreads>(p2);
    if (threadIdx.x == 0) {
        const double pi = 3.14159265358979323846;
        const double one[2] = {sqrt(pi) / (2.0 * S), -sqrt(pi / 2.0) / (2.0 * S)};
        const double vsq[2] = {sqrt(pi) * S / 2.0, sqrt(pi / 2.0) * S / 2.0};
        double mq = 0.0, eq = 0.0, mp = 0.0, ep = 0.0;
        const int ncorner = 1 << d;
        for (int c = 0; c < ncorner && N >= 2; ++c) {
            int idx = 0;
            double mass = 1.0, energy = 0.0;
            for (int l = 0; l < d; ++l) {
                const int bit = (c >> (d - 1 - l)) & 1;
                idx = idx * (N + 1) + 2 * bit;
                mass *= one[bit];
            }
            for (int l = 0; l < d; ++l) {
                double term = 1.0;
                for (int m2 = 0; m2 < d; ++m2) {
                    const int bit = (c >> (d - 1 - m2)) & 1;
                    term *= (m2 == l) ? vsq[bit] : one[bit];
                }
                energy += term;
            }
            mq += mass * Q[idx];
            eq += energy * Q[idx];
            mp += mass * Qp[idx];
            ep += energy * Qp[idx];
        }
        out[0] = mq;
        out[1] = eq;
        out[2] = mp;
        out[3] = ep;
        out[4] = sqrt(sq2);
        out[5] = sqrt(sp2);
    }
}

constexpr int kWeakThreads = 256;

// Discrete weak form of the collision operator (Eq. weak with the quadrature of Section 4):
//   out[2t]   = sum_{i,j,m} qbar [phi_t(v') - phi_t(v_i)],
//   out[2t+1] = sum_{i,j,m} qbar (|phi_t(v')| + |phi_t(v_i)|),
// qbar = a_i a_j w_m Bconst |v_i - v_j|^gamma b(cos theta_ijm), for phi_t in {1, v_1, .., v_d, |v|^2}
// (t = 0..d+1), cos theta_ijm = (v_i - v_j) . sigma_m / |v_i - v_j| (0 when i = j).
// One thread per node pair, FP64 throughout; block sums are added to out with atomics.
__global__ void __launch_bounds__(kWeakThreads) k_weak_moments(const double *__restrict__ a,
                                                               const double *__restrict__ vnode, int N, int d,
                                                               int M, const double *__restrict__ sig,
                                                               const double *__restrict__ wsig, const Angular ang,
                                                               double gamma, int fast_gamma, double Bconst,
                                                               double *__restrict__ out)
{
    const int nnode = (d == 2) ? N * N : N * N * N;
    const long long npairs = (long long)nnode * nnode;
    double acc[10];
    for (int t = 0; t < 10; ++t) acc[t] = 0.0;
    for (long long pr = blockIdx.x * (long long)blockDim.x + threadIdx.x; pr < npairs;
         pr += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(pr / nnode), j = (int)(pr - (long long)i * nnode);
        const double aij = a[i] * a[j];
        if (aij == 0.0) continue;
        double vi[3] = {0, 0, 0}, vj[3] = {0, 0, 0}, g2 = 0.0;
        int ii = i, jj = j;
        for (int l = d - 1; l >= 0; --l) {
            vi[l] = vnode[ii % N];
            vj[l] = vnode[jj % N];
            ii /= N;
            jj /= N;
            g2 += (vi[l] - vj[l]) * (vi[l] - vj[l]);
        }
        const double g = sqrt(g2);
        double B;
        switch (fast_gamma) {
        case 0: B = Bconst; break;
        case 1: B = Bconst * g; break;
        case 2: B = Bconst * sqrt(g); break;
        default: B = (g2 > 0.0) ? Bconst * pow(g, gamma) : 0.0; break;
        }
        double vi2 = 0.0;
        for (int l = 0; l < d; ++l) vi2 += vi[l] * vi[l];
        const double ginv = g > 0.0 ? 1.0 / g : 0.0;
        for (int m = 0; m < M; ++m) {
            double bang = 1.0;
            if (ang.n) {
                double c = 0.0;
                for (int l = 0; l < d; ++l) c += (vi[l] - vj[l]) * sig[m * d + l];
                c *= ginv;
                bang = ang.c[ang.n - 1];
                for (int t = ang.n - 2; t >= 0; --t) bang = bang * c + ang.c[t];
            }
            const double q = aij * B * wsig[m] * bang;
            double vp2 = 0.0;
            for (int l = 0; l < d; ++l) {
                const double vp = 0.5 * (vi[l] + vj[l]) + 0.5 * g * sig[m * d + l];
                vp2 += vp * vp;
                acc[2 + 2 * l] += q * (vp - vi[l]);
                acc[3 + 2 * l] += fabs(q) * (fabs(vp) + fabs(vi[l]));
            }
            acc[1] += 2.0 * fabs(q);  // phi = 1: the difference is exactly zero
            acc[2 + 2 * d] += q * (vp2 - vi2);
            acc[3 + 2 * d] += fabs(q) * (vp2 + vi2);
        }
    }
    __shared__ double part[kWeakThreads / 32][10];
    for (int t = 0; t < 2 * (d + 2); ++t) {
        double v = acc[t];
        for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
        if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5][t] = v;
    }
    __syncthreads();
    if (threadIdx.x < 2 * (d + 2)) {
        double v = 0.0;
        for (int w = 0; w < kWeakThreads / 32; ++w) v += part[w][threadIdx.x];
        atomicAdd(out + threadIdx.x, v);
    }
}

// y = x + c k (an RK stage argument).
__global__ void k_axpy(const double *__restrict__ x, const double *__restrict__ k, double c, double *__restrict__ y,
                       long long n)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        y[i] = fma(c, k[i], x[i]);
}

// f += dt/6 (k1 + 2 k2 + 2 k3 + k4) (the classical fourth-order Runge-Kutta update).
__global__ void k_rk4_update(double *__restrict__ f, const double *__restrict__ k1, const double *__restrict__ k2,
                             const double *__restrict__ k3, const double *__restrict__ k4, double dt, long long n)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        f[i] += (dt / 6.0) * (k1[i] + 2.0 * (k2[i] + k3[i]) + k4[i]);
}

int grid_for(long long total)
{
    long long b = (total + kThreads - 1) / kThreads;
    if (b < 1) b = 1;
    if (b > 4096) b = 4096;
    return (int)b;
}

}  // namespace

cudaError_t launch_axis_pass(const double *in, Dims3 in_dims, int ax, const double *A, int m,
                             double *out, cudaStream_t s)
{
    Dims3 od = in_dims;
    od.e[ax] = m;
    k_axis_pass<<<grid_for((long long)od.e[0] * od.e[1] * od.e[2] * kSplit), kThreads, 0, s>>>(in, in_dims,
                                                                                              ax, A, m, out);
    return cudaGetLastError();
}

cudaError_t launch_recon_last(const double *in, Dims3 in_dims, const double *A, int m,
                              const double *scale, int d, double *a, float *af, cudaStream_t s)
{
    k_recon_last<<<grid_for((long long)in_dims.e[0] * in_dims.e[1] * m), kThreads, 0, s>>>(
        in, in_dims, A, m, scale, d, a, af);
    return cudaGetLastError();
}

cudaError_t launch_loss(const double *a, const float *a32, const double *vnode, const float *vnode32,
                        const float *vnode32_lo, int N,
                        int d, int M,
                        const double *sig, const double *wsig, const float *sig32, const float *wsig32,
                        const Angular &ang, double angmax, double Wsig, double gamma,
                        int fast_gamma, double Bw, const double *inv_mu2, double S, int r, double *h,
                        double *ub, unsigned long long *hist, cudaStream_t s)
{
    const int nnode = (d == 2) ? N * N : N * N * N;
    if (vnode32 && d == 2)
        k_loss<float, 2><<<nnode, kLossThreads, 0, s>>>(a, a32, vnode32, vnode32_lo, N, M, sig32, wsig32, ang, angmax,
                                                        Wsig, gamma, fast_gamma, Bw, inv_mu2, S, r, h, ub, hist);
    else if (vnode32)
        k_loss<float, 3><<<nnode, kLossThreads, 0, s>>>(a, a32, vnode32, vnode32_lo, N, M, sig32, wsig32, ang, angmax,
                                                        Wsig, gamma, fast_gamma, Bw, inv_mu2, S, r, h, ub, hist);
    else if (d == 2)
        k_loss<double, 2><<<nnode, kLossThreads, 0, s>>>(a, nullptr, vnode, nullptr, N, M, sig, wsig, ang, angmax,
                                                         Wsig, gamma, fast_gamma, Bw, inv_mu2, S, r, h, ub, hist);
    else
        k_loss<double, 3><<<nnode, kLossThreads, 0, s>>>(a, nullptr, vnode, nullptr, N, M, sig, wsig, ang, angmax,
                                                         Wsig, gamma, fast_gamma, Bw, inv_mu2, S, r, h, ub, hist);
    return cudaGetLastError();
}

cudaError_t launch_bound_reduce(const double *ub, int n, const unsigned long long *hist, double eps, double *B,
                                double *tau, cudaStream_t s)
{
    k_bound_reduce<<<1, kReduceThreads, 0, s>>>(ub, n, hist, eps, B, tau);
    return cudaGetLastError();
}

cudaError_t launch_axis_pass_fixed(const unsigned long long *in, Dims3 in_dims, int ax, const double *A,
                                   int m, const double *B, double scale, double *out, cudaStream_t s)
{
    Dims3 od = in_dims;
    od.e[ax] = m;
    k_axis_pass_fixed<<<grid_for((long long)od.e[0] * od.e[1] * od.e[2] * kSplit), kThreads, 0, s>>>(
        in, in_dims, ax, A, m, B, scale, out);
    return cudaGetLastError();
}

cudaError_t launch_final(const double *G, Dims3 g_dims, const double *D, const double *H,
                         Dims3 h_dims, const double *E, int m, double *Q, double *Qplus,
                         double *Qcopy, cudaStream_t s)
{
    k_final<<<grid_for((long long)g_dims.e[0] * g_dims.e[1] * m * kSplit), kThreads, 0, s>>>(G, g_dims, D, H, h_dims,
                                                                                            E, m, Q, Qplus, Qcopy);
    return cudaGetLastError();
}

cudaError_t launch_axpy(const double *x, const double *k, double c, double *y, long long n, cudaStream_t s)
{
    k_axpy<<<grid_for(n), kThreads, 0, s>>>(x, k, c, y, n);
    return cudaGetLastError();
}

cudaError_t launch_rk4_update(double *f, const double *k1, const double *k2, const double *k3, const double *k4,
                              double dt, long long n, cudaStream_t s)
{
    k_rk4_update<<<grid_for(n), kThreads, 0, s>>>(f, k1, k2, k3, k4, dt, n);
    return cudaGetLastError();
}

cudaError_t launch_weak_moments(const double *a, const double *vnode, int N, int d, int M, const double *sig,
                                const double *wsig, const Angular &ang, double gamma, int fast_gamma, double Bconst,
                                double *out, cudaStream_t s)
{
    k_weak_moments<<<4 * 152, kWeakThreads, 0, s>>>(a, vnode, N, d, M, sig, wsig, ang, gamma, fast_gamma, Bconst,
                                                    out);
    return cudaGetLastError();
}

cudaError_t launch_moments(const double *Q, const double *Qplus, int d, int N, double S,
                           double *out, cudaStream_t s)
{
    k_moments<<<1, kThreads, 0, s>>>(Q, Qplus, d, N, S, out);
    return cudaGetLastError();
}

}  // namespace pgb
