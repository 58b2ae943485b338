// Inverse evaluation of a mapped-Chebyshev expansion at arbitrary velocities:
//   u_N(v) = sum_k u~_k prod_l T~_{k_l}(v_l),  T~_k(v) = mu(xi)^4 T_k(xi) / sqrt(c_k),  xi = xi(v)
// (Eq. fN_Expansion with the trial functions of Eq. 1DCheby).  Given the weak-form
// coefficients Q_k of the collision operator it returns Q_N(v), the trial-space function whose
// coefficients they are (the trial and test functions are biorthonormal), so errors against a
// closed-form Q can be measured on a grid of velocities without leaving the device.
//
// One thread per point.  The sum over the (N+1)^d coefficients is a nested Clenshaw
// recurrence, one level per axis: no table of T_k values, O((N+1)^d) FMAs per point, and
// every thread of a warp reads the same coefficient at the same time (a broadcast load).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>

#include "host.cuh"

#define PG_API extern "C" __attribute__((visibility("default")))

using namespace pgbh;

namespace {

constexpr double kSqrt2OverPi = 0.79788456080286535588;  // 1/sqrt(c_k), k >= 1
constexpr double kInvSqrtPi = 0.56418958354775628695;    // 1/sqrt(c_0)

// sum_{k_L..k_{D-1}} u[k_L, ..] prod_{l >= L} T_{k_l}(x_l) / sqrt(c_{k_l}): Clenshaw along axis L
// over the values of the inner sums.  sum_{k>=1} a_k T_k(x) = x b_1 - b_2 with
// b_k = a_k + 2 x b_{k+1} - b_{k+2}.
template <int L, int D>
__device__ double nested_clenshaw(const double *__restrict__ u, int N, const double *x)
{
    int stride = 1;
    for (int l = L + 1; l < D; ++l) stride *= N + 1;
    const double two_x = 2.0 * x[L];
    double b1 = 0.0, b2 = 0.0, a0 = 0.0;
    for (int k = N; k >= 0; --k) {
        double a;
        if constexpr (L == D - 1)
            a = __ldg(u + k);
        else
            a = nested_clenshaw<L + 1, D>(u + (size_t)k * stride, N, x);
        if (k == 0) {
            a0 = a;
        } else {
            const double t = fma(two_x, b1, a - b2);
            b2 = b1;
            b1 = t;
        }
    }
    return kSqrt2OverPi * fma(x[L], b1, -b2) + kInvSqrtPi * a0;
}

// xi(v) and mu(xi)^4 = (1 - xi^2)^(1+r) / S^2 (Eq. 1D_mu_function), with 1 - xi^2 in a form
// without cancellation: sech^2(v/S) for the logarithmic map xi = tanh(v/S), S^2/(S^2 + v^2) for
// the algebraic map xi = v / sqrt(S^2 + v^2).
__device__ void map_point(double v, double S, int r, double &xi, double &mu4)
{
    double om;
    if (r == 0) {
        const double t = v / S;
        xi = tanh(t);
        const double ch = cosh(t);
        om = 1.0 / (ch * ch);
        mu4 = om / (S * S);
    } else {
        const double h = hypot(S, v);
        xi = v / h;
        om = S / h;
        om *= om;
        mu4 = om * om / (S * S);
    }
}

template <int D>
__global__ void k_evaluate(int N, double S, int r, const double *__restrict__ u, long long npts,
                           const double *__restrict__ pts, double *__restrict__ out)
{
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < npts; p += stride) {
        double x[D];
        double w = 1.0;
        for (int l = 0; l < D; ++l) {
            double m4;
            map_point(pts[p * D + l], S, r, x[l], m4);
            w *= m4;
        }
        out[p] = w * nested_clenshaw<0, D>(u, N, x);
    }
}

}  // namespace

PG_API int pg_boltz_evaluate(pg_boltz_plan_t *p, const double *coef_dev, long long npts, const double *pts_dev,
                             double *out_dev)
{
    if (!p) return set_error(PG_ERR_ARG, "plan is NULL");
    if (p->batch) return set_error(PG_ERR_STATE, "evaluation is not available on batched plans");
    if (npts < 0) return set_error(PG_ERR_ARG, "npts must be >= 0");
    if (npts == 0) return PG_OK;
    if (!coef_dev || !pts_dev || !out_dev) return set_error(PG_ERR_ARG, "NULL device pointer");
    DeviceGuard guard(p->device);
    if (!guard.ok) return set_error(PG_ERR_CUDA, "cannot select the plan's device");
    const int threads = 256;
    const long long want = (npts + threads - 1) / threads;
    int sms = 152;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, p->device);
    const int blocks = (int)std::min<long long>(want, 8LL * sms);
    if (p->d == 2)
        k_evaluate<2><<<blocks, threads, 0, p->stream>>>(p->N, p->S, p->r, coef_dev, npts, pts_dev, out_dev);
    else
        k_evaluate<3><<<blocks, threads, 0, p->stream>>>(p->N, p->S, p->r, coef_dev, npts, pts_dev, out_dev);
    return cuda_check(cudaGetLastError(), "evaluation kernel");
}
