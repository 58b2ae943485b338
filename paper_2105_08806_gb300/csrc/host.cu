// Host-side internals shared by the plain and the batched plans: error state, device
// allocation with fault injection, and the quadrature / sphere / transform tables.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "host.cuh"

#define PG_API extern "C" __attribute__((visibility("default")))

namespace {
thread_local std::string g_last_error;
std::atomic<int> g_fail_alloc_countdown{0};
}  // namespace

namespace pgbh {

int set_error(int code, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_last_error = buf;
    return code;
}

int cuda_check(cudaError_t e, const char *what)
{
    if (e == cudaSuccess) return PG_OK;
    return set_error(PG_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

// Gauss-Legendre nodes and weights on [-1, 1] (Newton iteration on P_n).
void gauss_legendre(int n, std::vector<double> &x, std::vector<double> &w)
{
    x.assign(n, 0.0);
    w.assign(n, 0.0);
    for (int i = 0; i < (n + 1) / 2; ++i) {
        double z = std::cos(kPi * (i + 0.75) / (n + 0.5));
        double dp = 0.0;
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = z;
            for (int k = 2; k <= n; ++k) {
                double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
                p0 = p1;
                p1 = p2;
            }
            dp = n * (z * p1 - p0) / (z * z - 1.0);
            double dz = p1 / dp;
            z -= dz;
            if (std::fabs(dz) < 1e-16) break;
        }
        double p0 = 1.0, p1 = z;
        for (int k = 2; k <= n; ++k) {
            double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
            p0 = p1;
            p1 = p2;
        }
        dp = n * (z * p1 - p0) / (z * z - 1.0);
        x[i] = -z;
        x[n - 1 - i] = z;
        w[i] = w[n - 1 - i] = 2.0 / ((1.0 - z * z) * dp * dp);
    }
}


int grid_size(int N, double sigma)
{
    int n = (int)std::ceil(sigma * (2 * N + 1));
    return n + (n % 2);
}

double kernel_beta(int w, double sigma) { return 0.97 * kPi * (1.0 - 0.5 / sigma) * w; }

int width_for(double tol, double sigma)
{
    double per_w = 0.9 * std::sqrt(2.0 * (1.0 - 1.0 / sigma));
    int w = (int)std::ceil((-std::log10(tol) - 0.8) / per_w);
    return std::max(w, pgb::kMinWidth);
}

// Tap a of the kernel as a function of the offset y in [-1, 1]: t = (y + 1 + 2a - w)/w.
static long double kernel_tap(int w, double beta, int a, long double y)
{
    const long double t = (y + 1.0L + 2.0L * a - w) / w;
    const long double om = 1.0L - t * t;
    return om > 0.0L ? expl((long double)beta * (sqrtl(om) - 1.0L)) : 0.0L;
}

// Interpolate each tap at the P = kernel_poly_terms(w) Chebyshev points of [-1, 1] (coefficients
// of T_j by the discrete cosine sums, then expanded in powers of y through
// T_{j+1} = 2y T_j - T_{j-1}), all in long double; split into even and odd parts.
void kernel_poly(int w, double beta, double *c)
{
    const int P = pgb::kernel_poly_terms(w), NE = (P + 1) / 2, NO = P / 2;
    const long double pi = 3.141592653589793238462643383279502884L;
    std::vector<long double> g(P), cheb(P), mono(P), Tm(P), T0(P), T1(P);
    for (int a = 0; a < (w + 1) / 2; ++a) {
        for (int k = 0; k < P; ++k) g[k] = kernel_tap(w, beta, a, cosl(pi * (k + 0.5L) / P));
        for (int j = 0; j < P; ++j) {
            long double acc = 0.0L;
            for (int k = 0; k < P; ++k) acc += g[k] * cosl(pi * j * (k + 0.5L) / P);
            cheb[j] = acc * (j == 0 ? 1.0L : 2.0L) / P;
        }
        std::fill(mono.begin(), mono.end(), 0.0L);
        std::fill(T0.begin(), T0.end(), 0.0L);
        std::fill(T1.begin(), T1.end(), 0.0L);
        T0[0] = 1.0L;  // T_0
        if (P > 1) T1[1] = 1.0L;  // T_1
        for (int j = 0; j < P; ++j) {
            const std::vector<long double> &Tj = (j == 0) ? T0 : T1;
            for (int k = 0; k < P; ++k) mono[k] += cheb[j] * Tj[k];
            if (j >= 1) {  // T_{j+1} = 2 y T_j - T_{j-1} into Tm, then shift
                for (int k = 0; k < P; ++k) Tm[k] = (k > 0 ? 2.0L * T1[k - 1] : 0.0L) - T0[k];
                T0 = T1;
                T1 = Tm;
            }
        }
        for (int k = 0; k < NE; ++k) c[a * P + k] = (double)mono[2 * k];
        for (int k = 0; k < NO; ++k) c[a * P + NE + k] = (double)mono[2 * k + 1];
    }
}

// psi_hat(k) = int psi(x) cos(k x) dx with psi(x) = exp(beta (sqrt(1 - (x/alpha)^2) - 1)),
// |x| < alpha = w pi / n.  With x = alpha sin(theta) the integrand is smooth:
// alpha int_{-pi/2}^{pi/2} exp(beta (cos theta - 1)) cos(k alpha sin theta) cos theta dtheta.
std::vector<double> kernel_ft(int N, int w, double beta, int n)
{
    std::vector<double> gx, gw;
    gauss_legendre(256, gx, gw);
    const double alpha = w * kPi / n;
    std::vector<double> out(N + 1);
    for (int k = 0; k <= N; ++k) {
        double acc = 0.0;
        for (size_t t = 0; t < gx.size(); ++t) {
            double th = 0.5 * kPi * gx[t];
            acc += gw[t] * std::exp(beta * (std::cos(th) - 1.0)) * std::cos(k * alpha * std::sin(th)) *
                   std::cos(th);
        }
        out[k] = alpha * 0.5 * kPi * acc;
    }
    return out;
}

void sphere_points(int d, int M, int kind, std::vector<double> &pts, std::vector<double> &wts)
{
    pts.assign((size_t)M * d, 0.0);
    if (d == 2) {
        for (int m = 0; m < M; ++m) {
            double th = 2.0 * kPi * m / M;
            pts[2 * m] = std::cos(th);
            pts[2 * m + 1] = std::sin(th);
        }
        wts.assign(M, 2.0 * kPi / M);
        return;
    }
    const double golden = kPi * (3.0 - std::sqrt(5.0));
    if (kind == PG_SPHERE_FIBONACCI) {
        for (int m = 0; m < M; ++m) {
            double z = 1.0 - (2.0 * m + 1.0) / M;
            double rho = std::sqrt(1.0 - z * z);
            pts[3 * m] = rho * std::cos(m * golden);
            pts[3 * m + 1] = rho * std::sin(m * golden);
            pts[3 * m + 2] = z;
        }
    } else {
        const int h = M / 2;
        for (int m = 0; m < h; ++m) {
            double z = 1.0 - (2.0 * m + 1.0) / h;
            double rho = std::sqrt(1.0 - z * z);
            double x = rho * std::cos(m * golden), y = rho * std::sin(m * golden);
            pts[3 * m] = x;
            pts[3 * m + 1] = y;
            pts[3 * m + 2] = z;
            pts[3 * (m + h)] = -x;
            pts[3 * (m + h) + 1] = -y;
            pts[3 * (m + h) + 2] = -z;
        }
    }
    wts.assign(M, 4.0 * kPi / M);
}

double map_v(double phi, double S, int r)
{
    // xi = -cos(phi); r = 1: v = S xi / sqrt(1 - xi^2) = -S cot(phi); r = 0: v = S atanh(xi) = S ln tan(phi/2)
    if (r == 1) return -S * std::cos(phi) / std::sin(phi);
    return S * std::log(std::tan(0.5 * phi));
}

NodeTables node_tables(int N, double S, int r)
{
    NodeTables t;
    t.R.assign((size_t)N * (N + 1), 0.0);
    t.E.assign((size_t)(N + 1) * N, 0.0);
    t.scale_a.assign(N, 0.0);
    t.inv_mu2.assign(N, 0.0);
    t.v.assign(N, 0.0);
    const double wnode = kPi / (N + 1);
    for (int i = 0; i < N; ++i) {
        const double phi = kPi * (i + 1) / (N + 1);
        const double mu2 = ipow(std::sin(phi), 1 + r) / S;
        t.scale_a[i] = wnode * mu2;
        t.inv_mu2[i] = 1.0 / mu2;
        t.v[i] = map_v(phi, S, r);
        for (int k = 0; k <= N; ++k) {
            const double tk = std::cos(k * (kPi - phi)) / std::sqrt(k == 0 ? kPi : 0.5 * kPi);
            t.R[(size_t)i * (N + 1) + k] = tk;
            t.E[(size_t)k * N + i] = tk;
        }
    }
    return t;
}

std::vector<double> transform_matrix(int N, int n, int w, double beta)
{
    const int nf = n / 2 + 1;
    std::vector<double> ph = kernel_ft(N, w, beta, n);
    std::vector<double> D((size_t)(N + 1) * nf);
    for (int k = 0; k <= N; ++k) {
        const double ck = std::sqrt(k == 0 ? kPi : 0.5 * kPi);
        for (int g = 0; g < nf; ++g) {
            const long long kg = ((long long)k * g) % n;
            D[(size_t)k * nf + g] = (2.0 * kPi / n) * std::cos(2.0 * kPi * (double)kg / n) / (ck * ph[k]);
        }
    }
    return D;
}

pgb::Dims3 dims_of(int d, int a, int b, int c)
{
    pgb::Dims3 x;
    if (d == 2) {
        x.e[0] = 1;
        x.e[1] = b;
        x.e[2] = c;
    } else {
        x.e[0] = a;
        x.e[1] = b;
        x.e[2] = c;
    }
    return x;
}

int dev_alloc(pg_boltz_plan_t *p, void **ptr, size_t bytes)
{
    *ptr = nullptr;
    int c = g_fail_alloc_countdown.load();
    if (c > 0) {
        if (g_fail_alloc_countdown.fetch_sub(1) == 1)
            return set_error(PG_ERR_NOMEM, "device allocation of %zu bytes failed (injected)", bytes);
    }
    cudaError_t e = cudaMalloc(ptr, bytes < 16 ? 16 : bytes);
    if (e != cudaSuccess) {
        *ptr = nullptr;
        cudaGetLastError();
        return set_error(e == cudaErrorMemoryAllocation ? PG_ERR_NOMEM : PG_ERR_CUDA,
                         "cudaMalloc(%zu) failed: %s", bytes, cudaGetErrorString(e));
    }
    p->allocs.push_back(*ptr);
    p->device_bytes += bytes;
    return PG_OK;
}

int upload_bytes(pg_boltz_plan_t *p, void **dst, const void *src, size_t bytes)
{
    int rc = dev_alloc(p, dst, bytes);
    if (rc) return rc;
    cudaError_t e = cudaMemcpy(*dst, src, bytes, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return set_error(PG_ERR_CUDA, "upload failed: %s", cudaGetErrorString(e));
    return PG_OK;
}

void free_plan(pg_boltz_plan_t *p)
{
    if (!p) return;
    for (cudaEvent_t &e : p->ev)
        if (e) cudaEventDestroy(e);
    if (p->batch) pg_free_batch(p->batch);
    if (p->rk_exec) cudaGraphExecDestroy(p->rk_exec);
    if (p->rk_graph) cudaGraphDestroy(p->rk_graph);
    if (p->rk_cap_stream) cudaStreamDestroy(p->rk_cap_stream);
    for (void *q : p->allocs) cudaFree(q);
    p->allocs.clear();
    delete p;
}

}  // namespace pgbh

int pgb::record_error(int code, const char *msg) { return pgbh::set_error(code, "%s", msg); }

PG_API const char *pg_boltz_last_error(void) { return g_last_error.c_str(); }

PG_API void pg_boltz_debug_fail_alloc(int countdown) { g_fail_alloc_countdown.store(countdown > 0 ? countdown : 0); }
