// Host-side internals shared by the plain and the batched plans (not part of the ABI):
// error state, device guard, the plan record, device allocation, and the quadrature,
// sphere-set and transform tables of Sections 4.1-4.2.
#pragma once

#include <cuda_runtime.h>

#include <cstddef>
#include <vector>

#include "pg_boltz.h"
#include "pgb_internal.cuh"

namespace pgbh {

constexpr double kPi = 3.14159265358979323846;

// Record a formatted error for pg_boltz_last_error; returns code.
int set_error(int code, const char *fmt, ...);
// PG_OK for cudaSuccess, else PG_ERR_CUDA with "what: <cuda error>".
int cuda_check(cudaError_t e, const char *what);

// Make `dev` current for the lifetime of the guard and restore the caller's device.
struct DeviceGuard {
    int prev = -1;
    bool ok = true;
    explicit DeviceGuard(int dev)
    {
        if (cudaGetDevice(&prev) != cudaSuccess) {
            ok = false;
            return;
        }
        if (prev != dev && cudaSetDevice(dev) != cudaSuccess) ok = false;
    }
    ~DeviceGuard()
    {
        int cur = -1;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

inline double ipow(double x, int k)
{
    double r = 1.0;
    for (int i = 0; i < k; ++i) r *= x;
    return r;
}

// Gauss-Legendre nodes and weights on [-1, 1].
void gauss_legendre(int n, std::vector<double> &x, std::vector<double> &w);
// Spreading-kernel width for precision tol at oversampling sigma, and its shape parameter.
int width_for(double tol, double sigma);
double kernel_beta(int w, double sigma);
// Even periodic grid size n >= sigma (2N + 1).
int grid_size(int N, double sigma);
// Piecewise polynomial form of the kernel for the FP64 spreading kernels: ceil(w/2) blocks of
// kernel_poly_terms(w) coefficients (layout of SpreadArgs::kpoly).
void kernel_poly(int w, double beta, double *c);
// psi_hat(k), k = 0..N, of the exponential-of-semicircle kernel of width w on a grid of n cells.
std::vector<double> kernel_ft(int N, int w, double beta, int n);
// Sphere quadrature (points M x d, weights M), Section 4.1.
void sphere_points(int d, int M, int kind, std::vector<double> &pts, std::vector<double> &wts);
// v(xi) at xi = -cos(phi) for the map with tail parameter r.
double map_v(double phi, double S, int r);

// Interior-node tables of one axis (Section 4.2, M_v = N + 2): R[i][k] = T_k(xi_i)/sqrt(c_k)
// (N x (N+1)), E = R^T, scale_a[i] = (pi/(N+1)) mu(xi_i)^2, inv_mu2[i] = 1/mu(xi_i)^2, v[i] = v(xi_i).
struct NodeTables {
    std::vector<double> R, E, scale_a, inv_mu2, v;
};
NodeTables node_tables(int N, double S, int r);
// Cosine transform with deconvolution: D[k][g] = (2 pi/n) cos(2 pi k g/n) / (sqrt(c_k) psi_hat(k)),
// (N+1) x (n/2+1).
std::vector<double> transform_matrix(int N, int n, int w, double beta);

pgb::Dims3 dims_of(int d, int a, int b, int c);

}  // namespace pgbh

struct BatchState;

// Everything a plan owns.  Plain plans use the fields below; batched plans keep their
// state in `batch` (see batched.cu).
struct pg_boltz_plan_s {
    pg_boltz_info_t info{};
    int device = 0;
    cudaStream_t stream = nullptr;
    int d = 2, N = 2, M = 2, r = 1, prec = PG_PREC_FP64, Mp = 0;
    double S = 1.0, gamma = 0.0, tol = 1e-6, sigma_up = 2.0;
    int n = 0, nf = 0, w = 0;
    double beta = 0.0;
    int nnode = 0;
    long long npairs = 0;
    int fast_gamma = 0;
    double Bconst = 0.0, Wsig = 0.0;
    int nslab = 1, rows_per_slab = 0, spread_blocks = 0, spread_threads = 256;
    size_t spread_smem = 0;
    size_t device_bytes = 0;
    std::vector<void *> allocs;
    std::vector<double> proj_v;  // host copy of projection node velocities
    bool have_q = false;
    int last_launches = 0;
    pgb::SpreadArgs sargs{};   // spreading-kernel arguments (fixed at plan time)
    pgb::Angular ang{};        // angular factor b(cos theta) of the collision kernel (n = 0: VHS)
    double angmax = 1.0;       // bound of the even part of b on [-1, 1]
    // optional per-stage timing: events recorded on the plan's stream around the stages
    bool timing = false;
    cudaEvent_t ev[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
    bool ev_recorded = false;

    // device tables
    double *R = nullptr;       // N x (N+1): T_k(xi_i)/sqrt(c_k), interior nodes
    double *E = nullptr;       // (N+1) x N: transpose of R
    double *Dm = nullptr;      // (N+1) x nf: cosine transform + deconvolution
    double *Pm = nullptr;      // (N+1) x Mp: projection
    double *scale_a = nullptr; // N: (pi/(N+1)) mu_i^2
    double *inv_mu2 = nullptr; // N: 1/mu_i^2
    double *v64 = nullptr;     // N node velocities
    float *v32 = nullptr;
    float *v32lo = nullptr;  // v - (double)v32: the FP32 nodes' rounding
    double grid_scale_corr = 1.0;  // FP32 plans: exact / FP32 constant factors of the strengths
    int queued = 0;                // FP32 one-slab plans: point queues beside the tile (SpreadArgs::queued)
    double *sig64 = nullptr, *wsig64 = nullptr;  // M x d, M
    float *sig32 = nullptr, *wsig32 = nullptr;
    // workspace
    double *tA = nullptr, *tB = nullptr, *tC = nullptr, *tD = nullptr;
    double *a64 = nullptr;
    float *a32 = nullptr;
    double *h = nullptr, *Qplus = nullptr, *Qlast = nullptr, *mom = nullptr;
    int *carry = nullptr;      // FP32 spreading: per-block carry counters
    double *kpoly = nullptr;   // FP64 spreading: the kernel polynomial (kPolyCoefF64 doubles)
    double *ub = nullptr;      // N^d per-node strength bounds
    double *bound = nullptr;   // scalar B >= sum_p |q_p| (follows the grid in one allocation)
    unsigned long long *grid = nullptr;  // folded grid, int64 fixed point
    double *tau = nullptr;     // scalar screening threshold (follows the bound)
    unsigned long long *hist = nullptr;  // screening histogram (follows tau)
    double screen_eps = 0.0;   // skipped strength budget relative to B (0: no screening)
    // RK4 time stepping: stage slopes k1..k4 and the stage argument, (N+1)^d each
    double *rk = nullptr;
    cudaStream_t rk_cap_stream = nullptr;
    cudaGraph_t rk_graph = nullptr;
    cudaGraphExec_t rk_exec = nullptr;
    double *rk_f = nullptr;
    double rk_dt = 0.0;
    BatchState *batch = nullptr;  // non-null for batched plans
};

namespace pgbh {

// cudaMalloc tracked by the plan (freed by free_plan); honours pg_boltz_debug_fail_alloc.
int dev_alloc(pg_boltz_plan_t *p, void **ptr, size_t bytes);
int upload_bytes(pg_boltz_plan_t *p, void **dst, const void *src, size_t bytes);
template <typename T>
int upload(pg_boltz_plan_t *p, T **dst, const std::vector<T> &src)
{
    return upload_bytes(p, reinterpret_cast<void **>(dst), src.data(), src.size() * sizeof(T));
}
void free_plan(pg_boltz_plan_t *p);

}  // namespace pgbh

// Release a batched plan's state (batched.cu).
void pg_free_batch(BatchState *b);
// Per-call timing of batched plans (batched.cu); ms_out[2] receives the whole call.
int pg_batched_timing(pg_boltz_plan_t *p, int enable);
int pg_batched_elapsed(pg_boltz_plan_t *p, double *ms_out);
