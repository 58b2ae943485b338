// Host side of the collision-operator library: plan construction (quadrature
// nodes, sphere sets, transform matrices, spreading-kernel parameters), the
// C ABI entry points and the launch sequence of one evaluation.
//
// Quadrature (Section 4.1-4.2): M_v = N + 2 Chebyshev-Gauss-Lobatto nodes per
// axis, xi_i = -cos(pi i/(N+1)), i = 0..N+1, weight pi/(N+1) (halved at the ends).
// The end nodes map to v = -inf, +inf where f_N = mu^4 P vanishes, so only the N
// interior nodes i = 1..N carry weight.  With phi_i = pi i/(N+1):
//   T_k(xi_i) = cos(k (pi - phi_i)),  1 - xi_i^2 = sin^2 phi_i,
//   mu(xi_i)^2 = sin(phi_i)^(1+r) / S                       (Eq. 1D_mu_function)
//   v_i = -S cot(phi_i)            (r = 1, Eq. algebraic)
//   v_i =  S ln tan(phi_i / 2)     (r = 0, Eq. logarithmic)
// a_i = W_i g_i = prod_l (pi/(N+1)) mu(xi_{i_l})^2 P_i with P_i = sum_k f~_k T_k(xi_i)/sqrt(c_k).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "host.cuh"

#define PG_API extern "C" __attribute__((visibility("default")))

using namespace pgbh;

namespace {

int build_plan(pg_boltz_plan_t *p, const pg_boltz_opts_t &o)
{
    const int d = p->d, N = p->N, M = p->M;
    p->nnode = (d == 2) ? N * N : N * N * N;
    p->npairs = pgb::unordered_pairs(p->nnode);
    p->fast_gamma = (p->gamma == 0.0) ? 0 : (p->gamma == 1.0) ? 1 : (p->gamma == 0.5) ? 2 : 3;
    p->Bconst = 1.0 / (d == 2 ? 2.0 * kPi : 4.0 * kPi);
    p->ang.n = o.angular_terms;
    for (int t = 0; t < o.angular_terms; ++t) p->ang.c[t] = o.angular_coef[t];
    p->angmax = 1.0;
    if (p->ang.n) {
        p->angmax = 0.0;
        for (int t = 0; t < p->ang.n; t += 2) p->angmax += std::fabs(p->ang.c[t]);
    }

    // ---- transform / spreading parameters
    p->sigma_up = (o.upsampfac > 0.0) ? o.upsampfac : 2.0;
    p->n = grid_size(N, p->sigma_up);
    p->nf = p->n / 2 + 1;
    p->w = width_for(p->tol, p->sigma_up);
    const int wmax = (p->prec == PG_PREC_FP32) ? pgb::kMaxWidthF32 : pgb::kMaxWidthF64;
    if (p->w > wmax) {
        if (p->prec == PG_PREC_FP32) p->w = wmax;  // FP32 spreading cannot resolve more anyway
        else return set_error(PG_ERR_ARG, "tol %g needs kernel width %d > %d", p->tol, p->w, wmax);
    }
    p->beta = kernel_beta(p->w, p->sigma_up);
    p->Mp = (o.proj_nodes > 0) ? o.proj_nodes : 4 * (N + 1);

    // ---- node tables and the cosine transform with deconvolution
    NodeTables nt = node_tables(N, p->S, p->r);
    std::vector<float> vf(nt.v.begin(), nt.v.end()), vflo(nt.v.size());
    for (size_t k = 0; k < vflo.size(); ++k) vflo[k] = (float)(nt.v[k] - (double)vf[k]);
    std::vector<double> D = transform_matrix(N, p->n, p->w, p->beta);
    // ---- projection (Chebyshev-Gauss): P[k][p] = (pi/Mp) mu_p^-4 T_k(xi_p) / sqrt(c_k)
    const int Mp = p->Mp;
    std::vector<double> P((size_t)(N + 1) * Mp);
    p->proj_v.assign(Mp, 0.0);
    for (int q = 0; q < Mp; ++q) {
        const double phi = (2.0 * q + 1.0) * kPi / (2.0 * Mp);
        const double mu_m4 = p->S * p->S / ipow(std::sin(phi), 2 * (1 + p->r));
        p->proj_v[q] = map_v(phi, p->S, p->r);
        for (int k = 0; k <= N; ++k)
            P[(size_t)k * Mp + q] = (kPi / Mp) * mu_m4 * std::cos(k * (kPi - phi)) / std::sqrt(k == 0 ? kPi : 0.5 * kPi);
    }
    // ---- sphere set
    std::vector<double> sp, sw;
    sphere_points(d, M, p->info.sphere, sp, sw);
    p->Wsig = 0.0;
    for (double x : sw) p->Wsig += x;
    std::vector<float> spf(sp.begin(), sp.end()), swf(sw.begin(), sw.end());

    int rc;
    if ((rc = upload(p, &p->R, nt.R)) || (rc = upload(p, &p->E, nt.E)) || (rc = upload(p, &p->Dm, D)) ||
        (rc = upload(p, &p->Pm, P)) || (rc = upload(p, &p->scale_a, nt.scale_a)) ||
        (rc = upload(p, &p->inv_mu2, nt.inv_mu2)) || (rc = upload(p, &p->v64, nt.v)) ||
        (rc = upload(p, &p->v32, vf)) || (rc = upload(p, &p->v32lo, vflo)) || (rc = upload(p, &p->sig64, sp)) ||
        (rc = upload(p, &p->wsig64, sw)) || (rc = upload(p, &p->sig32, spf)) || (rc = upload(p, &p->wsig32, swf)))
        return rc;

    // ---- workspace
    const long long modes = (long long)ipow(N + 1, d);
    const long long nfd1 = (long long)ipow(p->nf, d - 1);
    const long long mpd1 = (long long)ipow(Mp, d - 1);
    const long long big = std::max({modes, (long long)(N + 1) * nfd1, (long long)(N + 1) * mpd1});
    const long long grid_cells = nfd1 * p->nf;
    if ((rc = dev_alloc(p, (void **)&p->tA, big * 8)) || (rc = dev_alloc(p, (void **)&p->tB, big * 8)) ||
        (rc = dev_alloc(p, (void **)&p->tC, modes * 8)) || (rc = dev_alloc(p, (void **)&p->tD, modes * 8)) ||
        (rc = dev_alloc(p, (void **)&p->a64, (size_t)p->nnode * 8)) ||
        (rc = dev_alloc(p, (void **)&p->a32, (size_t)p->nnode * 4)) ||
        (rc = dev_alloc(p, (void **)&p->h, (size_t)p->nnode * 8)) ||
        (rc = dev_alloc(p, (void **)&p->grid, grid_cells * 8 + 16 + pgb::kScreenBins * 8)) ||
        (rc = dev_alloc(p, (void **)&p->ub, (size_t)p->nnode * 8)) ||
        (rc = dev_alloc(p, (void **)&p->Qplus, modes * 8)) || (rc = dev_alloc(p, (void **)&p->Qlast, modes * 8)) ||
        (rc = dev_alloc(p, (void **)&p->rk, 5 * modes * 8)) ||
        (rc = dev_alloc(p, (void **)&p->mom, 16 * 8)))
        return rc;
    // one allocation: [grid | B | tau | screening histogram], cleared by one memset per call
    p->bound = reinterpret_cast<double *>(p->grid + grid_cells);
    p->tau = p->bound + 1;
    p->hist = reinterpret_cast<unsigned long long *>(p->tau + 1);

    // ---- spreading launch shape
    cudaDeviceProp prop;
    cudaError_t e = cudaGetDeviceProperties(&prop, p->device);
    if (e != cudaSuccess) return set_error(PG_ERR_CUDA, "cudaGetDeviceProperties: %s", cudaGetErrorString(e));
    const size_t elem = (p->prec == PG_PREC_FP32) ? 4 : 12;  // 32-bit words per cell: FP32 one, FP64 three
    // block tiles: rows of (nf^(d-2) x ncol) cells, the last axis padded with unfolded columns
    const int cpad = pgb::tile_col_pad(p->w), ncol = p->nf + 2 * cpad;
    const size_t plane = (size_t)ipow(p->nf, d - 2) * ncol;
    const bool f32 = (p->prec == PG_PREC_FP32);
    // leave room for the kernels' static shared memory (FP64: the kernel polynomial)
    // (and 16 bytes for rounding the tile up to 16 bytes)
    const size_t max_smem = prop.sharedMemPerBlockOptin - 1024 - 16 - (f32 ? 0 : sizeof(double) * pgb::kPolyCoefF64);
    const int max_threads = f32 ? pgb::kMaxThreadsF32 : pgb::max_threads_f64(d);
    int rows_fit = (int)std::min<size_t>(p->nf, max_smem / (plane * elem));
    size_t qbytes = 0;
    if (rows_fit < p->nf) {
        // slabbed grid: the warps' point queues (one block per SM, max_threads threads unless
        // set) share the block's shared memory with the slab
        const int thr = (o.spread_threads > 0) ? o.spread_threads : max_threads;
        qbytes = pgb::spread_queue_bytes(thr, d, f32);
        rows_fit = (max_smem > qbytes) ? (int)std::min<size_t>(p->nf, (max_smem - qbytes) / (plane * elem)) : 0;
    }
    if (rows_fit < 1) return set_error(PG_ERR_ARG, "folded grid plane of %zu cells does not fit shared memory", plane);
    p->nslab = (p->nf + rows_fit - 1) / rows_fit;
    p->rows_per_slab = (p->nf + p->nslab - 1) / p->nslab;
    p->nslab = (p->nf + p->rows_per_slab - 1) / p->rows_per_slab;  // no empty trailing slab
    p->spread_smem = pgb::tile_bytes((size_t)p->rows_per_slab * plane, f32) + (p->nslab > 1 ? qbytes : 0);
    int per_sm = (int)(prop.sharedMemPerMultiprocessor / (p->spread_smem + 1024 + prop.reservedSharedMemPerBlock));
    per_sm = std::max(per_sm, 1);
    if (o.spread_threads > 0) {
        p->spread_threads = o.spread_threads;
    } else if (f32) {
        // FP32: one block of 1024 threads per SM (measured fastest; more, smaller blocks
        // multiply the tile clears and flushes)
        p->spread_threads = max_threads;
        per_sm = 1;
    } else {
        // about 1024 resident threads per SM
        int t = (1024 / per_sm) / 32 * 32;
        p->spread_threads = std::max(128, std::min(max_threads, t));
    }
    if (p->nslab > 1 && o.spread_threads <= 0) p->spread_threads = max_threads;  // the queues were sized for it
    if (p->spread_threads % 32 || p->spread_threads > max_threads)
        return set_error(PG_ERR_ARG, "spread_threads must be a multiple of 32 and <= %d", max_threads);
    if (p->nslab > 1 && pgb::spread_queue_bytes(p->spread_threads, d, f32) > qbytes)
        return set_error(PG_ERR_STATE, "internal: point queues larger than reserved");
    // FP32 one-slab grids: the warps also queue their points that add something and spread full
    // queues (every lane busy), when the queues fit beside the tile
    p->queued = 0;
    if (f32 && p->nslab == 1) {
        const size_t qq = pgb::spread_queue_bytes(p->spread_threads, d, true);
        if (p->spread_smem + qq <= max_smem) {
            p->queued = 1;
            p->spread_smem += qq;
        }
    }
    per_sm = std::min(per_sm, prop.maxThreadsPerMultiProcessor / p->spread_threads);
    if (o.spread_blocks_per_sm > 0) per_sm = std::min(per_sm, o.spread_blocks_per_sm);
    per_sm = std::max(per_sm, 1);
    long long blocks = (long long)prop.multiProcessorCount * per_sm;
    blocks = std::max<long long>(blocks / p->nslab, 1) * p->nslab;
    const long long need = ((p->npairs + p->spread_threads - 1) / p->spread_threads) * p->nslab;
    blocks = std::min(blocks, need);
    p->spread_blocks = (int)blocks;
    // the pair schedule permutes thread starts by a multiplier prime to every smaller count
    if ((blocks / p->nslab) * p->spread_threads >= 1000003)
        return set_error(PG_ERR_ARG, "spreading launch of %lld threads per slab exceeds the pair schedule's range",
                         (blocks / p->nslab) * p->spread_threads);
    const long long tile_cells = (long long)p->rows_per_slab * (long long)plane;
    if (f32) {  // per-block carry counters of the FP32 tiles (global memory, cleared by each block)
        int rc2 = dev_alloc(p, (void **)&p->carry, (size_t)blocks * tile_cells * sizeof(int));
        if (rc2) return rc2;
    } else {
        std::vector<double> kp(pgb::kPolyCoefF64, 0.0);
        kernel_poly(p->w, p->beta, kp.data());
        int rc2 = upload(p, &p->kpoly, kp);
        if (rc2) return rc2;
    }

    // ---- spreading-kernel arguments
    pgb::SpreadArgs &ka = p->sargs;
    ka.d = d;
    ka.N = N;
    ka.M = M;
    ka.r = p->r;
    ka.nnode = p->nnode;
    ka.npairs = p->npairs;
    ka.n = p->n;
    ka.nf = p->nf;
    ka.rows_per_slab = p->rows_per_slab;
    ka.nslab = p->nslab;
    ka.fast_gamma = p->fast_gamma;
    ka.S = p->S;
    ka.gamma = p->gamma;
    ka.Bconst = p->Bconst;
    ka.beta = p->beta;
    ka.grid_scale = p->n / (2.0 * kPi);
    ka.vnode = f32 ? (const void *)p->v32 : (const void *)p->v64;
    ka.vnode_lo = f32 ? p->v32lo : nullptr;
    ka.a = f32 ? (const void *)p->a32 : (const void *)p->a64;
    ka.sig = f32 ? (const void *)p->sig32 : (const void *)p->sig64;
    ka.wsig = f32 ? (const void *)p->wsig32 : (const void *)p->wsig64;
    ka.Wsig = p->Wsig;
    ka.wmax_frac = *std::max_element(sw.begin(), sw.end()) / p->Wsig;
    // FP32 strengths carry Bconst, the (common) sphere weight and 1/S as rounded FP32 constants
    p->grid_scale_corr = f32 ? pgb::fp32_strength_correction(p->Bconst, sw[0], p->S, d) : 1.0;
    ka.bound = p->bound;
    ka.tau = p->tau;
    ka.grid = p->grid;
    ka.simple_fold = (p->w <= p->n / 2) ? 1 : 0;
    ka.cpad = cpad;
    ka.ncol = ncol;
    ka.tile_cells = (int)tile_cells;
    ka.carry = p->carry;
    ka.queued = p->queued;
    ka.nang_even = p->ang.n ? (p->ang.n + 1) / 2 : 0;
    for (int k = 0; k < ka.nang_even; ++k) ka.ang_even[k] = p->ang.c[2 * k];
    ka.angmax = p->angmax;
    ka.kpoly = p->kpoly;
    pgb::fill_spread_consts(ka);
    return PG_OK;
}

int validate(const pg_boltz_opts_t &o)
{
    if (o.d != 2 && o.d != 3) return set_error(PG_ERR_ARG, "d must be 2 or 3 (got %d)", o.d);
    if (o.N < 2 || o.N > (o.d == 2 ? 512 : 128)) return set_error(PG_ERR_ARG, "N out of range (got %d)", o.N);
    if (o.M < 2 || (o.M % 2)) return set_error(PG_ERR_ARG, "M must be even and >= 2 (got %d)", o.M);
    if (!(o.S > 0.0) || !std::isfinite(o.S)) return set_error(PG_ERR_ARG, "S must be positive (got %g)", o.S);
    if (!(o.kernel_gamma >= 0.0 && o.kernel_gamma <= 1.0))
        return set_error(PG_ERR_ARG, "kernel_gamma must be in [0, 1] (got %g)", o.kernel_gamma);
    if (!(o.tol >= 1e-15 && o.tol <= 1e-2)) return set_error(PG_ERR_ARG, "tol must be in [1e-15, 1e-2] (got %g)", o.tol);
    if (o.map_log != 0 && o.map_log != 1) return set_error(PG_ERR_ARG, "map_log must be 0 or 1");
    if (o.precision < PG_PREC_AUTO || o.precision > PG_PREC_FP32) return set_error(PG_ERR_ARG, "bad precision");
    if (o.sphere < PG_SPHERE_AUTO || o.sphere > PG_SPHERE_FIBONACCI) return set_error(PG_ERR_ARG, "bad sphere kind");
    if (o.upsampfac != 0.0 && !(o.upsampfac >= 1.5 && o.upsampfac <= 4.0))
        return set_error(PG_ERR_ARG, "upsampfac must be in [1.5, 4] (got %g)", o.upsampfac);
    if (o.proj_nodes < 0 || o.proj_nodes > 4096) return set_error(PG_ERR_ARG, "proj_nodes out of range");
    if (o.screen != 0 && o.screen != 1) return set_error(PG_ERR_ARG, "screen must be 0 or 1");
    if (o.angular_terms < 0 || o.angular_terms > pgb::kMaxAngular)
        return set_error(PG_ERR_ARG, "angular_terms must be in [0, %d] (got %d)", pgb::kMaxAngular, o.angular_terms);
    if (o.angular_terms > 0) {
        if (!o.angular_coef) return set_error(PG_ERR_ARG, "angular_coef is NULL");
        for (int t = 0; t < o.angular_terms; ++t)
            if (!std::isfinite(o.angular_coef[t])) return set_error(PG_ERR_ARG, "angular_coef[%d] is not finite", t);
    }
    return PG_OK;
}

// Contract every axis but the last of `in` (shape `dims`, the last d axes live) with A,
// alternating between t1 and t2; returns the buffer holding the result and updates dims.
int leading_passes(pg_boltz_plan_t *p, const double *in, pgb::Dims3 &dims, const double *A, int m,
                   double *t1, double *t2, const double **out, int *launches)
{
    const double *cur = in;
    double *bufs[2] = {t1, t2};
    int which = 0;
    for (int ax = 3 - p->d; ax < 2; ++ax) {
        int rc = cuda_check(pgb::launch_axis_pass(cur, dims, ax, A, m, bufs[which], p->stream), "axis pass");
        if (rc) return rc;
        ++*launches;
        dims.e[ax] = m;
        cur = bufs[which];
        which ^= 1;
    }
    *out = cur;
    return PG_OK;
}

}  // namespace

// ============================================================================ ABI

PG_API pg_boltz_plan_t *pg_boltz_plan_ex(const pg_boltz_opts_t *opts)
{
    set_error(PG_OK, "%s", "");
    if (!opts) {
        set_error(PG_ERR_ARG, "opts is NULL");
        return nullptr;
    }
    pg_boltz_opts_t o = *opts;
    if (validate(o)) return nullptr;
    pg_boltz_plan_t *p = new (std::nothrow) pg_boltz_plan_t();
    if (!p) {
        set_error(PG_ERR_NOMEM, "host allocation failed");
        return nullptr;
    }
    if (cudaGetDevice(&p->device) != cudaSuccess) {
        cudaGetLastError();
        set_error(PG_ERR_CUDA, "no CUDA device available");
        delete p;
        return nullptr;
    }
    p->d = o.d;
    p->N = o.N;
    p->M = o.M;
    p->S = o.S;
    p->gamma = o.kernel_gamma;
    p->tol = o.tol;
    p->r = o.map_log ? 0 : 1;
    p->prec = (o.precision == PG_PREC_AUTO) ? (o.tol < 1e-8 ? PG_PREC_FP64 : PG_PREC_FP32) : o.precision;
    p->info.sphere = (o.d == 3) ? (o.sphere == PG_SPHERE_AUTO ? PG_SPHERE_ANTIPODAL : o.sphere) : PG_SPHERE_AUTO;
    p->screen_eps = o.screen ? 0.05 * o.tol : 0.0;
    if (build_plan(p, o)) {
        free_plan(p);
        return nullptr;
    }
    pg_boltz_info_t &in = p->info;
    in.d = p->d;
    in.N = p->N;
    in.M = p->M;
    in.r = p->r;
    in.precision = p->prec;
    in.S = p->S;
    in.kernel_gamma = p->gamma;
    in.tol = p->tol;
    in.upsampfac = p->sigma_up;
    in.n_grid = p->n;
    in.n_fold = p->nf;
    in.kernel_width = p->w;
    in.kernel_beta = p->beta;
    in.slabs = p->nslab;
    in.spread_blocks = p->spread_blocks;
    in.spread_threads = p->spread_threads;
    in.spread_smem_bytes = p->spread_smem;
    in.pairs = p->npairs;
    in.points = p->npairs * p->M;
    in.proj_nodes = p->Mp;
    in.launches_per_collide = 3 + 3 * p->d;
    in.kernels_per_collide = 2 + 3 * p->d;
    in.device_bytes = p->device_bytes;
    return p;
}

PG_API pg_boltz_plan_t *pg_boltz_plan(int d, int N, int M, double S, double kernel_gamma, double tol)
{
    pg_boltz_opts_t o;
    std::memset(&o, 0, sizeof(o));
    o.d = d;
    o.N = N;
    o.M = M;
    o.S = S;
    o.kernel_gamma = kernel_gamma;
    o.tol = tol;
    return pg_boltz_plan_ex(&o);
}

PG_API int pg_boltz_set_stream(pg_boltz_plan_t *plan, void *cuda_stream)
{
    if (!plan) return set_error(PG_ERR_ARG, "plan is NULL");
    plan->stream = static_cast<cudaStream_t>(cuda_stream);
    return PG_OK;
}

PG_API int pg_boltz_collide(pg_boltz_plan_t *p, const double *f_dev, double *Q_dev)
{
    if (!p) return set_error(PG_ERR_ARG, "plan is NULL");
    if (p->batch) return set_error(PG_ERR_STATE, "batched plans take pg_boltz_collide_batched");
    if (!f_dev || !Q_dev) return set_error(PG_ERR_ARG, "f or Q is NULL");
    const long long modes = (long long)ipow(p->N + 1, p->d);
    const char *fb = reinterpret_cast<const char *>(f_dev);
    const char *qb = reinterpret_cast<const char *>(Q_dev);
    if (fb < qb + modes * 8 && qb < fb + modes * 8) return set_error(PG_ERR_ARG, "f and Q overlap");
    DeviceGuard guard(p->device);
    if (!guard.ok) return set_error(PG_ERR_CUDA, "cannot select the plan's device");
    const int d = p->d, N = p->N;
    int launches = 0, rc;
    const bool f32 = (p->prec == PG_PREC_FP32);

    auto mark = [&](int k) {
        if (p->timing) cudaEventRecord(p->ev[k], p->stream);
    };
    mark(0);
    // 1. reconstruct a_i = W_i mu_i^2 sum_k f~_k T_k(xi_i)/sqrt(c_k)   (Section 4.2)
    pgb::Dims3 dims = dims_of(d, N + 1, N + 1, N + 1);
    const double *cur = nullptr;
    if ((rc = leading_passes(p, f_dev, dims, p->R, N, p->tA, p->tB, &cur, &launches))) return rc;
    if ((rc = cuda_check(pgb::launch_recon_last(cur, dims, p->R, N, p->scale_a, d, p->a64, f32 ? p->a32 : nullptr,
                                                p->stream), "reconstruct")))
        return rc;
    ++launches;
    mark(1);
    // 2. clear the fixed-point grid and its bound; loss weights h_i = a_i L_i / mu_i^2 (Eq. Qminus,
    //    inner sum over v_*, sigma) and the strength bound B >= sum_p |q_p|
    const size_t grid_bytes = (size_t)ipow(p->nf, d) * 8;
    if ((rc = cuda_check(cudaMemsetAsync(p->grid, 0, grid_bytes + 16 + pgb::kScreenBins * 8, p->stream),
                         "memset grid")))
        return rc;
    ++launches;
    if ((rc = cuda_check(pgb::launch_loss(p->a64, f32 ? p->a32 : nullptr, p->v64, f32 ? p->v32 : nullptr, p->v32lo, N,
                                          d, p->M, p->sig64, p->wsig64, p->sig32, p->wsig32, p->ang, p->angmax,
                                          p->Wsig, p->gamma, p->fast_gamma, p->Bconst * p->Wsig, p->inv_mu2, p->S, p->r, p->h, p->ub,
                                          p->screen_eps > 0.0 ? p->hist : nullptr, p->stream),
                         "loss")))
        return rc;
    ++launches;
    if ((rc = cuda_check(pgb::launch_bound_reduce(p->ub, p->nnode, p->screen_eps > 0.0 ? p->hist : nullptr,
                                                  p->screen_eps, p->bound, p->tau, p->stream),
                         "bound")))
        return rc;
    ++launches;
    mark(2);
    // 3. spread the M N^(2d) post-collision points onto the folded grid   (Eq. num_fast_k, Eq. nufft)
    const pgb::SpreadArgs &sa = p->sargs;
    auto launch = f32 ? (d == 2 ? pgb::launch_spread_f32_d2 : pgb::launch_spread_f32_d3)
                      : (d == 2 ? pgb::launch_spread_f64_d2 : pgb::launch_spread_f64_d3);
    cudaError_t e = launch(sa, p->w, p->spread_blocks, p->spread_threads, p->spread_smem, p->stream);
    if ((rc = cuda_check(e, "spread"))) return rc;
    ++launches;
    mark(3);
    // 4. cosine transform + deconvolution of the grid (first pass converts from fixed point),
    //    forward Chebyshev transform of the loss
    pgb::Dims3 gd = dims_of(d, p->nf, p->nf, p->nf);
    const int ax0 = 3 - d;
    if ((rc = cuda_check(pgb::launch_axis_pass_fixed(p->grid, gd, ax0, p->Dm, N + 1, p->bound, p->grid_scale_corr,
                                                     p->tA, p->stream),
                         "transform pass")))
        return rc;
    ++launches;
    gd.e[ax0] = N + 1;
    const double *gcur = p->tA;
    if (d == 3) {
        if ((rc = cuda_check(pgb::launch_axis_pass(p->tA, gd, 1, p->Dm, N + 1, p->tB, p->stream), "transform pass")))
            return rc;
        ++launches;
        gd.e[1] = N + 1;
        gcur = p->tB;
    }
    pgb::Dims3 hd = dims_of(d, N, N, N);
    const double *hcur = nullptr;
    if ((rc = leading_passes(p, p->h, hd, p->E, N + 1, p->tC, p->tD, &hcur, &launches))) return rc;
    // 5. Q = Q+ - Q-
    if ((rc = cuda_check(pgb::launch_final(gcur, gd, p->Dm, hcur, hd, p->E, N + 1, Q_dev, p->Qplus, p->Qlast, p->stream),
                         "final")))
        return rc;
    ++launches;
    mark(4);
    p->ev_recorded = p->timing;
    p->last_launches = launches;
    p->info.launches_per_collide = launches;
    p->info.kernels_per_collide = launches - 1;  // one memset
    p->have_q = true;
    return PG_OK;
}

namespace {

// One RK4 step of df~/dt = Q(f~) on stream s: four evaluations and the update.
int rk4_step(pg_boltz_plan_t *p, double *f, double dt, cudaStream_t s)
{
    const long long n = (long long)ipow(p->N + 1, p->d);
    double *k1 = p->rk, *k2 = k1 + n, *k3 = k2 + n, *k4 = k3 + n, *y = k4 + n;
    cudaStream_t keep = p->stream;
    const bool timing = p->timing;
    p->stream = s;
    p->timing = false;
    int rc = pg_boltz_collide(p, f, k1);
    if (!rc) rc = cuda_check(pgb::launch_axpy(f, k1, 0.5 * dt, y, n, s), "rk4 stage");
    if (!rc) rc = pg_boltz_collide(p, y, k2);
    if (!rc) rc = cuda_check(pgb::launch_axpy(f, k2, 0.5 * dt, y, n, s), "rk4 stage");
    if (!rc) rc = pg_boltz_collide(p, y, k3);
    if (!rc) rc = cuda_check(pgb::launch_axpy(f, k3, dt, y, n, s), "rk4 stage");
    if (!rc) rc = pg_boltz_collide(p, y, k4);
    if (!rc) rc = cuda_check(pgb::launch_rk4_update(f, k1, k2, k3, k4, dt, n, s), "rk4 update");
    p->stream = keep;
    p->timing = timing;
    return rc;
}

}  // namespace

PG_API int pg_boltz_rk4(pg_boltz_plan_t *p, double *f_dev, double dt, int nsteps)
{
    if (!p) return set_error(PG_ERR_ARG, "plan is NULL");
    if (p->batch) return set_error(PG_ERR_STATE, "RK4 stepping takes a single plan");
    if (!f_dev || nsteps < 0 || !std::isfinite(dt)) return set_error(PG_ERR_ARG, "bad f, dt or nsteps");
    DeviceGuard guard(p->device);
    if (!guard.ok) return set_error(PG_ERR_CUDA, "cannot select the plan's device");
    int rc;
    if (!p->rk_exec || p->rk_f != f_dev || p->rk_dt != dt) {
        // capture one step once per (f, dt), then replay it
        if (p->rk_exec) {
            cudaGraphExecDestroy(p->rk_exec);
            p->rk_exec = nullptr;
        }
        if (p->rk_graph) {
            cudaGraphDestroy(p->rk_graph);
            p->rk_graph = nullptr;
        }
        if (!p->rk_cap_stream &&
            (rc = cuda_check(cudaStreamCreateWithFlags(&p->rk_cap_stream, cudaStreamNonBlocking), "capture stream")))
            return rc;
        if ((rc = cuda_check(cudaStreamBeginCapture(p->rk_cap_stream, cudaStreamCaptureModeThreadLocal), "begin capture")))
            return rc;
        rc = rk4_step(p, f_dev, dt, p->rk_cap_stream);
        cudaGraph_t g = nullptr;
        cudaError_t e = cudaStreamEndCapture(p->rk_cap_stream, &g);
        if (rc) {
            if (g) cudaGraphDestroy(g);
            return rc;
        }
        if ((rc = cuda_check(e, "end capture"))) return rc;
        p->rk_graph = g;
        if ((rc = cuda_check(cudaGraphInstantiate(&p->rk_exec, p->rk_graph, 0), "graph instantiate"))) return rc;
        p->rk_f = f_dev;
        p->rk_dt = dt;
    }
    for (int s = 0; s < nsteps; ++s)
        if ((rc = cuda_check(cudaGraphLaunch(p->rk_exec, p->stream), "graph launch"))) return rc;
    return PG_OK;
}

PG_API int pg_boltz_conservation(pg_boltz_plan_t *p, const double *f_dev, double *out_host)
{
    if (!p || !f_dev || !out_host) return set_error(PG_ERR_ARG, "NULL argument");
    if (p->batch) return set_error(PG_ERR_STATE, "conservation diagnostics take a single plan");
    DeviceGuard guard(p->device);
    if (!guard.ok) return set_error(PG_ERR_CUDA, "cannot select the plan's device");
    const int d = p->d, N = p->N;
    int launches = 0, rc;
    pgb::Dims3 dims = dims_of(d, N + 1, N + 1, N + 1);
    const double *cur = nullptr;
    if ((rc = leading_passes(p, f_dev, dims, p->R, N, p->tA, p->tB, &cur, &launches))) return rc;
    if ((rc = cuda_check(pgb::launch_recon_last(cur, dims, p->R, N, p->scale_a, d, p->a64, nullptr, p->stream),
                         "reconstruct")))
        return rc;
    const int nout = 2 * (d + 2);
    if ((rc = cuda_check(cudaMemsetAsync(p->mom, 0, nout * sizeof(double), p->stream), "memset"))) return rc;
    if ((rc = cuda_check(pgb::launch_weak_moments(p->a64, p->v64, N, d, p->M, p->sig64, p->wsig64, p->ang,
                                                  p->gamma, p->fast_gamma, p->Bconst, p->mom, p->stream),
                         "weak moments")))
        return rc;
    double tmp[10];
    if ((rc = cuda_check(cudaMemcpyAsync(tmp, p->mom, nout * sizeof(double), cudaMemcpyDeviceToHost, p->stream),
                         "copy")))
        return rc;
    if ((rc = cuda_check(cudaStreamSynchronize(p->stream), "sync"))) return rc;
    std::memcpy(out_host, tmp, nout * sizeof(double));
    return PG_OK;
}

PG_API int pg_boltz_moments(pg_boltz_plan_t *p, double *out_host)
{
    if (!p || !out_host) return set_error(PG_ERR_ARG, "NULL argument");
    if (!p->have_q) return set_error(PG_ERR_STATE, "no pg_boltz_collide has run on this plan");
    DeviceGuard guard(p->device);
    if (!guard.ok) return set_error(PG_ERR_CUDA, "cannot select the plan's device");
    int rc;
    if ((rc = cuda_check(pgb::launch_moments(p->Qlast, p->Qplus, p->d, p->N, p->S, p->mom, p->stream), "moments")))
        return rc;
    double tmp[6];
    if ((rc = cuda_check(cudaMemcpyAsync(tmp, p->mom, sizeof(tmp), cudaMemcpyDeviceToHost, p->stream), "moments copy")))
        return rc;
    if ((rc = cuda_check(cudaStreamSynchronize(p->stream), "moments sync"))) return rc;
    std::memcpy(out_host, tmp, sizeof(tmp));
    return PG_OK;
}

PG_API int pg_boltz_set_timing(pg_boltz_plan_t *p, int enable)
{
    if (!p) return set_error(PG_ERR_ARG, "plan is NULL");
    if (p->batch) return pg_batched_timing(p, enable);
    DeviceGuard guard(p->device);
    if (!guard.ok) return set_error(PG_ERR_CUDA, "cannot select the plan's device");
    if (enable && !p->ev[0]) {
        for (cudaEvent_t &e : p->ev) {
            int rc = cuda_check(cudaEventCreate(&e), "cudaEventCreate");
            if (rc) return rc;
        }
    }
    p->timing = enable != 0;
    p->ev_recorded = false;
    return PG_OK;
}

PG_API int pg_boltz_stage_times(pg_boltz_plan_t *p, double *ms_out)
{
    if (!p || !ms_out) return set_error(PG_ERR_ARG, "NULL argument");
    if (p->batch) return pg_batched_elapsed(p, ms_out);
    if (!p->ev_recorded) return set_error(PG_ERR_STATE, "no timed pg_boltz_collide since timing was enabled");
    DeviceGuard guard(p->device);
    if (!guard.ok) return set_error(PG_ERR_CUDA, "cannot select the plan's device");
    int rc = cuda_check(cudaEventSynchronize(p->ev[4]), "cudaEventSynchronize");
    if (rc) return rc;
    for (int k = 0; k < 4; ++k) {
        float ms = 0.0f;
        if ((rc = cuda_check(cudaEventElapsedTime(&ms, p->ev[k], p->ev[k + 1]), "cudaEventElapsedTime"))) return rc;
        ms_out[k] = ms;
    }
    return PG_OK;
}

PG_API int pg_boltz_project_nodes(const pg_boltz_plan_t *p, double *v_host, int *count_out)
{
    if (!p) return set_error(PG_ERR_ARG, "plan is NULL");
    if (p->batch) return set_error(PG_ERR_STATE, "projection is not available on batched plans");
    if (count_out) *count_out = p->Mp;
    if (v_host) std::memcpy(v_host, p->proj_v.data(), sizeof(double) * p->Mp);
    return PG_OK;
}

PG_API int pg_boltz_project(pg_boltz_plan_t *p, const double *fvals_dev, double *ftilde_dev)
{
    if (!p) return set_error(PG_ERR_ARG, "plan is NULL");
    if (p->batch) return set_error(PG_ERR_STATE, "projection is not available on batched plans");
    if (!fvals_dev || !ftilde_dev) return set_error(PG_ERR_ARG, "NULL device pointer");
    DeviceGuard guard(p->device);
    if (!guard.ok) return set_error(PG_ERR_CUDA, "cannot select the plan's device");
    const int d = p->d, N = p->N, Mp = p->Mp;
    pgb::Dims3 dims = dims_of(d, Mp, Mp, Mp);
    const double *cur = fvals_dev;
    double *bufs[2] = {p->tA, p->tB};
    int which = 0;
    for (int ax = 3 - d; ax < 3; ++ax) {
        double *dst = (ax == 2) ? ftilde_dev : bufs[which];
        int rc = cuda_check(pgb::launch_axis_pass(cur, dims, ax, p->Pm, N + 1, dst, p->stream), "projection pass");
        if (rc) return rc;
        dims.e[ax] = N + 1;
        cur = dst;
        which ^= 1;
    }
    return PG_OK;
}

// v(xi_2) = -L with xi_2 = -cos(pi/(N+1)): for r = 1, v = S xi / sqrt(1 - xi^2) gives
// S = L sin(phi) / cos(phi) with phi = pi/(N+1); for r = 0, v = S atanh(xi) gives S = L / atanh(cos phi).
PG_API int pg_boltz_adaptive_scale(int N, double L, int map_log, double *S_out)
{
    if (!S_out) return set_error(PG_ERR_ARG, "S_out is NULL");
    if (N < 2) return set_error(PG_ERR_ARG, "need N >= 2");
    if (!std::isfinite(L) || L <= 0.0) return set_error(PG_ERR_ARG, "L must be finite and > 0");
    const double phi = kPi / (N + 1);
    *S_out = map_log ? L / std::atanh(std::cos(phi)) : L * std::tan(phi);
    return PG_OK;
}

PG_API int pg_boltz_kernel_poly(int w, double upsampfac, double *coef_out, int capacity, int *terms_out,
                                double *beta_out)
{
    if (!coef_out || !terms_out || !beta_out) return set_error(PG_ERR_ARG, "NULL argument");
    if (w < pgb::kMinWidth || w > pgb::kMaxWidthF64)
        return set_error(PG_ERR_ARG, "w must be in [%d, %d] (got %d)", pgb::kMinWidth, pgb::kMaxWidthF64, w);
    const double sigma = (upsampfac == 0.0) ? 2.0 : upsampfac;
    if (!(sigma >= 1.5 && sigma <= 4.0)) return set_error(PG_ERR_ARG, "upsampfac must be in [1.5, 4] (got %g)", upsampfac);
    const int P = pgb::kernel_poly_terms(w), need = (w + 1) / 2 * P;
    if (capacity < need) return set_error(PG_ERR_ARG, "capacity %d below %d coefficients", capacity, need);
    double c[pgb::kPolyCoefF64];
    const double beta = kernel_beta(w, sigma);
    kernel_poly(w, beta, c);
    std::copy(c, c + need, coef_out);
    *terms_out = P;
    *beta_out = beta;
    return PG_OK;
}

PG_API int pg_boltz_info(const pg_boltz_plan_t *p, pg_boltz_info_t *out)
{
    if (!p || !out) return set_error(PG_ERR_ARG, "NULL argument");
    *out = p->info;
    out->device_bytes = p->device_bytes;
    return PG_OK;
}

PG_API void pg_boltz_destroy(pg_boltz_plan_t *p)
{
    if (!p) return;
    DeviceGuard guard(p->device);
    cudaStreamSynchronize(p->stream);
    free_plan(p);
}
