/*
 * pg_boltz.h -- C ABI of the GB300 (sm_103a) library that evaluates the
 * Petrov-Galerkin mapped-Chebyshev collision operator of arXiv 2105.08806
 * with the fast (non-uniform FFT) algorithm of its Section 4.2.
 *
 * The operator (Section 3, Eq. Qk_component, discretised as in Section 4):
 *
 *   Q_k = sum_{i,j} sum_m W_i W_j w_m B(|v_i - v_j|) g_i g_j [That_k(v'_ijm) - That_k(v_i)],
 *   0 <= k_l <= N,  l = 1..d,
 *
 * over the N interior Chebyshev-Gauss-Lobatto nodes per axis of M_v = N + 2
 * (Section 4.2), with g_i = f_N(v_i)/mu(xi_i)^2, v' = (v_i+v_j)/2 + |v_i-v_j| sigma_m/2,
 * That_k the test functions of Eq. 1DCheby and B = |g|^gamma / |S^{d-1}| (VHS,
 * Section 3.1).  The gain sum is evaluated as a type-1 non-uniform cosine
 * transform (Eq. num_fast_k, Eq. nufft): exponential-of-semicircle spreading onto
 * a folded, oversampled cosine grid, a d-dimensional cosine transform and a
 * deconvolution; the loss is Eq. Qminus.
 *
 * Conventions for every entry point:
 *  - Arrays of modes are (N+1)^d doubles in C order over (k_1, ..., k_d),
 *    k_d fastest.  "Device" pointers are CUDA global-memory pointers of the
 *    current device; "host" pointers are ordinary host memory.
 *  - Return codes: PG_OK (0) or a negative PG_ERR_* code; functions returning a
 *    pointer return NULL on failure.  pg_boltz_last_error() (thread-local) then
 *    holds a one-line reason.  No function aborts, prints or exits.
 *  - A plan owns every device buffer it allocates and is freed by
 *    pg_boltz_destroy.  Caller arrays stay owned by the caller.
 *  - A plan is not thread-safe: use one plan per host thread / stream.
 *  - Work is enqueued on the plan's stream (default: the legacy default
 *    stream) and the calls return after enqueue, except where noted.
 */
#ifndef PG_BOLTZ_H
#define PG_BOLTZ_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Status codes. */
#define PG_OK 0
#define PG_ERR_ARG (-1)     /* invalid argument or NULL handle            */
#define PG_ERR_NOMEM (-2)   /* host or device allocation failed           */
#define PG_ERR_CUDA (-3)    /* a CUDA runtime call or launch failed       */
#define PG_ERR_TIMEOUT (-4) /* a bounded device-side wait gave up         */
#define PG_ERR_STATE (-5)   /* call not valid in the plan's current state */

/* Arithmetic of the spreading stage. */
#define PG_PREC_AUTO 0 /* tol < 1e-8 -> FP64, else FP32                          */
#define PG_PREC_FP64 1 /* FP64 point generation, spreading and transform         */
#define PG_PREC_FP32 2 /* FP32 point generation and shared-memory spreading (exact
                          integer sums), FP32 loss pair terms summed as float pairs;
                          FP64 global grid, cosine transform, deconvolution, moments */

/* Sphere quadrature for d = 3 (d = 2 always uses M uniform polar angles, Section 4.1). */
#define PG_SPHERE_AUTO 0      /* antipodal Fibonacci set (M even)                  */
#define PG_SPHERE_ANTIPODAL 1 /* M/2 golden-angle points and their negatives       */
#define PG_SPHERE_FIBONACCI 2 /* plain M-point golden-angle set                    */

typedef struct pg_boltz_plan_s pg_boltz_plan_t;

/* Extended plan options.  Zero-initialise, then set d, N, M, S, kernel_gamma, tol. */
typedef struct {
    int d;               /* velocity dimension, 2 or 3                                   */
    int N;               /* highest mode per axis (modes 0..N), N >= 2                   */
    int M;               /* sphere points M_sigma, M >= 2 and even                       */
    double S;            /* map scale S > 0 (Eq. 1D_mapping)                             */
    double kernel_gamma; /* VHS exponent, 0 <= gamma <= 1 (Section 3.1)                  */
    double tol;          /* requested transform precision, 1e-15 <= tol <= 1e-2          */
    int map_log;         /* 0: algebraic map r = 1 (default); 1: logarithmic map r = 0
                            (Section 2.1 Remark)                                          */
    int precision;       /* PG_PREC_*                                                    */
    int sphere;          /* PG_SPHERE_*                                                  */
    double upsampfac;    /* grid oversampling sigma, 0 -> 2.0, range [1.5, 4]             */
    int proj_nodes;      /* Chebyshev-Gauss nodes per axis for pg_boltz_project, 0 -> 4(N+1) */
    int spread_threads;  /* threads per spreading block, 0 -> automatic                  */
    int spread_blocks_per_sm; /* spreading blocks per SM, 0 -> automatic                 */
    int screen;          /* 1: skip the node pairs with the smallest strength bounds, as many
                            as keep their summed bound below 0.05 tol B (B >= the sum of all
                            point strengths); 0 (default): spread every pair.               */
    int angular_terms;   /* 0 (default): VHS kernel B = |g|^gamma / |S^{d-1}|.  1..8: the kernel
                            B(|g|, cos theta) = |g|^gamma b(cos theta) / |S^{d-1}| of
                            Eq. collision_form with b(c) = sum_{p < angular_terms}
                            angular_coef[p] c^p, cos theta = (v - v_*) . sigma / |v - v_*|
                            (0 when v = v_*).  The loss sum then runs over the sphere set per
                            node pair (O(M N^(2d)), as Section 4.2 states for general kernels).
                            Plain plans only.                                               */
    const double *angular_coef; /* host array of angular_terms finite values, copied at plan time */
} pg_boltz_opts_t;

/* Read-only description of a plan (pg_boltz_info). */
typedef struct {
    int d, N, M, r, precision, sphere;
    double S, kernel_gamma, tol, upsampfac;
    int n_grid;            /* periodic oversampled grid size n (even)                      */
    int n_fold;            /* folded cosine grid cells per axis, n/2 + 1                    */
    int kernel_width;      /* spreading kernel width w (grid cells)                         */
    double kernel_beta;    /* exponential-of-semicircle shape parameter                     */
    int slabs;             /* shared-memory slabs of the folded grid along axis 1           */
    int spread_blocks, spread_threads;
    size_t spread_smem_bytes;
    long long points;      /* non-uniform points spread per evaluation, M x pairs            */
    long long pairs;       /* node pairs spread per evaluation: each unordered pair {i, j} of
                              the N^d interior nodes once, N^d (N^d + 1) / 2 (the orders (i, j)
                              and (j, i) add the same points with the same strength)          */
    int proj_nodes;
    int launches_per_collide; /* kernels + memsets enqueued by one pg_boltz_collide          */
    size_t device_bytes;   /* device memory owned by the plan                               */
    int kernels_per_collide; /* kernel launches (memsets excluded) of one collide              */
} pg_boltz_info_t;

/*
 * Create a plan with the defaults: algebraic map (r = 1), M_v = N + 2 CGL
 * nodes (Section 4.2), uniform circle (d = 2) or antipodal Fibonacci sphere
 * (d = 3), oversampling 2, precision chosen from tol (PG_PREC_AUTO).
 * Uploads all tables and allocates the workspace on the current device.
 * Returns NULL on error (PG_ERR_ARG / PG_ERR_NOMEM / PG_ERR_CUDA in last_error).
 */
pg_boltz_plan_t *pg_boltz_plan(int d, int N, int M, double S, double kernel_gamma, double tol);

/* Same as pg_boltz_plan with every option of pg_boltz_opts_t. */
pg_boltz_plan_t *pg_boltz_plan_ex(const pg_boltz_opts_t *opts);

/* Set the CUDA stream (a cudaStream_t, NULL = legacy default stream) for later calls. */
int pg_boltz_set_stream(pg_boltz_plan_t *plan, void *cuda_stream);

/*
 * Q_k for the coefficients f~_k of f_N (Eq. fN_Expansion, Section 4.2 fast algorithm).
 * f_dev, Q_dev: caller-owned device arrays of (N+1)^d doubles (C order); they must not
 * overlap.  Asynchronous on the plan's stream.  The plan's workspace is reused by the
 * next call on the same plan, so calls on one plan must not overlap in time.
 */
int pg_boltz_collide(pg_boltz_plan_t *plan, const double *f_dev, double *Q_dev);

/*
 * Time integration of the Petrov-Galerkin ODE system df~_k/dt = Q_k (Eq. spectral_ODE) with
 * the classical fourth-order Runge-Kutta method (the paper's choice, Section 5.1.2 uses
 * dt = 0.02): nsteps steps of size dt applied to f_dev in place ((N+1)^d doubles, device).
 * FP64 state and updates; the evaluations use the plan's precision.  The first call for a
 * given (f_dev, dt) captures one step (four evaluations and the updates) into a CUDA graph,
 * later calls replay it.  Asynchronous on the plan's stream.  Not for batched plans.
 */
int pg_boltz_rk4(pg_boltz_plan_t *plan, double *f_dev, double dt, int nsteps);

/*
 * Conservation of the discrete operator in weak form (Eq. weak and Eq. consv, with the
 * quadrature of Section 4), in FP64 on the device, for the coefficients f_dev:
 *   out_host[2t]   = sum_{i,j,m} qbar [phi_t(v') - phi_t(v_i)],
 *   out_host[2t+1] = sum_{i,j,m} qbar (|phi_t(v')| + |phi_t(v_i)|)   (a scale for [2t]),
 * phi_0 = 1, phi_1..phi_d = v_1..v_d, phi_{d+1} = |v|^2; out_host holds 2(d+2) doubles.  Mass is
 * conserved exactly; momentum and energy when the sphere set is antipodal.  Overwrites the
 * plan's reconstruction buffers (so pg_boltz_moments refers to no collide afterwards only if
 * none follows).  Synchronises the plan's stream.
 */
int pg_boltz_conservation(pg_boltz_plan_t *plan, const double *f_dev, double *out_host);

/*
 * FP64 diagnostics of the last pg_boltz_collide, copied to host (synchronises the
 * plan's stream).  out_host[0..5]:
 *   [0] sum_k a_k Q_k, [1] sum_k b_k Q_k  where 1 = sum a_k That_k, |v|^2 = sum b_k That_k
 *       (Section 3.3 proof; exact identities for r = 1, N >= 2: mass and energy of Q),
 *   [2] sum_k a_k Q+_k, [3] sum_k b_k Q+_k (the same functionals of the gain term),
 *   [4] ||Q||_2, [5] ||Q+||_2.
 */
int pg_boltz_moments(pg_boltz_plan_t *plan, double *out_host);

/*
 * Per-stage timing of pg_boltz_collide (no counterpart in the paper, which reports
 * whole-evaluation CPU seconds in Section 5.1.1 Test 04).  enable != 0 makes every later
 * collide record CUDA events on the plan's stream between its stages; 0 stops it.
 * Creates the events on first use.  Returns PG_OK / PG_ERR_ARG / PG_ERR_CUDA.
 */
int pg_boltz_set_timing(pg_boltz_plan_t *plan, int enable);

/*
 * Durations in milliseconds of the stages of the last timed collide (waits for it):
 *   ms_out[0] reconstruction of f_N at the nodes, [1] loss sums,
 *   [2] grid clear + spreading, [3] cosine transform, deconvolution, loss transform, combine.
 * PG_ERR_STATE if no collide ran since timing was enabled.
 */
int pg_boltz_stage_times(pg_boltz_plan_t *plan, double *ms_out);

/*
 * Velocities v(xi_p) of the proj_nodes Chebyshev-Gauss projection nodes
 * xi_p = -cos((2p-1) pi / (2 Mp)), p = 1..Mp, written to v_host[0..Mp-1].
 * *count_out receives Mp.  Host-only, no device work.
 */
int pg_boltz_project_nodes(const pg_boltz_plan_t *plan, double *v_host, int *count_out);

/*
 * f~_k = (f, That_k) (Eq. MultiD_spectral_coef) by Chebyshev-Gauss quadrature.
 * fvals_dev: device array of Mp^d doubles, f at the tensor grid of the projection
 * nodes (C order); ftilde_dev: device array of (N+1)^d doubles.  Asynchronous.
 */
int pg_boltz_project(pg_boltz_plan_t *plan, const double *fvals_dev, double *ftilde_dev);

/*
 * Inverse transform at arbitrary velocities: u_N(v) = sum_k u~_k prod_l T~_{k_l}(v_l) with the
 * trial functions T~_k = mu^4 T_k(xi(v)) / sqrt(c_k) of the plan's map and S (Eq. fN_Expansion,
 * Eq. 1DCheby).  Applied to f~ it gives f_N(v); applied to the Q_k of pg_boltz_collide it gives
 * Q_N(v), the trial-space function with those weak-form coefficients.
 * coef_dev: device array of (N+1)^d doubles (C order, the layout of pg_boltz_collide);
 * pts_dev: device array of npts x d doubles (row-major, one velocity per row, any finite value);
 * out_dev: device array of npts doubles.  Caller owns all three.  npts = 0 is a no-op.
 * Asynchronous on the plan's stream.  PG_ERR_ARG for npts < 0 or NULL pointers,
 * PG_ERR_STATE on batched plans.
 */
int pg_boltz_evaluate(pg_boltz_plan_t *plan, const double *coef_dev, long long npts, const double *pts_dev,
                      double *out_dev);

/*
 * Adaptive map scale (Section 5, the choice of S stated before the 2D examples): the S for
 * which the first interior node xi_2 = -cos(pi/(N+1)) of the M_v = N + 2 Chebyshev-Gauss-Lobatto
 * nodes maps to v = -L (and, by symmetry, the last interior node to +L):
 *   algebraic map (map_log = 0):   S = L tan(pi/(N+1))
 *   logarithmic map (map_log = 1): S = L / atanh(cos(pi/(N+1)))
 * Host-only.  *S_out receives S.  PG_ERR_ARG for N < 2, L not finite or <= 0, S_out NULL.
 */
int pg_boltz_adaptive_scale(int N, double L, int map_log, double *S_out);

/*
 * The FP64 spreading kernels' form of the exponential-of-semicircle kernel of the type-1 NUFFT
 * (Eq. nufft): psi(t) = exp(beta (sqrt(1 - t^2) - 1)) for |t| < 1, t = (grid index - x) 2/w.
 * A point at grid coordinate x touches indices s .. s+w-1, s = floor(x - w/2) + 1; with the
 * offset y = 2 (s - x) + w - 1 in (-1, 1], tap a (t = (y + 1 + 2a - w)/w) equals, up to about
 * exp(-beta), E_a(y^2) + y O_a(y^2) for a < ceil(w/2), and tap w-1-a equals E_a(y^2) - y O_a(y^2).
 * For width w in [2, 16] and oversampling upsampfac in [1.5, 4] (0 -> 2) this writes beta to
 * *beta_out, the number of terms P (w + 3 for w < 12, else w + 1) to *terms_out and
 * ceil(w/2) * P coefficients to coef_out (host array of `capacity` doubles): block a holds the
 * (P+1)/2 coefficients of E_a, then the P/2 of O_a, lowest power first (for odd w the middle
 * tap's O is zero by symmetry).  Host-only.  PG_ERR_ARG for w or upsampfac out of range, NULL
 * pointers, or capacity below ceil(w/2) * P.
 */
int pg_boltz_kernel_poly(int w, double upsampfac, double *coef_out, int capacity, int *terms_out,
                         double *beta_out);

/* Describe the plan (host-only). */
int pg_boltz_info(const pg_boltz_plan_t *plan, pg_boltz_info_t *out);

/* Free the plan and its device memory.  NULL-safe.  Synchronises the plan's stream. */
void pg_boltz_destroy(pg_boltz_plan_t *plan);

/*
 * Batched plans: ncell independent operators of one dimension d (one velocity distribution
 * per spatial cell of an inhomogeneous solver; each cell is an instance of Section 4.2 with its
 * own N_c, M_c, S_c, gamma_c).  N[c], M[c], S[c], kernel_gamma[c]: host arrays of ncell values
 * (2 <= N_c <= 200 in 2D, <= 40 in 3D; M_c even; the cell's folded grid must fit shared memory).
 * The _ex form reads d, tol, map_log, precision, sphere, upsampfac, spread_threads,
 * spread_blocks_per_sm and screen from opts (its N, M, S, kernel_gamma are ignored).
 * NULL on error.  Other entry points accept a batched plan where noted.
 */
pg_boltz_plan_t *pg_boltz_plan_batched(int d, int ncell, const int *N, const int *M, const double *S,
                                       const double *kernel_gamma, double tol);
pg_boltz_plan_t *pg_boltz_plan_batched_ex(const pg_boltz_opts_t *opts, int ncell, const int *N, const int *M,
                                          const double *S, const double *kernel_gamma);

/*
 * Q for every cell of a batched plan.  f_packed_dev / Q_packed_dev: device arrays holding the
 * cells' (N_c+1)^d coefficient arrays one after the other in cell order (offsets from
 * pg_boltz_batched_offsets); they must not overlap.  Asynchronous on the plan's stream.  The
 * launch sequence (prep, persistent spreading over a work queue of (cell, pair range) items,
 * finalisation) is captured into a CUDA graph on the first call for a given (f, Q) pair and
 * replayed afterwards (pg_boltz_batched_use_graph(plan, 0) launches directly instead).
 */
int pg_boltz_collide_batched(pg_boltz_plan_t *plan, const double *f_packed_dev, double *Q_packed_dev);

/* Offsets (in doubles) of each cell in the packed arrays: offsets_host[0..ncell], last = total. */
int pg_boltz_batched_offsets(const pg_boltz_plan_t *plan, long long *offsets_host);

/* 1 (default): replay a captured CUDA graph in pg_boltz_collide_batched; 0: direct launches. */
int pg_boltz_batched_use_graph(pg_boltz_plan_t *plan, int enable);

/*
 * Autotuner of a batched plan's persistent spreading launch (no counterpart in the paper, which
 * evaluates one operator at a time): runs pg_boltz_collide_batched's launch sequence on the
 * caller's f_packed_dev / Q_packed_dev (Q is overwritten), first for threads per block in
 * {128, 256, 512, 1024} and every blocks-per-SM count the kernel's occupancy allows (FP32 plans:
 * at most the block count the plan sized its carry counters for), then at the fastest shape for
 * work items of 2^15, 2^16, ..., 2^19 points (the node-pair ranges the blocks take from the
 * global counter); `trials` timed runs each after one warm-up.  Keeps the fastest shape and item
 * size for later calls (the next call captures a new graph).  The results do not depend on
 * either (exact fixed-point sums).  Synchronises the plan's stream.  Optional outputs (host):
 * threads per block, blocks, points per work item, best time in ms of one call.
 * PG_ERR_ARG for NULL or overlapping arrays or trials outside [1, 100]; PG_ERR_STATE on plain plans.
 */
int pg_boltz_batched_autotune(pg_boltz_plan_t *plan, const double *f_packed_dev, double *Q_packed_dev, int trials,
                              int *threads_out, int *blocks_out, long long *item_points_out, double *ms_out);

/*
 * Measured throughput (atomic additions per second, whole GPU) of 32-bit integer atomic adds
 * to shared memory at random addresses of a 16,900-cell tile -- the operation that bounds
 * the spreading kernels.  No counterpart in the paper; used as the measured roofline of
 * spreading.  Allocates and frees 64 bytes; synchronises cuda_stream.  PG_OK / PG_ERR_CUDA.
 */
int pg_boltz_probe_shared_atomics(void *cuda_stream, double *rate_out);

/*
 * Measured peaks of the whole GPU for the spreading kernels' rooflines (no counterpart in the
 * paper): rates_out[0] = FP32 fused multiply-adds per second, rates_out[1] = FP64 fused
 * multiply-adds per second (independent chains in every thread of two 1024-thread blocks per
 * SM), rates_out[2] = 32-bit integer shared-memory atomic adds per second with every lane of a
 * warp on its own bank (no conflicts).  rates_out: host array of 3 doubles.  Allocates and frees
 * 64 bytes; synchronises cuda_stream.  PG_OK, PG_ERR_ARG (NULL) or PG_ERR_CUDA.
 */
int pg_boltz_probe_pipes(void *cuda_stream, double *rates_out);

/*
 * The FP32 spreading kernels' grid coordinates, for testing them: for each of the n velocities
 * v_dev[i] (device, FP32) of one mapped axis, the grid coordinate x = n_grid z / (2 pi) of
 * z = arccos(xi(v)) (Section 2.1 maps: map_log 0 algebraic r = 1, 1 logarithmic r = 0, scale S)
 * as the kernels form it: an integer cell cell_dev[i] and a fraction frac_dev[i] in [0, 1)
 * (x = cell + frac), and m2_dev[i] = mu(xi(v))^-2 in FP32.  cell_dev, frac_dev, m2_dev: device
 * arrays of n doubles.  n_grid: the (even) periodic grid size.  Asynchronous on cuda_stream.
 * PG_OK, PG_ERR_ARG or PG_ERR_CUDA.
 */
int pg_boltz_grid_coords_f32(const float *v_dev, long long n, double S, int map_log, int n_grid, double *cell_dev,
                             double *frac_dev, double *m2_dev, void *cuda_stream);

/*
 * Size of the library-owned static device array used by pg_boltz_project_noalloc
 * (4 MiB of doubles, held on every GPU that loads the library until process exit).
 */
#define PG_BOLTZ_NOALLOC_SCRATCH_BYTES (4u << 20)

/*
 * pg_boltz_project without any allocation.  The paper has no counterpart; this is a
 * library facility for callers that cannot allocate device memory -- applications whose
 * own pool or arena owns all device memory and forbids library calls to cudaMalloc, or
 * bindings that can only pass pointers they already hold -- and therefore cannot create
 * a plan (plans allocate their tables and workspace).
 *
 * Computes the same coefficients as pg_boltz_project on a plan with the same d, N, S, map
 * and proj_nodes = Mp (nodes from pg_boltz_project_nodes), up to rounding.
 *   d: 2 or 3; N >= 2; S > 0; map_log: 0 algebraic (r = 1), 1 logarithmic (r = 0); Mp >= 1.
 *   fvals_dev: device array of Mp^d doubles (f at the tensor grid of the nodes, C order).
 *   ftilde_dev: device array of (N+1)^d doubles, written.
 *   cuda_stream: a cudaStream_t (NULL = legacy default stream); the call is asynchronous.
 * Scratch: (N+1) Mp + (N+1) Mp^(d-1) [+ (N+1)^2 Mp when d = 3] doubles of the static array of
 * PG_BOLTZ_NOALLOC_SCRATCH_BYTES; larger requests return PG_ERR_ARG (see pg_boltz_last_error).
 * It calls no cudaMalloc, cudaFree or other allocating routine.  Every call looks up the
 * array's device address with cudaGetSymbolAddress on the current device (no cache, so a
 * device reset or a change of context needs no special care); the first call in a context may
 * load the library's device code there, so make it before any stream capture.  All calls share the array,
 * which keeps the last call's contents (every value a call reads it has written itself, so
 * nothing needs clearing); calls that overlap on the GPU (different streams, or another
 * host thread) race on it and must be serialised by the caller.
 * Returns PG_OK, PG_ERR_ARG or PG_ERR_CUDA.
 */
int pg_boltz_project_noalloc(int d, int N, double S, int map_log, int Mp, const double *fvals_dev,
                             double *ftilde_dev, void *cuda_stream);

/*
 * Host-side fault injection for tests: the countdown-th device allocation made by a
 * later plan creation fails with PG_ERR_NOMEM (0 disables).  Process-wide; no device work.
 */
void pg_boltz_debug_fail_alloc(int countdown);

/* Thread-local text of the last error ("" when none); valid until the next call. */
const char *pg_boltz_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* PG_BOLTZ_H */
