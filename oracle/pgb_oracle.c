/*
 * FP64 CPU oracle for the weak-form collision operator of the Petrov-Galerkin
 * mapped-Chebyshev spectral method (arXiv 2105.08806).
 *
 * TEST INFRASTRUCTURE ONLY. Only tests/, __graft_entry__.smoke() and bench.py's
 * cpu_baseline / reference leg may load this library. It shares no code, header,
 * table or constant with the CUDA library under paper_2105_08806_gb300/.
 *
 * What it computes (Section 3, Eq. Qk_component, with the quadrature of Section 4.1):
 *
 *   Q_k = sum_{i,j interior nodes} sum_m  qbar_{ijm} [ That_k(v'_{ijm}) - That_k(v_i) ]
 *   qbar_{ijm} = W_i W_j w_m B(|v_i - v_j|, cos theta_{ijm}) g_i g_j,
 *   cos theta_{ijm} = <(v_i - v_j)/|v_i - v_j|, sigma_m>                 (Eq. collision_form)
 *   v'_{ijm}   = (v_i + v_j)/2 + |v_i - v_j| sigma_m / 2                  (Section 1)
 *   That_k(v)  = prod_l mu(xi(v_l))^{-2} T_{k_l}(xi(v_l)) / sqrt(c_{k_l})  (Section 2.1, Eq. 1DCheby)
 *
 * The gain part sum qbar That_k(v') is evaluated directly for every requested
 * mode: no NUFFT, no spreading, no transform.  The loss part follows Eq. Qminus:
 * the inner (v_*, sigma) sum is formed first and then multiplied by That_k(v_i).
 * The nodes v_i, the weights, g_i = f_N(v_i)/mu(xi_i)^2 and the sphere set are
 * prepared by oracle.py (numpy) and passed in.
 *
 * Chebyshev polynomials come from the three-term recurrence of Section 2.1; the
 * maps are the logarithmic (r = 0, Eq. logarithmic) and algebraic (r = 1,
 * Eq. algebraic) maps of Section 2.1 Remark; mu from Eq. 1D_mu_function.
 *
 * Work is split over the outer node index i across POSIX threads; each thread
 * keeps private accumulators that are summed in thread order at the end.
 */
#include <math.h>
#include <pthread.h>
#include <stdlib.h>
#include <string.h>

#define ORACLE_MAX_D 3

typedef struct {
    int d, Nn, M, r, nmodes, kmax;
    const double *v1d;   /* Nn interior node velocities, one axis (same on every axis) */
    const double *g;     /* Nn^d values g_i, C-order (last axis fastest)               */
    double Wnode;        /* product quadrature weight of one node, W_i = W_j           */
    const double *sig;   /* M x d sphere points                                        */
    const double *wsig;  /* M sphere weights                                           */
    double S, gamma, Bconst;
    int nb;              /* angular polynomial terms (0: b = 1)                        */
    const double *bcoef; /* b(cos theta) = sum_p bcoef[p] cos^p theta                  */
    const int *modes;    /* nmodes x d mode multi-indices                              */
    /* weak functionals */
    int nphi;
    const int *phi;      /* nphi x 3: (kind, a, b), see phi_eval                       */
} prob_t;

typedef struct {
    const prob_t *p;
    int i_begin, i_end;
    double *gain;   /* nmodes */
    double *lossw;  /* Nn^d : inner loss sums per outer node */
    double *wk;     /* nphi x 2 */
} work_t;

/* xi(v) for the map with tail parameter r (Section 2.1 Remark). */
static double map_xi(double v, double S, int r)
{
    if (r == 0) return tanh(v / S);
    return v / sqrt(S * S + v * v);
}

/* mu(xi)^{-2} with mu = (1-xi^2)^{(1+r)/4} / sqrt(S)  (Eq. 1D_mu_function). */
static double mu_m2(double xi, double S, int r)
{
    double one_m = (1.0 - xi) * (1.0 + xi);
    return S / pow(one_m, 0.5 * (1.0 + r));
}

/* That_k(v) for k = 0..kmax along one axis, written into out[0..kmax]. */
static void that_1d(double v, double S, int r, int kmax, double *out)
{
    double xi = map_xi(v, S, r);
    double m2 = mu_m2(xi, S, r);
    double tkm1 = 1.0, tk = xi;
    out[0] = m2 * tkm1 / sqrt(M_PI);
    if (kmax >= 1) out[1] = m2 * tk / sqrt(M_PI / 2.0);
    for (int k = 1; k < kmax; ++k) {
        double tkp1 = 2.0 * xi * tk - tkm1;   /* T_{k+1} = 2 xi T_k - T_{k-1} */
        out[k + 1] = m2 * tkp1 / sqrt(M_PI / 2.0);
        tkm1 = tk;
        tk = tkp1;
    }
}

/* Collision kernel B = Bconst |g|^gamma (VHS, Section 3.1); gamma = 0 gives Bconst even at g = 0. */
static double kernel_B(double grel, double gamma, double Bconst)
{
    if (gamma == 0.0) return Bconst;
    return Bconst * pow(grel, gamma);
}

/* Angular factor b(cos theta) of B(|g|, cos theta) = Bconst |g|^gamma b(cos theta) (Eq. collision_form),
 * cos theta = <(v - v_*)/|v - v_*|, sigma>; taken as 0 when v = v_*.  nb = 0: b = 1 (VHS). */
static double angular_b(const prob_t *p, const double *vi, const double *vj, double grel, const double *sig)
{
    if (p->nb == 0) return 1.0;
    double c = 0.0;
    if (grel > 0.0) {
        for (int l = 0; l < p->d; ++l) c += (vi[l] - vj[l]) * sig[l];
        c /= grel;
    }
    double b = 0.0, cp = 1.0;
    for (int t = 0; t < p->nb; ++t) {
        b += p->bcoef[t] * cp;
        cp *= c;
    }
    return b;
}

/* Weak-form test functions used for conservation and moment checks:
 * kind 0: 1;  kind 1: v_a;  kind 2: |v|^2;  kind 3: v_a v_b;  kind 4: v_a |v|^2;
 * kind 5: v_a^2 v_b^2;  kind 6: |v|^4. */
static double phi_eval(const int *ph, const double *v, int d)
{
    double n2 = 0.0;
    for (int l = 0; l < d; ++l) n2 += v[l] * v[l];
    switch (ph[0]) {
    case 0: return 1.0;
    case 1: return v[ph[1]];
    case 2: return n2;
    case 3: return v[ph[1]] * v[ph[2]];
    case 4: return v[ph[1]] * n2;
    case 5: return v[ph[1]] * v[ph[1]] * v[ph[2]] * v[ph[2]];
    default: return n2 * n2;
    }
}

static void node_coords(const prob_t *p, long idx, double *v)
{
    for (int l = p->d - 1; l >= 0; --l) {
        v[l] = p->v1d[idx % p->Nn];
        idx /= p->Nn;
    }
}

static void *worker(void *arg)
{
    work_t *w = (work_t *)arg;
    const prob_t *p = w->p;
    const int d = p->d;
    long nnode = 1;
    for (int l = 0; l < d; ++l) nnode *= p->Nn;
    double *tab = (double *)malloc(sizeof(double) * (size_t)d * (p->kmax + 1));
    double vi[ORACLE_MAX_D], vj[ORACLE_MAX_D], vp[ORACLE_MAX_D];

    for (long i = w->i_begin; i < w->i_end; ++i) {
        node_coords(p, i, vi);
        double inner = 0.0;
        for (long j = 0; j < nnode; ++j) {
            node_coords(p, j, vj);
            double gap2 = 0.0;
            for (int l = 0; l < d; ++l) gap2 += (vi[l] - vj[l]) * (vi[l] - vj[l]);
            double grel = sqrt(gap2);
            double B = kernel_B(grel, p->gamma, p->Bconst);
            double pair = p->Wnode * p->Wnode * B * p->g[i] * p->g[j];
            for (int m = 0; m < p->M; ++m) {
                double qbar = pair * p->wsig[m] * angular_b(p, vi, vj, grel, p->sig + m * d);
                inner += qbar;
                for (int l = 0; l < d; ++l)
                    vp[l] = 0.5 * (vi[l] + vj[l]) + 0.5 * grel * p->sig[m * d + l];
                if (p->nmodes > 0) {
                    for (int l = 0; l < d; ++l)
                        that_1d(vp[l], p->S, p->r, p->kmax, tab + (size_t)l * (p->kmax + 1));
                    for (int t = 0; t < p->nmodes; ++t) {
                        double val = 1.0;
                        for (int l = 0; l < d; ++l)
                            val *= tab[(size_t)l * (p->kmax + 1) + p->modes[t * d + l]];
                        w->gain[t] += qbar * val;
                    }
                }
                for (int t = 0; t < p->nphi; ++t) {
                    double fp = phi_eval(p->phi + 3 * t, vp, d);
                    double fv = phi_eval(p->phi + 3 * t, vi, d);
                    w->wk[2 * t] += qbar * (fp - fv);
                    w->wk[2 * t + 1] += qbar * (fabs(fp) + fabs(fv));
                }
            }
        }
        w->lossw[i] = inner;
    }
    free(tab);
    return NULL;
}

static int run(prob_t *p, long i_lo, long i_hi, int nthreads, double *gain, double *lossw, double *wk)
{
    long span = i_hi - i_lo;
    if (span < 1) return 0;
    if (nthreads < 1) nthreads = 1;
    if (nthreads > span) nthreads = (int)span;
    pthread_t *th = (pthread_t *)calloc((size_t)nthreads, sizeof(pthread_t));
    work_t *ws = (work_t *)calloc((size_t)nthreads, sizeof(work_t));
    if (!th || !ws) { free(th); free(ws); return -2; }
    int rc = 0;
    for (int t = 0; t < nthreads; ++t) {
        ws[t].p = p;
        ws[t].i_begin = (int)(i_lo + span * t / nthreads);
        ws[t].i_end = (int)(i_lo + span * (t + 1) / nthreads);
        ws[t].gain = (double *)calloc((size_t)(p->nmodes > 0 ? p->nmodes : 1), sizeof(double));
        ws[t].wk = (double *)calloc((size_t)(2 * (p->nphi > 0 ? p->nphi : 1)), sizeof(double));
        ws[t].lossw = lossw;  /* disjoint rows per thread */
        if (!ws[t].gain || !ws[t].wk) rc = -2;
    }
    if (rc == 0) {
        for (int t = 0; t < nthreads; ++t) pthread_create(&th[t], NULL, worker, &ws[t]);
        for (int t = 0; t < nthreads; ++t) pthread_join(th[t], NULL);
        for (int t = 0; t < nthreads; ++t) {
            for (int k = 0; k < p->nmodes; ++k) gain[k] += ws[t].gain[k];
            for (int k = 0; k < 2 * p->nphi; ++k) wk[k] += ws[t].wk[k];
        }
    }
    for (int t = 0; t < nthreads; ++t) { free(ws[t].gain); free(ws[t].wk); }
    free(th);
    free(ws);
    return rc;
}

/*
 * Gain and loss parts of Q_k for the requested modes.
 *   gain[t] = sum_{i,j,m} qbar That_{k_t}(v')                       (Eq. Qplus, discretised)
 *   loss[t] = sum_i That_{k_t}(v_i) * sum_{j,m} qbar                (Eq. Qminus, discretised)
 * The outer sum runs over the node indices i_lo <= i < i_hi (the full operator when
 * i_lo = 0, i_hi = Nn^d; a partial range is a bounded sample of the same work).
 * Returns 0, or -1 on bad arguments, -2 when memory runs out.
 */
int pgb_oracle_collide(int d, int Nn, const double *v1d, const double *g, double Wnode,
                       int M, const double *sig, const double *wsig,
                       double S, int r, double gamma, double Bconst, int nb, const double *bcoef,
                       int nmodes, const int *modes, long i_lo, long i_hi,
                       double *gain, double *loss, int nthreads)
{
    if (d < 1 || d > ORACLE_MAX_D || Nn < 1 || M < 1 || nmodes < 1 || (r != 0 && r != 1) || nb < 0 ||
        (nb > 0 && !bcoef))
        return -1;
    prob_t p;
    memset(&p, 0, sizeof(p));
    p.d = d; p.Nn = Nn; p.M = M; p.r = r; p.nmodes = nmodes;
    p.v1d = v1d; p.g = g; p.Wnode = Wnode; p.sig = sig; p.wsig = wsig;
    p.S = S; p.gamma = gamma; p.Bconst = Bconst; p.nb = nb; p.bcoef = bcoef; p.modes = modes;
    p.kmax = 0;
    for (int t = 0; t < nmodes * d; ++t) if (modes[t] > p.kmax) p.kmax = modes[t];
    long nnode = 1;
    for (int l = 0; l < d; ++l) nnode *= Nn;
    double *lossw = (double *)calloc((size_t)nnode, sizeof(double));
    if (!lossw) return -2;
    if (i_lo < 0 || i_hi > nnode || i_lo > i_hi) { free(lossw); return -1; }
    memset(gain, 0, sizeof(double) * (size_t)nmodes);
    int rc = run(&p, i_lo, i_hi, nthreads, gain, lossw, NULL);
    if (rc == 0) {
        double *tab = (double *)malloc(sizeof(double) * (size_t)d * (p.kmax + 1));
        double vi[ORACLE_MAX_D];
        memset(loss, 0, sizeof(double) * (size_t)nmodes);
        for (long i = i_lo; i < i_hi; ++i) {
            node_coords(&p, i, vi);
            for (int l = 0; l < d; ++l) that_1d(vi[l], S, r, p.kmax, tab + (size_t)l * (p.kmax + 1));
            for (int t = 0; t < nmodes; ++t) {
                double val = 1.0;
                for (int l = 0; l < d; ++l) val *= tab[(size_t)l * (p.kmax + 1) + modes[t * d + l]];
                loss[t] += lossw[i] * val;
            }
        }
        free(tab);
    }
    free(lossw);
    return rc;
}

/*
 * Weak-form functionals  sum_{i,j,m} qbar [phi(v') - phi(v_i)]  (Eq. weak, discretised)
 * for the test functions listed in phi (nphi x 3 ints, see phi_eval).  out[2t] is the
 * functional, out[2t+1] the scale sum qbar (|phi(v')| + |phi(v_i)|) used to normalise it.
 */
int pgb_oracle_weak(int d, int Nn, const double *v1d, const double *g, double Wnode,
                    int M, const double *sig, const double *wsig,
                    double S, int r, double gamma, double Bconst, int nb, const double *bcoef,
                    int nphi, const int *phi, double *out, int nthreads)
{
    if (d < 1 || d > ORACLE_MAX_D || Nn < 1 || M < 1 || nphi < 1 || nb < 0 || (nb > 0 && !bcoef)) return -1;
    prob_t p;
    memset(&p, 0, sizeof(p));
    p.d = d; p.Nn = Nn; p.M = M; p.r = r; p.nmodes = 0;
    p.v1d = v1d; p.g = g; p.Wnode = Wnode; p.sig = sig; p.wsig = wsig;
    p.S = S; p.gamma = gamma; p.Bconst = Bconst; p.nb = nb; p.bcoef = bcoef; p.nphi = nphi; p.phi = phi;
    long nnode = 1;
    for (int l = 0; l < d; ++l) nnode *= Nn;
    double *lossw = (double *)calloc((size_t)nnode, sizeof(double));
    if (!lossw) return -2;
    memset(out, 0, sizeof(double) * 2 * (size_t)nphi);
    int rc = run(&p, 0, nnode, nthreads, NULL, lossw, out);
    free(lossw);
    return rc;
}
