/*
 * RSOT oracle -- TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow, FP64 CPU statement of what the semi-discrete entropic dual
 * evaluation computes.  Only the test suite, the smoke check and the CPU
 * baseline leg of the benchmark may load this library; the product path
 * never does.  It shares no code, header or constant with the CUDA path.
 *
 * Notation (Sec. 2-3): quadrature points x_q with masses m_q, targets y_j
 * with weights nu_j, potentials psi_j, regularisation eps, cost
 * c(x,y) = 1/2 |x - y|^2.
 *
 *   s_qj      = (psi_j - c(x_q, y_j)) / eps + ln nu_j
 *   J(psi)    = sum_q m_q eps ln sum_j exp(s_qj) - sum_j psi_j nu_j     (Eq. discretized_functional)
 *   dJ/dpsi_k = sum_q m_q p_qk - nu_k,  p_qk = exp(s_qk) / sum_j exp(s_qj)
 *                                                       (Eq. discretized_gradient, Eq. final_plan_density)
 *
 * The loop structure is Algorithm 2: for every quadrature point, gather
 * I_q = { j : c(x_q, y_j) < C } (here by testing every j: no index), form
 * S_q, add eps ln S_q m_q to J and scatter m_q T_qj / S_q into the gradient;
 * then subtract sum psi nu and nu.  A cutoff C = +inf gives the dense
 * evaluation.  Two readings are applied:
 *   - ln S_q is evaluated as max_j s_qj + ln sum_j exp(s_qj - max), the same
 *     number without the underflow of exp(s) at small eps;  the guard
 *     "S_q > 0" of Algorithm 2 therefore becomes "I_q is not empty".
 *   - sums use Neumaier compensation; the point loop is split over OpenMP
 *     threads with thread-local gradients merged in thread order
 *     (Remark 4.1, the paper's own shared-memory scheme).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef struct {
    double s;
    double c;
} nsum_t;

static void nadd(nsum_t *a, double v)
{
    double t = a->s + v;
    if (fabs(a->s) >= fabs(v))
        a->c += (a->s - t) + v;
    else
        a->c += (v - t) + a->s;
    a->s = t;
}

static double nval(const nsum_t *a) { return a->s + a->c; }

static double cost(int d, const double *x, const double *y)
{
    double r = 0.0;
    for (int k = 0; k < d; ++k) {
        double t = x[k] - y[k];
        r += t * t;
    }
    return 0.5 * r;
}

static int nthreads_of(int requested)
{
#ifdef _OPENMP
    return requested > 0 ? requested : omp_get_max_threads();
#else
    (void)requested;
    return 1;
#endif
}

int oracle_threads_used(int requested) { return nthreads_of(requested); }

/*
 * Algorithm 2 (dense when cutoff = +inf).
 * x: nq*d row-major, mass: nq, y: n*d row-major, nu: n, psi: n.
 * Membership: c(x_q, y_j) < cutoff, or, when alpha and beta are given,
 * c(x_q, y_j) < alpha_q + beta_j (a cutoff per pair, separable).
 * Outputs: *J_out, grad_out[n]; optional pairs_out = sum_q |I_q|,
 * empty_out = number of points with an empty I_q.
 * Returns 0 on success, -1 on bad arguments, -2 on allocation failure.
 */
static int dual_grad_impl(int d, int64_t nq, const double *x, const double *mass,
                          int64_t n, const double *y, const double *nu, const double *psi,
                          double eps, double cutoff, const double *alpha, const double *beta,
                          int threads, double *J_out, double *grad_out, int64_t *pairs_out,
                          int64_t *empty_out)
{
    if (d < 1 || d > 3 || nq < 0 || n < 1 || !(eps > 0.0))
        return -1;
    int T = nthreads_of(threads);
    nsum_t *gpart = (nsum_t *)calloc((size_t)T * (size_t)n, sizeof(nsum_t));
    nsum_t *jpart = (nsum_t *)calloc((size_t)T, sizeof(nsum_t));
    int64_t *ppart = (int64_t *)calloc((size_t)T, sizeof(int64_t));
    int64_t *epart = (int64_t *)calloc((size_t)T, sizeof(int64_t));
    double *sbuf = (double *)malloc((size_t)T * (size_t)n * sizeof(double));
    unsigned char *inbuf = (unsigned char *)malloc((size_t)T * (size_t)n);
    if (!gpart || !jpart || !ppart || !epart || !sbuf || !inbuf) {
        free(gpart); free(jpart); free(ppart); free(epart); free(sbuf); free(inbuf);
        return -2;
    }

#ifdef _OPENMP
#pragma omp parallel num_threads(T)
#endif
    {
#ifdef _OPENMP
        int t = omp_get_thread_num();
#else
        int t = 0;
#endif
        nsum_t *g = gpart + (size_t)t * (size_t)n;
        double *s = sbuf + (size_t)t * (size_t)n;
        unsigned char *in = inbuf + (size_t)t * (size_t)n;
#ifdef _OPENMP
#pragma omp for schedule(static)
#endif
        for (int64_t q = 0; q < nq; ++q) {
            const double *xq = x + q * d;
            /* I_q and the exponents s_qj */
            double smax = -INFINITY;
            int64_t cnt = 0;
            for (int64_t j = 0; j < n; ++j) {
                double c = cost(d, xq, y + j * d);
                in[j] = (unsigned char)(alpha ? c < alpha[q] + beta[j] : c < cutoff);
                if (in[j]) {
                    s[j] = (psi[j] - c) / eps + log(nu[j]);
                    if (s[j] > smax)
                        smax = s[j];
                    ++cnt;
                }
            }
            ppart[t] += cnt;
            if (cnt == 0) {          /* S_q = 0: the point is skipped */
                epart[t] += 1;
                continue;
            }
            /* S_q = sum_{j in I_q} nu_j exp((psi_j - c)/eps), max-shifted */
            nsum_t S = {0.0, 0.0};
            for (int64_t j = 0; j < n; ++j)
                if (in[j])
                    nadd(&S, exp(s[j] - smax));
            double lnS = smax + log(nval(&S));
            nadd(&jpart[t], mass[q] * eps * lnS);
            /* scatter m_q T_qj / S_q */
            for (int64_t j = 0; j < n; ++j)
                if (in[j])
                    nadd(&g[j], mass[q] * exp(s[j] - lnS));
        }
    }

    nsum_t J = {0.0, 0.0};
    for (int t = 0; t < T; ++t)
        nadd(&J, nval(&jpart[t]));
    for (int64_t j = 0; j < n; ++j)
        nadd(&J, -psi[j] * nu[j]);
    for (int64_t j = 0; j < n; ++j) {
        nsum_t a = {0.0, 0.0};
        for (int t = 0; t < T; ++t)
            nadd(&a, nval(&gpart[(size_t)t * (size_t)n + (size_t)j]));
        nadd(&a, -nu[j]);
        grad_out[j] = nval(&a);
    }
    *J_out = nval(&J);
    if (pairs_out) {
        int64_t p = 0;
        for (int t = 0; t < T; ++t) p += ppart[t];
        *pairs_out = p;
    }
    if (empty_out) {
        int64_t e = 0;
        for (int t = 0; t < T; ++t) e += epart[t];
        *empty_out = e;
    }
    free(gpart); free(jpart); free(ppart); free(epart); free(sbuf); free(inbuf);
    return 0;
}

int oracle_dual_grad(int d, int64_t nq, const double *x, const double *mass,
                     int64_t n, const double *y, const double *nu, const double *psi,
                     double eps, double cutoff, int threads,
                     double *J_out, double *grad_out, int64_t *pairs_out, int64_t *empty_out)
{
    return dual_grad_impl(d, nq, x, mass, n, y, nu, psi, eps, cutoff, NULL, NULL, threads,
                          J_out, grad_out, pairs_out, empty_out);
}

/* Algorithm 2 with I_q = { j : c(x_q, y_j) < alpha_q + beta_j }. */
int oracle_dual_grad_sep(int d, int64_t nq, const double *x, const double *mass,
                         int64_t n, const double *y, const double *nu, const double *psi,
                         double eps, const double *alpha, const double *beta, int threads,
                         double *J_out, double *grad_out, int64_t *pairs_out, int64_t *empty_out)
{
    if (!alpha || !beta)
        return -1;
    return dual_grad_impl(d, nq, x, mass, n, y, nu, psi, eps, INFINITY, alpha, beta, threads,
                          J_out, grad_out, pairs_out, empty_out);
}

/*
 * Nearest target of every point: j_out[q] = argmin_j c(x_q, y_j) (the lowest
 * index among equal costs), c_out[q] = that cost.  Brute force in FP64.
 */
int oracle_nearest(int d, int64_t nq, const double *x, int64_t n, const double *y, int threads,
                   int64_t *j_out, double *c_out)
{
    if (d < 1 || d > 3 || nq < 0 || n < 1)
        return -1;
    int T = nthreads_of(threads);
#ifdef _OPENMP
#pragma omp parallel for num_threads(T) schedule(static)
#endif
    for (int64_t q = 0; q < nq; ++q) {
        double best = INFINITY;
        int64_t bj = 0;
        for (int64_t j = 0; j < n; ++j) {
            double c = cost(d, x + q * d, y + j * d);
            if (c < best) {
                best = c;
                bj = j;
            }
        }
        j_out[q] = bj;
        c_out[q] = best;
    }
    (void)T;
    return 0;
}

/*
 * The plan density p_j(x_q | psi) of Eq. final_plan_density for every pair,
 * P[q*n + j] (dense, small inputs only).
 */
int oracle_plan(int d, int64_t nq, const double *x, int64_t n, const double *y,
                const double *nu, const double *psi, double eps, double *P)
{
    if (d < 1 || d > 3 || n < 1 || !(eps > 0.0))
        return -1;
    for (int64_t q = 0; q < nq; ++q) {
        double *row = P + q * n;
        double smax = -INFINITY;
        for (int64_t j = 0; j < n; ++j) {
            row[j] = (psi[j] - cost(d, x + q * d, y + j * d)) / eps + log(nu[j]);
            if (row[j] > smax)
                smax = row[j];
        }
        nsum_t S = {0.0, 0.0};
        for (int64_t j = 0; j < n; ++j)
            nadd(&S, exp(row[j] - smax));
        double lnS = smax + log(nval(&S));
        for (int64_t j = 0; j < n; ++j)
            row[j] = exp(row[j] - lnS);
    }
    return 0;
}

/*
 * Per-point log partition L_q = ln sum_j nu_j exp((psi_j - c(x_q, y_j))/eps),
 * the quantity whose eps-multiple is integrated in Eq. discretized_functional
 * (and whose exponential is the denominator of Eq. final_plan_density),
 * max-shifted.  Dense only.
 */
/* L_q = ln S_trunc(x_q) = ln sum_{j : c(x_q, y_j) < cutoff} nu_j exp((psi_j - c)/eps)
 * (-inf for an empty I_q; cutoff = +inf: every j). */
int oracle_point_lse_cut(int d, int64_t nq, const double *x, int64_t n, const double *y,
                         const double *nu, const double *psi, double eps, double cutoff,
                         int threads, double *L)
{
    if (d < 1 || d > 3 || n < 1 || !(eps > 0.0))
        return -1;
    int T = nthreads_of(threads);
#ifdef _OPENMP
#pragma omp parallel for num_threads(T) schedule(static)
#endif
    for (int64_t q = 0; q < nq; ++q) {
        double smax = -INFINITY;
        for (int64_t j = 0; j < n; ++j) {
            double c = cost(d, x + q * d, y + j * d);
            if (!(c < cutoff))
                continue;
            double s = (psi[j] - c) / eps + log(nu[j]);
            if (s > smax)
                smax = s;
        }
        if (smax == -INFINITY) {
            L[q] = -INFINITY;
            continue;
        }
        nsum_t S = {0.0, 0.0};
        for (int64_t j = 0; j < n; ++j) {
            double c = cost(d, x + q * d, y + j * d);
            if (c < cutoff)
                nadd(&S, exp((psi[j] - c) / eps + log(nu[j]) - smax));
        }
        L[q] = smax + log(nval(&S));
    }
    return 0;
}

int oracle_point_lse(int d, int64_t nq, const double *x, int64_t n, const double *y,
                     const double *nu, const double *psi, double eps, int threads, double *L)
{
    return oracle_point_lse_cut(d, nq, x, n, y, nu, psi, eps, INFINITY, threads, L);
}

/* Covering cost C_0 = max_q min_j c(x_q, y_j) over the quadrature points
 * (App. B, the discrete counterpart of the max over the domain). */
int oracle_covering_cost(int d, int64_t nq, const double *x, int64_t n, const double *y,
                         int threads, double *C0_out)
{
    if (d < 1 || d > 3 || n < 1)
        return -1;
    int T = nthreads_of(threads);
    double best = 0.0;
#ifdef _OPENMP
#pragma omp parallel for num_threads(T) schedule(static) reduction(max : best)
#endif
    for (int64_t q = 0; q < nq; ++q) {
        double mn = INFINITY;
        for (int64_t j = 0; j < n; ++j) {
            double c = cost(d, x + q * d, y + j * d);
            if (c < mn)
                mn = c;
        }
        if (mn > best)
            best = mn;
    }
    *C0_out = best;
    return 0;
}

/*
 * Softmax refinement (Eq. softmax_refinement_formula): with the coarse
 * potential psi_c on coarse targets (y_c, nu_c),
 *   psi_k^init = -eps ln sum_q m_q exp(-c(x_q, y_k)/eps) / S_c(x_q),
 *   S_c(x) = sum_j nu_c_j exp((psi_c_j - c(x, y_c_j))/eps),
 * the source integral taken with the quadrature masses.  Both sums are
 * evaluated in the log domain with a max shift.
 */
int oracle_softmax_refine(int d, int64_t nq, const double *x, const double *mass,
                          int64_t nc, const double *yc, const double *nuc, const double *psic,
                          int64_t nf, const double *yf, double eps, int threads, double *psi_out)
{
    if (d < 1 || d > 3 || nc < 1 || nf < 1 || !(eps > 0.0))
        return -1;
    int T = nthreads_of(threads);
    double *lnS = (double *)malloc((size_t)(nq > 0 ? nq : 1) * sizeof(double));
    if (!lnS)
        return -2;
#ifdef _OPENMP
#pragma omp parallel for num_threads(T) schedule(static)
#endif
    for (int64_t q = 0; q < nq; ++q) {
        double smax = -INFINITY;
        for (int64_t j = 0; j < nc; ++j) {
            double s = (psic[j] - cost(d, x + q * d, yc + j * d)) / eps + log(nuc[j]);
            if (s > smax)
                smax = s;
        }
        nsum_t S = {0.0, 0.0};
        for (int64_t j = 0; j < nc; ++j)
            nadd(&S, exp((psic[j] - cost(d, x + q * d, yc + j * d)) / eps + log(nuc[j]) - smax));
        lnS[q] = smax + log(nval(&S));
    }
#ifdef _OPENMP
#pragma omp parallel for num_threads(T) schedule(static)
#endif
    for (int64_t k = 0; k < nf; ++k) {
        double tmax = -INFINITY;
        for (int64_t q = 0; q < nq; ++q) {
            if (!(mass[q] > 0.0))
                continue;
            double t = log(mass[q]) - cost(d, x + q * d, yf + k * d) / eps - lnS[q];
            if (t > tmax)
                tmax = t;
        }
        nsum_t A = {0.0, 0.0};
        for (int64_t q = 0; q < nq; ++q) {
            if (!(mass[q] > 0.0))
                continue;
            nadd(&A, exp(log(mass[q]) - cost(d, x + q * d, yf + k * d) / eps - lnS[q] - tmax));
        }
        psi_out[k] = -eps * (tmax + log(nval(&A)));
    }
    free(lnS);
    return 0;
}

/*
 * Transport maps of Sec. 6.3 for every quadrature point (dense):
 *   T_bary(x_q) = sum_j p_qj y_j        (Eq. barycentric_map_registration)
 *   j*(q)       = argmax_j s_qj,  s_qj = (psi_j - c(x_q, y_j))/eps + ln nu_j
 *                                       (Eq. modal_map_registration; the
 *                                       first maximal j on ties)
 * p_qj is the plan density of Eq. final_plan_density, max-shifted; the
 * weighted sum uses Neumaier compensation per coordinate.
 * Outputs: Tbary[q*d + k] (may be NULL), jstar[q] (may be NULL).
 */
int oracle_transport_maps(int d, int64_t nq, const double *x, int64_t n, const double *y,
                          const double *nu, const double *psi, double eps, int threads,
                          double *Tbary, int64_t *jstar)
{
    if (d < 1 || d > 3 || n < 1 || !(eps > 0.0))
        return -1;
    int T = nthreads_of(threads);
#ifdef _OPENMP
#pragma omp parallel for num_threads(T) schedule(static)
#endif
    for (int64_t q = 0; q < nq; ++q) {
        double smax = -INFINITY;
        int64_t arg = 0;
        for (int64_t j = 0; j < n; ++j) {
            double s = (psi[j] - cost(d, x + q * d, y + j * d)) / eps + log(nu[j]);
            if (s > smax) {
                smax = s;
                arg = j;
            }
        }
        if (jstar)
            jstar[q] = arg;
        if (!Tbary)
            continue;
        nsum_t S = {0.0, 0.0}, W[3] = {{0.0, 0.0}, {0.0, 0.0}, {0.0, 0.0}};
        for (int64_t j = 0; j < n; ++j) {
            double e = exp((psi[j] - cost(d, x + q * d, y + j * d)) / eps + log(nu[j]) - smax);
            nadd(&S, e);
            for (int k = 0; k < d; ++k)
                nadd(&W[k], e * y[j * d + k]);
        }
        for (int k = 0; k < d; ++k)
            Tbary[q * d + k] = nval(&W[k]) / nval(&S);
    }
    return 0;
}

/*
 * Conditional centroids of the plan (Eq. barycenter_fixed_point):
 *   T_j = (1/nu_j) sum_q m_q p_qj x_q,   and the transported mass
 *   a_j = sum_q m_q p_qj (= nu_j at the optimum, Eq. gradient_compact_expanded).
 * Dense.  Outputs: T[j*d + k], a[j] (may be NULL).
 */
int oracle_centroids(int d, int64_t nq, const double *x, const double *mass, int64_t n,
                     const double *y, const double *nu, const double *psi, double eps,
                     double *Tc, double *a_out)
{
    if (d < 1 || d > 3 || n < 1 || !(eps > 0.0))
        return -1;
    nsum_t *A = (nsum_t *)calloc((size_t)n * 4, sizeof(nsum_t));
    double *row = (double *)malloc((size_t)n * sizeof(double));
    if (!A || !row) {
        free(A);
        free(row);
        return -2;
    }
    for (int64_t q = 0; q < nq; ++q) {
        double smax = -INFINITY;
        for (int64_t j = 0; j < n; ++j) {
            row[j] = (psi[j] - cost(d, x + q * d, y + j * d)) / eps + log(nu[j]);
            if (row[j] > smax)
                smax = row[j];
        }
        nsum_t S = {0.0, 0.0};
        for (int64_t j = 0; j < n; ++j)
            nadd(&S, exp(row[j] - smax));
        const double lnS = smax + log(nval(&S));
        for (int64_t j = 0; j < n; ++j) {
            const double w = mass[q] * exp(row[j] - lnS);   /* m_q p_qj */
            nadd(&A[j * 4 + 3], w);
            for (int k = 0; k < d; ++k)
                nadd(&A[j * 4 + k], w * x[q * d + k]);
        }
    }
    for (int64_t j = 0; j < n; ++j) {
        for (int k = 0; k < d; ++k)
            Tc[j * d + k] = nval(&A[j * 4 + k]) / nu[j];
        if (a_out)
            a_out[j] = nval(&A[j * 4 + 3]);
    }
    free(A);
    free(row);
    return 0;
}
