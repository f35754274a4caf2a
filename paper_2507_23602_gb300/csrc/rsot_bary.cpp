// Wasserstein barycenter with fixed uniform weights by the damped Lloyd
// iteration of Sec. 6.2 (Eq. damped_lloyd):
//   y_j <- (1 - theta) y_j + theta sum_i lambda_i T_ij,
//   T_ij = (1/nu_j) sum_q m_q^i p^i_qj x^i_q          (Eq. barycenter_fixed_point)
// where p^i is the optimal plan between source i and the current support
// (rsot_solve, warm-started from the previous iteration's potential), stopped
// when the RMS displacement of the support falls below tol_rms.
#include <math.h>
#include <string.h>

#include <chrono>
#include <vector>

#include "../../include/rsot.h"

extern "C" rsot_status rsot_barycenter(int K, const rsot_source_level *src, const double *lambda,
                                       int64_t n, double *y_inout, const double *nu,
                                       const rsot_options *opt, double theta, int max_iter,
                                       double tol_rms, rsot_barycenter_stats *stats) {
    if (K < 1 || !src || !lambda || n < 1 || !y_inout || !nu || !opt) return RSOT_ERR_ARG;
    if (!(theta > 0.0 && theta <= 1.0) || max_iter < 1 || !(tol_rms >= 0.0)) return RSOT_ERR_ARG;
    const int d = src[0].d;
    for (int i = 0; i < K; ++i)
        if (src[i].d != d || !(lambda[i] >= 0.0)) return RSOT_ERR_ARG;
    const auto t0 = std::chrono::steady_clock::now();
    double t_solve = 0.0, t_cent = 0.0;
    std::vector<std::vector<double>> psi(K, std::vector<double>(n, 0.0));
    std::vector<double> y(y_inout, y_inout + n * d), ybar(n * d), T(n * d);
    rsot_status st = RSOT_OK;
    int it = 0, solve_iters = 0, solve_evals = 0, converged = 0;
    double rms = INFINITY;
    for (; it < max_iter; ++it) {
        std::fill(ybar.begin(), ybar.end(), 0.0);
        for (int i = 0; i < K && !st; ++i) {
            rsot_problem *p = nullptr;
            st = rsot_create(d, src[i].nq, src[i].x, src[i].mass, n, y.data(), nu, 0, &p);
            if (st) break;
            rsot_options o = *opt;
            if (it > 0) o.eps_start = 0.0;   // warm start: the support moved little
            rsot_solve_stats ss;
            auto a = std::chrono::steady_clock::now();
            rsot_status s = rsot_solve(p, psi[i].data(), &o, &ss);
            auto b = std::chrono::steady_clock::now();
            t_solve += std::chrono::duration<double>(b - a).count();
            solve_iters += ss.iters;
            solve_evals += ss.evals;
            if (s && s != RSOT_ERR_NOT_CONVERGED && s != RSOT_ERR_LINESEARCH) st = s;
            if (!st) st = rsot_centroids(p, psi[i].data(), o.eps, T.data(), nullptr);
            t_cent += std::chrono::duration<double>(std::chrono::steady_clock::now() - b).count();
            rsot_destroy(p);
            if (st) break;
            for (int64_t k = 0; k < n * d; ++k) ybar[k] += lambda[i] * T[k];
        }
        if (st) break;
        double ss = 0.0;
        for (int64_t k = 0; k < n * d; ++k) {
            const double ynew = (1.0 - theta) * y[k] + theta * ybar[k];
            ss += (ynew - y[k]) * (ynew - y[k]);
            y[k] = ynew;
        }
        rms = sqrt(ss / (double)n);
        if (rms <= tol_rms) {
            converged = 1;
            ++it;
            break;
        }
    }
    if (!st) memcpy(y_inout, y.data(), sizeof(double) * n * d);
    if (stats) {
        stats->iterations = it;
        stats->rms_last = rms;
        stats->converged = converged;
        stats->solve_iters = solve_iters;
        stats->solve_evals = solve_evals;
        stats->seconds_solve = t_solve;
        stats->seconds_centroids = t_cent;
        stats->seconds_total =
            std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    }
    return st;
}
