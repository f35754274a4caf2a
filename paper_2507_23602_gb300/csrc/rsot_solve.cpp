// Host driver: FP64 L-BFGS with a strong-Wolfe line search (Algorithm 1),
// the eps-schedule with warm start (Sec. 4.2), the L1 gradient stop
// (Remark 3.3), and mixed -> FP64 refinement of the last stage.
//
// The L-BFGS details are not fixed by the paper.  This driver uses
//   * the two-loop recursion with memory m and a diagonal initial matrix
//     H0 = gamma * diag(eps / nu_j): near the optimum the Hessian diagonal of
//     J is (1/eps) sum_q m_q p_qj (1 - p_qj) ~ nu_j / eps, so this H0 makes
//     the very first step a Newton-like step; gamma = s^T y / y^T D y;
//   * a strong-Wolfe line search (c1 = 1e-4, c2 = 0.9): expansion by 2x, then
//     sectioning with a safeguarded cubic fit;
//   * where J differs from J(0) only by its evaluation noise (|dJ| <= tolJ,
//     tolJ = 1e-13 |J| for FP64, 1e-6 |J| for mixed precision), Hager &
//     Zhang's approximate Wolfe test sigma d0 <= d <= (2 c1 - 1) d0
//     replaces sufficient decrease.
// With MIXED precision and refine_fp64, the last stage switches to FP64
// evaluations when it converges under mixed precision or when the mixed
// line search stalls, and finishes there.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <deque>
#include <vector>

#include "../../include/rsot.h"

namespace rsot {
int64_t num_targets(const rsot_problem *p);
void copy_nu(const rsot_problem *p, double *out);
}  // namespace rsot

namespace {

struct Evaluator {
    rsot_problem *p;
    int64_t n;
    double eps;
    double tail;
    rsot_precision prec;
    int evals = 0;
    int64_t pairs = 0;
    rsot_status last = RSOT_OK;

    rsot_status operator()(const std::vector<double> &psi, double &J, std::vector<double> &g) {
        double radius = 0.0;
        if (tail > 0.0) {
            rsot_status s = rsot_radius_for_tail(p, psi.data(), eps, tail, &radius);
            if (s) return last = s;
        }
        int64_t pr = 0;
        rsot_status s = rsot_eval_dual_grad(p, psi.data(), eps, radius, prec, &J, g.data(), &pr);
        ++evals;
        pairs += pr;
        return last = s;
    }
};

double dot(const std::vector<double> &a, const std::vector<double> &b) {
    double s = 0.0;
    for (size_t i = 0; i < a.size(); ++i) s += a[i] * b[i];
    return s;
}

double norm1(const std::vector<double> &a) {
    double s = 0.0;
    for (double v : a) s += fabs(v);
    return s;
}

struct Pair {
    std::vector<double> s, y;
    double rho;
};

// Minimiser of the cubic matching (a,fa,da), (b,fb,db); NaN if none.
double cubic_step(double a, double fa, double da, double b, double fb, double db) {
    const double t = da + db - 3.0 * (fa - fb) / (a - b);
    const double r = t * t - da * db;
    if (!(r >= 0.0) || a == b) return NAN;
    const double s = (b > a ? 1.0 : -1.0) * sqrt(r);
    const double den = db - da + 2.0 * s;
    if (den == 0.0) return NAN;
    return b - (b - a) * (db + s - t) / den;
}

struct Trial {
    double a, f, d;
    std::vector<double> g;
};

// Strong-Wolfe line search along p from (x, f0, g0); on success x_new, f, g are set.
rsot_status wolfe_search(Evaluator &ev, const std::vector<double> &x, double f0,
                         const std::vector<double> &g0, const std::vector<double> &p, double noise,
                         std::vector<double> &x_new, double &f_new, std::vector<double> &g_new) {
    const double c1 = 1e-4, c2 = 0.9;
    const double d0 = dot(g0, p);
    const size_t n = x.size();
    std::vector<double> xt(n), gt(n);
    int budget = 30;

    auto eval = [&](double a, Trial &t) -> rsot_status {
        for (size_t i = 0; i < n; ++i) xt[i] = x[i] + a * p[i];
        double f;
        rsot_status s = ev(xt, f, gt);
        if (s) return s;
        t.a = a;
        t.f = f;
        t.d = dot(gt, p);
        t.g = gt;
        --budget;
        return RSOT_OK;
    };
    auto accept = [&](const Trial &t) {
        for (size_t i = 0; i < n; ++i) x_new[i] = x[i] + t.a * p[i];
        f_new = t.f;
        g_new = t.g;
        return RSOT_OK;
    };
    auto flat_ok = [&](const Trial &t) {
        return fabs(t.f - f0) <= noise && c2 * d0 <= t.d && t.d <= (2.0 * c1 - 1.0) * d0;
    };
    auto strong = [&](const Trial &t) { return fabs(t.d) <= -c2 * d0; };
    auto armijo = [&](const Trial &t) { return t.f <= f0 + c1 * t.a * d0; };

    Trial lo{0.0, f0, d0, g0}, hi{}, cur{};
    double a = 1.0;
    bool bracketed = false;
    // expansion phase
    while (budget > 0) {
        rsot_status s = eval(a, cur);
        if (s) return s;
        if (flat_ok(cur)) return accept(cur);
        if (!armijo(cur) || (lo.a > 0.0 && cur.f >= lo.f)) {
            hi = cur;
            bracketed = true;
            break;
        }
        if (strong(cur)) return accept(cur);
        if (cur.d >= 0.0) {
            hi = lo;
            lo = cur;
            bracketed = true;
            break;
        }
        lo = cur;
        a *= 2.0;
    }
    if (!bracketed) return RSOT_ERR_LINESEARCH;
    // sectioning phase: lo satisfies Armijo and has the lowest f so far
    while (budget > 0) {
        const double left = std::min(lo.a, hi.a), right = std::max(lo.a, hi.a);
        const double w = right - left;
        if (w <= 1e-16 * std::max(1.0, right)) break;
        double at = cubic_step(lo.a, lo.f, lo.d, hi.a, hi.f, hi.d);
        if (!(at > left + 0.1 * w && at < right - 0.1 * w)) at = 0.5 * (left + right);
        rsot_status s = eval(at, cur);
        if (s) return s;
        if (flat_ok(cur)) return accept(cur);
        if (!armijo(cur) || cur.f >= lo.f) {
            hi = cur;
        } else {
            if (strong(cur)) return accept(cur);
            if (cur.d * (hi.a - lo.a) >= 0.0) hi = lo;
            lo = cur;
        }
    }
    // no strong-Wolfe point: take the best Armijo point if it moved
    if (lo.a > 0.0 && lo.f < f0) return accept(lo);
    return RSOT_ERR_LINESEARCH;
}

// One L-BFGS run at fixed eps and precision.
rsot_status lbfgs_stage(Evaluator &ev, std::vector<double> &x, double &f, std::vector<double> &g,
                        bool have_fg, double tol, int m, int max_iter, const std::vector<double> &D,
                        int &iters, int verbose) {
    const size_t n = x.size();
    if (!have_fg) {
        rsot_status s = ev(x, f, g);
        if (s) return s;
    }
    std::deque<Pair> hist;
    std::vector<double> q(n), p(n), alpha(m), xn(n), gn(n);
    const double noise_rel = ev.prec == RSOT_FP64 ? 1e-13 : 1e-6;
    for (int it = 0;; ++it) {
        const double gl1 = norm1(g);
        if (verbose)
            fprintf(stderr, "[rsot] eps=%.3g %s it=%d J=%.15g |g|_1=%.3e evals=%d\n", ev.eps,
                    ev.prec == RSOT_FP64 ? "fp64" : "mixed", it, f, gl1, ev.evals);
        if (gl1 <= tol) return RSOT_OK;
        if (it >= max_iter) return RSOT_ERR_NOT_CONVERGED;
        // two-loop recursion with H0 = gamma D
        q = g;
        const int k = (int)hist.size();
        for (int i = k - 1; i >= 0; --i) {
            alpha[i] = hist[i].rho * dot(hist[i].s, q);
            for (size_t t = 0; t < n; ++t) q[t] -= alpha[i] * hist[i].y[t];
        }
        double gamma = 1.0;
        if (k > 0) {
            const Pair &l = hist.back();
            double yDy = 0.0;
            for (size_t t = 0; t < n; ++t) yDy += l.y[t] * D[t] * l.y[t];
            gamma = (1.0 / l.rho) / yDy;
        }
        for (size_t t = 0; t < n; ++t) q[t] *= gamma * D[t];
        for (int i = 0; i < k; ++i) {
            const double b = hist[i].rho * dot(hist[i].y, q);
            for (size_t t = 0; t < n; ++t) q[t] += (alpha[i] - b) * hist[i].s[t];
        }
        for (size_t t = 0; t < n; ++t) p[t] = -q[t];
        if (dot(g, p) >= 0.0) {   // not a descent direction: restart along -D g
            hist.clear();
            for (size_t t = 0; t < n; ++t) p[t] = -D[t] * g[t];
        }
        const double noise = noise_rel * std::max(fabs(f), 1e-300);
        rsot_status s = wolfe_search(ev, x, f, g, p, noise, xn, f, gn);
        if (s) return s;
        Pair pr;
        pr.s.resize(n);
        pr.y.resize(n);
        for (size_t t = 0; t < n; ++t) {
            pr.s[t] = xn[t] - x[t];
            pr.y[t] = gn[t] - g[t];
        }
        const double sy = dot(pr.s, pr.y);
        if (sy > 0.0) {
            pr.rho = 1.0 / sy;
            hist.push_back(std::move(pr));
            if ((int)hist.size() > m) hist.pop_front();
        }
        x.swap(xn);
        g.swap(gn);
        ++iters;
    }
}

}  // namespace

extern "C" {

void rsot_default_options(rsot_options *o) {
    if (!o) return;
    memset(o, 0, sizeof(*o));
    o->eps = 1e-2;
    o->eps_start = 0.0;
    o->eps_factor = 0.5;
    o->tail = 0.0;
    o->tol_l1 = 1e-6;
    o->stage_tol_l1 = 0.0;
    o->precision = RSOT_MIXED;
    o->refine_fp64 = 1;
    o->lbfgs_m = 10;
    o->max_iter = 10000;
    o->verbose = 0;
}

rsot_status rsot_solve(rsot_problem *p, double *psi_inout, const rsot_options *opt,
                       rsot_solve_stats *stats) {
    if (!p || !psi_inout || !opt) return RSOT_ERR_ARG;
    if (!(opt->eps > 0.0) || !(opt->tol_l1 > 0.0) || opt->tail < 0.0 || opt->tail >= 1.0)
        return RSOT_ERR_ARG;
    if (opt->precision != RSOT_FP64 && opt->precision != RSOT_MIXED) return RSOT_ERR_ARG;
    const auto t0 = std::chrono::steady_clock::now();
    const int64_t n = rsot::num_targets(p);
    std::vector<double> nu(n);
    rsot::copy_nu(p, nu.data());
    // eps stages
    std::vector<double> eps_list;
    if (opt->eps_start > opt->eps && opt->eps_factor > 0.0 && opt->eps_factor < 1.0) {
        for (double e = opt->eps_start; e > opt->eps * (1.0 + 1e-12); e *= opt->eps_factor)
            eps_list.push_back(e);
    }
    eps_list.push_back(opt->eps);

    const int m = opt->lbfgs_m > 0 ? opt->lbfgs_m : 10;
    const int max_iter = opt->max_iter > 0 ? opt->max_iter : 10000;
    const double stage_tol = opt->stage_tol_l1 > 0.0 ? opt->stage_tol_l1 : opt->tol_l1;

    std::vector<double> x(psi_inout, psi_inout + n), g(n), D(n);
    double f = 0.0;
    int iters = 0, evals = 0, stages = 0;
    int64_t pairs = 0;
    rsot_status st = RSOT_OK;
    for (size_t si = 0; si < eps_list.size(); ++si) {
        const double eps = eps_list[si];
        const bool last = si + 1 == eps_list.size();
        const double tol = last ? opt->tol_l1 : stage_tol;
        for (int64_t j = 0; j < n; ++j) D[j] = eps / nu[j];
        Evaluator ev{p, n, eps, opt->tail, (rsot_precision)opt->precision};
        ++stages;
        st = lbfgs_stage(ev, x, f, g, false, tol, m, max_iter, D, iters, opt->verbose);
        evals += ev.evals;
        pairs += ev.pairs;
        const bool refine = last && opt->precision == RSOT_MIXED && opt->refine_fp64;
        if (refine && (st == RSOT_OK || st == RSOT_ERR_LINESEARCH)) {
            Evaluator ev64{p, n, eps, opt->tail, RSOT_FP64};
            st = lbfgs_stage(ev64, x, f, g, false, tol, m, max_iter, D, iters, opt->verbose);
            evals += ev64.evals;
            pairs += ev64.pairs;
        }
        if (st != RSOT_OK && !(st == RSOT_ERR_LINESEARCH && !last)) break;
        st = RSOT_OK;
    }
    std::copy(x.begin(), x.end(), psi_inout);
    if (stats) {
        stats->J = f;
        stats->grad_l1 = norm1(g);
        stats->iters = iters;
        stats->evals = evals;
        stats->stages = stages;
        stats->pairs = pairs;
        stats->seconds =
            std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    }
    return st;
}

}  // extern "C"
