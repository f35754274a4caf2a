// Host driver: FP64 L-BFGS with a strong-Wolfe line search (Algorithm 1),
// the eps-schedule with warm start (Sec. 4.2), the L1 gradient stop
// (Remark 3.3), and mixed -> FP64 refinement of the last stage.  The L-BFGS
// itself is the resumable machine of rsot_lbfgs.h; here one problem drives it
// with one GPU evaluation per request.
//
// The L-BFGS details are not fixed by the paper.  The machine uses
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
// With MIXED precision and refine_fp64, the last stage runs mixed evaluations
// down to mixed_tol_l1 (default 1e-5, above the FP32 rounding floor of the
// gradient), then refines on reference evaluations, always dense (the stop
// holds for the untruncated J whatever truncation the mixed phase used; the
// correction absorbs the difference).  The reference is the
// compensated evaluation (rsot_df.cu), stopped at tol - B with B = 6.5e-7
// sum m_q its certified gradient error, so that ||grad J||_1 <= tol holds.  At
// about ten mixed evaluations per compensated one, one correction (as below)
// runs mixed L-BFGS on the corrected objective until its rounding noise stops
// it, then L-BFGS on compensated evaluations finishes.  Where B leaves too
// little room under tol (or on request) the reference is FP64, three hundred
// times dearer than a mixed evaluation; then a reference and a mixed
// evaluation at the iterate give the
// systematic mixed-precision error, mixed L-BFGS continues on the corrected
// objective (at most 200 iterations per correction) until the FP64 gradient
// meets tol, and when a correction no longer halves the FP64 gradient (tol
// below the mixed noise floor) plain FP64 L-BFGS finishes.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <deque>
#include <vector>

#include "../../include/rsot.h"
#include "rsot_lbfgs.h"

namespace rsot {
int64_t num_targets(const rsot_problem *p);
int64_t num_points(const rsot_problem *p);
double mass_sum(const rsot_problem *p);
void copy_nu(const rsot_problem *p, double *out);
int pair_kernel_of(const rsot_problem *p);
void pair_kernel_for_gradient(rsot_problem *p, double grad_l1);
void set_in_solve(rsot_problem *p, int on);
}  // namespace rsot

namespace {

// evaluations and pairs by precision over one solve
struct PrecCount {
    int evals[3] = {0, 0, 0};
    int64_t pairs[3] = {0, 0, 0};
};

// Cutoff of a truncated evaluation (Sec. 4.1): none (dense), the psi-aware
// cutoffs of a tail tolerance, or one of the paper's global cutoffs C_int,
// C_pw, C_geom (rsot_truncation_cutoff).
struct Truncation {
    double tail = 0.0, tau_int = 0.0, delta_pw = 0.0, tau_geom = 0.0;
};

// Kept fraction of all pairs above which a truncated evaluation of the
// psi-aware cutoffs costs about as much as a dense one (the block-skip passes
// take 0.77 of the dense time at 16.5 % kept and 1.4 times at 83 %): an
// eps-stage whose first truncated evaluation keeps more runs dense.  The dense
// functional differs from the truncated one by at most the tail tolerance.
constexpr double kTailDenseFraction = 0.35;

struct Evaluator {
    rsot_problem *p;
    int64_t n;
    double eps;
    Truncation tr;
    rsot_precision prec;
    PrecCount *count = nullptr;
    int evals = 0;
    int64_t pairs = 0;
    int64_t skipped = 0;      // points left without a target (C_pw, C_geom), summed
    rsot_status last = RSOT_OK;
    bool have_prev = false;   // ln D and J of the previous evaluation (C_int, C_geom)
    double lnD_prev = 0.0, J_prev = 0.0;
    bool probed = false;      // tail mode: the first evaluation has chosen the form
    bool tail_dense = false;  // tail mode: this evaluator's evaluations run dense

    rsot_status operator()(const std::vector<double> &psi, double &J, std::vector<double> &g) {
        int64_t pr = 0;
        rsot_status s;
        if (tr.tail > 0.0 && tail_dense) {
            s = rsot_eval_dual_grad(p, psi.data(), eps, 0.0, prec, &J, g.data(), &pr);
        } else if (tr.tail > 0.0) {
            // the psi-aware cutoffs of that tail tolerance (Sec. 4.1, App. B)
            s = rsot_eval_dual_grad_tail(p, psi.data(), eps, tr.tail, prec, &J, g.data(), &pr);
            if (!s && !probed) {
                probed = true;
                const double all = (double)rsot::num_points(p) * (double)n;
                if ((double)pr > kTailDenseFraction * all) {
                    // most pairs kept: this evaluator runs dense from here on.  An
                    // FP64 one evaluates this point again dense, so that its line
                    // searches see one functional at FP64 resolution; a mixed or
                    // compensated one keeps the truncated result, whose difference
                    // from the dense one (the tail tolerance, ~1e-12 relative) lies
                    // far below its own rounding bound
                    tail_dense = true;
                    if (prec == RSOT_FP64) {
                        count_eval(pr);
                        s = rsot_eval_dual_grad(p, psi.data(), eps, 0.0, prec, &J, g.data(), &pr);
                    }
                }
            }
        } else {
            double radius = 0.0;   // dense
            double C = NAN;
            if (tr.tau_int > 0.0 && have_prev) {
                // C_int (Eq. truncation_cutoff_int) with D and J of the previous
                // evaluation, kept above the covering cost so that every point keeps
                // its nearest target
                double C0 = 0.0;
                if ((s = rsot_covering_cost(p, &C0))) return last = s;
                if ((s = rsot_truncation_cutoff(p, psi.data(), eps, RSOT_CUTOFF_INTEGRAL, tr.tau_int,
                                                J_prev, lnD_prev, &C)))
                    return last = s;
                if (isfinite(C)) C = std::max(C, C0 * (1.0 + 1e-5) + 1e-12);
            } else if (tr.delta_pw > 0.0) {
                // C_pw of the current potential (Eq. cost_cutoff_delta)
                if ((s = rsot_truncation_cutoff(p, psi.data(), eps, RSOT_CUTOFF_POINTWISE, tr.delta_pw,
                                                0.0, 0.0, &C)))
                    return last = s;
            } else if (tr.tau_geom > 0.0 && have_prev) {
                // C_geom (Eq. truncation_cutoff_geom) with J of the previous evaluation
                if ((s = rsot_truncation_cutoff(p, psi.data(), eps, RSOT_CUTOFF_GEOMETRIC, tr.tau_geom,
                                                J_prev, 0.0, &C)))
                    return last = s;
            }
            // a cutoff at or below 0 keeps no pair (every point is skipped)
            if (isfinite(C)) radius = C > 0.0 ? sqrt(2.0 * C) : 1e-150;
            s = rsot_eval_dual_grad(p, psi.data(), eps, radius, prec, &J, g.data(), &pr);
            if (s == RSOT_ERR_EMPTY_NEIGHBORHOOD && (tr.delta_pw > 0.0 || tr.tau_geom > 0.0)) {
                // Algorithm 2 skips points whose truncated sum is empty
                int64_t empty = 0;
                s = rsot_last_eval(p, &J, g.data(), &pr, &empty);
                skipped += empty;
            }
            if (!s && (tr.tau_int > 0.0 || tr.tau_geom > 0.0)) {
                double lnD = INFINITY;
                if (tr.tau_int > 0.0 && (s = rsot_log_integrated_D(p, &lnD))) return last = s;
                lnD_prev = lnD;
                J_prev = J;
                have_prev = J != 0.0;
            }
        }
        count_eval(pr);
        return last = s;
    }

    void count_eval(int64_t pr) {
        ++evals;
        pairs += pr;
        if (count) {
            ++count->evals[prec];
            count->pairs[prec] += pr;
        }
    }
};

// Mixed-precision evaluation plus a linear correction measured once against
// FP64 at psi0: J'(psi) = J_m(psi) + dJ + b.(psi - psi0), g'(psi) = g_m(psi) + b,
// with b = g_64(psi0) - g_m(psi0), dJ = J_64(psi0) - J_m(psi0).  The
// systematic part of the FP32 rounding (per-target constants) is nearly
// constant near the minimiser, so J' has FP64 accuracy there and the
// minimiser of J' is refined by mixed evaluations only.
struct CorrectedEvaluator {
    Evaluator &mixed;
    std::vector<double> b, psi0;
    double dJ = 0.0;
    int64_t n;
    double eps;
    rsot_precision prec = RSOT_MIXED;
    int evals = 0;

    rsot_status operator()(const std::vector<double> &psi, double &J, std::vector<double> &g) {
        rsot_status s = mixed(psi, J, g);
        ++evals;
        if (s) return s;
        double lin = 0.0;
        for (int64_t j = 0; j < n; ++j) {
            g[j] += b[j];
            lin += b[j] * (psi[j] - psi0[j]);
        }
        J += dJ + lin;
        return RSOT_OK;
    }
};

// iterations without halving the corrected objective's gradient after which
// a correction's mixed run stops at its rounding noise
constexpr int kCorrStallWindow = 25;
// largest tail tolerance at which the compensated reference evaluations are
// truncated (its bound stays far below any useful tolerance)
constexpr double kRefTailMax = 1e-8;
// tail of the compensated reference evaluations of an untruncated solve of at
// least kRefTailMinPairs pairs: their bound (1e-12 sum(nu) (2 sum(m) + sum(nu)))
// joins the certified one, and the evaluator falls back to dense evaluations
// where most pairs are kept.  Smaller problems keep dense references: the cell
// list that a first truncated evaluation builds costs them more than it saves
// (measured: 256 batched problems of up to 1.6e10 pairs refined in 8.6 s
// instead of 6.4 s; the 5.2e10-pair cube solved in 3.15 s instead of 3.29 s).
constexpr double kRefTailDense = 1e-12;
constexpr double kRefTailMinPairs = 2e10;

double norm1(const std::vector<double> &a) {
    double s = 0.0;
    for (double v : a) s += fabs(v);
    return s;
}

// Drive one L-BFGS run with GPU evaluations until it stops.
template <class Ev>
rsot_status run_machine(Ev &ev, rsot::LbfgsMachine &mc, int verbose, rsot_problem *p) {
    std::vector<double> g(ev.n);
    double f = 0.0;
    while (mc.wants_eval()) {
        rsot_status s = ev(mc.trial(), f, g);
        if (s) return s;
        mc.feed(f, g);
        // tensor-core pair kernels only while the gradient is far above their noise
        rsot::pair_kernel_for_gradient(p, mc.grad_l1());
        if (verbose && !mc.wants_eval())
            fprintf(stderr, "[rsot] eps=%.3g %s stop after %d it: J=%.15g |g|_1=%.3e evals=%d\n",
                    ev.eps, ev.prec == RSOT_FP64 ? "fp64" : ev.prec == RSOT_MIXED ? "mixed" : "compensated", mc.iters(), mc.f(),
                    mc.grad_l1(), ev.evals);
    }
    return mc.status();
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
    o->mixed_tol_l1 = 1e-5;
    o->refine_precision = RSOT_COMPENSATED;
}

rsot_status rsot_solve(rsot_problem *p, double *psi_inout, const rsot_options *opt,
                       rsot_solve_stats *stats) {
    if (!p || !psi_inout || !opt) return RSOT_ERR_ARG;
    if (!(opt->eps > 0.0) || !(opt->tol_l1 > 0.0) || opt->tail < 0.0 || opt->tail >= 1.0)
        return RSOT_ERR_ARG;
    if (opt->precision != RSOT_FP64 && opt->precision != RSOT_MIXED &&
        opt->precision != RSOT_COMPENSATED)
        return RSOT_ERR_ARG;
    if (opt->refine_precision != RSOT_FP64 && opt->refine_precision != RSOT_COMPENSATED)
        return RSOT_ERR_ARG;
    if (opt->tau_int < 0.0 || opt->delta_pw < 0.0 || opt->tau_geom < 0.0) return RSOT_ERR_ARG;
    if ((opt->tail > 0.0) + (opt->tau_int > 0.0) + (opt->delta_pw > 0.0) + (opt->tau_geom > 0.0) > 1)
        return RSOT_ERR_ARG;   // one truncation at a time
    Truncation trunc;
    trunc.tail = opt->tail;
    trunc.tau_int = opt->tau_int;
    trunc.delta_pw = opt->delta_pw;
    trunc.tau_geom = opt->tau_geom;
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
    // intermediate eps stages only warm-start the next one: 100 tol_l1 unless given
    const double stage_tol = opt->stage_tol_l1 > 0.0 ? opt->stage_tol_l1 : rsot::kStageTolFactor * opt->tol_l1;
    // reference evaluations of the final stop: compensated with its certified
    // bound subtracted from tol where the bound leaves room, else FP64.  The
    // compensated references are truncated at the psi-aware cutoffs of the
    // solve's tail (or of kRefTailDense for a large untruncated solve) and the
    // truncation's own bound joins: per point at most tail * sum(nu) of the kept
    // mass is lost, so ||grad J~ - grad J||_1 <= tail * sum(nu) * (2 sum(m) +
    // sum(nu)); the stop then holds for the untruncated J
    const double msum = rsot::mass_sum(p);
    double nusum = 0.0;
    for (int64_t j = 0; j < n; ++j) nusum += nu[j];
    const bool untruncated = !(opt->tail > 0.0) && !(opt->tau_int > 0.0) && !(opt->delta_pw > 0.0) &&
                             !(opt->tau_geom > 0.0) &&
                             (double)rsot::num_points(p) * (double)n >= kRefTailMinPairs;
    const double ref_tail = (opt->tail > 0.0 && opt->tail <= kRefTailMax) ? opt->tail
                            : untruncated                               ? kRefTailDense
                                                                        : 0.0;
    Truncation ref_trunc;
    ref_trunc.tail = ref_tail;
    const double comp_bound =
        RSOT_COMPENSATED_GRAD_REL * msum + ref_tail * nusum * (2.0 * msum + nusum);
    const bool comp_ref = opt->refine_precision == RSOT_COMPENSATED && comp_bound <= 0.8 * opt->tol_l1;
    const rsot_precision ref_prec = comp_ref ? RSOT_COMPENSATED : RSOT_FP64;
    const double ref_tol = comp_ref ? opt->tol_l1 - comp_bound : opt->tol_l1;
    const double ref_noise = comp_ref ? 1e-6 : 1e-13;

    rsot::pair_kernel_for_gradient(p, INFINITY);
    rsot::set_in_solve(p, 1);   // mixed iterations may take the tensor-core form
    std::vector<double> x(psi_inout, psi_inout + n), g(n, 0.0), D(n);
    double f = 0.0;
    int iters = 0, evals = 0, stages = 0;
    int64_t pairs = 0;
    PrecCount pc;
    rsot_status st = RSOT_OK;
    for (size_t si = 0; si < eps_list.size(); ++si) {
        const double eps = eps_list[si];
        const bool last = si + 1 == eps_list.size();
        const double tol = last ? opt->tol_l1 : stage_tol;
        for (int64_t j = 0; j < n; ++j) D[j] = eps / nu[j];
        // a COMPENSATED solve whose bound leaves no room finishes in FP64
        const rsot_precision prec = (opt->precision == RSOT_COMPENSATED && last && !comp_ref)
                                        ? RSOT_FP64
                                        : (rsot_precision)opt->precision;
        Evaluator ev{p, n, eps, trunc, prec, &pc};
        rsot::LbfgsMachine mc;
        double tol_run = tol;
        if (last && opt->precision == RSOT_MIXED && opt->refine_fp64)
            tol_run = std::max(tol, opt->mixed_tol_l1 > 0.0 ? opt->mixed_tol_l1 : 1e-5);
        if (last && prec == RSOT_COMPENSATED) tol_run = ref_tol;
        mc.start(x, tol_run, m, max_iter, D, prec == RSOT_FP64 ? 1e-13 : 1e-6);
        // mixed evaluations: stop at their rounding floor instead of the cap
        if (prec == RSOT_MIXED) mc.set_stall_window(rsot::kMixedStallWindow);
        ++stages;
        st = run_machine(ev, mc, opt->verbose, p);
        x = mc.x();
        f = mc.f();
        g = mc.g();
        iters += mc.iters();
        evals += ev.evals;
        pairs += ev.pairs;
        const bool refine = last && opt->precision == RSOT_MIXED && opt->refine_fp64;
        const bool refine_ok = st == RSOT_OK || st == RSOT_ERR_LINESEARCH || st == RSOT_ERR_NOT_CONVERGED;
        if (refine && refine_ok && ref_prec == RSOT_COMPENSATED) {
            // a compensated evaluation costs about ten mixed ones.  One correction
            // first: the compensated and the mixed gradient at the iterate give
            // the systematic mixed error, and mixed L-BFGS on the corrected
            // objective runs until its own rounding noise stops it (no halving
            // in kCorrStallWindow iterations); then L-BFGS on compensated
            // evaluations finishes from there (the D-scaled first step is
            // Newton-like near the optimum: a few iterations)
            // reference evaluations: dense, or truncated at the solve's tail with
            // its bound inside comp_bound (the stop then holds for the
            // untruncated J); a truncated mixed phase differs by tail-level
            // terms, which the correction absorbs
            Evaluator evc{p, n, eps, ref_trunc, RSOT_COMPENSATED, &pc};
            Evaluator evm{p, n, eps, trunc, RSOT_MIXED, &pc};
            const int kernel_before = rsot::pair_kernel_of(p);
            rsot_set_pair_kernel(p, RSOT_PAIRS_FP32);
            double fc = 0.0, fm = 0.0;
            std::vector<double> gc(n), gm(n);
            st = evc(x, fc, gc);
            if (!st) st = evm(x, fm, gm);
            const bool corrected = !st && norm1(gc) > ref_tol;
            if (corrected) {
                CorrectedEvaluator ce{evm, std::vector<double>(n), x, fc - fm, n, eps};
                for (int64_t j = 0; j < n; ++j) ce.b[j] = gc[j] - gm[j];
                rsot::LbfgsMachine mcc;
                mcc.start_from(x, fc, gc, 0.5 * ref_tol, m, std::min(max_iter, 200), D, 1e-6);
                mcc.set_stall_window(kCorrStallWindow);
                const rsot_status sc = run_machine(ce, mcc, opt->verbose, p);
                if (sc && sc != RSOT_ERR_LINESEARCH && sc != RSOT_ERR_NOT_CONVERGED) st = sc;
                iters += mcc.iters();
                x = mcc.x();
            }
            rsot_set_pair_kernel(p, (rsot_pair_kernel)kernel_before);
            if (!st) {
                rsot::LbfgsMachine mcr;
                if (corrected)
                    mcr.start(x, ref_tol, m, max_iter, D, ref_noise);
                else
                    mcr.start_from(x, fc, gc, ref_tol, m, max_iter, D, ref_noise);
                st = run_machine(evc, mcr, opt->verbose, p);
                x = mcr.x();
                f = mcr.f();
                g = mcr.g();
                iters += mcr.iters();
            }
            evals += evc.evals + evm.evals;
            pairs += evc.pairs + evm.pairs;
        } else if (refine && refine_ok) {
            // corrected refinement: one reference and one mixed evaluation per
            // correction, mixed L-BFGS on the corrected objective in between
            Evaluator ev64{p, n, eps, Truncation(), ref_prec, &pc};   // dense reference, as above
            Evaluator evm{p, n, eps, trunc, RSOT_MIXED, &pc};
            // the refinement works below the random rounding noise of the
            // tensor-core exponents (rms ~2e-5 per pair, several 1e-6 in the L1
            // norm of a large gradient): its mixed evaluations take the FP32
            // kernels, whose noise is four times lower
            const int kernel_before = rsot::pair_kernel_of(p);
            rsot_set_pair_kernel(p, RSOT_PAIRS_FP32);
            bool done = false;
            st = RSOT_OK;
            // each correction runs at most 200 mixed iterations; corrections stop when
            // the FP64 gradient no longer halves (the mixed random noise floor is near)
            double last64 = INFINITY;
            for (int corr = 0; corr < 6 && !done; ++corr) {
                double f64 = 0.0, fm = 0.0;
                std::vector<double> g64(n), gm(n);
                if ((st = ev64(x, f64, g64))) break;
                f = f64;
                g = g64;
                const double n64 = norm1(g64);
                if (n64 <= ref_tol) {
                    done = true;
                    break;
                }
                if (n64 > 0.5 * last64) break;
                last64 = n64;
                if ((st = evm(x, fm, gm))) break;
                CorrectedEvaluator ce{evm, std::vector<double>(n), x, f64 - fm, n, eps};
                for (int64_t j = 0; j < n; ++j) ce.b[j] = g64[j] - gm[j];
                rsot::LbfgsMachine mcc;
                mcc.start_from(x, f64, g64, 0.5 * ref_tol, m, std::min(max_iter, 200), D, 1e-6);
                rsot_status sc = run_machine(ce, mcc, opt->verbose, p);
                if (sc && sc != RSOT_ERR_LINESEARCH && sc != RSOT_ERR_NOT_CONVERGED) {
                    st = sc;
                    break;
                }
                iters += mcc.iters();
                x = mcc.x();
            }
            if (!done && st == RSOT_OK) {
                // fall back to L-BFGS on reference evaluations from the corrected iterate
                rsot::LbfgsMachine mc64;
                mc64.start(x, ref_tol, m, max_iter, D, ref_noise);
                st = run_machine(ev64, mc64, opt->verbose, p);
                x = mc64.x();
                f = mc64.f();
                g = mc64.g();
                iters += mc64.iters();
            }
            rsot_set_pair_kernel(p, (rsot_pair_kernel)kernel_before);
            evals += ev64.evals + evm.evals;
            pairs += ev64.pairs + evm.pairs;
        }
        if (st != RSOT_OK && !(st == RSOT_ERR_LINESEARCH && !last)) break;
        st = RSOT_OK;
    }
    rsot::pair_kernel_for_gradient(p, INFINITY);
    rsot::set_in_solve(p, 0);
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
        for (int k = 0; k < 3; ++k) {
            stats->evals_prec[k] = pc.evals[k];
            stats->pairs_prec[k] = pc.pairs[k];
        }
    }
    return st;
}

}  // extern "C"
