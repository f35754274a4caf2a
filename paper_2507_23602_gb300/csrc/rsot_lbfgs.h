// Resumable FP64 L-BFGS with a strong-Wolfe line search (host only).
//
// Algorithm 1 of the paper: L-BFGS steps whose line search calls the dual
// evaluation several times, until ||grad J||_1 <= tol (Remark 3.3).  The
// machine never calls the objective itself: it exposes the next point to
// evaluate (trial()) and takes the result (feed()), so that one driver can
// advance many independent problems in lockstep, each evaluation round being
// one batched GPU launch.
//
// Details (the paper leaves them open):
//   * two-loop recursion with memory m and H0 = gamma * diag(D), D_j = eps / nu_j
//     (the Hessian diagonal of J near the optimum is ~ nu_j / eps), gamma =
//     s^T y / y^T D y of the newest pair; curvature pairs kept when s^T y > 0;
//   * strong-Wolfe search (c1 = 1e-4, c2 = 0.9): step 1, doubled while the
//     function decreases with a negative slope, then sectioning of the bracket
//     with a safeguarded cubic fit; Hager & Zhang's approximate Wolfe test
//     (sigma d0 <= d <= (2 c1 - 1) d0) replaces sufficient decrease where J
//     moves less than its evaluation noise (noise_rel |J|);
//   * a failed search first restarts from the scaled gradient (curvature
//     history dropped, at most 5 times per run), then reports failure.
#pragma once

#include <math.h>

#include <algorithm>
#include <deque>
#include <vector>

#include "../../include/rsot.h"

namespace rsot {

// iterations without halving the gradient's L1 norm after which a run on
// mixed-precision evaluations stops at their rounding floor (a refinement on
// reference evaluations takes over)
inline constexpr int kMixedStallWindow = 300;

// default tolerance of intermediate eps stages, as a multiple of the final one
// (their solutions only warm-start the next stage, Sec. 4.2)
inline constexpr double kStageTolFactor = 100.0;

class LbfgsMachine {
   public:
    enum State { kIdle, kNeedF0, kSearch, kDone };

    void start(const std::vector<double> &x0, double tol, int m, int max_iter,
               const std::vector<double> &D, double noise_rel) {
        x_ = x0;
        n_ = x0.size();
        tol_ = tol;
        m_ = m;
        max_iter_ = max_iter;
        D_ = D;
        noise_rel_ = noise_rel;
        hist_.clear();
        iters_ = 0;
        evals_ = 0;
        restarts_ = 0;
        best_l1_ = INFINITY;
        best_iter_ = 0;
        status_ = RSOT_OK;
        xt_ = x_;
        state_ = kNeedF0;
    }

    // Noisy evaluations (mixed precision): stop with RSOT_ERR_LINESEARCH when
    // the gradient's L1 norm has not halved within `window` iterations -- the
    // rounding floor of the evaluation is reached.  0 (default): never.
    void set_stall_window(int window) { stall_window_ = window; }

    // Continue from a known (x, f, g) (e.g. after a change of precision).
    void start_from(const std::vector<double> &x, double f, const std::vector<double> &g, double tol,
                    int m, int max_iter, const std::vector<double> &D, double noise_rel) {
        start(x, tol, m, max_iter, D, noise_rel);
        f_ = f;
        g_ = g;
        next_iteration();
    }

    bool wants_eval() const { return state_ == kNeedF0 || state_ == kSearch; }
    bool done() const { return state_ == kDone; }
    const std::vector<double> &trial() const { return xt_; }

    void feed(double f, const std::vector<double> &g) {
        ++evals_;
        if (state_ == kNeedF0) {
            f_ = f;
            g_ = g;
            next_iteration();
            return;
        }
        if (state_ != kSearch) return;
        Trial cur;
        cur.a = a_try_;
        cur.f = f;
        cur.g = g;
        cur.d = dot(g, p_);
        --budget_;
        if (flat_ok(cur)) return accept(cur);
        if (!bracketed_) {
            if (!armijo(cur) || (lo_.a > 0.0 && cur.f >= lo_.f)) {
                hi_ = cur;
                bracketed_ = true;
            } else if (strong(cur)) {
                return accept(cur);
            } else if (cur.d >= 0.0) {
                hi_ = lo_;
                lo_ = cur;
                bracketed_ = true;
            } else {
                lo_ = cur;
                if (budget_ <= 0) return finish_search();
                propose(2.0 * cur.a);
                return;
            }
        } else {
            if (!armijo(cur) || cur.f >= lo_.f) {
                hi_ = cur;
            } else {
                if (strong(cur)) return accept(cur);
                if (cur.d * (hi_.a - lo_.a) >= 0.0) hi_ = lo_;
                lo_ = cur;
            }
        }
        // next point inside the bracket
        const double left = std::min(lo_.a, hi_.a), right = std::max(lo_.a, hi_.a);
        const double w = right - left;
        if (budget_ <= 0 || w <= 1e-16 * std::max(1.0, right)) return finish_search();
        double at = cubic_step(lo_.a, lo_.f, lo_.d, hi_.a, hi_.f, hi_.d);
        if (!(at > left + 0.1 * w && at < right - 0.1 * w)) at = 0.5 * (left + right);
        propose(at);
    }

    rsot_status status() const { return status_; }
    const std::vector<double> &x() const { return x_; }
    const std::vector<double> &g() const { return g_; }
    double f() const { return f_; }
    int iters() const { return iters_; }
    int evals() const { return evals_; }
    double grad_l1() const { return norm1(g_); }

   private:
    struct Trial {
        double a = 0.0, f = 0.0, d = 0.0;
        std::vector<double> g;
    };
    struct Pair {
        std::vector<double> s, y;
        double rho;
    };

    static double dot(const std::vector<double> &a, const std::vector<double> &b) {
        double s = 0.0;
        for (size_t i = 0; i < a.size(); ++i) s += a[i] * b[i];
        return s;
    }
    static double norm1(const std::vector<double> &a) {
        double s = 0.0;
        for (double v : a) s += fabs(v);
        return s;
    }
    static double cubic_step(double a, double fa, double da, double b, double fb, double db) {
        const double t = da + db - 3.0 * (fa - fb) / (a - b);
        const double r = t * t - da * db;
        if (!(r >= 0.0) || a == b) return NAN;
        const double s = (b > a ? 1.0 : -1.0) * sqrt(r);
        const double den = db - da + 2.0 * s;
        if (den == 0.0) return NAN;
        return b - (b - a) * (db + s - t) / den;
    }

    bool flat_ok(const Trial &t) const {
        return fabs(t.f - f0_) <= noise_ && kC2 * d0_ <= t.d && t.d <= (2.0 * kC1 - 1.0) * d0_;
    }
    bool strong(const Trial &t) const { return fabs(t.d) <= -kC2 * d0_; }
    bool armijo(const Trial &t) const { return t.f <= f0_ + kC1 * t.a * d0_; }

    void propose(double a) {
        a_try_ = a;
        for (size_t i = 0; i < n_; ++i) xt_[i] = x_[i] + a * p_[i];
        state_ = kSearch;
    }

    void finish_search() {
        if (lo_.a > 0.0 && lo_.f < f0_) return accept(lo_);
        // no acceptable step: drop the curvature history and retry along
        // -D g (a few times per run) before reporting a failed search
        if (!hist_.empty() && restarts_ < kMaxRestarts) {
            ++restarts_;
            hist_.clear();
            return next_iteration();
        }
        status_ = RSOT_ERR_LINESEARCH;
        state_ = kDone;
    }

    void accept(const Trial &t) {
        Pair pr;
        pr.s.resize(n_);
        pr.y.resize(n_);
        for (size_t i = 0; i < n_; ++i) {
            pr.s[i] = t.a * p_[i];
            pr.y[i] = t.g[i] - g_[i];
            x_[i] += pr.s[i];
        }
        const double sy = dot(pr.s, pr.y);
        if (sy > 0.0) {
            pr.rho = 1.0 / sy;
            hist_.push_back(std::move(pr));
            if ((int)hist_.size() > m_) hist_.pop_front();
        }
        f_ = t.f;
        g_ = t.g;
        ++iters_;
        next_iteration();
    }

    void next_iteration() {
        if (!(isfinite(f_))) {
            status_ = RSOT_ERR_NONFINITE;
            state_ = kDone;
            return;
        }
        if (norm1(g_) <= tol_) {
            status_ = RSOT_OK;
            state_ = kDone;
            return;
        }
        if (iters_ >= max_iter_) {
            status_ = RSOT_ERR_NOT_CONVERGED;
            state_ = kDone;
            return;
        }
        if (stall_window_ > 0) {
            const double gn = norm1(g_);
            if (gn < 0.5 * best_l1_) {
                best_l1_ = gn;
                best_iter_ = iters_;
            } else if (iters_ - best_iter_ >= stall_window_) {
                status_ = RSOT_ERR_LINESEARCH;
                state_ = kDone;
                return;
            }
        }
        // two-loop recursion
        std::vector<double> q = g_;
        const int k = (int)hist_.size();
        std::vector<double> alpha(k);
        for (int i = k - 1; i >= 0; --i) {
            alpha[i] = hist_[i].rho * dot(hist_[i].s, q);
            for (size_t t = 0; t < n_; ++t) q[t] -= alpha[i] * hist_[i].y[t];
        }
        double gamma = 1.0;
        if (k > 0) {
            const Pair &l = hist_.back();
            double yDy = 0.0;
            for (size_t t = 0; t < n_; ++t) yDy += l.y[t] * D_[t] * l.y[t];
            gamma = (1.0 / l.rho) / yDy;
        }
        for (size_t t = 0; t < n_; ++t) q[t] *= gamma * D_[t];
        for (int i = 0; i < k; ++i) {
            const double b = hist_[i].rho * dot(hist_[i].y, q);
            for (size_t t = 0; t < n_; ++t) q[t] += (alpha[i] - b) * hist_[i].s[t];
        }
        p_.resize(n_);
        for (size_t t = 0; t < n_; ++t) p_[t] = -q[t];
        if (dot(g_, p_) >= 0.0) {   // not a descent direction: restart along -D g
            hist_.clear();
            for (size_t t = 0; t < n_; ++t) p_[t] = -D_[t] * g_[t];
        }
        f0_ = f_;
        d0_ = dot(g_, p_);
        noise_ = noise_rel_ * std::max(fabs(f_), 1e-300);
        lo_ = Trial();
        lo_.a = 0.0;
        lo_.f = f_;
        lo_.d = d0_;
        lo_.g = g_;
        hi_ = Trial();
        bracketed_ = false;
        budget_ = 30;
        propose(1.0);
    }

    static constexpr double kC1 = 1e-4, kC2 = 0.9;
    static constexpr int kMaxRestarts = 5;
    int restarts_ = 0;
    int stall_window_ = 0, best_iter_ = 0;
    double best_l1_ = INFINITY;
    size_t n_ = 0;
    double tol_ = 0.0, noise_rel_ = 0.0, noise_ = 0.0;
    int m_ = 10, max_iter_ = 10000;
    std::vector<double> x_, g_, p_, xt_, D_;
    double f_ = 0.0, f0_ = 0.0, d0_ = 0.0, a_try_ = 1.0;
    std::deque<Pair> hist_;
    Trial lo_, hi_;
    bool bracketed_ = false;
    int budget_ = 0;
    int iters_ = 0, evals_ = 0;
    rsot_status status_ = RSOT_OK;
    State state_ = kIdle;
};

}  // namespace rsot
