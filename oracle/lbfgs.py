"""FP64 L-BFGS with a strong-Wolfe line search -- TEST INFRASTRUCTURE ONLY.

Algorithm 1 minimises J(psi) with L-BFGS steps whose line search calls the
dual evaluation several times, stopping when ||grad J||_1 <= delta_tol
(Remark 3.3).  The paper does not fix the L-BFGS details; this oracle takes the
textbook method (Nocedal & Wright, Numerical Optimization, 2nd ed.):

  * two-loop recursion (their Algorithm 7.4) with memory m = 10 and the
    initial matrix H_0 = (s^T y / y^T y) I of their Eq. 7.20;
  * line search for the strong Wolfe conditions, c1 = 1e-4, c2 = 0.9, by
    bracketing (their Algorithm 3.5) and zoom (their Algorithm 3.6) with a
    safeguarded cubic interpolation step;
  * a curvature pair is stored only when s^T y > 0;
  * where the function values at the trial and the base point differ only by
    round-off (|f - f0| <= 1e-14 |f0|), the approximate Wolfe conditions of
    Hager & Zhang (SIAM J. Optim. 16, 2005),
    sigma phi'(0) <= phi'(a) <= (2 c1 - 1) phi'(0), replace the sufficient
    decrease test, which round-off makes meaningless that close to the minimum.

It is written independently of the product's C++ driver and shares no code
with it.
"""
from __future__ import annotations

import dataclasses
from collections import deque
from typing import Callable, Tuple

import numpy as np


@dataclasses.dataclass
class Result:
    x: np.ndarray
    f: float
    g: np.ndarray
    iters: int
    evals: int
    status: str          # "converged" | "max_iter" | "linesearch_failed"
    history: list


def _cubic_min(a0, f0, d0, a1, f1, d1):
    """Minimiser of the cubic through (a0,f0,d0), (a1,f1,d1); None if none."""
    if a0 == a1:
        return None
    d1_ = d0 + d1 - 3.0 * (f0 - f1) / (a0 - a1)
    rad = d1_ * d1_ - d0 * d1
    if rad < 0.0:
        return None
    d2 = np.sign(a1 - a0) * np.sqrt(rad)
    den = d1 - d0 + 2.0 * d2
    if den == 0.0:
        return None
    return a1 - (a1 - a0) * (d1 + d2 - d1_) / den


def _line_search(fun, x, f0, g0, p, a_init, c1, c2, max_evals=40):
    d0 = float(g0 @ p)
    evals = 0

    def phi(a):
        nonlocal evals
        evals += 1
        f, g = fun(x + a * p)
        return f, g, float(g @ p)

    def approx_wolfe(f, d):
        return (abs(f - f0) <= 1e-14 * abs(f0) and c2 * d0 <= d <= (2.0 * c1 - 1.0) * d0)

    def zoom(lo, f_lo, d_lo, hi, f_hi, d_hi):
        while evals < max_evals:
            a = _cubic_min(lo, f_lo, d_lo, hi, f_hi, d_hi)
            w = abs(hi - lo)
            left, right = min(lo, hi), max(lo, hi)
            if a is None or not np.isfinite(a) or a < left + 0.1 * w or a > right - 0.1 * w:
                a = 0.5 * (lo + hi)
            f, g, d = phi(a)
            if approx_wolfe(f, d):
                return a, f, g
            if f > f0 + c1 * a * d0 or f >= f_lo:
                hi, f_hi, d_hi = a, f, d
            else:
                if abs(d) <= -c2 * d0:
                    return a, f, g
                if d * (hi - lo) >= 0.0:
                    hi, f_hi, d_hi = lo, f_lo, d_lo
                lo, f_lo, d_lo = a, f, d
        return None

    a_prev, f_prev, d_prev = 0.0, f0, d0
    a = a_init
    first = True
    while evals < max_evals:
        f, g, d = phi(a)
        if approx_wolfe(f, d):
            return (a, f, g), evals
        if f > f0 + c1 * a * d0 or (not first and f >= f_prev):
            r = zoom(a_prev, f_prev, d_prev, a, f, d)
            return r, evals
        if abs(d) <= -c2 * d0:
            return (a, f, g), evals
        if d >= 0.0:
            r = zoom(a, f, d, a_prev, f_prev, d_prev)
            return r, evals
        a_prev, f_prev, d_prev = a, f, d
        a = 2.0 * a
        first = False
    return None, evals


def minimize(fun: Callable[[np.ndarray], Tuple[float, np.ndarray]], x0, tol_l1: float,
             m: int = 10, max_iter: int = 10000, c1: float = 1e-4, c2: float = 0.9) -> Result:
    """Minimise fun (returning (f, grad)) from x0 until ||grad||_1 <= tol_l1."""
    x = np.array(x0, dtype=np.float64, copy=True)
    f, g = fun(x)
    evals = 1
    hist = deque(maxlen=m)
    history = []
    for it in range(max_iter + 1):
        gn1 = float(np.sum(np.abs(g)))
        history.append((f, gn1))
        if gn1 <= tol_l1:
            return Result(x, f, g, it, evals, "converged", history)
        if it == max_iter:
            break
        # two-loop recursion
        q = g.copy()
        alphas = []
        for s, y, rho in reversed(hist):
            a = rho * float(s @ q)
            alphas.append(a)
            q -= a * y
        if hist:
            s, y, _ = hist[-1]
            q *= float(s @ y) / float(y @ y)
        for (s, y, rho), a in zip(hist, reversed(alphas)):
            b = rho * float(y @ q)
            q += (a - b) * s
        p = -q
        if float(g @ p) >= 0.0:
            hist.clear()
            p = -g
        a_init = 1.0
        res, ne = _line_search(fun, x, f, g, p, a_init, c1, c2)
        evals += ne
        if res is None:
            return Result(x, f, g, it, evals, "linesearch_failed", history)
        a, f_new, g_new = res
        s = a * p
        yv = g_new - g
        sy = float(s @ yv)
        if sy > 0.0:
            hist.append((s, yv, 1.0 / sy))
        x = x + s
        f, g = f_new, g_new
    return Result(x, f, g, max_iter, evals, "max_iter", history)
