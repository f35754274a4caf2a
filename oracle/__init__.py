"""RSOT oracle -- TEST INFRASTRUCTURE ONLY.

Plain FP64 CPU statements of what the method computes, used to check the CUDA
path.  Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package; the product library never does, and the
two share no code (the only common module is ``rsot_inputs``, which builds
inputs and holds none of the method's arithmetic).

Contents
  * ``dual_grad``      -- Algorithm 2, dense (cutoff=inf) or truncated with the
                          strict predicate c(x_q, y_j) < C tested for every j
                          (Eq. discretized_functional / discretized_gradient).
  * ``dual_grad_sep``  -- the same with a separable cutoff per pair,
                          c(x_q, y_j) < alpha_q + beta_j.
  * ``nearest``        -- the nearest target of every point (brute force).
  * ``plan``           -- the plan density p_j(x_q | psi), Eq. final_plan_density.
  * ``point_lse``      -- the per-point log partition L_q of Eq. discretized_functional.
  * ``integrated_D``   -- ln D(psi, C) = ln sum_q m_q / S_trunc(x_q) of Eq.
                          truncation_cutoff_int.
  * ``covering_cost``  -- C_0 of App. B over the quadrature points.
  * ``softmax_refine`` -- Eq. softmax_refinement_formula.
  * ``truncation``     -- the cutoffs C_pw, C_int, C_geom (Sec. 4.1, App. B) and
                          the pointwise tail reading used for the cell-list radius.
  * ``lbfgs``          -- a separate FP64 L-BFGS with a strong-Wolfe line search
                          and the L1 gradient stop (Algorithm 1, Remark 3.3).
  * ``maps``           -- barycentric / modal maps and the barycenter centroid
                          (Sec. 6.2-6.3).

Every function here has at least one pin in ``tests/test_oracle_pins.py`` that
does not go back to the oracle itself.
"""
from __future__ import annotations

import ctypes
import math
import os

import numpy as np

from . import build as _build

_lib = None


def _load():
    global _lib
    if _lib is None:
        path = _build.build()
        lib = ctypes.CDLL(path)
        dp = ctypes.POINTER(ctypes.c_double)
        i64p = ctypes.POINTER(ctypes.c_int64)
        lib.oracle_dual_grad.argtypes = [ctypes.c_int, ctypes.c_int64, dp, dp, ctypes.c_int64,
                                         dp, dp, dp, ctypes.c_double, ctypes.c_double,
                                         ctypes.c_int, dp, dp, i64p, i64p]
        lib.oracle_plan.argtypes = [ctypes.c_int, ctypes.c_int64, dp, ctypes.c_int64, dp, dp,
                                    dp, ctypes.c_double, dp]
        lib.oracle_covering_cost.argtypes = [ctypes.c_int, ctypes.c_int64, dp, ctypes.c_int64,
                                             dp, ctypes.c_int, dp]
        lib.oracle_softmax_refine.argtypes = [ctypes.c_int, ctypes.c_int64, dp, dp,
                                              ctypes.c_int64, dp, dp, dp, ctypes.c_int64, dp,
                                              ctypes.c_double, ctypes.c_int, dp]
        lib.oracle_point_lse.argtypes = [ctypes.c_int, ctypes.c_int64, dp, ctypes.c_int64, dp,
                                         dp, dp, ctypes.c_double, ctypes.c_int, dp]
        lib.oracle_point_lse_cut.argtypes = [ctypes.c_int, ctypes.c_int64, dp, ctypes.c_int64, dp,
                                             dp, dp, ctypes.c_double, ctypes.c_double, ctypes.c_int,
                                             dp]
        lib.oracle_threads_used.argtypes = [ctypes.c_int]
        lib.oracle_transport_maps.argtypes = [ctypes.c_int, ctypes.c_int64, dp, ctypes.c_int64, dp,
                                              dp, dp, ctypes.c_double, ctypes.c_int, dp,
                                              ctypes.POINTER(ctypes.c_int64)]
        lib.oracle_centroids.argtypes = [ctypes.c_int, ctypes.c_int64, dp, dp, ctypes.c_int64, dp,
                                         dp, dp, ctypes.c_double, dp, dp]
        lib.oracle_dual_grad_sep.argtypes = [ctypes.c_int, ctypes.c_int64, dp, dp, ctypes.c_int64,
                                             dp, dp, dp, ctypes.c_double, dp, dp, ctypes.c_int, dp,
                                             dp, i64p, i64p]
        lib.oracle_nearest.argtypes = [ctypes.c_int, ctypes.c_int64, dp, ctypes.c_int64, dp,
                                       ctypes.c_int, i64p, dp]
        _lib = lib
    return _lib


def _f64(a):
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a, a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def threads_used(threads: int = 0) -> int:
    return int(_load().oracle_threads_used(int(threads)))


def dual_grad(x, mass, y, nu, psi, eps, cutoff=math.inf, threads=0):
    """(J, grad, pairs, empty) of Algorithm 2.  cutoff=inf -> dense J^h."""
    lib = _load()
    x, xp = _f64(x)
    y, yp = _f64(y)
    mass, mp = _f64(mass)
    nu, nup = _f64(nu)
    psi, pp = _f64(psi)
    d = x.shape[1] if x.ndim == 2 else 1
    n = y.shape[0]
    grad = np.empty(n)
    J = ctypes.c_double()
    pairs = ctypes.c_int64()
    empty = ctypes.c_int64()
    rc = lib.oracle_dual_grad(d, x.shape[0], xp, mp, n, yp, nup, pp, float(eps), float(cutoff),
                              int(threads), ctypes.byref(J),
                              grad.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                              ctypes.byref(pairs), ctypes.byref(empty))
    if rc != 0:
        raise ValueError(f"oracle_dual_grad failed ({rc})")
    return J.value, grad, pairs.value, empty.value


def dual_grad_sep(x, mass, y, nu, psi, eps, alpha, beta, threads=0):
    """(J, grad, pairs, empty) of Algorithm 2 with the separable cutoff
    I_q = {j : c(x_q, y_j) < alpha_q + beta_j} (see truncation.separable_cutoffs)."""
    lib = _load()
    x, xp = _f64(x)
    y, yp = _f64(y)
    mass, mp = _f64(mass)
    nu, nup = _f64(nu)
    psi, pp = _f64(psi)
    alpha, ap = _f64(alpha)
    beta, bp = _f64(beta)
    d = x.shape[1] if x.ndim == 2 else 1
    n = y.shape[0]
    grad = np.empty(n)
    J = ctypes.c_double()
    pairs = ctypes.c_int64()
    empty = ctypes.c_int64()
    rc = lib.oracle_dual_grad_sep(d, x.shape[0], xp, mp, n, yp, nup, pp, float(eps), ap, bp,
                                  int(threads), ctypes.byref(J),
                                  grad.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                  ctypes.byref(pairs), ctypes.byref(empty))
    if rc != 0:
        raise ValueError(f"oracle_dual_grad_sep failed ({rc})")
    return J.value, grad, pairs.value, empty.value


def nearest(x, y, threads=0):
    """(j, c): the nearest target of every point (lowest index among equal
    costs) and its cost c(x_q, y_j), brute force in FP64."""
    lib = _load()
    x, xp = _f64(x)
    y, yp = _f64(y)
    nq, d = x.shape
    js = np.zeros(nq, dtype=np.int64)
    cs = np.zeros(nq)
    rc = lib.oracle_nearest(d, nq, xp, y.shape[0], yp, int(threads),
                            js.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                            cs.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    if rc:
        raise ValueError(f"oracle_nearest failed ({rc})")
    return js, cs


def plan(x, y, nu, psi, eps):
    """Dense (nq, n) matrix of p_j(x_q | psi)."""
    lib = _load()
    x, xp = _f64(x)
    y, yp = _f64(y)
    nu, nup = _f64(nu)
    psi, pp = _f64(psi)
    d = x.shape[1]
    P = np.empty((x.shape[0], y.shape[0]))
    rc = lib.oracle_plan(d, x.shape[0], xp, y.shape[0], yp, nup, pp, float(eps),
                         P.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    if rc != 0:
        raise ValueError("oracle_plan failed")
    return P


def point_lse(x, y, nu, psi, eps, threads=0):
    """L_q = ln sum_j nu_j exp((psi_j - c(x_q, y_j))/eps) for every q."""
    lib = _load()
    x, xp = _f64(x)
    y, yp = _f64(y)
    nu, nup = _f64(nu)
    psi, pp = _f64(psi)
    out = np.empty(x.shape[0])
    rc = lib.oracle_point_lse(x.shape[1], x.shape[0], xp, y.shape[0], yp, nup, pp, float(eps),
                              int(threads), out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    if rc != 0:
        raise ValueError("oracle_point_lse failed")
    return out


def integrated_D(x, mass, y, nu, psi, eps, cutoff=math.inf, threads=0):
    """ln D(psi, C) with D = sum_q m_q / S_trunc(x_q, psi; C), the discrete
    integral of the inverse truncated sum (Sec. 4.1, Eq. truncation_cutoff_int);
    +inf when some point with m_q > 0 has an empty I_q."""
    lib = _load()
    x, xp = _f64(x)
    y, yp = _f64(y)
    nu, nup = _f64(nu)
    psi, pp = _f64(psi)
    L = np.empty(x.shape[0])
    rc = lib.oracle_point_lse_cut(x.shape[1], x.shape[0], xp, y.shape[0], yp, nup, pp, float(eps),
                                  float(cutoff), int(threads),
                                  L.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    if rc != 0:
        raise ValueError("oracle_point_lse_cut failed")
    mass = np.asarray(mass, dtype=np.float64)
    keep = mass > 0
    if np.any(~np.isfinite(L[keep])):
        return math.inf
    v = np.log(mass[keep]) - L[keep]
    vmax = float(np.max(v))
    return vmax + math.log(float(np.sum(np.exp(v - vmax))))


def covering_cost(x, y, threads=0):
    lib = _load()
    x, xp = _f64(x)
    y, yp = _f64(y)
    out = ctypes.c_double()
    rc = lib.oracle_covering_cost(x.shape[1], x.shape[0], xp, y.shape[0], yp, int(threads),
                                  ctypes.byref(out))
    if rc != 0:
        raise ValueError("oracle_covering_cost failed")
    return out.value


def softmax_refine(x, mass, y_coarse, nu_coarse, psi_coarse, y_fine, eps, threads=0):
    lib = _load()
    x, xp = _f64(x)
    mass, mp = _f64(mass)
    yc, ycp = _f64(y_coarse)
    nuc, nucp = _f64(nu_coarse)
    psic, pcp = _f64(psi_coarse)
    yf, yfp = _f64(y_fine)
    out = np.empty(yf.shape[0])
    rc = lib.oracle_softmax_refine(x.shape[1], x.shape[0], xp, mp, yc.shape[0], ycp, nucp, pcp,
                                   yf.shape[0], yfp, float(eps), int(threads),
                                   out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    if rc != 0:
        raise ValueError("oracle_softmax_refine failed")
    return out


def transport_maps(x, y, nu, psi, eps, threads=0):
    """Sec. 6.3: barycentric map T_bary(x_q) = sum_j p_qj y_j (Eq.
    barycentric_map_registration) and modal assignment j*(q) = argmax_j s_qj
    (Eq. modal_map_registration, first maximum on ties).  Returns (T_bary [nq, d],
    jstar [nq] int64)."""
    lib = _load()
    x, xp = _f64(x)
    y, yp = _f64(y)
    nu, nup = _f64(nu)
    psi, pp = _f64(psi)
    nq, d = x.shape
    T = np.zeros((nq, d))
    js = np.zeros(nq, dtype=np.int64)
    rc = lib.oracle_transport_maps(d, nq, xp, y.shape[0], yp, nup, pp, float(eps), int(threads),
                                   T.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                   js.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)))
    if rc:
        raise ValueError(f"oracle_transport_maps failed ({rc})")
    return T, js


def centroids(x, mass, y, nu, psi, eps):
    """Eq. barycenter_fixed_point: T_j = (1/nu_j) sum_q m_q p_qj x_q and the
    transported mass a_j = sum_q m_q p_qj.  Returns (T [n, d], a [n])."""
    lib = _load()
    x, xp = _f64(x)
    mass, mp = _f64(mass)
    y, yp = _f64(y)
    nu, nup = _f64(nu)
    psi, pp = _f64(psi)
    nq, d = x.shape
    n = y.shape[0]
    T = np.zeros((n, d))
    a = np.zeros(n)
    rc = lib.oracle_centroids(d, nq, xp, mp, n, yp, nup, pp, float(eps),
                              T.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                              a.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    if rc:
        raise ValueError(f"oracle_centroids failed ({rc})")
    return T, a
