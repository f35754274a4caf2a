"""Truncation cutoffs -- TEST INFRASTRUCTURE ONLY (part of the oracle).

Sec. 4.1 and App. B define the cost cutoff C used in I_q = {j : c(x_q,y_j) < C}.

  * pointwise  C_pw  = M + eps ln(nu_max / delta_thr)               (Eq. cost_cutoff_delta)
  * integrated C_int = M + eps ln(eps D / (tau |J|))                  (Eq. truncation_cutoff_int)
  * geometric  C_geom = max(C_0, C_0 + Gamma + eps ln(eps / (nu_min tau |J|)))
                                                                     (Eq. truncation_cutoff_geom, App. B)
  * tail (the reading used for a single global cell-list radius):
        C_tail = C_0 + Gamma + eps ln(1 / (nu_min tail))
    App. B's geometric argument applied per point instead of integrated:
    with C > C_0 every point keeps its nearest target, so
        S_trunc(x) >= nu_min exp((m - C_0)/eps)   and
        sum_{excluded} nu_j exp((psi_j - c)/eps) <= exp((M - C)/eps),
    hence the excluded mass is at most ``tail`` times S_trunc(x) at every
    point, |J - J_trunc| <= eps * tail * sum_q m_q, and per target
    |dJ/dpsi_j - dJ_trunc/dpsi_j| <= tail * (sum_q m_q p~_qj + nu_j).

  * separable (psi-aware, per pair; the cell-list pruning uses it):
        c(x_q, y_j) < alpha_q + beta_j,
        alpha_q = c(x_q, y_n) - psi_n - eps ln nu_n   (n = n(q), a nearest target of x_q),
        beta_j  = psi_j + eps ln(1 / tail).
    The same geometric argument with the point's own nearest target as the
    anchor: s_qn = (psi_n - c(x_q, y_n))/eps + ln nu_n is a term of S_trunc(x_q)
    (its pair is kept: alpha_q + beta_n - c_qn = eps ln(1/(nu_n tail)) > 0), and
    every excluded term has exp(s_qj) <= tail nu_j exp(s_qn), so the excluded
    mass is at most
    tail * sum_j nu_j * S_trunc(x) at every point: the guarantees of C_tail
    with sum nu in place of 1.  alpha_q + beta_j <= C_tail for every pair, so
    the separable cutoff keeps a subset of the global one's pairs.

M = max psi, m = min psi, Gamma = M - m, C_0 = max_q min_j c(x_q, y_j).
"""
from __future__ import annotations

import math

import numpy as np


def cutoff_pointwise(psi, nu, eps, delta_thr):
    return float(np.max(psi)) + eps * math.log(float(np.max(nu)) / delta_thr)


def cutoff_integrated(psi, eps, tau, D, J):
    return float(np.max(psi)) + eps * math.log(eps * D / (tau * abs(J)))


def cutoff_geometric(psi, nu, eps, tau, J, C0):
    gamma = float(np.max(psi) - np.min(psi))
    c = C0 + gamma + eps * math.log(eps / (float(np.min(nu)) * tau * abs(J)))
    return max(C0, c)


def cutoff_tail(psi, nu, eps, tail, C0):
    gamma = float(np.max(psi) - np.min(psi))
    return C0 + gamma + eps * math.log(1.0 / (float(np.min(nu)) * tail))


def radius_of_cutoff(C):
    """c(x,y) = |x-y|^2 / 2 < C  <=>  |x - y| < sqrt(2 C)."""
    return math.sqrt(2.0 * C)


def separable_cutoffs(x, y, nu, psi, eps, tail):
    """(alpha [nq], beta [n]) of the separable cutoff c(x_q, y_j) < alpha_q + beta_j."""
    from . import nearest
    jn, cn = nearest(x, y)
    psi = np.asarray(psi, dtype=np.float64)
    nu = np.asarray(nu, dtype=np.float64)
    alpha = cn - psi[jn] - eps * np.log(nu[jn])
    beta = psi + eps * math.log(1.0 / tail)
    return alpha, beta
