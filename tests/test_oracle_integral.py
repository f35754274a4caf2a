"""Pins of the oracle's integrated cutoff (Sec. 4.1, Eq. truncation_cutoff_int,
App. B): D(psi, C) = sum_q m_q / S_trunc(x_q, psi; C) and
C_int = M + eps ln(eps D / (tau |J|)).  No GPU."""
import math

import numpy as np
import pytest
from scipy.special import logsumexp

import oracle
from oracle import truncation


def rand_case(seed, d, nq, n, eps, scale):
    rng = np.random.default_rng(seed)
    x = rng.uniform(0, 1, (nq, d))
    m = rng.uniform(0.5, 1.5, nq)
    m /= m.sum()
    y = rng.uniform(0, 1, (n, d))
    nu = rng.uniform(0.5, 1.5, n)
    nu /= nu.sum()
    return x, m, y, nu, scale * rng.standard_normal(n), eps


def test_single_target_closed_form():
    """N = 1: S(x_q) = nu exp((psi - c_q)/eps), so ln D = ln sum_q m_q exp((c_q - psi)/eps) - ln nu."""
    x, m, y, nu, psi, eps = rand_case(1, 2, 500, 1, 0.05, 0.0)
    nu = np.array([0.7])
    psi = np.array([0.013])
    c = 0.5 * ((x - y[0]) ** 2).sum(1)
    ref = logsumexp(np.log(m) + (c - psi[0]) / eps) - math.log(0.7)
    assert abs(oracle.integrated_D(x, m, y, nu, psi, eps) - ref) <= 1e-12 * abs(ref)


def test_definition_by_brute_force():
    x, m, y, nu, psi, eps = rand_case(2, 3, 200, 30, 0.02, 0.02)
    C = 0.2
    c = 0.5 * ((x[:, None, :] - y[None, :, :]) ** 2).sum(-1)
    s = np.where(c < C, (psi[None, :] - c) / eps + np.log(nu)[None, :], -np.inf)
    L = logsumexp(s, axis=1)
    assert np.all(np.isfinite(L))
    ref = logsumexp(np.log(m) - L)
    assert abs(oracle.integrated_D(x, m, y, nu, psi, eps, cutoff=C) - ref) <= 1e-12 * abs(ref)
    # an empty point with mass makes D infinite; without mass it does not count
    C = 0.03
    empty = ~(c < C).any(1)
    assert empty.any() and not empty.all()
    assert oracle.integrated_D(x, m, y, nu, psi, eps, cutoff=C) == math.inf
    m2 = np.where(empty, 0.0, m)
    s = np.where(c < C, (psi[None, :] - c) / eps + np.log(nu)[None, :], -np.inf)
    ref = logsumexp(np.log(m2[~empty]) - logsumexp(s[~empty], axis=1))
    assert abs(oracle.integrated_D(x, m2, y, nu, psi, eps, cutoff=C) - ref) <= 1e-12 * abs(ref)


def test_D_decreases_with_the_cutoff():
    x, m, y, nu, psi, eps = rand_case(3, 2, 400, 50, 0.01, 0.01)
    Ds = [oracle.integrated_D(x, m, y, nu, psi, eps, cutoff=C) for C in (0.03, 0.06, 0.12, math.inf)]
    assert all(a >= b - 1e-12 for a, b in zip(Ds, Ds[1:]))


@pytest.mark.parametrize("seed,d,eps,scale,tau", [
    (4, 2, 0.01, 0.02, 1e-3),
    (5, 3, 0.005, 0.01, 1e-6),
    (6, 2, 0.02, 0.05, 1e-9),
])
def test_integrated_bound_holds_at_a_consistent_cutoff(seed, d, eps, scale, tau):
    """App. B: a cutoff with C >= M + eps ln(eps D(psi, C) / (tau |J|)) keeps
    |J - J~| <= tau |J| (normalised measures)."""
    x, m, y, nu, psi, eps = rand_case(seed, d, 600, 80, eps, scale)
    J, _, _, _ = oracle.dual_grad(x, m, y, nu, psi, eps)
    # RHS(C) = M + eps ln(eps D(C) / (tau |J|)) does not increase with C (D decreases),
    # so C = RHS(RHS(inf)) satisfies C >= RHS(C)
    rhs = lambda C: truncation.cutoff_integrated(
        psi, eps, tau, math.exp(oracle.integrated_D(x, m, y, nu, psi, eps, cutoff=C)), J)
    C = rhs(rhs(math.inf)) * (1 + 1e-12)
    lnD = oracle.integrated_D(x, m, y, nu, psi, eps, cutoff=C)
    assert C >= truncation.cutoff_integrated(psi, eps, tau, math.exp(lnD), J)
    Jt, _, pt, et = oracle.dual_grad(x, m, y, nu, psi, eps, cutoff=C)
    assert et == 0 and pt < 600 * 80
    assert abs(J - Jt) <= tau * abs(J)
    # the bound's own estimate eps exp((M - C)/eps) D dominates the error
    assert abs(J - Jt) <= eps * math.exp((np.max(psi) - C) / eps + lnD) * (1 + 1e-9)
