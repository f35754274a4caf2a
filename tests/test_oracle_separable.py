"""Pins of the oracle's separable (psi-aware) truncation: Algorithm 2 with
I_q = {j : c(x_q, y_j) < alpha_q + beta_j}, alpha_q = c(x_q, y_n) - psi_n -
eps ln nu_n with n the nearest target of x_q, beta_j = psi_j + eps ln(1/tail)
(the geometric argument of App. B anchored at each point's nearest target).
No GPU; nothing here calls the oracle to check the oracle."""
import math

import numpy as np
import pytest
from scipy.special import logsumexp

import oracle
from oracle import truncation


def rand_case(seed, d, nq, n, eps, scale, nu_spread=0.5):
    rng = np.random.default_rng(seed)
    x = rng.uniform(0, 1, (nq, d))
    m = rng.uniform(0.5, 1.5, nq)
    m /= m.sum()
    y = rng.uniform(0, 1, (n, d))
    nu = rng.uniform(1 - nu_spread, 1 + nu_spread, n)
    nu /= nu.sum()
    psi = scale * rng.standard_normal(n)
    return x, m, y, nu, psi, eps


def brute_sep(x, m, y, nu, psi, eps, alpha, beta):
    """The definition in numpy: masked log-sum-exp and softmax, no loops."""
    c = 0.5 * ((x[:, None, :] - y[None, :, :]) ** 2).sum(-1)
    keep = c < alpha[:, None] + beta[None, :]
    s = np.where(keep, (psi[None, :] - c) / eps + np.log(nu)[None, :], -np.inf)
    ok = keep.any(1)
    L = logsumexp(s[ok], axis=1)
    J = eps * (m[ok] * L).sum() - psi @ nu
    P = np.exp(s[ok] - L[:, None])
    g = m[ok] @ P - nu
    return J, g, int(keep.sum()), int((~ok).sum())


@pytest.mark.parametrize("d", [2, 3])
def test_nearest_matches_kdtree(d):
    from scipy.spatial import cKDTree
    rng = np.random.default_rng(d)
    x = rng.uniform(0, 1, (3000, d))
    y = rng.uniform(0, 1, (500, d))
    j, c = oracle.nearest(x, y)
    dist, jj = cKDTree(y).query(x)
    assert np.array_equal(j, jj)
    assert np.allclose(c, 0.5 * dist ** 2, rtol=1e-13, atol=1e-16)


def test_nearest_takes_the_lowest_index_on_ties():
    x = np.array([[0.5, 0.5], [0.0, 0.0]])
    y = np.array([[0.9, 0.9], [0.5, 0.5], [0.5, 0.5], [0.0, 0.0], [0.0, 0.0]])
    j, c = oracle.nearest(x, y)
    assert list(j) == [1, 3] and list(c) == [0.0, 0.0]


@pytest.mark.parametrize("d,tail", [(2, 1e-3), (3, 1e-8)])
def test_separable_matches_the_definition(d, tail):
    x, m, y, nu, psi, eps = rand_case(10 + d, d, 300, 60, 0.01, 0.02)
    a, b = truncation.separable_cutoffs(x, y, nu, psi, eps, tail)
    Jo, go, po, eo = oracle.dual_grad_sep(x, m, y, nu, psi, eps, a, b)
    Jb, gb, pb, eb = brute_sep(x, m, y, nu, psi, eps, a, b)
    assert (po, eo) == (pb, eb)
    assert abs(Jo - Jb) <= 1e-13 * abs(Jb)
    assert np.max(np.abs(go - gb)) <= 1e-14


def test_uniform_separable_cutoff_is_the_scalar_cutoff():
    x, m, y, nu, psi, eps = rand_case(3, 2, 400, 50, 0.02, 0.01)
    C = 0.03
    r1 = oracle.dual_grad(x, m, y, nu, psi, eps, cutoff=C)
    r2 = oracle.dual_grad_sep(x, m, y, nu, psi, eps, np.full(400, C), np.zeros(50))
    assert r1[0] == r2[0] and np.array_equal(r1[1], r2[1]) and r1[2:] == r2[2:]


@pytest.mark.parametrize("seed,d,eps,scale,tail,nu_spread", [
    (1, 2, 0.01, 0.03, 1e-2, 0.5),
    (2, 3, 0.005, 0.01, 1e-4, 0.9),
    (3, 2, 0.002, 0.05, 1e-6, 0.9),
    (4, 3, 0.02, 0.0, 1e-3, 0.0),
])
def test_tail_guarantee_against_dense(seed, d, eps, scale, tail, nu_spread):
    """0 <= J - J~ <= eps tail sum(nu) sum(m) and, per target,
    |g - g~| <= tail (sum(nu) (g~ + nu) + nu sum(m)); no point loses its
    nearest target, and the truncation actually removes pairs."""
    x, m, y, nu, psi, eps = rand_case(seed, d, 800, 120, eps, scale, nu_spread)
    a, b = truncation.separable_cutoffs(x, y, nu, psi, eps, tail)
    Jd, gd, _, _ = oracle.dual_grad(x, m, y, nu, psi, eps)
    Jt, gt, pt, et = oracle.dual_grad_sep(x, m, y, nu, psi, eps, a, b)
    assert et == 0
    assert pt < 800 * 120
    sm, snu = m.sum(), nu.sum()
    assert -1e-15 <= Jd - Jt <= eps * tail * snu * sm + 1e-15
    assert np.all(np.abs(gd - gt) <= tail * (snu * (gt + nu) + nu * sm) + 1e-16)


def test_separable_keeps_a_subset_of_the_global_tail_cutoff():
    x, m, y, nu, psi, eps = rand_case(8, 2, 600, 90, 0.005, 0.02, 0.9)
    tail = 1e-6
    a, b = truncation.separable_cutoffs(x, y, nu, psi, eps, tail)
    C0 = oracle.covering_cost(x, y)
    Ct = truncation.cutoff_tail(psi, nu, eps, tail, C0)
    assert np.all(a[:, None] + b[None, :] <= Ct * (1 + 1e-14))
    _, _, p_sep, _ = oracle.dual_grad_sep(x, m, y, nu, psi, eps, a, b)
    _, _, p_glob, _ = oracle.dual_grad(x, m, y, nu, psi, eps, cutoff=Ct)
    assert p_sep < p_glob
