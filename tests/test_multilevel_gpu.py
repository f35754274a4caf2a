"""Multilevel parts (Sec. 5): weighted k-means, softmax refinement against the
oracle, and the combined multilevel solve."""
import numpy as np
import pytest

import oracle
from oracle import lbfgs
import rsot_inputs as ri

pytestmark = pytest.mark.gpu


def rs():
    import paper_2507_23602_gb300 as m
    return m


@pytest.mark.parametrize("d,n,k", [(2, 3000, 50), (3, 5000, 128)])
def test_kmeans_clusters_and_weights(d, n, k):
    rng = np.random.default_rng(d + n)
    y = rng.uniform(0, 1, (n, d))
    w = rng.uniform(0.5, 1.5, n)
    C, W, a = rs().kmeans(y, w, k, iters=30, seed=6)
    assert np.all((a >= 0) & (a < k))
    # cluster weights are the summed weights (mass conservation, Sec. 5.2)
    assert np.allclose(W, np.bincount(a, weights=w, minlength=k), rtol=1e-12, atol=0)
    assert abs(W.sum() - w.sum()) <= 1e-9 * w.sum()
    # centres are the weighted centroids of the final clusters
    for t in range(d):
        ref = np.bincount(a, weights=w * y[:, t], minlength=k) / np.maximum(W, 1e-300)
        nz = W > 0
        assert np.allclose(C[nz, t], ref[nz], rtol=0, atol=1e-12)
    # after 30 Lloyd iterations nearly every point is nearest to its own centre
    D = ((y[:, None, :] - C[None, :, :]) ** 2).sum(-1)
    assert np.mean(np.argmin(D, 1) == a) > 0.97
    # deterministic
    C2, W2, a2 = rs().kmeans(y, w, k, iters=30, seed=6)
    assert np.array_equal(a, a2) and np.array_equal(C, C2)


def test_softmax_refine_matches_oracle():
    p = ri.make_problem(2, 12, 300, 0.02, src_seed=11, src_k=3, tgt_seed=12, nu_seed=13)
    rng = np.random.default_rng(3)
    psi_c = 0.02 * rng.standard_normal(p.n)
    y_f = rng.uniform(0, 1, (900, 2))
    P = rs().Problem(p.x, p.mass, p.y, p.nu)
    try:
        g = P.softmax_refine(psi_c, p.eps, y_f)
    finally:
        P.close()
    o = oracle.softmax_refine(p.x, p.mass, p.y, p.nu, psi_c, y_f, p.eps)
    assert np.max(np.abs(g - o)) <= 1e-4 * p.eps


def test_softmax_refine_fixed_point_at_the_optimum():
    p = ri.make_problem(3, 6, 200, 0.05, src_seed=21, src_k=2, tgt_seed=22, nu_seed=23)
    res = lbfgs.minimize(lambda q: oracle.dual_grad(p.x, p.mass, p.y, p.nu, q, p.eps)[:2],
                         np.zeros(p.n), 1e-12)
    P = rs().Problem(p.x, p.mass, p.y, p.nu)
    try:
        g = P.softmax_refine(res.x, p.eps, p.y)
    finally:
        P.close()
    assert np.max(np.abs(g - res.x)) <= 1e-4 * p.eps


def test_multilevel_solve_reaches_tolerance_and_matches_single_level():
    eps = 5e-3
    mix = ri.random_mixture(2, 3, 31)
    src = []
    for n in (12, 24, 48):
        v, c = ri.unit_square_tri_mesh(n)
        src.append(ri.source_measure(v, c, ri.tri_rule_deg2(), ri.mixture_density(mix, v)))
    y = ri.sample_mixture(ri.random_mixture(2, 2, 32), 4096, 33)
    nu = np.full(4096, 1 / 4096)
    tg = []
    for k in (256, 1024):
        C, W, _ = rs().kmeans(y, nu, k, iters=20, seed=6)
        keep = W > 0
        tg.append((C[keep], W[keep] / W[keep].sum()))
    tg.append((y, nu))
    psi, st = rs().multilevel_solve(src, tg, [2e-2, 1e-2, eps], tol_l1=1e-6,
                                    precision=rs().MIXED, refine_fp64=True)
    assert st["transfer"] == [0, 2, 2]
    assert st["grad_l1"] <= 1e-6
    xf, mf = src[-1]
    _, go, _, _ = oracle.dual_grad(xf, mf, y, nu, psi, eps)
    assert np.sum(np.abs(go)) <= 1e-6 * (1 + 1e-9)
    P = rs().Problem(xf, mf, y, nu)
    try:
        psi1, st1 = P.solve(eps=eps, tol_l1=1e-6, precision=rs().MIXED)
    finally:
        P.close()
    a, b = psi - psi @ nu, psi1 - psi1 @ nu
    assert np.max(np.abs(a - b)) <= 1e-3 * eps
