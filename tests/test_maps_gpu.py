"""Transport maps (Sec. 6.3), conditional centroids (Eq. barycenter_fixed_point)
and the damped Lloyd barycenter (Eq. damped_lloyd) on the GPU against the
oracle, through the C ABI.

Tolerances, from the arithmetic (FP32 pair exponents r = c_j + x'.w_j, log2
domain, three FMA with |terms| <= K = k (|y'|^2 + 2 |x'||y'|) + |b|, k =
log2(e)/(2 eps)): each exponent errs by <= 4 2^-24 K, so each plan weight by a
relative ln2 4 2^-24 K =: delta.
  T_bary: |T - T_o| <= delta max_j |y_j - T_o| (weights renormalised), x2 margin;
  modal map: where the indices differ, the oracle's score of the GPU's choice
             is within 2 delta of the maximum;
  centroids: a_j = sum_q m_q p_qj and nu_j T_j as the gradient (1e-6 absolute).
"""
import math

import numpy as np
import pytest

import oracle
from oracle import lbfgs

pytestmark = pytest.mark.gpu


def rs():
    import paper_2507_23602_gb300 as m
    return m


def case(seed, d, nq, n, eps, scale):
    rng = np.random.default_rng(seed)
    x = rng.uniform(0, 1, (nq, d))
    m = rng.uniform(0.5, 1.5, nq)
    m /= m.sum()
    y = rng.uniform(0, 1, (n, d))
    nu = rng.uniform(0.5, 1.5, n)
    nu /= nu.sum()
    return x, m, y, nu, scale * rng.standard_normal(n), eps


def delta_of(x, y, nu, psi, eps):
    k = math.log2(math.e) / (2 * eps)
    o = 0.5 * (np.minimum(x.min(0), y.min(0)) + np.maximum(x.max(0), y.max(0)))
    ry = np.max(np.linalg.norm(y - o, axis=1))
    rx = np.max(np.linalg.norm(x - o, axis=1))
    b = np.max(np.abs((psi - psi[0]) / eps + np.log(nu))) * math.log2(math.e)
    K = k * (ry * ry + 2 * rx * ry) + b
    return math.log(2) * 4 * 2.0 ** -24 * K


@pytest.mark.parametrize("d,nq,n,eps,scale", [
    (2, 3000, 700, 0.02, 0.02),
    (3, 2500, 1300, 0.005, 0.005),
    (3, 1025, 257, 0.1, 0.05),
    (2, 7, 3, 0.05, 0.05),
])
def test_transport_maps_parity(d, nq, n, eps, scale):
    x, m, y, nu, psi, eps = case(d * 100 + n, d, nq, n, eps, scale)
    To, jo = oracle.transport_maps(x, y, nu, psi, eps)
    P = rs().Problem(x, m, y, nu)
    try:
        T, js = P.transport_maps(psi, eps)
    finally:
        P.close()
    delta = delta_of(x, y, nu, psi, eps)
    spread = np.max(np.linalg.norm(y[None, :, :] - To[:, None, :], axis=2), axis=1)
    assert np.all(np.abs(T - To).max(axis=1) <= 2 * delta * spread + 1e-12)
    d2 = ((x[:, None, :] - y[None, :, :]) ** 2).sum(-1)
    s = (psi[None, :] - 0.5 * d2) / eps + np.log(nu)[None, :]
    q = np.arange(nq)
    assert np.all(s[q, js] >= s[q, jo] - 2 * delta)
    assert np.mean(js == jo) >= 0.99


def test_modal_map_of_zero_potential_is_nearest_target():
    from scipy.spatial import cKDTree
    x, m, y, nu, psi, eps = case(5, 3, 4000, 500, 0.01, 0.0)
    nu = np.full(500, 1 / 500)
    P = rs().Problem(x, m, y, nu)
    try:
        _, js = P.transport_maps(psi, eps, bary=False)
    finally:
        P.close()
    dist, nn = cKDTree(y).query(x, k=2)
    clear = dist[:, 1] - dist[:, 0] > 1e-5
    assert np.array_equal(js[clear], nn[clear, 0])


@pytest.mark.parametrize("d,nq,n,eps,scale", [
    (2, 3000, 700, 0.02, 0.02),
    (3, 4100, 1500, 0.005, 0.005),
    (2, 50, 9, 0.05, 0.05),
])
def test_centroids_parity(d, nq, n, eps, scale):
    x, m, y, nu, psi, eps = case(d * 7 + nq, d, nq, n, eps, scale)
    To, ao = oracle.centroids(x, m, y, nu, psi, eps)
    P = rs().Problem(x, m, y, nu)
    try:
        for kind in (rs().PAIRS_AUTO, rs().PAIRS_FP32):
            P.set_pair_kernel(kind)
            T, a = P.centroids(psi, eps)
            assert np.max(np.abs(a - ao)) <= 1e-6
            assert np.max(np.abs(nu[:, None] * (T - To))) <= 1e-6
            # the identity sum_j nu_j T_j = sum_q m_q x_q of the plan's rows
            assert np.allclose(nu @ T, m @ x, atol=1e-6)
    finally:
        P.close()


def test_barycenter_lloyd_matches_an_oracle_driven_loop():
    """Three damped Lloyd updates for two 2-D sources; the reference loop
    solves each RSOT problem with the oracle's L-BFGS (FP64) and forms the
    oracle's centroids."""
    rng = np.random.default_rng(11)
    srcs = []
    for s in range(2):
        x = rng.uniform(0, 1, (1500, 2)) * 0.5 + 0.25 * s
        mm = rng.uniform(0.5, 1.5, 1500)
        srcs.append((x, mm / mm.sum()))
    lam = np.array([0.4, 0.6])
    n, eps, theta = 40, 0.01, 0.5
    y0 = rng.uniform(0.2, 0.8, (n, 2))
    nu = np.full(n, 1 / n)
    y, st = rs().barycenter(srcs, lam, y0, nu, theta=theta, max_iter=3, tol_rms=0.0, eps=eps,
                            tol_l1=1e-9, raise_on_error=False)
    assert st["iterations"] == 3
    yr = y0.copy()
    psis = [np.zeros(n), np.zeros(n)]
    for it in range(3):
        ybar = np.zeros_like(yr)
        for i, (x, mm) in enumerate(srcs):
            res = lbfgs.minimize(lambda q: oracle.dual_grad(x, mm, yr, nu, q, eps)[:2], psis[i],
                                 tol_l1=1e-10)
            psis[i] = res.x
            T, _ = oracle.centroids(x, mm, yr, nu, res.x, eps)
            ybar += lam[i] * T
        yr = (1 - theta) * yr + theta * ybar
    # centroids carry the FP32 plan error of the mixed path (a few 1e-6 relative)
    assert np.max(np.abs(y - yr)) <= 1e-4, np.max(np.abs(y - yr))
