"""Pins of the oracle's transport maps (Sec. 6.3) and conditional centroids
(Eq. barycenter_fixed_point) against closed forms, invariants and library
routines -- no GPU."""
import math

import numpy as np
import pytest

import oracle


def rand_case(seed, d, nq, n, eps, scale):
    rng = np.random.default_rng(seed)
    x = rng.uniform(0, 1, (nq, d))
    m = rng.uniform(0.5, 1.5, nq)
    m /= m.sum()
    y = rng.uniform(0, 1, (n, d))
    nu = rng.uniform(0.5, 1.5, n)
    nu /= nu.sum()
    psi = scale * rng.standard_normal(n)
    return x, m, y, nu, psi, eps


def test_single_target_maps_everything_to_it():
    x, m, y, nu, psi, eps = rand_case(1, 3, 200, 1, 0.05, 0.0)
    nu = np.ones(1)
    T, js = oracle.transport_maps(x, y, nu, psi, eps)
    assert np.all(js == 0)
    assert np.allclose(T, y[0], atol=1e-15)
    C, a = oracle.centroids(x, m, y, nu, psi, eps)
    assert np.allclose(C[0], m @ x, rtol=1e-14)        # the source's centre of mass
    assert abs(a[0] - 1.0) <= 1e-14


def test_two_targets_closed_form():
    """p_2 = 1 / (1 + exp(s_1 - s_2)) with s_j = (psi_j - |x - y_j|^2/2)/eps + ln nu_j,
    so T_bary = y_1 + p_2 (y_2 - y_1)."""
    rng = np.random.default_rng(2)
    x = rng.uniform(0, 1, (300, 2))
    y = np.array([[0.2, 0.3], [0.7, 0.6]])
    nu = np.array([0.3, 0.7])
    psi = np.array([0.01, -0.02])
    eps = 0.03
    T, js = oracle.transport_maps(x, y, nu, psi, eps)
    d2 = ((x[:, None, :] - y[None, :, :]) ** 2).sum(-1)
    s1 = (psi[0] - 0.5 * d2[:, 0]) / eps + math.log(nu[0])
    s2 = (psi[1] - 0.5 * d2[:, 1]) / eps + math.log(nu[1])
    p2 = 0.5 * (1.0 + np.tanh(0.5 * (s2 - s1)))       # logistic via tanh
    assert np.allclose(T, y[0] + p2[:, None] * (y[1] - y[0]), atol=1e-13)
    assert np.array_equal(js, (s2 > s1).astype(np.int64))


def test_coincident_targets():
    """All targets at one place: T_bary is that place and the mode follows
    psi_j + eps ln nu_j only (first index on ties)."""
    x, m, y, nu, psi, eps = rand_case(3, 2, 100, 6, 0.02, 0.0)
    y[:] = [0.4, 0.55]
    psi = np.array([0.0, 0.01, 0.01, -0.3, 0.005, 0.0])
    nu = np.full(6, 1 / 6)
    T, js = oracle.transport_maps(x, y, nu, psi, eps)
    assert np.allclose(T, y[0], atol=1e-15)
    assert np.all(js == 1)


def test_modal_map_is_nearest_target_for_zero_potential():
    """psi = 0, equal nu: the modal map is the Voronoi (nearest-target) map."""
    from scipy.spatial import cKDTree
    x, m, y, nu, psi, eps = rand_case(4, 3, 2000, 150, 0.01, 0.0)
    nu = np.full(150, 1 / 150)
    _, js = oracle.transport_maps(x, y, nu, psi, eps)
    _, nn = cKDTree(y).query(x)
    assert np.array_equal(js, nn)


def test_barycentric_map_tends_to_the_modal_map():
    """As eps -> 0 the plan concentrates on argmax_j s_qj (Sec. 6.3)."""
    x, m, y, nu, psi, _ = rand_case(5, 2, 400, 40, 0.0, 0.01)
    for eps in (1e-4, 1e-5):
        T, js = oracle.transport_maps(x, y, nu, psi, eps)
        d2 = ((x[:, None, :] - y[None, :, :]) ** 2).sum(-1)
        s = (psi[None, :] - 0.5 * d2) / eps + np.log(nu)[None, :]
        top2 = np.sort(s, axis=1)[:, -2:]
        clear = top2[:, 1] - top2[:, 0] > 40.0          # the runner-up weighs < e^-40
        assert clear.sum() > 200
        assert np.allclose(T[clear], y[js[clear]], atol=1e-12)


def test_maps_and_centroids_are_dual():
    """Remark conditional_expectations: sum_q m_q T_bary(x_q) = sum_j a_j y_j and
    sum_j nu_j T_j = sum_q m_q x_q (rows of the plan sum to 1), with
    a_j = dJ/dpsi_j + nu_j (Eq. gradient_compact_expanded)."""
    for d in (2, 3):
        x, m, y, nu, psi, eps = rand_case(6 + d, d, 700, 90, 0.02, 0.02)
        T, _ = oracle.transport_maps(x, y, nu, psi, eps)
        C, a = oracle.centroids(x, m, y, nu, psi, eps)
        _, g, _, _ = oracle.dual_grad(x, m, y, nu, psi, eps)
        assert np.allclose(a, g + nu, atol=1e-15)
        assert np.allclose(m @ T, a @ y, atol=1e-13)
        assert np.allclose(nu @ C, m @ x, atol=1e-13)


def test_centroids_tend_to_laguerre_cell_centroids():
    """eps -> 0: T_j -> (1/nu_j) sum of m_q x_q over the points whose mode is j."""
    x, m, y, nu, psi, _ = rand_case(9, 2, 3000, 25, 0.0, 0.01)
    eps = 1e-7
    C, a = oracle.centroids(x, m, y, nu, psi, eps)
    _, js = oracle.transport_maps(x, y, nu, psi, eps)
    d2 = ((x[:, None, :] - y[None, :, :]) ** 2).sum(-1)
    s = (psi[None, :] - 0.5 * d2) / eps + np.log(nu)[None, :]
    top2 = np.sort(s, axis=1)[:, -2:]
    clear = top2[:, 1] - top2[:, 0] > 40.0
    checked = 0
    for j in range(25):
        sel = js == j
        if not sel.any() or not clear[sel].all():
            continue
        ref = (m[sel, None] * x[sel]).sum(0) / nu[j]
        assert np.allclose(C[j], ref, atol=1e-10)
        assert abs(a[j] - m[sel].sum()) <= 1e-12
        checked += 1
    assert checked >= 5


def test_centroids_of_a_point_mass():
    """All mass at one point x0: T_j = x0 a_j / nu_j."""
    x, m, y, nu, psi, eps = rand_case(10, 3, 50, 12, 0.05, 0.03)
    x[:] = [0.3, 0.2, 0.9]
    C, a = oracle.centroids(x, m, y, nu, psi, eps)
    assert np.allclose(C, x[0][None, :] * (a / nu)[:, None], rtol=1e-13)
