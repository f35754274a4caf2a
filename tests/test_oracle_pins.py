"""Pins of the FP64 oracle against facts the paper and the mathematics fix.

None of these checks goes back to the oracle's own formulas: each compares it
with a closed form, an invariant, a bound, a library routine or brute force,
chosen so that a dropped term, a wrong sign, a swapped index or a transposed
operand in the oracle fails at least one of them.
"""
import math

import numpy as np
import pytest
import scipy.special
from scipy.spatial import cKDTree

import oracle
from oracle import lbfgs, truncation
import rsot_inputs as ri


def tiny_problem(seed, d=2, nq=40, n=7, eps=0.05, psi_scale=0.05):
    rng = np.random.default_rng(seed)
    x = rng.uniform(0, 1, (nq, d))
    m = rng.uniform(0.5, 1.5, nq)
    m /= m.sum()
    y = rng.uniform(0, 1, (n, d))
    nu = rng.uniform(0.5, 1.5, n)
    nu /= nu.sum()
    psi = psi_scale * rng.standard_normal(n)
    return x, m, y, nu, psi, eps


# ---------------------------------------------------------------- inputs ---

def test_tri_rule_integrates_quadratics_exactly():
    """Degree-2 exactness of the 3-point rule on the structured square mesh."""
    verts, cells = ri.unit_square_tri_mesh(5)
    x, w, _, _ = ri.quadrature(verts, cells, ri.tri_rule_deg2())
    for a in range(3):
        for b in range(3 - a):
            exact = 1.0 / ((a + 1) * (b + 1))
            assert abs(np.sum(w * x[:, 0] ** a * x[:, 1] ** b) - exact) < 1e-14
    # and not degree 3 on a single cell (so the rule is really degree 2)
    v = np.array([[0.0, 0.0], [1.0, 0.0], [0.0, 1.0]])
    xx, ww, _, _ = ri.quadrature(v, np.array([[0, 1, 2]]), ri.tri_rule_deg2())
    assert abs(np.sum(ww * xx[:, 0] ** 3) - 1.0 / 20.0) > 1e-4


def test_tet_rule_integrates_quadratics_exactly():
    verts, cells = ri.unit_cube_tet_mesh(3)
    x, w, _, _ = ri.quadrature(verts, cells, ri.tet_rule_deg2())
    assert x.shape[0] == 27 * 6 * 4
    for a in range(3):
        for b in range(3 - a):
            for c in range(3 - a - b):
                exact = 1.0 / ((a + 1) * (b + 1) * (c + 1))
                got = np.sum(w * x[:, 0] ** a * x[:, 1] ** b * x[:, 2] ** c)
                assert abs(got - exact) < 1e-14


def test_config_sizes():
    p = ri.small_2d()
    assert p.nq == 24576 and p.n == 512 and p.d == 2
    assert abs(p.mass.sum() - 1) < 1e-14 and abs(p.nu.sum() - 1) < 1e-14
    assert np.all(p.mass > 0)
    verts, cells = ri.unit_cube_tet_mesh(32)
    assert cells.shape[0] * 4 == 786432


def test_p1_density_is_interpolated():
    """A linear density is reproduced exactly by the P1 interpolant."""
    verts, cells = ri.unit_square_tri_mesh(4)
    rho_v = 1.0 + verts[:, 0] + 2.0 * verts[:, 1]
    x, m = ri.source_measure(verts, cells, ri.tri_rule_deg2(), rho_v, normalize=False)
    _, w, _, _ = ri.quadrature(verts, cells, ri.tri_rule_deg2())
    assert np.allclose(m, w * (1.0 + x[:, 0] + 2.0 * x[:, 1]), rtol=1e-14, atol=0)


# ------------------------------------------------------------- softmax ----

def test_plan_rows_sum_to_one():
    """sum_j p_j(x|psi) = 1 at every x (Remark 'Plan Density Interpretation')."""
    x, m, y, nu, psi, eps = tiny_problem(1, nq=30, n=9)
    P = oracle.plan(x, y, nu, psi, eps)
    assert np.all(P >= 0)
    assert np.max(np.abs(P.sum(1) - 1.0)) < 1e-14


def test_plan_matches_library_softmax():
    """p_qj equals scipy's softmax of (psi_j - c_qj)/eps + ln nu_j over j."""
    x, m, y, nu, psi, eps = tiny_problem(2, d=3, nq=11, n=6)
    P = oracle.plan(x, y, nu, psi, eps)
    C = 0.5 * ((x[:, None, :] - y[None, :, :]) ** 2).sum(-1)
    ref = scipy.special.softmax((psi[None, :] - C) / eps + np.log(nu)[None, :], axis=1)
    assert np.allclose(P, ref, rtol=1e-13, atol=1e-300)


def test_plan_coincident_targets():
    """All targets at one place: p_qj = softmax_j(psi_j/eps + ln nu_j), any q."""
    x, m, y, nu, psi, eps = tiny_problem(3, n=5)
    y[:] = y[0]
    P = oracle.plan(x, y, nu, psi, eps)
    ref = scipy.special.softmax(psi / eps + np.log(nu))
    assert np.allclose(P, ref[None, :], rtol=1e-13)


def test_point_lse_matches_library_logsumexp_and_J():
    """L_q equals scipy's logsumexp of (psi_j - c_qj)/eps with weights nu_j,
    and sum_q m_q eps L_q - psi.nu reproduces J."""
    x, m, y, nu, psi, eps = tiny_problem(20, d=3, nq=40, n=9, eps=0.02)
    L = oracle.point_lse(x, y, nu, psi, eps)
    C = 0.5 * ((x[:, None, :] - y[None, :, :]) ** 2).sum(-1)
    ref = scipy.special.logsumexp((psi[None, :] - C) / eps, b=nu[None, :], axis=1)
    assert np.allclose(L, ref, rtol=1e-14, atol=1e-13)
    J, _, _, _ = oracle.dual_grad(x, m, y, nu, psi, eps)
    assert abs(np.sum(m * eps * L) - psi @ nu - J) < 1e-15


# ----------------------------------------------------- dual value / grad ---

def test_single_target_closed_form():
    """N = 1, nu = 1: J = sum_q m_q (psi - c_q) - psi = -sum_q m_q c_q, grad = 0."""
    x, m, y, nu, psi, eps = tiny_problem(4, nq=50, n=1)
    nu = np.ones(1)
    for p in (0.0, 0.3, -2.0):
        J, g, pairs, empty = oracle.dual_grad(x, m, y, nu, np.array([p]), eps)
        c = 0.5 * np.sum((x - y[0]) ** 2, axis=1)
        assert abs(J - (-np.sum(m * c))) < 1e-15
        assert abs(g[0]) < 1e-15
        assert pairs == 50 and empty == 0


@pytest.mark.parametrize("seed,d", [(5, 2), (6, 3)])
def test_gradient_mass_balance(seed, d):
    """sum_k dJ/dpsi_k = sum_q m_q - sum_k nu_k = 0 (Eq. gradient_compact_expanded)."""
    x, m, y, nu, psi, eps = tiny_problem(seed, d=d, nq=200, n=17)
    J, g, _, _ = oracle.dual_grad(x, m, y, nu, psi, eps)
    assert abs(g.sum()) < 1e-15
    assert np.all(g + nu >= 0)            # received masses are non-negative


@pytest.mark.parametrize("c", [-3.0, 0.5, 7.0])
def test_shift_invariance(c):
    """J(psi + c 1) = J(psi), grad unchanged, when sum m = sum nu = 1 (App. A)."""
    x, m, y, nu, psi, eps = tiny_problem(7, nq=120, n=11)
    J0, g0, _, _ = oracle.dual_grad(x, m, y, nu, psi, eps)
    J1, g1, _, _ = oracle.dual_grad(x, m, y, nu, psi + c, eps)
    assert abs(J1 - J0) < 1e-13 * max(1.0, abs(c))
    assert np.max(np.abs(g1 - g0)) < 1e-14


def test_shift_changes_J_when_masses_unbalanced():
    """With sum m != sum nu: J(psi + c1) = J(psi) + c (sum m - sum nu)."""
    x, m, y, nu, psi, eps = tiny_problem(8, nq=60, n=5)
    m2 = 1.3 * m
    J0, _, _, _ = oracle.dual_grad(x, m2, y, nu, psi, eps)
    J1, _, _, _ = oracle.dual_grad(x, m2, y, nu, psi + 0.25, eps)
    assert abs((J1 - J0) - 0.25 * (1.3 - 1.0)) < 1e-14


@pytest.mark.parametrize("seed,d,eps", [(9, 2, 0.05), (10, 3, 0.02), (11, 2, 0.2)])
def test_gradient_central_differences(seed, d, eps):
    """J is C-infinity: grad matches central differences to O(h^2)."""
    x, m, y, nu, psi, _ = tiny_problem(seed, d=d, nq=150, n=8, eps=eps)
    J, g, _, _ = oracle.dual_grad(x, m, y, nu, psi, eps)
    rng = np.random.default_rng(seed + 100)
    for _ in range(3):
        v = rng.standard_normal(psi.shape)
        errs = []
        for h in (4e-4 * eps, 2e-4 * eps):
            Jp, _, _, _ = oracle.dual_grad(x, m, y, nu, psi + h * v, eps)
            Jm, _, _, _ = oracle.dual_grad(x, m, y, nu, psi - h * v, eps)
            errs.append(abs((Jp - Jm) / (2 * h) - g @ v))
        assert errs[1] < 1e-8 * max(1.0, abs(g @ v) * 1e3)
        # second order: halving h divides the error by ~4 (until round-off)
        assert errs[1] < 1e-11 or 3.0 < errs[0] / errs[1] < 5.0
    # coordinate-wise too: a transposed index would show here
    for k in range(len(psi)):
        e = np.zeros_like(psi)
        e[k] = 1e-4 * eps
        Jp, _, _, _ = oracle.dual_grad(x, m, y, nu, psi + e, eps)
        Jm, _, _, _ = oracle.dual_grad(x, m, y, nu, psi - e, eps)
        assert abs((Jp - Jm) / (2e-4 * eps) - g[k]) < 1e-8


def test_convexity_along_lines():
    x, m, y, nu, psi, eps = tiny_problem(12, nq=100, n=9)
    rng = np.random.default_rng(3)
    v = rng.standard_normal(psi.shape)
    ts = np.linspace(-1, 1, 21) * 0.1
    Js = np.array([oracle.dual_grad(x, m, y, nu, psi + t * v, eps)[0] for t in ts])
    assert np.all(Js[:-2] - 2 * Js[1:-1] + Js[2:] >= -1e-14)


def test_lse_sandwich():
    """max_j s <= LSE_j s <= max_j s + ln N gives bounds on J (App. A)."""
    x, m, y, nu, psi, eps = tiny_problem(13, d=3, nq=80, n=12, eps=0.03)
    J, _, _, _ = oracle.dual_grad(x, m, y, nu, psi, eps)
    C = 0.5 * ((x[:, None, :] - y[None, :, :]) ** 2).sum(-1)
    smax = np.max((psi[None, :] - C) / eps + np.log(nu)[None, :], axis=1)
    lo = np.sum(m * eps * smax) - psi @ nu
    assert lo <= J <= lo + eps * math.log(len(nu)) + 1e-15
    # the paper's own lower bound (App. A): J + psi.nu >= sum_q m_q max_j (psi_j - c_qj + eps ln nu_j)
    assert J + psi @ nu >= np.sum(m * np.max(psi[None, :] - C + eps * np.log(nu)[None, :], axis=1)) - 1e-15


def test_laguerre_limit_small_eps():
    """As eps -> 0 with psi fixed, dJ/dpsi_j -> (mass of the Laguerre cell of j) - nu_j
    (Remark 'Connection to Power Diagrams'); brute-force argmax on a tiny input."""
    rng = np.random.default_rng(14)
    x = rng.uniform(0, 1, (300, 2))
    m = np.full(300, 1 / 300)
    y = rng.uniform(0, 1, (6, 2))
    nu = np.full(6, 1 / 6)
    psi = 0.05 * rng.standard_normal(6)
    C = 0.5 * ((x[:, None, :] - y[None, :, :]) ** 2).sum(-1)
    U = psi[None, :] - C
    srt = np.sort(U, axis=1)
    assert np.min(srt[:, -1] - srt[:, -2]) > 5e-5      # distinct maxima
    owner = np.argmax(U, axis=1)
    lag = np.bincount(owner, weights=m, minlength=6) - nu
    errs = []
    for eps in (1e-1, 1e-2, 1e-3, 1e-4, 1e-6, 1e-7):
        _, g, _, _ = oracle.dual_grad(x, m, y, nu, psi, eps)
        errs.append(np.max(np.abs(g - lag)))
    assert all(errs[i + 1] <= errs[i] + 1e-15 for i in range(len(errs) - 1))
    assert errs[-1] < 1e-12


# ------------------------------------------- 1-D two-target closed form ---

def _two_target_case(mesh_n, eps, a, b, psi, nu):
    """Uniform density on the unit square, targets (a, 1/2) and (b, 1/2): the
    problem reduces to 1-D in x_1 (the x_2 part of the cost is common)."""
    verts, cells = ri.unit_square_tri_mesh(mesh_n)
    x, m = ri.source_measure(verts, cells, ri.tri_rule_deg2(), np.ones(len(verts)))
    y = np.array([[a, 0.5], [b, 0.5]])
    return x, m, y


def _softplus(t):
    return np.logaddexp(0.0, t)


def _exact_two_target(eps, a, b, psi, nu):
    import mpmath
    mpmath.mp.dps = 40
    alpha = (psi[1] - psi[0] + 0.5 * (a * a - b * b)) / eps + math.log(nu[1] / nu[0])
    beta = (b - a) / eps
    g2 = (float(_softplus(alpha + beta)) - float(_softplus(alpha))) / beta - nu[1]
    sp = mpmath.quad(lambda t: mpmath.log1p(mpmath.exp(alpha + beta * t)), [0, 0.5, 1])
    J = (psi[0] - 0.5 * ((1 - a) ** 3 + a ** 3) / 3.0 - 0.5 / 12.0 + eps * math.log(nu[0])
         + eps * float(sp) - psi @ nu)
    return J, np.array([-g2, g2])


def test_two_target_1d_closed_form_and_convergence_order():
    eps, a, b = 0.05, 0.3, 0.7
    psi = np.array([0.01, -0.02])
    nu = np.array([0.4, 0.6])
    Jx, gx = _exact_two_target(eps, a, b, psi, nu)
    errJ, errg = [], []
    for n in (8, 16, 32, 64):
        x, m, y = _two_target_case(n, eps, a, b, psi, nu)
        J, g, _, _ = oracle.dual_grad(x, m, y, nu, psi, eps)
        errJ.append(abs(J - Jx))
        errg.append(abs(g[1] - gx[1]))
    assert errJ[-1] < 1e-6 and errg[-1] < 1e-6
    # degree-2 rule: global error O(h^3); accept an observed order >= 2.5
    for e in (errJ, errg):
        rates = [math.log2(e[i] / e[i + 1]) for i in range(len(e) - 1)]
        assert min(rates[1:]) > 2.5, rates


def test_two_target_solve_matches_exact_minimiser():
    """L-BFGS on the embedded 2-target problem converges to the root of
    softplus(alpha+beta) - softplus(alpha) = beta nu_2."""
    from scipy.optimize import brentq
    eps, a, b = 0.05, 0.3, 0.7
    nu = np.array([0.4, 0.6])
    beta = (b - a) / eps
    alpha = brentq(lambda t: _softplus(t + beta) - _softplus(t) - beta * nu[1], -50, 50, xtol=1e-15)
    dpsi_exact = eps * (alpha - math.log(nu[1] / nu[0])) - 0.5 * (a * a - b * b)
    x, m, y = _two_target_case(64, eps, a, b, np.zeros(2), nu)
    res = lbfgs.minimize(lambda p: oracle.dual_grad(x, m, y, nu, p, eps)[:2], np.zeros(2), 1e-13)
    assert res.status == "converged"
    assert abs((res.x[1] - res.x[0]) - dpsi_exact) < 1e-6


# ------------------------------------------------------------ truncation ---

def test_cutoff_infinite_is_dense_and_zero_is_empty():
    x, m, y, nu, psi, eps = tiny_problem(15, nq=70, n=10)
    Jd, gd, pd, ed = oracle.dual_grad(x, m, y, nu, psi, eps)
    assert pd == 700 and ed == 0
    J0, g0, p0, e0 = oracle.dual_grad(x, m, y, nu, psi, eps, cutoff=0.0)
    assert p0 == 0 and e0 == 70
    assert J0 == pytest.approx(-psi @ nu, abs=1e-16)
    assert np.allclose(g0, -nu, atol=0)


def test_truncation_pairs_match_brute_force_count():
    x, m, y, nu, psi, eps = tiny_problem(16, d=3, nq=90, n=25)
    C = 0.5 * ((x[:, None, :] - y[None, :, :]) ** 2).sum(-1)
    for cut in (0.01, 0.05, 0.2):
        _, _, pairs, empty = oracle.dual_grad(x, m, y, nu, psi, eps, cutoff=cut)
        assert pairs == int(np.sum(C < cut))
        assert empty == int(np.sum(~np.any(C < cut, axis=1)))


def test_covering_cost_matches_kdtree():
    rng = np.random.default_rng(17)
    x = rng.uniform(0, 1, (500, 3))
    y = rng.uniform(0, 1, (60, 3))
    dist, _ = cKDTree(y).query(x)
    assert oracle.covering_cost(x, y) == pytest.approx(0.5 * np.max(dist) ** 2, rel=1e-14)


@pytest.mark.parametrize("tail", [1e-2, 1e-4])
def test_tail_cutoff_error_bounds(tail):
    """With C = C_0 + Gamma + eps ln(1/(nu_min tail)) no point loses all its
    targets, |J - J_trunc| <= eps tail sum m, and per target
    |g - g_trunc| <= tail (sum_q m_q p~_qj + nu_j)."""
    p = ri.make_problem(2, 12, 200, 0.01, src_seed=21, src_k=3, tgt_seed=22, nu_seed=23)
    rng = np.random.default_rng(24)
    psi = 0.02 * rng.standard_normal(p.n)
    C0 = oracle.covering_cost(p.x, p.y)
    C = truncation.cutoff_tail(psi, p.nu, p.eps, tail, C0)
    assert C > C0
    Jd, gd, pd, _ = oracle.dual_grad(p.x, p.mass, p.y, p.nu, psi, p.eps)
    Jt, gt, pt, et = oracle.dual_grad(p.x, p.mass, p.y, p.nu, psi, p.eps, cutoff=C)
    assert et == 0 and pt < pd
    assert 0.0 <= Jd - Jt <= p.eps * tail + 1e-16
    recv_t = gt + p.nu
    assert np.all(np.abs(gd - gt) <= tail * (recv_t + p.nu) + 1e-16)
    assert np.sum(np.abs(gd - gt)) <= 2 * tail + 1e-15


def test_pointwise_cutoff_drops_only_small_terms():
    """C_pw guarantees every dropped term nu_j exp((psi_j - c)/eps) < delta_thr."""
    x, m, y, nu, psi, eps = tiny_problem(18, nq=60, n=20, eps=0.01)
    dthr = 1e-6
    C = truncation.cutoff_pointwise(psi, nu, eps, dthr)
    Cm = 0.5 * ((x[:, None, :] - y[None, :, :]) ** 2).sum(-1)
    dropped = Cm >= C
    terms = nu[None, :] * np.exp((psi[None, :] - Cm) / eps)
    assert np.all(terms[dropped] <= dthr * (1 + 1e-12))


def test_geometric_cutoff_relative_error():
    """C_geom(tau) keeps |J - J_trunc| <= tau |J| (App. B)."""
    p = ri.make_problem(2, 10, 150, 0.02, src_seed=31, src_k=3, tgt_seed=32)
    psi = 0.03 * np.random.default_rng(33).standard_normal(p.n)
    Jd, _, _, _ = oracle.dual_grad(p.x, p.mass, p.y, p.nu, psi, p.eps)
    C0 = oracle.covering_cost(p.x, p.y)
    for tau in (1e-2, 1e-4):
        C = truncation.cutoff_geometric(psi, p.nu, p.eps, tau, Jd, C0)
        Jt, _, _, et = oracle.dual_grad(p.x, p.mass, p.y, p.nu, psi, p.eps, cutoff=C)
        assert et == 0
        assert abs(Jd - Jt) <= tau * abs(Jd)


# ------------------------------------------------------ softmax refinement ---

def test_softmax_refinement_fixed_point():
    """At the minimiser of the coarse problem the marginal condition
    int nu_k exp((psi_k - c)/eps)/S dmu = nu_k holds, so refining onto the
    same targets returns psi itself (Eq. softmax_refinement_formula)."""
    p = ri.make_problem(2, 10, 40, 0.05, src_seed=41, src_k=2, tgt_seed=42, nu_seed=43)
    fun = lambda q: oracle.dual_grad(p.x, p.mass, p.y, p.nu, q, p.eps)[:2]
    res = lbfgs.minimize(fun, np.zeros(p.n), 1e-12)
    assert res.status == "converged"
    psi_ref = oracle.softmax_refine(p.x, p.mass, p.y, p.nu, res.x, p.y, p.eps)
    assert np.max(np.abs(psi_ref - res.x)) < 1e-9


def test_softmax_refinement_single_coarse_target():
    """One coarse target (nu = 1): S_c(x) = exp((psi - c(x,y_c))/eps), so the
    formula is -eps ln sum_q m_q exp((c(x_q,y_c) - c(x_q,y_k))/eps) + psi."""
    x, m, y, nu, psi, eps = tiny_problem(19, nq=50, n=4)
    yc = np.array([[0.4, 0.6]])
    out = oracle.softmax_refine(x, m, yc, np.ones(1), np.array([0.07]), y, eps)
    cc = 0.5 * np.sum((x - yc[0]) ** 2, axis=1)
    for k in range(len(y)):
        ck = 0.5 * np.sum((x - y[k]) ** 2, axis=1)
        ref = -eps * scipy.special.logsumexp((cc - ck) / eps, b=m) + 0.07
        assert out[k] == pytest.approx(ref, abs=1e-13)


# ---------------------------------------------------------------- L-BFGS ---

def test_lbfgs_quadratic():
    rng = np.random.default_rng(50)
    A = rng.standard_normal((12, 12))
    A = A @ A.T + 12 * np.eye(12)
    bvec = rng.standard_normal(12)
    res = lbfgs.minimize(lambda z: (0.5 * z @ A @ z - bvec @ z, A @ z - bvec), np.zeros(12), 1e-10)
    assert res.status == "converged"
    assert np.allclose(res.x, np.linalg.solve(A, bvec), atol=1e-10)


def test_lbfgs_rosenbrock():
    def f(z):
        a, b = z
        return ((1 - a) ** 2 + 100 * (b - a * a) ** 2,
                np.array([-2 * (1 - a) - 400 * a * (b - a * a), 200 * (b - a * a)]))
    res = lbfgs.minimize(f, np.array([-1.2, 1.0]), 1e-10)
    assert res.status == "converged"
    assert np.allclose(res.x, [1.0, 1.0], atol=1e-8)


def test_oracle_solve_small_problem_reaches_tolerance():
    p = ri.make_problem(2, 8, 30, 0.02, src_seed=61, src_k=3, tgt_seed=62)
    fun = lambda q: oracle.dual_grad(p.x, p.mass, p.y, p.nu, q, p.eps)[:2]
    res = lbfgs.minimize(fun, np.zeros(p.n), 1e-9)
    assert res.status == "converged"
    assert np.sum(np.abs(res.g)) <= 1e-9
