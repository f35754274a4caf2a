"""Parity of the compensated evaluation (double-float pair exponents,
ex2.approx, compensated sums) with the FP64 oracle, dense and truncated,
through the C ABI; and solves whose stop it certifies.

Tolerances are the evaluator's error budget (per-term relative errors of
ex2.approx and of the compensated sums, independent of sizes, eps and
potentials):
  gradient : |g_j - g_o,j| <= 6.0e-7 (g_o,j + nu_j) per entry, and
             ||g - g_o||_1 <= COMPENSATED_GRAD_REL sum_q m_q (= 6.5e-7 sum m)
  J        : |J - J_o| <= 3e-7 eps sum_q m_q + FP64 rounding of the
             assembled terms (1e-12 (|J_o| + sum |psi_j| nu_j))
  L_q      : |L - L_o| <= 4e-7 + 1e-12 |L_o|
"""
import numpy as np
import pytest

import oracle
import rsot_inputs as ri

pytestmark = pytest.mark.gpu

ENTRY_REL = 6.0e-7


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


def check_against(J, g, Jo, go, m, nu, psi, eps):
    err = np.abs(g - go)
    assert np.all(err <= ENTRY_REL * (go + nu) + 1e-17), np.max(err / (go + nu))
    assert err.sum() <= rs().COMPENSATED_GRAD_REL * m.sum(), err.sum()
    jtol = 3e-7 * eps * m.sum() + 1e-12 * (abs(Jo) + np.abs(psi) @ nu)
    assert abs(J - Jo) <= jtol, (J, Jo, abs(J - Jo), jtol)


@pytest.mark.parametrize("d,nq,n,eps,scale", [
    (2, 3000, 700, 0.02, 0.02),          # ragged tails on both sides
    (3, 2500, 1300, 0.005, 0.005),
    (3, 1025, 257, 1e-4, 1e-4),          # small eps: |exponents| ~ 1e4
    (2, 1, 1, 0.05, 0.0),                # one point, one target
    (3, 5, 2000, 0.01, 0.3),             # few points, large potentials
    (2, 4097, 3, 1e-3, 0.0),
])
def test_dense_parity(d, nq, n, eps, scale):
    x, m, y, nu, psi, eps = case(d * 1000 + nq + n, d, nq, n, eps, scale)
    Jo, go, _, _ = oracle.dual_grad(x, m, y, nu, psi, eps)
    P = rs().Problem(x, m, y, nu)
    try:
        J, g, pairs = P.eval(psi, eps, 0.0, rs().COMPENSATED)
        assert pairs == nq * n
        check_against(J, g, Jo, go, m, nu, psi, eps)
        L = P.point_log_partition()
        Lo = oracle.point_lse(x, y, nu, psi, eps)
        assert np.all(np.abs(L - Lo) <= 4e-7 + 1e-12 * np.abs(Lo))
    finally:
        P.close()


def test_zero_masses_and_coincident_points():
    x, m, y, nu, psi, eps = case(7, 3, 2048, 600, 0.01, 0.01)
    m[::3] = 0.0
    x[100:200] = x[100]
    y[50:60] = y[50]
    Jo, go, _, _ = oracle.dual_grad(x, m, y, nu, psi, eps)
    P = rs().Problem(x, m, y, nu)
    try:
        J, g, _ = P.eval(psi, eps, 0.0, rs().COMPENSATED)
        check_against(J, g, Jo, go, m, nu, psi, eps)
    finally:
        P.close()


@pytest.mark.parametrize("d,nq,n,eps,radius", [
    (2, 3000, 900, 0.01, 0.25),
    (3, 2600, 1100, 0.004, 0.3),
    (3, 1500, 400, 1e-4, 0.35),
])
def test_truncated_parity_same_pairs_as_fp64(d, nq, n, eps, radius):
    x, m, y, nu, psi, eps = case(d * 31 + nq, d, nq, n, eps, eps)
    C = 0.5 * radius * radius
    Jo, go, po, eo = oracle.dual_grad(x, m, y, nu, psi, eps, cutoff=C)
    assert eo == 0
    P = rs().Problem(x, m, y, nu)
    try:
        J, g, pairs = P.eval(psi, eps, radius, rs().COMPENSATED)
        # the oracle tests c < C in the caller's frame, the GPU paths in the
        # translated one: FP64 rounding may move a pair at the cutoff
        assert abs(pairs - po) <= 16 + 1e-6 * po
        check_against(J, g, Jo, go, m, nu, psi, eps)
        J64, g64, p64 = P.eval(psi, eps, radius, rs().FP64)
        assert p64 == pairs                  # the same membership test as the FP64 path
        check_against(J, g, J64, g64, m, nu, psi, eps)
    finally:
        P.close()


def test_truncated_empty_neighbourhood_is_reported():
    x, m, y, nu, psi, eps = case(5, 2, 500, 40, 0.01, 0.0)
    x[0] = [5.0, 5.0]                     # far from every target
    radius = 0.5
    Jo, go, po, eo = oracle.dual_grad(x, m, y, nu, psi, eps, cutoff=0.5 * radius * radius)
    assert eo >= 1
    P = rs().Problem(x, m, y, nu)
    try:
        with pytest.raises(rs().RsotError) as ei:
            P.eval(psi, eps, radius, rs().COMPENSATED)
        assert ei.value.status == 4
        J, g, pairs = P.eval(psi, eps, radius, rs().COMPENSATED, allow_empty=True)
        assert abs(pairs - po) <= 16 + 1e-6 * po
        check_against(J, g, Jo, go, m, nu, psi, eps)
    finally:
        P.close()


def test_full_size_cube_against_the_fp64_path():
    """786,432 points x 65,536 targets (the unit-cube workload): the
    compensated gradient against the FP64 path's (itself within 1e-10 of the
    oracle), L1 within the certified bound, at a potential away from 0."""
    p = ri.cube_3d()
    rng = np.random.default_rng(3)
    psi = 2e-3 * rng.standard_normal(p.n)
    P = rs().Problem(p.x, p.mass, p.y, p.nu)
    try:
        J64, g64, _ = P.eval(psi, p.eps, 0.0, rs().FP64)
        J, g, _ = P.eval(psi, p.eps, 0.0, rs().COMPENSATED)
        check_against(J, g, J64, g64, p.mass, p.nu, psi, p.eps)
        # the mixed path's error is far above the compensated one here
        Jm, gm, _ = P.eval(psi, p.eps, 0.0, rs().MIXED)
        assert np.abs(g - g64).sum() < 0.2 * np.abs(gm - g64).sum()
    finally:
        P.close()


def test_solve_with_compensated_refinement_certifies_tolerance():
    """Default refinement: the returned potential's exact (oracle) gradient
    meets tol_l1 with no slack."""
    p = ri.make_problem(3, 10, 2000, 5e-3, src_seed=71, src_k=3, tgt_seed=72, tgt_k=2, nu_seed=73)
    P = rs().Problem(p.x, p.mass, p.y, p.nu)
    try:
        psi, st = P.solve(eps=p.eps, eps_start=0.1, eps_factor=0.5, tol_l1=1e-6,
                          precision=rs().MIXED, refine_fp64=True)
        assert st.status == 0
        assert st.grad_l1 <= 1e-6 - rs().COMPENSATED_GRAD_REL * p.mass.sum()
        _, go, _, _ = oracle.dual_grad(p.x, p.mass, p.y, p.nu, psi, p.eps)
        assert np.sum(np.abs(go)) <= 1e-6
    finally:
        P.close()


def test_compensated_solve_and_fp64_reference_option():
    p = ri.make_problem(2, 16, 300, 0.01, src_seed=81, src_k=2, tgt_seed=82)
    P = rs().Problem(p.x, p.mass, p.y, p.nu)
    try:
        psi, st = P.solve(eps=p.eps, tol_l1=2e-6, precision=rs().COMPENSATED)
        assert st.status == 0
        _, go, _, _ = oracle.dual_grad(p.x, p.mass, p.y, p.nu, psi, p.eps)
        assert np.sum(np.abs(go)) <= 2e-6
        # tol below the certified bound's room: the last stage finishes in FP64
        psi2, st2 = P.solve(eps=p.eps, tol_l1=5e-7, precision=rs().COMPENSATED)
        assert st2.status == 0
        _, go2, _, _ = oracle.dual_grad(p.x, p.mass, p.y, p.nu, psi2, p.eps)
        assert np.sum(np.abs(go2)) <= 5e-7 * (1 + 1e-9)
        # FP64 reference evaluations on request
        psi3, st3 = P.solve(eps=p.eps, tol_l1=1e-6, refine_precision=rs().FP64)
        assert st3.status == 0
        _, go3, _, _ = oracle.dual_grad(p.x, p.mass, p.y, p.nu, psi3, p.eps)
        assert np.sum(np.abs(go3)) <= 1e-6 * (1 + 1e-9)
    finally:
        P.close()


@pytest.mark.parametrize("d", [2, 3])
def test_truncated_pairs_at_the_cutoff_match_fp64(d):
    """Points and targets on lattices with the cutoff radius a lattice distance:
    many pairs sit at the cutoff, where the exponent test of the truncated
    compensated passes is undecided and the FP64 expression decides, so the
    kept pairs equal the FP64 path's exactly (the oracle tests in the caller's
    frame, so it may differ by those boundary pairs only)."""
    k = 24 if d == 2 else 10
    g = np.arange(k) / k
    x = np.stack(np.meshgrid(*([g] * d), indexing="ij"), -1).reshape(-1, d)
    gy = np.arange(k // 2) / (k // 2) + 0.5 / k
    y = np.stack(np.meshgrid(*([gy] * d), indexing="ij"), -1).reshape(-1, d)
    rng = np.random.default_rng(90 + d)
    m = rng.uniform(0.5, 1.5, x.shape[0])
    m /= m.sum()
    nu = rng.uniform(0.5, 1.5, y.shape[0])
    nu /= nu.sum()
    psi = np.zeros(y.shape[0])
    eps = 0.01
    radius = np.sqrt(d) * 1.5 / k           # the distance of many lattice pairs
    C = 0.5 * radius * radius
    Jo, go, po, eo = oracle.dual_grad(x, m, y, nu, psi, eps, cutoff=C)
    d2 = ((x[:, None, :] - y[None, :, :]) ** 2).sum(-1) * 0.5
    at_cut = int(np.sum(np.abs(d2 - C) <= 1e-12))
    assert at_cut > 100                       # the case really tests the band
    P = rs().Problem(x, m, y, nu)
    try:
        J64, g64, p64 = P.eval(psi, eps, radius, rs().FP64, allow_empty=True)
        J, g, pairs = P.eval(psi, eps, radius, rs().COMPENSATED, allow_empty=True)
        assert pairs == p64
        assert abs(pairs - po) <= at_cut
        assert np.abs(g - g64).sum() <= rs().COMPENSATED_GRAD_REL * m.sum()
    finally:
        P.close()
