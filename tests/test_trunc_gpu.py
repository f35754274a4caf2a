"""Parity of the truncated (cell-list) CUDA path with the oracle's truncated
evaluation (Algorithm 2 with I_q = {j : c(x_q, y_j) < C}, every j tested).

Tolerances: as for the dense path (mixed: J 1e-5 relative, gradient 1e-6
absolute per entry; FP64: 1e-10).  Pairs within FP32 rounding of the cutoff
may be classified differently by the two sides (their terms are bounded by the
tail), so the pair counts must agree to a few boundary pairs.
"""
import math

import numpy as np
import pytest

import oracle
from oracle import truncation
import rsot_inputs as ri

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


def tensor_tols(m, nu, eps, Jo):
    """Bounds of the tensor-core pair kernel forced onto any problem (its
    exponents err by rms ~2e-5 in log2 units): five standard deviations of the
    resulting gradient / J errors, never below the mixed path's own bounds."""
    g_tol = max(1e-6, 5 * 1.4e-5 * math.sqrt(m.max() * nu.max()))
    j_tol = max(1e-5 * abs(Jo), 5 * eps * math.log(2) * 2e-5 * math.sqrt(np.sum(m * m)))
    return g_tol, j_tol


def compare(P, x, m, y, nu, psi, eps, radius, precs=(1, 0), allow_empty=False):
    """The FP64 path, and the mixed path with the automatic, FP32 and forced
    tensor-core pair kernels, against the oracle's truncated evaluation."""
    C = 0.5 * radius * radius
    Jo, go, po, eo = oracle.dual_grad(x, m, y, nu, psi, eps, cutoff=C)
    out = {}
    runs = [(prec, kind) for prec in precs
            for kind in ((None,) if prec == 0 else
                         (rs().PAIRS_AUTO, rs().PAIRS_FP32, rs().PAIRS_TENSOR))]
    try:
        for prec, kind in runs:
            if kind is not None:
                P.set_pair_kernel(kind)
            J, g, pairs = P.eval(psi, eps, radius, prec, allow_empty=allow_empty)
            assert abs(pairs - po) <= 16 + 1e-6 * po, (kind, pairs, po)
            if prec == 0:
                assert abs(J - Jo) <= 1e-10 * abs(Jo)
                assert np.max(np.abs(g - go)) <= 1e-10 * max(np.max(np.abs(go)), np.max(nu))
            elif kind == rs().PAIRS_TENSOR:
                g_tol, j_tol = tensor_tols(m, nu, eps, Jo)
                assert abs(J - Jo) <= j_tol, (J, Jo, j_tol)
                assert np.max(np.abs(g - go)) <= g_tol, (np.max(np.abs(g - go)), g_tol)
            else:
                assert abs(J - Jo) <= 1e-5 * abs(Jo), (kind, J, Jo)
                assert np.max(np.abs(g - go)) <= 1e-6, (kind, np.max(np.abs(g - go)))
            if kind in (None, rs().PAIRS_AUTO):
                out[prec] = (J, g, pairs)
    finally:
        P.set_pair_kernel(rs().PAIRS_AUTO)
    return out, (Jo, go, po, eo)


@pytest.mark.parametrize("d,nq,n,eps,scale,tail", [
    (2, 5000, 1500, 0.01, 0.01, 1e-12),
    (3, 6000, 2000, 0.005, 0.005, 1e-12),
    (3, 3000, 700, 0.02, 0.02, 1e-4),
    (2, 2100, 300, 0.002, 0.002, 1e-8),
])
def test_trunc_parity_tail_radius(d, nq, n, eps, scale, tail):
    x, m, y, nu, psi, eps = case(d * 31 + nq, d, nq, n, eps, scale)
    P = rs().Problem(x, m, y, nu)
    try:
        R = P.radius_for_tail(psi, eps, tail)
        C0 = oracle.covering_cost(x, y)
        Ro = truncation.radius_of_cutoff(truncation.cutoff_tail(psi, nu, eps, tail, C0))
        assert abs(R - Ro) <= 1e-6 * Ro
        res, (Jo, go, po, eo) = compare(P, x, m, y, nu, psi, eps, R)
        assert eo == 0
        assert po < x.shape[0] * y.shape[0]      # the radius really truncates
        # against the dense oracle: within the tail bound (plus FP32 noise)
        Jd, gd, _, _ = oracle.dual_grad(x, m, y, nu, psi, eps)
        J64, g64, _ = res[0]
        assert abs(J64 - Jd) <= eps * tail + 1e-12 * abs(Jd)
        assert np.all(np.abs(g64 - gd) <= tail * (g64 + 2 * nu) + 1e-13)
    finally:
        P.close()


def test_trunc_small_radius_reports_empty_points_and_skips_them():
    x, m, y, nu, psi, eps = case(77, 2, 3000, 200, 0.01, 0.01)
    P = rs().Problem(x, m, y, nu)
    try:
        R = 0.02   # far below the covering radius of 200 targets
        with pytest.raises(rs().RsotError) as ei:
            P.eval(psi, eps, R, 1)
        assert ei.value.status == 4
        res, (Jo, go, po, eo) = compare(P, x, m, y, nu, psi, eps, R, allow_empty=True)
        assert eo > 0
    finally:
        P.close()


def test_trunc_huge_radius_is_dense():
    x, m, y, nu, psi, eps = case(78, 3, 2000, 500, 0.02, 0.02)
    P = rs().Problem(x, m, y, nu)
    try:
        for prec in (0, 1):
            Jd, gd, pd = P.eval(psi, eps, 0.0, prec)
            Jt, gt, pt = P.eval(psi, eps, 10.0, prec)
            assert Jd == Jt and np.array_equal(gd, gt) and pd == pt == 2000 * 500
    finally:
        P.close()


def test_trunc_radius_changes_reuse_the_grid_and_repeat_bitwise():
    x, m, y, nu, psi, eps = case(79, 3, 4100, 1300, 0.01, 0.01)
    P = rs().Problem(x, m, y, nu)
    try:
        for R in (0.35, 0.2, 0.5, 0.2):
            compare(P, x, m, y, nu, psi, eps, R, precs=(1,))
        a = P.eval(psi, eps, 0.3, 1)
        b = P.eval(psi, eps, 0.3, 1)
        assert a[0] == b[0] and np.array_equal(a[1], b[1]) and a[2] == b[2]
        L = P.point_log_partition()
        # L_q of the truncated evaluation: ln of the truncated sum, caller's order
        Ld = oracle.point_lse(x, y, nu, psi, eps)
        assert np.all(L <= Ld + 1e-4)
    finally:
        P.close()


def test_trunc_mixture_workload_reduced_mesh():
    """Cube workload (mixture targets, random nu) on a 12^3 mesh, eps 1e-3, tail 1e-12."""
    p = ri.cube_3d(mesh_n=12, n_targets=8192, eps=1e-3)
    psi = 0.002 * np.random.default_rng(80).standard_normal(p.n)
    P = rs().Problem(p.x, p.mass, p.y, p.nu)
    try:
        R = P.radius_for_tail(psi, p.eps, 1e-12)
        compare(P, p.x, p.mass, p.y, p.nu, psi, p.eps, R, precs=(1,))
    finally:
        P.close()


def test_trunc_full_size_against_dense_gpu():
    """Full cube workload: the truncated evaluation at tail 1e-12 agrees with the
    dense one within the tail bound plus the mixed-precision tolerance, and its
    mass balance holds."""
    p = ri.cube_3d()
    psi = 0.002 * np.random.default_rng(81).standard_normal(p.n)
    P = rs().Problem(p.x, p.mass, p.y, p.nu)
    try:
        R = P.radius_for_tail(psi, p.eps, 1e-12)
        Jt, gt, pt = P.eval(psi, p.eps, R, 1)
        Jd, gd, pd = P.eval(psi, p.eps, 0.0, 1)
        assert pt < pd
        assert abs(Jt - Jd) <= 1e-5 * abs(Jd)
        assert np.max(np.abs(gt - gd)) <= 1e-6
        assert abs(gt.sum()) <= 5e-7
        # the FP32 truncated kernels count the same pairs up to boundary rounding
        P.set_pair_kernel(rs().PAIRS_FP32)
        Jf, gf, pf = P.eval(psi, p.eps, R, 1)
        assert abs(pf - pt) <= 1e-6 * pt
        assert abs(Jf - Jt) <= 1e-5 * abs(Jt)
        assert np.max(np.abs(gf - gt)) <= 1e-6
    finally:
        P.close()


def test_trunc_excluded_exponent_overflow():
    """A target with a potential far above the others, outside the radius of
    most points: its excluded terms' exponentials overflow FP32 in those points'
    shifts (weight 0 times inf in the tensor-core passes), which must drop them
    (exact redo in pass 1, the stage again in pass 2) and match the oracle."""
    x, m, y, nu, psi, eps = case(82, 2, 4000, 900, 0.01, 0.01)
    y[0] = (0.05, 0.05)
    psi[0] = 5.0              # (psi_0 - c) / eps ~ 480 >> 88 for every point
    P = rs().Problem(x, m, y, nu)
    try:
        res, (Jo, go, po, eo) = compare(P, x, m, y, nu, psi, eps, 0.3)
        assert eo == 0
        # most points exclude target 0, and its own cell takes most of the mass
        far = np.sum(np.sum((x - y[0]) ** 2, axis=1) >= 0.09)
        assert far > 0.5 * x.shape[0]
        J, g, pairs = res[1]
        assert np.isfinite(J) and np.all(np.isfinite(g))
    finally:
        P.close()
