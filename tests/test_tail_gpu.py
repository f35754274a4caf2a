"""Parity of the psi-aware truncated evaluation (rsot_eval_dual_grad_tail:
I_q = {j : c(x_q, y_j) < alpha_q + beta_j}, alpha_q from each point's nearest
target, beta_j = psi_j + eps ln(1/tail)) with the oracle's separable
Algorithm 2, in every precision, through the C ABI.

Tolerances: FP64 1e-10 (J relative, gradient relative to its scale); mixed
1e-5 relative J, 1e-6 absolute per gradient entry (the tensor-core pair kernel
forced: its error model); compensated its proven bound.  The oracle tests
c < alpha + beta in the caller's frame, the GPU in the translated one: pairs
within FP64 rounding of a cutoff may differ (FP64 / compensated: a few; mixed
kernels decide in FP32: 16 + 1e-6 of the count).  Against the dense oracle the
truncation stays within its tail guarantee."""
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
    g_tol = max(1e-6, 5 * 1.4e-5 * math.sqrt(m.max() * nu.max()))
    j_tol = max(1e-5 * abs(Jo), 5 * eps * math.log(2) * 2e-5 * math.sqrt(np.sum(m * m)))
    return g_tol, j_tol


def check_all(P, x, m, y, nu, psi, eps, tail):
    a, b = truncation.separable_cutoffs(x, y, nu, psi, eps, tail)
    Jo, go, po, eo = oracle.dual_grad_sep(x, m, y, nu, psi, eps, a, b)
    assert eo == 0
    scale = max(np.max(np.abs(go)), np.max(nu))
    J64, g64, p64 = P.eval_tail(psi, eps, tail, rs().FP64)
    assert abs(p64 - po) <= 4
    assert abs(J64 - Jo) <= 1e-10 * abs(Jo)
    assert np.max(np.abs(g64 - go)) <= 1e-10 * scale
    Jc, gc, pc = P.eval_tail(psi, eps, tail, rs().COMPENSATED)
    assert pc == p64                                   # the FP64 path's own test
    assert np.abs(gc - g64).sum() <= rs().COMPENSATED_GRAD_REL * m.sum()
    assert abs(Jc - J64) <= 3e-7 * eps * m.sum() + 1e-12 * abs(J64)
    for kind in (rs().PAIRS_AUTO, rs().PAIRS_FP32, rs().PAIRS_TENSOR):
        P.set_pair_kernel(kind)
        J, g, pairs = P.eval_tail(psi, eps, tail, rs().MIXED)
        assert abs(pairs - po) <= 16 + 1e-6 * po, (kind, pairs, po)
        if kind == rs().PAIRS_TENSOR:
            g_tol, j_tol = tensor_tols(m, nu, eps, Jo)
        else:
            g_tol, j_tol = 1e-6, 1e-5 * abs(Jo)
        assert abs(J - Jo) <= j_tol, (kind, J, Jo)
        assert np.max(np.abs(g - go)) <= g_tol, (kind, np.max(np.abs(g - go)))
    P.set_pair_kernel(rs().PAIRS_AUTO)
    return (J64, g64, p64), (Jo, go, po)


@pytest.mark.parametrize("d,nq,n,eps,scale,tail", [
    (2, 5000, 1500, 0.01, 0.01, 1e-12),
    (3, 6000, 2000, 0.005, 0.005, 1e-12),
    (3, 3000, 700, 0.02, 0.05, 1e-4),
    (2, 2100, 300, 0.002, 0.002, 1e-8),
    (3, 1025, 257, 0.001, 0.01, 1e-6),
])
def test_tail_parity(d, nq, n, eps, scale, tail):
    x, m, y, nu, psi, eps = case(d * 37 + nq, d, nq, n, eps, scale)
    P = rs().Problem(x, m, y, nu)
    try:
        (J64, g64, p64), (Jo, go, po) = check_all(P, x, m, y, nu, psi, eps, tail)
        assert po < x.shape[0] * y.shape[0]
        # fewer pairs than the global tail radius, within the same guarantee
        R = P.radius_for_tail(psi, eps, tail)
        _, _, pr = P.eval(psi, eps, R, rs().FP64)
        assert p64 <= pr
        Jd, gd, _, _ = oracle.dual_grad(x, m, y, nu, psi, eps)
        assert -1e-12 * abs(Jd) <= Jd - J64 <= eps * tail * nu.sum() * m.sum() + 1e-12 * abs(Jd)
        assert np.all(np.abs(g64 - gd) <= tail * (nu.sum() * (g64 + nu) + nu * m.sum()) + 1e-13)
    finally:
        P.close()


def test_tail_nearest_target_ties_and_point_log_partition():
    """Coincident targets (ties broken by the lowest index on both sides) and
    the per-point log partition of a truncated evaluation."""
    x, m, y, nu, psi, eps = case(91, 2, 3000, 400, 0.01, 0.01)
    y[200:210] = y[3]
    P = rs().Problem(x, m, y, nu)
    try:
        check_all(P, x, m, y, nu, psi, eps, 1e-6)
        P.eval_tail(psi, eps, 1e-6, rs().FP64)
        L = P.point_log_partition()
        Ld = oracle.point_lse(x, y, nu, psi, eps)
        assert np.all(L <= Ld + 1e-12) and np.all(Ld - L <= 1e-6 * nu.sum() + 1e-12)
    finally:
        P.close()


def test_tail_cube_reduced_mesh():
    """Cube workload (mixture targets, random nu) on a 12^3 mesh, eps 1e-3, tail 1e-12."""
    p = ri.cube_3d(mesh_n=12, n_targets=8192, eps=1e-3)
    psi = 0.002 * np.random.default_rng(82).standard_normal(p.n)
    P = rs().Problem(p.x, p.mass, p.y, p.nu)
    try:
        check_all(P, p.x, p.mass, p.y, p.nu, psi, p.eps, 1e-12)
    finally:
        P.close()


def test_tail_full_size_against_dense_gpu():
    """Full cube workload at tail 1e-12: within the tail guarantee of the dense
    FP64-accurate (compensated) evaluation, fewer pairs than the global radius,
    and the mixed kernels agree with the compensated ones."""
    p = ri.cube_3d()
    psi = 0.002 * np.random.default_rng(83).standard_normal(p.n)
    P = rs().Problem(p.x, p.mass, p.y, p.nu)
    try:
        Jd, gd, _ = P.eval(psi, p.eps, 0.0, rs().COMPENSATED)
        Jc, gc, pc = P.eval_tail(psi, p.eps, 1e-12, rs().COMPENSATED)
        R = P.radius_for_tail(psi, p.eps, 1e-12)
        _, _, pr = P.eval(psi, p.eps, R, rs().MIXED)
        assert pc < pr
        assert abs(Jd - Jc) <= 1e-12 * abs(Jd) + 6e-7 * p.eps
        assert np.abs(gd - gc).sum() <= 2 * rs().COMPENSATED_GRAD_REL
        Jm, gm, pm = P.eval_tail(psi, p.eps, 1e-12, rs().MIXED)
        assert abs(pm - pc) <= 16 + 1e-6 * pc
        assert abs(Jm - Jc) <= 1e-5 * abs(Jc)
        assert np.max(np.abs(gm - gc)) <= 1e-6
    finally:
        P.close()


def test_solve_with_tail_meets_tolerance_against_dense():
    p = ri.make_problem(3, 10, 2000, 5e-3, src_seed=71, src_k=3, tgt_seed=72, tgt_k=2, nu_seed=73)
    P = rs().Problem(p.x, p.mass, p.y, p.nu)
    try:
        tail = 1e-10
        psi, st = P.solve(eps=p.eps, eps_start=0.1, eps_factor=0.5, tol_l1=1e-6, tail=tail)
        assert st.status == 0
        # the refinement's compensated reference evaluations are truncated at the
        # tail, its bound subtracted from tol: the dense gradient meets tol
        # (certified); the truncated one within the tail bound of it
        _, gd, _, _ = oracle.dual_grad(p.x, p.mass, p.y, p.nu, psi, p.eps)
        assert np.abs(gd).sum() <= 1e-6
        a, b = truncation.separable_cutoffs(p.x, p.y, p.nu, psi, p.eps, tail)
        _, gt, _, _ = oracle.dual_grad_sep(p.x, p.mass, p.y, p.nu, psi, p.eps, a, b)
        assert np.abs(gt).sum() <= 1e-6 + 3 * tail
    finally:
        P.close()


def test_tail_solve_runs_dense_where_most_pairs_are_kept():
    """A tail-mode evaluator whose first (truncated) evaluation keeps more than
    35 % of all pairs runs dense from then on (the dense functional lies within
    the tail tolerance of the truncated one); an FP64 evaluator evaluates that
    first point again dense.  A single-stage FP64 solve has one evaluator: it
    equals the dense solve bitwise, with one more evaluation, the truncated
    probe at the start point."""
    eps = 1e-2      # psi = 0 keeps 83 % of the pairs at tail 1e-12
    p = ri.make_problem(3, 10, 2000, eps, src_seed=74, src_k=3, tgt_seed=75, tgt_k=2, nu_seed=76)
    P = rs().Problem(p.x, p.mass, p.y, p.nu)
    try:
        allp = p.x.shape[0] * p.y.shape[0]
        _, _, pr0 = P.eval_tail(np.zeros(p.y.shape[0]), eps, 1e-12, rs().FP64)
        assert 0.35 * allp < pr0 < allp
        sd, std = P.solve(eps=eps, tol_l1=1e-8, precision=rs().FP64)
        st_, stt = P.solve(eps=eps, tol_l1=1e-8, precision=rs().FP64, tail=1e-12)
        assert std.status == 0 and stt.status == 0
        assert np.array_equal(sd, st_)
        assert stt.evals == std.evals + 1
        assert stt.pairs == std.pairs + pr0
        # where the start point keeps fewer pairs the solve stays truncated
        eps2 = 3e-3     # psi = 0 keeps 28 %
        _, _, pr1 = P.eval_tail(np.zeros(p.y.shape[0]), eps2, 1e-12, rs().FP64)
        assert pr1 < 0.35 * allp
        _, st2 = P.solve(eps=eps2, tol_l1=1e-8, precision=rs().FP64, tail=1e-12)
        assert st2.status == 0 and st2.pairs < 0.5 * st2.evals * allp
    finally:
        P.close()
