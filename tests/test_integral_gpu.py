"""The integral cutoff of Sec. 4.1 (Eq. truncation_cutoff_int) on the GPU:
ln D = ln sum_q m_q / S_trunc(x_q) of the last evaluation against the oracle,
and solves whose evaluations are truncated at C_int.

Tolerances: ln D inherits the per-point log partitions' errors -- 1e-10
relative for FP64, 1e-6 absolute for the mixed path (its L_q errs by a few
1e-7), 1e-6 for the compensated one."""
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


@pytest.mark.parametrize("d,nq,n,eps,scale,radius", [
    (2, 3000, 700, 0.01, 0.02, 0.0),
    (3, 2600, 900, 0.005, 0.01, 0.0),
    (2, 3000, 700, 0.01, 0.02, 0.35),
    (3, 2600, 900, 0.005, 0.01, 0.4),
])
def test_log_integrated_D_parity(d, nq, n, eps, scale, radius):
    x, m, y, nu, psi, eps = case(d * 11 + n, d, nq, n, eps, scale)
    C = 0.5 * radius * radius if radius > 0 else math.inf
    ref = oracle.integrated_D(x, m, y, nu, psi, eps, cutoff=C)
    assert math.isfinite(ref)
    P = rs().Problem(x, m, y, nu)
    try:
        for prec, tol in ((rs().FP64, 1e-10 * abs(ref)), (rs().MIXED, 1e-6), (rs().COMPENSATED, 1e-6)):
            P.eval(psi, eps, radius, prec)
            v = P.log_integrated_D()
            assert abs(v - ref) <= tol, (prec, v, ref)
    finally:
        P.close()


def test_log_integrated_D_is_infinite_with_an_empty_point():
    x, m, y, nu, psi, eps = case(5, 2, 500, 40, 0.01, 0.0)
    x[0] = [5.0, 5.0]
    P = rs().Problem(x, m, y, nu)
    try:
        P.eval(psi, eps, 0.5, rs().FP64, allow_empty=True)
        assert P.log_integrated_D() == math.inf
    finally:
        P.close()


def test_solve_with_the_integral_cutoff():
    """Every mixed evaluation after the first of a stage is truncated at C_int
    (tau = 1e-9); the refinement's reference evaluations are dense, so the dense
    gradient at the result meets tol."""
    p = ri.make_problem(3, 10, 2000, 5e-3, src_seed=71, src_k=3, tgt_seed=72, tgt_k=2, nu_seed=73)
    P = rs().Problem(p.x, p.mass, p.y, p.nu)
    try:
        tau = 1e-9
        psi, st = P.solve(eps=p.eps, eps_start=0.1, eps_factor=0.5, tol_l1=1e-6, tau_int=tau)
        assert st.status == 0
        assert st.pairs < st.evals * p.x.shape[0] * p.n      # the cutoff truncated
        J, gd, _, _ = oracle.dual_grad(p.x, p.mass, p.y, p.nu, psi, p.eps)
        assert np.abs(gd).sum() <= 1e-6
        with pytest.raises(rs().RsotError):
            P.solve(eps=p.eps, tol_l1=1e-6, tau_int=tau, tail=1e-8)
    finally:
        P.close()
