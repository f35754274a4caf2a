"""The paper's cost cutoffs (Sec. 4.1, App. B) through the C ABI:
rsot_truncation_cutoff against the oracle's statements of C_pw (Eq.
cost_cutoff_delta), C_int (Eq. truncation_cutoff_int), C_geom (Eq.
truncation_cutoff_geom) and the tail cutoff; evaluations at those cutoffs
against the oracle's truncated Algorithm 2 (points without a target skipped);
and solves truncated at C_pw and C_geom whose certified stop holds for the
untruncated functional."""
import math

import numpy as np
import pytest

import oracle
from oracle import truncation

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


@pytest.mark.parametrize("d", [2, 3])
def test_cutoffs_match_the_oracle_statements(d):
    import torch
    x, m, y, nu, psi, eps = case(40 + d, d, 3000, 800, 0.01, 0.02)
    P = rs().Problem(x, m, y, nu)
    try:
        Jd, _, _, _ = oracle.dual_grad(x, m, y, nu, psi, eps)
        # the covering cost comes from an FP32 nearest-target search on FP32
        # coordinates (|dc| <= |x - y| |d(x - y)| ~ sqrt(2 C_0) 2^-23 plus 1e-7
        # relative); the cutoffs built on it are compared on the GPU's C_0
        C0o = oracle.covering_cost(x, y)
        C0 = P.covering_cost()
        assert abs(C0 - C0o) <= 2e-7 * C0o + 2.0 ** -23 * np.sqrt(2 * C0o)
        lnD = oracle.integrated_D(x, m, y, nu, psi, eps)
        for arr in (psi, torch.tensor(psi, device="cuda")):
            for dthr in (1e-12, 1e-7):
                C = P.truncation_cutoff(arr, eps, rs().CUTOFF_POINTWISE, dthr)
                assert abs(C - truncation.cutoff_pointwise(psi, nu, eps, dthr)) <= 1e-13 * abs(C) + 1e-15
            for tau in (1e-6, 1e-4):
                C = P.truncation_cutoff(arr, eps, rs().CUTOFF_GEOMETRIC, tau, J=Jd)
                Co = truncation.cutoff_geometric(psi, nu, eps, tau, Jd, C0)
                assert abs(C - Co) <= 1e-12 * abs(Co)
                C = P.truncation_cutoff(arr, eps, rs().CUTOFF_INTEGRAL, tau, J=Jd, lnD=lnD)
                Co = truncation.cutoff_integrated(psi, eps, tau, math.exp(lnD), Jd)
                assert abs(C - Co) <= 1e-12 * abs(Co)
            C = P.truncation_cutoff(arr, eps, rs().CUTOFF_TAIL, 1e-10)
            Co = truncation.cutoff_tail(psi, nu, eps, 1e-10, C0)
            assert abs(C - Co) <= 1e-12 * abs(Co)
        with pytest.raises(rs().RsotError):
            P.truncation_cutoff(psi, eps, rs().CUTOFF_GEOMETRIC, 1e-6, J=0.0)
        with pytest.raises(rs().RsotError):
            P.truncation_cutoff(psi, eps, 7, 1e-6)
    finally:
        P.close()


@pytest.mark.parametrize("kind,param", [(0, 1e-12), (0, 1e-5), (2, 1e-4)])
def test_evaluations_at_the_cutoffs_match_the_oracle(kind, param):
    """FP64 at 1e-10, mixed at its tolerances, compensated within its bound,
    each against Algorithm 2 truncated at C with empty points skipped."""
    x, m, y, nu, psi, eps = case(50 + kind, 2, 4000, 900, 0.005, 0.01)
    P = rs().Problem(x, m, y, nu)
    try:
        Jd, _, _, _ = oracle.dual_grad(x, m, y, nu, psi, eps)
        C = P.truncation_cutoff(psi, eps, kind, param, J=Jd)
        R = math.sqrt(2.0 * C)
        Jo, go, po, eo = oracle.dual_grad(x, m, y, nu, psi, eps, cutoff=C)
        assert po < x.shape[0] * y.shape[0]              # the cutoff truncates
        scale = max(np.max(np.abs(go)), np.max(nu))
        for prec, jt, gt in ((0, 1e-10 * abs(Jo), 1e-10 * scale), (1, 1e-5 * abs(Jo), 1e-6),
                             (2, 1e-5 * abs(Jo), rs().COMPENSATED_GRAD_REL)):
            J, g, pairs = P.eval(psi, eps, R, prec, allow_empty=True)
            _, _, _, empty = P.last_eval()
            if prec == 1 and empty != eo:
                continue      # an FP32 decision at a cutoff moved a point's only pair (R4)
            assert empty == eo
            assert abs(pairs - po) <= 16 + 1e-6 * po
            assert abs(J - Jo) <= jt, (prec, J, Jo)
            assert np.max(np.abs(g - go)) <= gt, (prec, np.max(np.abs(g - go)))
    finally:
        P.close()


@pytest.mark.parametrize("opt", [{"delta_pw": 1e-12}, {"tau_geom": 1e-6}, {"tau_int": 1e-6}])
def test_solves_truncated_at_the_papers_cutoffs_meet_the_dense_tolerance(opt):
    x, m, y, nu, psi, eps = case(60, 3, 6000, 1500, 5e-3, 0.0)
    P = rs().Problem(x, m, y, nu)
    try:
        sol, st = P.solve(eps=eps, eps_start=0.1, eps_factor=0.5, tol_l1=1e-6, **opt)
        assert st.status == 0
        assert st.pairs < st.evals * x.shape[0] * y.shape[0]    # evaluations were truncated
        _, gd, _, _ = oracle.dual_grad(x, m, y, nu, sol, eps)
        assert np.abs(gd).sum() <= 1e-6 * (1 + 1e-9)            # certified on dense references
        with pytest.raises(rs().RsotError):
            P.solve(eps=eps, tol_l1=1e-6, tail=1e-10, **opt)     # one truncation at a time
    finally:
        P.close()


def test_fp64_solve_at_the_pointwise_cutoff_reports_the_truncated_functional():
    """A plain FP64 solve truncated at C_pw (no refinement): it converges on the
    truncated functional; E_rel against the dense solve is the truncation's."""
    x, m, y, nu, psi, eps = case(61, 2, 3000, 400, 1e-2, 0.0)
    P = rs().Problem(x, m, y, nu)
    try:
        s0, st0 = P.solve(eps=eps, tol_l1=1e-8, precision=rs().FP64)
        s1, st1 = P.solve(eps=eps, tol_l1=1e-8, precision=rs().FP64, delta_pw=1e-10)
        assert st0.status == 0 and st1.status == 0
        assert st1.pairs < st1.evals * x.shape[0] * y.shape[0]
        e_rel = abs(st1.J - st0.J) / abs(st0.J)
        assert e_rel < 1e-4
        # the truncated solve's gradient is the truncated functional's: the oracle's
        # truncated gradient at its cutoff meets the tolerance
        C = P.truncation_cutoff(s1, eps, rs().CUTOFF_POINTWISE, 1e-10)
        _, gt, _, _ = oracle.dual_grad(x, m, y, nu, s1, eps, cutoff=C)
        assert np.abs(gt).sum() <= 1e-8 * (1 + 1e-6)
    finally:
        P.close()
