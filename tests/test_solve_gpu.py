"""The host L-BFGS driver over GPU evaluations (Algorithm 1, Sec. 4.2)
against the oracle's own L-BFGS: both must reach ||grad J||_1 <= tol and
agree on the minimiser (up to the additive constant, Remark 3.3 / App. A)."""
import numpy as np
import pytest

import oracle
from oracle import lbfgs
import rsot_inputs as ri

pytestmark = pytest.mark.gpu


def rs():
    import paper_2507_23602_gb300 as m
    return m


def centred(psi, nu):
    return psi - psi @ nu


def test_small_2d_fp64_solve_matches_oracle_solve():
    p = ri.small_2d()
    P = rs().Problem(p.x, p.mass, p.y, p.nu)
    try:
        psi, st = P.solve(eps=p.eps, tol_l1=1e-8, precision=rs().FP64)
        assert st.status == 0 and st.grad_l1 <= 1e-8
        # the reported gradient norm is the oracle's too
        Jo, go, _, _ = oracle.dual_grad(p.x, p.mass, p.y, p.nu, psi, p.eps)
        assert np.sum(np.abs(go)) <= 1e-8 * (1 + 1e-9)
        assert abs(st.J - Jo) <= 1e-10 * abs(Jo)
    finally:
        P.close()
    res = lbfgs.minimize(lambda q: oracle.dual_grad(p.x, p.mass, p.y, p.nu, q, p.eps)[:2],
                         np.zeros(p.n), 1e-8)
    assert res.status == "converged"
    assert np.max(np.abs(centred(psi, p.nu) - centred(res.x, p.nu))) <= 1e-5


def test_mixed_solve_with_fp64_refinement_reaches_tolerance():
    p = ri.make_problem(3, 10, 2000, 5e-3, src_seed=71, src_k=3, tgt_seed=72, tgt_k=2, nu_seed=73)
    P = rs().Problem(p.x, p.mass, p.y, p.nu)
    try:
        psi, st = P.solve(eps=p.eps, eps_start=0.1, eps_factor=0.5, tol_l1=1e-6,
                          precision=rs().MIXED, refine_fp64=True)
        assert st.status == 0 and st.grad_l1 <= 1e-6
        assert st.stages == 6
        _, go, _, _ = oracle.dual_grad(p.x, p.mass, p.y, p.nu, psi, p.eps)
        assert np.sum(np.abs(go)) <= 1e-6 * (1 + 1e-9)
    finally:
        P.close()


def test_solve_warm_start_is_a_fixed_point():
    p = ri.make_problem(2, 16, 300, 0.02, src_seed=81, src_k=2, tgt_seed=82)
    P = rs().Problem(p.x, p.mass, p.y, p.nu)
    try:
        psi, st = P.solve(eps=p.eps, tol_l1=1e-9, precision=rs().FP64)
        psi2, st2 = P.solve(psi0=psi, eps=p.eps, tol_l1=1e-9, precision=rs().FP64)
        assert st2.iters == 0 and np.array_equal(psi, psi2)
    finally:
        P.close()


def test_solve_reports_iteration_cap():
    p = ri.make_problem(2, 16, 300, 0.01, src_seed=91, src_k=2, tgt_seed=92)
    P = rs().Problem(p.x, p.mass, p.y, p.nu)
    try:
        psi, st = P.solve(eps=p.eps, tol_l1=1e-12, max_iter=3, precision=rs().FP64,
                          raise_on_error=False)
        assert st.status == 5 and st.iters == 3
    finally:
        P.close()


def test_concurrent_solves_on_separate_handles_match_sequential():
    """Handles are independent: solves of two problems from two host threads (as
    the batched refinement runs them) give bitwise the results of sequential
    solves."""
    import threading
    probs = [ri.make_problem(2, 16, 300, 0.01, src_seed=81 + k, src_k=2, tgt_seed=82 + k) for k in range(2)]
    handles = [rs().Problem(q.x, q.mass, q.y, q.nu) for q in probs]
    try:
        seq = [h.solve(eps=q.eps, eps_start=0.1, tol_l1=1e-6)[0] for h, q in zip(handles, probs)]
        out = [None, None]

        def run(k):
            out[k] = handles[k].solve(eps=probs[k].eps, eps_start=0.1, tol_l1=1e-6)[0]
        ths = [threading.Thread(target=run, args=(k,)) for k in range(2)]
        for t in ths:
            t.start()
        for t in ths:
            t.join()
        for k in range(2):
            assert np.array_equal(out[k], seq[k])
    finally:
        for h in handles:
            h.close()
