"""Batched evaluation and solve (persistent multi-problem kernels, CUDA-graph
rounds, lockstep L-BFGS) against per-problem evaluations and the oracle."""
import numpy as np
import pytest

import oracle
import rsot_inputs as ri

pytestmark = pytest.mark.gpu


def rs():
    import paper_2507_23602_gb300 as m
    return m


def small_batch(seed0=300, count=6):
    probs, eps = [], []
    for i in range(count):
        rng = np.random.default_rng(seed0 + i)
        d = 2 + (i % 2)
        mesh = int(rng.integers(6, 14)) if d == 3 else int(rng.integers(20, 60))
        n = int(rng.integers(200, 3000))
        e = float(np.exp(rng.uniform(np.log(3e-3), np.log(1e-1))))
        p = ri.make_problem(d, mesh, n, e, src_seed=seed0 + i, src_k=3, tgt_seed=seed0 + 50 + i,
                            nu_seed=seed0 + 90 + i)
        probs.append(p)
        eps.append(e)
    return probs, np.array(eps)


def test_batch_eval_matches_single_problem_and_oracle():
    probs, eps = small_batch()
    B = rs().Batch([(p.x, p.mass, p.y, p.nu) for p in probs])
    rng = np.random.default_rng(1)
    psis = [0.02 * rng.standard_normal(p.n) for p in probs]
    try:
        J, g = B.eval(np.concatenate(psis), eps)
        for i, (p, psi) in enumerate(zip(probs, psis)):
            gi = B.split(g)[i]
            Jo, go, _, _ = oracle.dual_grad(p.x, p.mass, p.y, p.nu, psi, eps[i])
            assert abs(J[i] - Jo) <= 1e-5 * abs(Jo), (i, J[i], Jo)
            assert np.max(np.abs(gi - go)) <= 1e-6, i
        # an inactive problem is left untouched; the others do not change
        act = np.ones(len(probs), np.uint8)
        act[2] = 0
        J2, g2 = B.eval(np.concatenate(psis), eps, active=act)
        assert np.isnan(J2[2]) and np.all(np.isnan(B.split(g2)[2]))
        for i in (0, 1, 3, 4, 5):
            assert J2[i] == J[i] and np.array_equal(B.split(g2)[i], B.split(g)[i])
        # autotuned work-item size: same values within the mixed tolerance
        B.tune(np.concatenate(psis), eps)
        J3, g3 = B.eval(np.concatenate(psis), eps)
        assert np.all(np.abs(J3 - J) <= 1e-6 * np.abs(J))
        assert np.max(np.abs(g3 - g)) <= 1e-7
    finally:
        B.close()


def test_batch_pair_kernels_agree_with_the_oracle():
    """The batched tensor-core passes (forced) and the batched FP32 passes (forced,
    and the automatic choice for evaluations returned to the caller) meet the
    mixed bounds against the oracle."""
    probs, eps = small_batch(seed0=400, count=5)
    B = rs().Batch([(p.x, p.mass, p.y, p.nu) for p in probs])
    rng = np.random.default_rng(2)
    psis = [0.02 * rng.standard_normal(p.n) for p in probs]
    try:
        ref = [oracle.dual_grad(p.x, p.mass, p.y, p.nu, psi, eps[i])[:2]
               for i, (p, psi) in enumerate(zip(probs, psis))]
        for kind in (rs().PAIRS_TENSOR, rs().PAIRS_FP32, rs().PAIRS_AUTO):
            B.set_pair_kernel(kind)
            J, g = B.eval(np.concatenate(psis), eps)
            for i, (Jo, go) in enumerate(ref):
                p = probs[i]
                tol_g = 1e-6
                if kind == rs().PAIRS_TENSOR:   # the forced form's error model
                    tol_g = max(1e-6, 5 * 1.4e-5 * np.sqrt(p.mass.max() * p.nu.max()))
                assert abs(J[i] - Jo) <= 1e-5 * abs(Jo), (kind, i, J[i], Jo)
                assert np.max(np.abs(B.split(g)[i] - go)) <= tol_g, (kind, i)
    finally:
        B.close()


def test_batch_solve_mixed_with_refinement_reaches_tolerance():
    probs, eps = small_batch(400, 5)
    B = rs().Batch([(p.x, p.mass, p.y, p.nu) for p in probs])
    try:
        psi, st = B.solve(eps, eps_start=0.1, eps_factor=0.5, tol_l1=1e-6, precision=rs().MIXED,
                          refine_fp64=True)
        assert st["converged"] == len(probs), st
        assert st["rounds"] > 0
        for i, p in enumerate(probs):
            _, go, _, _ = oracle.dual_grad(p.x, p.mass, p.y, p.nu, B.split(psi)[i], eps[i])
            assert np.sum(np.abs(go)) <= 1e-6 * (1 + 1e-9), i
        # the plain FP64 path reaches the same minimisers (up to the constant)
        psi64, st64 = B.solve(eps, eps_start=0.1, eps_factor=0.5, tol_l1=1e-6,
                              precision=rs().FP64)
        assert st64["converged"] == len(probs)
        for i, p in enumerate(probs):
            a, b = B.split(psi)[i], B.split(psi64)[i]
            a = a - a @ p.nu
            b = b - b @ p.nu
            assert np.max(np.abs(a - b)) <= 1e-3 * eps[i] + 1e-7, i
    finally:
        B.close()
