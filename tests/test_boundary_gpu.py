"""Boundary conventions of the C ABI on the GPU:
  * outputs are written only on RSOT_OK (device and host gradient buffers keep
    their contents on RSOT_ERR_EMPTY_NEIGHBORHOOD and RSOT_ERR_NONFINITE), and
    rsot_last_eval returns the evaluation that skipped empty points, which
    matches the oracle's truncated Algorithm 2 with the same points skipped;
  * rsot_create with device_ptrs = 1 borrows mass and nu and gives the same
    results as the copying form;
  * a bounded device-side wait that runs out reports RSOT_ERR_TIMEOUT and
    leaves the context usable.
"""
import ctypes

import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu


def rs():
    import paper_2507_23602_gb300 as m
    return m


def case(seed, d, nq, n):
    rng = np.random.default_rng(seed)
    x = rng.uniform(0, 1, (nq, d))
    m = rng.uniform(0.5, 1.5, nq)
    m /= m.sum()
    y = rng.uniform(0, 1, (n, d))
    nu = rng.uniform(0.5, 1.5, n)
    nu /= nu.sum()
    return x, m, y, nu, 0.01 * rng.standard_normal(n)


@pytest.mark.parametrize("prec", [0, 1, 2])
def test_no_output_on_empty_neighbourhood_and_last_eval(prec):
    import torch
    x, m, y, nu, psi = case(3, 2, 4000, 300)
    eps, radius = 0.02, 0.03                        # leaves some points without a target
    Jo, go, po, eo = oracle.dual_grad(x, m, y, nu, psi, eps, cutoff=0.5 * radius * radius)
    assert eo > 0
    lib = rs().load()
    P = rs().Problem(x, m, y, nu)
    try:
        g_host = np.full(300, 7.0)
        g_dev = torch.full((300,), 7.0, dtype=torch.float64, device="cuda")
        for g in (g_host, g_dev):
            pg, keep = rs()._ptr(g)
            J = ctypes.c_double(-5.0)
            pairs = ctypes.c_int64(-5)
            st = lib.rsot_eval_dual_grad(P._h, rs()._ptr(psi)[0], eps, radius, prec,
                                         ctypes.byref(J), pg, ctypes.byref(pairs))
            assert st == rs().RSOT_ERR_EMPTY_NEIGHBORHOOD
            assert J.value == -5.0 and pairs.value == -5
        assert np.all(g_host == 7.0)
        assert bool(torch.all(g_dev == 7.0))
        J, g, pairs, empty = P.last_eval()
        if prec == 1:
            # FP32 may classify a pair at the cutoff the other way (R4); a point
            # whose only pair sits there can change between empty and kept
            assert abs(empty - eo) <= 2 and abs(pairs - po) <= 16 + 1e-6 * po
            if empty != eo:
                return
        else:
            assert empty == eo and abs(pairs - po) <= 4
        scale = max(np.max(np.abs(go)), np.max(nu))
        tol_g = 1e-10 * scale if prec == 0 else (1e-6 if prec == 1 else 6.5e-7)
        assert abs(J - Jo) <= (1e-10 if prec == 0 else 1e-5) * abs(Jo)
        assert np.max(np.abs(g - go)) <= tol_g
        # the binding's allow_empty form returns the same evaluation
        J2, g2, _ = P.eval(psi, eps, radius, prec, allow_empty=True)
        assert J2 == J and np.array_equal(g2, g)
    finally:
        P.close()


def test_no_output_on_nonfinite_potential():
    import torch
    x, m, y, nu, psi = case(4, 3, 2000, 500)
    P = rs().Problem(x, m, y, nu)
    try:
        J0, g0, _ = P.eval(psi, 0.02, 0.0, rs().MIXED)      # a completed evaluation first
        bad = psi.copy()
        bad[11] = np.inf
        for prec in (0, 1, 2):
            g_dev = torch.full((500,), 3.0, dtype=torch.float64, device="cuda")
            g_host = np.full(500, 3.0)
            for g in (g_dev, g_host):
                with pytest.raises(rs().RsotError) as ei:
                    P.eval(bad, 0.02, 0.0, prec, grad_out=g)
                assert ei.value.status == 3
            assert bool(torch.all(g_dev == 3.0)) and np.all(g_host == 3.0)
    finally:
        P.close()


def test_borrowed_device_inputs_match_copied_inputs():
    import torch
    x, m, y, nu, psi = case(5, 3, 6000, 1500)
    t = [torch.tensor(a, device="cuda") for a in (x, m, y, nu)]
    A = rs().Problem(x, m, y, nu)
    B = rs().Problem(*t, borrow=True)
    try:
        for prec in (0, 1, 2):
            Ja, ga, _ = A.eval(psi, 0.01, 0.0, prec)
            Jb, gb, _ = B.eval(psi, 0.01, 0.0, prec)
            assert Ja == Jb and np.array_equal(ga, gb), prec
        Ja, ga, pa = A.eval_tail(psi, 0.01, 1e-10, rs().MIXED)
        Jb, gb, pb = B.eval_tail(psi, 0.01, 1e-10, rs().MIXED)
        assert Ja == Jb and np.array_equal(ga, gb) and pa == pb
        sa = A.solve(eps=0.01, tol_l1=1e-6)[0]
        sb = B.solve(eps=0.01, tol_l1=1e-6)[0]
        assert np.array_equal(sa, sb)
    finally:
        A.close()
        B.close()
    # host memory cannot be borrowed
    with pytest.raises(rs().RsotError) as ei:
        rs().Problem(x, m, y, nu, borrow=True)
    assert ei.value.status == 1


def test_bounded_wait_runs_out_and_reports_timeout():
    import torch
    lib = rs().load()
    lib.rsot_selftest_wait_timeout.argtypes = [ctypes.c_longlong, ctypes.c_void_p]
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    assert lib.rsot_selftest_wait_timeout(1000, stream) == 7
    assert lib.rsot_selftest_wait_timeout(0, stream) == 1
    # the context is still usable: an evaluation after the timeout succeeds
    x, m, y, nu, psi = case(6, 2, 1000, 200)
    P = rs().Problem(x, m, y, nu)
    try:
        J, g, _ = P.eval(psi, 0.02, 0.0, rs().FP64)
        Jo, go, _, _ = oracle.dual_grad(x, m, y, nu, psi, 0.02)
        assert abs(J - Jo) <= 1e-10 * abs(Jo)
    finally:
        P.close()
