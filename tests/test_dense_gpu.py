"""Parity of the dense CUDA path with the FP64 oracle, through the C ABI.

Tolerances (written here, from the stated targets):
  FP64 path  : |J - J_o| <= 1e-10 |J_o|,  |g - g_o| <= 1e-10 s per entry, with
               s = max(max|g_o|, max nu) the scale of the terms of each entry
               (sum_q m_q p_qj ~ nu_j; max|g_o| alone vanishes at the optimum)
  mixed path : |J - J_o| <= 1e-5 |J_o|,   |g - g_o| <= 1e-6 per entry (absolute)
"""
import math

import numpy as np
import pytest

import oracle
import rsot_inputs as ri

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-10
MIX_J_TOL = 1e-5
MIX_G_TOL = 1e-6


def rs():
    import paper_2507_23602_gb300 as m
    return m


def random_case(seed, d, nq, n, eps, psi_scale):
    rng = np.random.default_rng(seed)
    x = rng.uniform(0, 1, (nq, d))
    m = rng.uniform(0.5, 1.5, nq)
    m /= m.sum()
    y = rng.uniform(0, 1, (n, d))
    nu = rng.uniform(0.5, 1.5, n)
    nu /= nu.sum()
    psi = psi_scale * rng.standard_normal(n)
    return x, m, y, nu, psi, eps


def tensor_tols(m, nu, eps, Jo):
    """Bounds for the tensor-core pair kernel forced onto any problem: its
    exponents err by rms ~2e-5 (log2 units, measured), i.e. a relative error
    of ~1.4e-5 per plan entry; a gradient entry sum_q m_q p_qj then errs by
    <= 1.4e-5 sqrt(m_max nu_max) per standard deviation and J by
    eps ln2 2e-5 sqrt(sum_q m_q^2).  Five deviations, never below the mixed
    path's own bounds (which the automatic choice meets)."""
    g_tol = max(MIX_G_TOL, 5 * 1.4e-5 * math.sqrt(m.max() * nu.max()))
    j_tol = max(MIX_J_TOL * abs(Jo), 5 * eps * math.log(2) * 2e-5 * math.sqrt(np.sum(m * m)))
    return g_tol, j_tol


def check(x, m, y, nu, psi, eps, precisions=(0, 1)):
    """FP64 path once; the mixed path with the automatic pair kernel, the FP32
    kernels, and the tensor-core kernels forced (with their error model)."""
    Jo, go, _, _ = oracle.dual_grad(x, m, y, nu, psi, eps)
    P = rs().Problem(x, m, y, nu)
    runs = [(prec, kind) for prec in precisions
            for kind in ((None,) if prec == 0 else
                         (rs().PAIRS_AUTO, rs().PAIRS_FP32, rs().PAIRS_TENSOR))]
    try:
        for prec, kind in runs:
            if kind is not None:
                P.set_pair_kernel(kind)
            J, g, pairs = P.eval(psi, eps, 0.0, prec)
            assert pairs == x.shape[0] * y.shape[0]
            if prec == 0:
                assert abs(J - Jo) <= FP64_TOL * abs(Jo), (J, Jo)
                assert np.max(np.abs(g - go)) <= FP64_TOL * max(np.max(np.abs(go)), np.max(nu))
            elif kind == rs().PAIRS_TENSOR:
                g_tol, j_tol = tensor_tols(m, nu, eps, Jo)
                assert abs(J - Jo) <= j_tol, (J, Jo, abs(J - Jo), j_tol)
                assert np.max(np.abs(g - go)) <= g_tol, (np.max(np.abs(g - go)), g_tol)
            else:
                assert abs(J - Jo) <= MIX_J_TOL * abs(Jo), (J, Jo, abs(J - Jo) / abs(Jo))
                assert np.max(np.abs(g - go)) <= MIX_G_TOL, np.max(np.abs(g - go))
            # point log partition of the same evaluation
            L = P.point_log_partition()
            Lo = oracle.point_lse(x, y, nu, psi, eps)
            tol = 1e-11 if prec == 0 else 2e-4
            assert np.max(np.abs(L - Lo) / np.maximum(1.0, np.abs(Lo))) <= tol
    finally:
        P.close()


@pytest.mark.parametrize("d,nq,n,eps,scale", [
    (2, 3000, 700, 0.05, 0.02),      # several point tiles, ragged tails both ways
    (2, 5000, 1300, 0.01, 0.01),
    (3, 4100, 1500, 0.02, 0.02),
    (3, 2500, 2049, 1e-3, 0.01),     # small eps: large exponent range
    (2, 1025, 257, 0.1, 0.1),
])
def test_dense_parity_random(d, nq, n, eps, scale):
    check(*random_case(d * 1000 + nq, d, nq, n, eps, scale))


@pytest.mark.parametrize("nq,n", [(1, 1), (1, 5), (7, 1), (3, 2), (1023, 3), (1024, 256), (2048, 1024)])
def test_dense_edge_sizes(nq, n):
    for d in (2, 3):
        x, m, y, nu, psi, eps = random_case(nq * 7 + n, d, nq, n, 0.05, 0.05)
        if n == 1:
            nu = np.ones(1)
        check(x, m, y, nu, psi, eps)


def test_dense_coincident_points_and_zero_mass():
    x, m, y, nu, psi, eps = random_case(5, 2, 2000, 300, 0.02, 0.02)
    x[100:200] = x[100]          # repeated quadrature points
    y[10:20] = y[10]             # coincident targets
    m[300:400] = 0.0             # zero-mass points
    m /= m.sum()
    check(x, m, y, nu, psi, eps)


def test_dense_large_potential_offset():
    """J is shift invariant; a large constant offset must not hurt the mixed path."""
    x, m, y, nu, psi, eps = random_case(6, 3, 3000, 800, 0.01, 0.01)
    check(x, m, y, nu, psi + 123.25, eps)


def test_small_2d_full_size():
    p = ri.small_2d()
    psi = 0.01 * np.random.default_rng(7).standard_normal(p.n)
    check(p.x, p.mass, p.y, p.nu, psi, p.eps)


def test_cube_3d_reduced_mesh_full_targets():
    """Cube workload with all 65,536 targets on a 16^3 mesh (98,304 points)."""
    p = ri.cube_3d(mesh_n=16, eps=1e-3)
    psi = 0.005 * np.random.default_rng(8).standard_normal(p.n)
    check(p.x, p.mass, p.y, p.nu, psi, p.eps, precisions=(1,))


def test_cube_3d_full_size_sampled_and_invariants():
    """Full 786,432 x 65,536 workload in the benchmark's launch configuration:
    sampled per-point log partitions against the oracle, the mass balance
    sum_j dJ/dpsi_j = 0, shift invariance, and agreement with the FP64 path."""
    p = ri.cube_3d()
    psi = 0.005 * np.random.default_rng(9).standard_normal(p.n)
    P = rs().Problem(p.x, p.mass, p.y, p.nu)
    try:
        J, g, pairs = P.eval(psi, p.eps, 0.0, 1)
        assert pairs == p.nq * p.n
        L = P.point_log_partition()
        idx = np.random.default_rng(10).choice(p.nq, 1500, replace=False)
        Lo = oracle.point_lse(p.x[idx], p.y, p.nu, psi, p.eps)
        assert np.max(np.abs(L[idx] - Lo) / np.maximum(1.0, np.abs(Lo))) <= 2e-4
        # J = sum_q m_q eps L_q - psi.nu with the GPU's own L_q
        assert abs(np.sum(p.mass * p.eps * L) - psi @ p.nu - J) <= 1e-9 * abs(J) + 1e-12
        # ex2.approx carries ~2^-22 relative error per term: the row sums of the
        # mixed plan deviate from 1 by that much, so the mass balance holds to ~1e-7
        assert abs(g.sum()) <= 5e-7
        J2, g2, _ = P.eval(psi + 0.75, p.eps, 0.0, 1)
        assert abs(J2 - J) <= MIX_J_TOL * abs(J)
        assert np.max(np.abs(g2 - g)) <= MIX_G_TOL
        J64, g64, _ = P.eval(psi, p.eps, 0.0, 0)
        assert abs(J - J64) <= MIX_J_TOL * abs(J64)
        assert np.max(np.abs(g - g64)) <= MIX_G_TOL
        assert abs(g64.sum()) <= 1e-12
    finally:
        P.close()


def test_repeated_evaluations_are_bitwise_identical():
    """No atomics and fixed reduction orders: results repeat exactly."""
    x, m, y, nu, psi, eps = random_case(11, 3, 6000, 2000, 0.01, 0.01)
    P = rs().Problem(x, m, y, nu)
    try:
        for prec, kind in ((0, None), (1, rs().PAIRS_TENSOR), (1, rs().PAIRS_FP32)):
            if kind is not None:
                P.set_pair_kernel(kind)
            J1, g1, _ = P.eval(psi, eps, 0.0, prec)
            J2, g2, _ = P.eval(psi, eps, 0.0, prec)
            assert J1 == J2 and np.array_equal(g1, g2)
    finally:
        P.close()


def test_tensor_pairs_fall_back_outside_f16_range():
    """At eps = 1e-7 the target operands w / P leave the f16 range: the
    tensor-core evaluation must hand both passes to the FP32 kernels (same
    per-pair arithmetic, other chunking) rather than overflow."""
    x, m, y, nu, psi, _ = random_case(14, 2, 3000, 700, 1.0, 1e-9)
    P = rs().Problem(x, m, y, nu)
    try:
        P.set_pair_kernel(rs().PAIRS_FP32)
        Jf, gf, _ = P.eval(psi, 1e-7, 0.0, 1)
        P.set_pair_kernel(rs().PAIRS_TENSOR)
        Jt, gt, _ = P.eval(psi, 1e-7, 0.0, 1)
        assert np.isfinite(Jt) and np.all(np.isfinite(gt))
        assert abs(Jt - Jf) <= 1e-9 * abs(Jf)
        assert np.max(np.abs(gt - gf)) <= 1e-9
    finally:
        P.close()


def test_tensor_pairs_passes_are_consistent():
    """Both tensor-core passes form bitwise the same exponents, so with one
    target (p = 1) the gradient vanishes to the FP32 rounding of the shifts,
    as with the FP32 kernels."""
    x, m, y, nu, psi, eps = random_case(16, 3, 20000, 1, 0.01, 0.0)
    nu = np.ones(1)
    P = rs().Problem(x, m, y, nu)
    try:
        for kind in (rs().PAIRS_TENSOR, rs().PAIRS_FP32):
            P.set_pair_kernel(kind)
            _, g, _ = P.eval(psi, eps, 0.0, 1)
            assert abs(g[0]) <= 1e-6, (kind, g[0])
    finally:
        P.close()


def test_automatic_pair_kernel_fp32_for_results_tensor_inside_solves():
    """RSOT_PAIRS_AUTO: an evaluation returned to the caller runs the FP32 pair
    kernels (FP32 pair arithmetic, FP64 reductions); a solve on the same handle
    takes the tensor-core form for its mixed iterations (its stop is certified
    on compensated evaluations) and still meets the tolerance."""
    p = ri.cube_3d(mesh_n=8, eps=1e-3)
    psi = 0.005 * np.random.default_rng(17).standard_normal(p.n)
    P = rs().Problem(p.x, p.mass, p.y, p.nu)
    try:
        assert p.mass.max() * p.nu.max() <= 2e-6
        P.kernel_timing(True)
        Ja, ga, _ = P.eval(psi, p.eps, 0.0, 1)
        names = set(P.kernel_times())
        assert {"lse_mixed", "grad_mixed"} <= names and not ({"lse_tc", "grad_tc"} & names)
        P.kernel_timing(True)
        sol, st = P.solve(eps=p.eps, eps_start=0.1, eps_factor=0.5, tol_l1=1e-6)
        names = set(P.kernel_times())
        P.kernel_timing(False)
        assert st.status == 0 and {"lse_tc", "grad_tc"} <= names
        _, go, _, _ = oracle.dual_grad(p.x, p.mass, p.y, p.nu, sol, p.eps)
        assert np.abs(go).sum() <= 1e-6 * (1 + 1e-9)
        # after the solve, evaluations return to the FP32 form
        Jb, gb, _ = P.eval(psi, p.eps, 0.0, 1)
        assert Jb == Ja and np.array_equal(gb, ga)
    finally:
        P.close()


def test_pair_kernel_argument_checked():
    x, m, y, nu, psi, eps = random_case(15, 2, 100, 10, 0.05, 0.05)
    P = rs().Problem(x, m, y, nu)
    try:
        with pytest.raises(rs().RsotError) as ei:
            P.set_pair_kernel(7)
        assert ei.value.status == 1
    finally:
        P.close()


def test_device_resident_inputs_and_outputs():
    import torch
    x, m, y, nu, psi, eps = random_case(12, 2, 4000, 900, 0.02, 0.02)
    dev = torch.device("cuda:0")
    P = rs().Problem(torch.tensor(x, device=dev), torch.tensor(m, device=dev),
                     torch.tensor(y, device=dev), torch.tensor(nu, device=dev))
    try:
        psi_d = torch.tensor(psi, device=dev)
        J, g, _ = P.eval(psi_d, eps, 0.0, 1)
        assert g.is_cuda
        Jh, gh, _ = P.eval(psi, eps, 0.0, 1)
        assert J == Jh and np.array_equal(g.cpu().numpy(), gh)
    finally:
        P.close()


def test_nonfinite_psi_and_bad_eps_are_rejected():
    x, m, y, nu, psi, eps = random_case(13, 2, 500, 50, 0.05, 0.05)
    P = rs().Problem(x, m, y, nu)
    try:
        bad = psi.copy()
        bad[3] = np.nan
        with pytest.raises(rs().RsotError) as ei:
            P.eval(bad, eps)
        assert ei.value.status == 3
        with pytest.raises(rs().RsotError) as ei:
            P.eval(psi, -1.0)
        assert ei.value.status == 1
    finally:
        P.close()
