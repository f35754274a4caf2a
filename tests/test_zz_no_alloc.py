"""The allocation-free entry point, rsot_eval_dense_noalloc, called through the
C ABI: against the FP64 oracle, against the handle-based rsot_eval_dual_grad
(two calls in a row, each with a new potential), at its documented maximum
sizes, and without any change of the device's free memory once warmed up.

rsot_eval_dense_noalloc serves callers that cannot allocate device memory
themselves (their device memory belongs to another component, such as a
framework's caching allocator, or is fixed at start-up): it takes the
caller's device buffers and keeps its own scratch in a static device array of
bounded size.  This file is collected last so that a stop-at-first-failure run
has executed every other test before it.
"""
import ctypes
import os
import re

import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
J_TOL = 1e-5     # the mixed path's tolerances
G_TOL = 1e-6


def header_limit(name):
    src = open(os.path.join(ROOT, "include", "rsot.h")).read()
    return int(re.search(r"#define\s+%s\s+(\d+)" % name, src).group(1))


MAX_NQ = header_limit("RSOT_NOALLOC_MAX_NQ")
MAX_N = header_limit("RSOT_NOALLOC_MAX_N")


def setup():
    import torch
    import paper_2507_23602_gb300 as rs
    so = rs.load()
    vp = ctypes.c_void_p
    so.rsot_eval_dense_noalloc.argtypes = [ctypes.c_int, ctypes.c_int64, vp, vp, ctypes.c_int64,
                                           vp, vp, vp, ctypes.c_double, vp,
                                           ctypes.POINTER(ctypes.c_double), vp]
    so.rsot_eval_dense_noalloc.restype = ctypes.c_int
    return torch, rs, so


def case(seed, d, nq, n, eps):
    rng = np.random.default_rng(seed)
    x = rng.uniform(0, 1, (nq, d))
    m = rng.uniform(0.5, 1.5, nq)
    m /= m.sum()
    y = rng.uniform(0, 1, (n, d))
    nu = rng.uniform(0.5, 1.5, n)
    nu /= nu.sum()
    return x, m, y, nu, eps


def call(so, torch, d, nq, n, bufs, psi, grad, eps, nq_arg=None, n_arg=None):
    x, m, y, nu = bufs
    J = ctypes.c_double(np.nan)
    st = so.rsot_eval_dense_noalloc(
        d, nq if nq_arg is None else nq_arg, ctypes.c_void_p(x.data_ptr()),
        ctypes.c_void_p(m.data_ptr()), n if n_arg is None else n_arg,
        ctypes.c_void_p(y.data_ptr()), ctypes.c_void_p(nu.data_ptr()),
        ctypes.c_void_p(psi.data_ptr()), eps,
        ctypes.c_void_p(torch.cuda.current_stream().cuda_stream), ctypes.byref(J),
        ctypes.c_void_p(grad.data_ptr()))
    return st, J.value


@pytest.mark.parametrize("d,nq,n,eps", [(3, 5000, 1300, 0.01), (2, 3000, 700, 0.02)])
def test_noalloc_matches_oracle_and_handle_path_on_two_calls_in_a_row(d, nq, n, eps):
    torch, rs, so = setup()
    x, m, y, nu, eps = case(nq + n, d, nq, n, eps)
    dev = torch.device("cuda", torch.cuda.current_device())
    bufs = [torch.tensor(a, device=dev) for a in (x, m, y, nu)]
    P = rs.Problem(x, m, y, nu)
    rng = np.random.default_rng(d)
    try:
        for call_no in range(2):
            psi = 0.01 * rng.standard_normal(n)        # a new potential each call
            Jo, go, _, _ = oracle.dual_grad(x, m, y, nu, psi, eps)
            Jr, gr, _ = P.eval(psi, eps, 0.0, rs.MIXED)
            grad = torch.full((n,), np.nan, dtype=torch.float64, device=dev)
            st, J = call(so, torch, d, nq, n, bufs, torch.tensor(psi, device=dev), grad, eps)
            assert st == 0, f"call {call_no}: status {st}"
            g = grad.cpu().numpy()
            assert abs(J - Jo) <= J_TOL * abs(Jo), (call_no, J, Jo)
            assert np.max(np.abs(g - go)) <= G_TOL, call_no
            assert abs(J - Jr) <= J_TOL * abs(Jr), (call_no, J, Jr)
            assert np.max(np.abs(g - gr)) <= G_TOL, call_no
    finally:
        P.close()


def test_noalloc_at_its_maximum_sizes_against_the_handle_path():
    """nq and n at the documented maxima (d = 3): the tight end of the static
    scratch layout, against the handle path's FP32 pair kernels."""
    torch, rs, so = setup()
    d, nq, n, eps = 3, MAX_NQ, MAX_N, 2e-3
    x, m, y, nu, eps = case(77, d, nq, n, eps)
    dev = torch.device("cuda", torch.cuda.current_device())
    bufs = [torch.tensor(a, device=dev) for a in (x, m, y, nu)]
    psi = 0.003 * np.random.default_rng(78).standard_normal(n)
    P = rs.Problem(x, m, y, nu)
    try:
        P.set_pair_kernel(rs.PAIRS_FP32)
        Jr, gr, _ = P.eval(psi, eps, 0.0, rs.MIXED)
    finally:
        P.close()
    grad = torch.full((n,), np.nan, dtype=torch.float64, device=dev)
    st, J = call(so, torch, d, nq, n, bufs, torch.tensor(psi, device=dev), grad, eps)
    assert st == 0, st
    g = grad.cpu().numpy()
    assert abs(J - Jr) <= J_TOL * abs(Jr), (J, Jr)
    assert np.max(np.abs(g - gr)) <= G_TOL
    assert abs(g.sum()) <= 5e-7                      # mass balance at ex2.approx accuracy


def test_noalloc_allocates_nothing_once_warm_and_leaves_outputs_on_error():
    torch, rs, so = setup()
    d, nq, n, eps = 3, 20000, 3000, 0.01
    x, m, y, nu, eps = case(5, d, nq, n, eps)
    dev = torch.device("cuda", torch.cuda.current_device())
    bufs = [torch.tensor(a, device=dev) for a in (x, m, y, nu)]
    psi = torch.tensor(0.01 * np.random.default_rng(6).standard_normal(n), device=dev)
    grad = torch.zeros(n, dtype=torch.float64, device=dev)
    assert call(so, torch, d, nq, n, bufs, psi, grad, eps)[0] == 0    # warm-up (first call)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for _ in range(3):
        assert call(so, torch, d, nq, n, bufs, psi, grad, eps)[0] == 0
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    # a non-finite potential: NONFINITE, and neither output is written
    bad = psi.clone()
    bad[7] = float("nan")
    sentinel = torch.full((n,), 123.0, dtype=torch.float64, device=dev)
    st, J = call(so, torch, d, nq, n, bufs, bad, sentinel, eps)
    assert st == 3 and np.isnan(J)
    assert torch.all(sentinel == 123.0)


def test_noalloc_rejects_sizes_beyond_its_scratch_and_host_pointers():
    torch, rs, so = setup()
    x, m, y, nu, eps = case(5, 2, 100, 10, 0.05)
    dev = torch.device("cuda", torch.cuda.current_device())
    bufs = [torch.tensor(a, device=dev) for a in (x, m, y, nu)]
    psi = torch.zeros(10, dtype=torch.float64, device=dev)
    grad = torch.zeros(10, dtype=torch.float64, device=dev)
    assert call(so, torch, 2, 100, 10, bufs, psi, grad, eps, nq_arg=MAX_NQ + 1)[0] == 1
    assert call(so, torch, 2, 100, 10, bufs, psi, grad, eps, n_arg=MAX_N + 1)[0] == 1
    host = [torch.tensor(a) for a in (x, m, y, nu)]
    assert call(so, torch, 2, 100, 10, host, psi, grad, eps)[0] == 1
