"""The allocation-free entry point, rsot_eval_dense_noalloc, called through the
C ABI, against the handle-based rsot_eval_dual_grad.

rsot_eval_dense_noalloc serves callers that must not allocate device memory
themselves (their device memory is owned by another component or fixed at
start-up): it takes the caller's device buffers and keeps its own scratch in a
static device array of bounded size.  This file is collected last so that a
stop-at-first-failure run has executed every other test before it.
"""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

MAX_NQ = 524288
MAX_N = 65536


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
def test_noalloc_matches_handle_path_on_two_calls_in_a_row(d, nq, n, eps):
    torch, rs, so = setup()
    x, m, y, nu, eps = case(nq + n, d, nq, n, eps)
    dev = torch.device("cuda", torch.cuda.current_device())
    bufs = [torch.tensor(a, device=dev) for a in (x, m, y, nu)]
    P = rs.Problem(x, m, y, nu)
    rng = np.random.default_rng(d)
    try:
        for call_no in range(2):
            psi = 0.01 * rng.standard_normal(n)        # a new potential each call
            Jr, gr, _ = P.eval(psi, eps, 0.0, rs.MIXED)
            grad = torch.full((n,), np.nan, dtype=torch.float64, device=dev)
            st, J = call(so, torch, d, nq, n, bufs, torch.tensor(psi, device=dev), grad, eps)
            assert st == 0, f"call {call_no}: status {st}"
            assert abs(J - Jr) <= 1e-5 * abs(Jr), (call_no, J, Jr)
            assert np.max(np.abs(grad.cpu().numpy() - gr)) <= 1e-6, call_no
    finally:
        P.close()


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
