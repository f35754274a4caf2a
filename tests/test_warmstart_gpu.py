"""Learned warm start, end to end at a reduced size: potentials from the
batched solver train the MLP (the library's kernels); on held-out problems
the warm-started solve must reach the same tolerance with fewer evaluations
than the plain eps-scheduled solve from psi = 0."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def test_warm_start_pipeline_small():
    from paper_2507_23602_gb300 import warmstart as ws
    kw = dict(mesh_n=16, n_targets=256, eps=5e-3)
    X, Y, _ = ws.generate(list(range(10000, 10096)), tol_l1=1e-5, chunk=48, **kw)
    assert X.shape == (96 * 256, 18) and np.all(np.isfinite(Y))
    net, hist, _ = ws.train(X, Y, epochs=30, rows=2048, lr=3e-3, width=128)
    assert hist[-1] < 0.5 * hist[0]
    res = ws.evaluate(net, list(range(20000, 20008)), tol_l1=1e-6, chunk=8, **kw)
    net.close()
    assert res["plain_converged"] == 8 and res["warm_converged"] == 8, res
    assert res["warm_max_grad_l1"] <= 1e-6
    assert res["warm_evals"] < res["plain_evals"], res
