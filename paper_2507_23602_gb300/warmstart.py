"""Learned warm start for the dual potential (host orchestration).

Every numerical step runs in librsot: the training potentials come from the
library's batched solver (Algorithm 1 with the eps-schedule of Sec. 4.2), and
the network is trained and evaluated with the library's MLP kernels.  This
module only assembles feature rows and drives the loops.

Features of target j of a problem with density parameters theta (16 values,
4 x (mu_x, mu_y, log sigma, weight logit)) are [theta, y_j]; the label is the
potential psi_j centred so that sum_j nu_j psi_j = 0 (J is invariant under
psi -> psi + c, App. A), divided by PSI_SCALE.
"""
from __future__ import annotations

import time
from typing import Dict, List, Sequence

import numpy as np

import rsot_inputs as ri

from . import MIXED, Batch, MLP, SolveOptions

PSI_SCALE = 0.05
IN_DIM = 18


def features(theta: np.ndarray, y: np.ndarray) -> np.ndarray:
    x = np.empty((y.shape[0], IN_DIM), dtype=np.float32)
    x[:, :16] = np.asarray(theta, dtype=np.float32)[None, :]
    x[:, 16:] = y
    return x


def centred(psi: np.ndarray, nu: np.ndarray) -> np.ndarray:
    return psi - psi @ nu


def generate(seeds: Sequence[int], mesh_n=64, n_targets=4096, eps=5e-3, tol_l1=1e-5,
             chunk=128, eps_start=0.1):
    """Solve the problems of `seeds` in batches (mixed precision, eps-schedule
    from eps_start) and return (features [S*n, 18] float32, labels [S*n] float32,
    seconds)."""
    X, Y = [], []
    t0 = time.perf_counter()
    for c0 in range(0, len(seeds), chunk):
        probs = [ri.warmstart_problem(s, mesh_n, n_targets, eps) for s in seeds[c0:c0 + chunk]]
        B = Batch([(p.x, p.mass, p.y, p.nu) for p, _ in probs])
        try:
            psi, st = B.solve(np.full(len(probs), eps), eps_start=eps_start, eps_factor=0.5,
                              tol_l1=tol_l1, precision=MIXED, refine_fp64=False,
                              raise_on_error=False)
        finally:
            B.close()
        for (p, th), ps in zip(probs, B.split(psi)):
            X.append(features(th, p.y))
            Y.append((centred(ps, p.nu) / PSI_SCALE).astype(np.float32))
    return np.concatenate(X), np.concatenate(Y), time.perf_counter() - t0


def train(X, Y, epochs=8, rows=8192, lr=2e-3, seed=0, width=256, log=None):
    """Adam on the library's MLP; X, Y are moved to the GPU once (torch)."""
    import torch
    dev = torch.device("cuda", torch.cuda.current_device())
    Xd = torch.as_tensor(X, device=dev)
    Yd = torch.as_tensor(Y, device=dev)
    net = MLP(IN_DIM, width, seed=seed)
    g = torch.Generator(device=dev)
    g.manual_seed(seed)
    n = Xd.shape[0]
    steps = max(1, n // rows)
    hist = []
    t0 = time.perf_counter()
    for ep in range(epochs):
        perm = torch.randperm(n, device=dev, generator=g)
        lr_ep = lr * 0.5 * (1.0 + np.cos(np.pi * ep / max(1, epochs)))   # cosine decay
        tot = 0.0
        for s in range(steps):
            idx = perm[s * rows:(s + 1) * rows]
            tot += net.train_step(Xd[idx], Yd[idx], lr_ep)
        hist.append(tot / steps)
        if log:
            log(f"epoch {ep} loss {hist[-1]:.4e}")
    return net, hist, time.perf_counter() - t0


def predict(net: MLP, theta, y, nu) -> np.ndarray:
    psi = net.forward(features(theta, y)).astype(np.float64) * PSI_SCALE
    return centred(psi, nu)


def evaluate(net: MLP, seeds: Sequence[int], mesh_n=64, n_targets=4096, eps=5e-3, tol_l1=1e-6,
             chunk=128, eps_start=0.1) -> Dict[str, float]:
    """Solve the held-out problems twice with the batched solver and its
    refinement (compensated reference evaluations) to tol_l1: from psi = 0 with the eps-schedule (the fallback and
    judge), and from the network's psi directly at eps.  Returns totals."""
    res = {"plain_seconds": 0.0, "warm_seconds": 0.0, "plain_rounds": 0, "warm_rounds": 0,
           "plain_evals": 0, "warm_evals": 0, "plain_converged": 0, "warm_converged": 0,
           "problems": 0, "warm_max_grad_l1": 0.0, "plain_max_grad_l1": 0.0}
    for c0 in range(0, len(seeds), chunk):
        probs = [ri.warmstart_problem(s, mesh_n, n_targets, eps) for s in seeds[c0:c0 + chunk]]
        B = Batch([(p.x, p.mass, p.y, p.nu) for p, _ in probs])
        epsv = np.full(len(probs), eps)
        try:
            _, st0 = B.solve(epsv, eps_start=eps_start, eps_factor=0.5, tol_l1=tol_l1,
                             precision=MIXED, refine_fp64=True, raise_on_error=False)
            psi0 = np.concatenate([predict(net, th, p.y, p.nu) for p, th in probs])
            _, st1 = B.solve(epsv, psi0=psi0, eps_start=0.0, tol_l1=tol_l1, precision=MIXED,
                             refine_fp64=True, raise_on_error=False)
        finally:
            B.close()
        for key, st in (("plain", st0), ("warm", st1)):
            res[key + "_seconds"] += st["seconds"]
            res[key + "_rounds"] += st["rounds"]
            res[key + "_evals"] += st["evals"]
            res[key + "_converged"] += st["converged"]
            res[key + "_max_grad_l1"] = max(res[key + "_max_grad_l1"], st["max_grad_l1"])
        res["problems"] += len(probs)
    return res
