"""MLP oracle -- TEST INFRASTRUCTURE ONLY.

A plain numpy FP64 statement of the warm-start network and of its gradient
by hand-written back-propagation: in_dim -> W (SiLU) -> W (SiLU) -> W (SiLU)
-> 1, loss = mean (f(x) - y)^2 / 2.  With ``emulate_bf16`` the operands are
rounded to bfloat16 (round to nearest even) at the places where the GPU
kernels round them (inputs, the three weight matrices, the hidden
activations, the stored pre-activations whose SiLU' the back-propagation
takes, and the back-propagated dZ), everything else in FP64; without it
the network is plain FP64 (the form pinned by finite differences).

The parameter block layout is the library's: W1 [W][in_pad], b1 [W],
W2 [W][W], b2, W3 [W][W], b3, w4 [W], b4 [1] with in_pad = in_dim rounded up
to 32.
"""
from __future__ import annotations

import numpy as np


def bf16(a):
    """Round to bfloat16 (nearest even) and return as float64."""
    a32 = np.asarray(a, dtype=np.float32)
    u = a32.view(np.uint32).astype(np.uint64)
    rounded = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return rounded.astype(np.uint32).view(np.float32).astype(np.float64)


def silu(z):
    return z / (1.0 + np.exp(-z))


def dsilu(z):
    s = 1.0 / (1.0 + np.exp(-z))
    return s * (1.0 + z * (1.0 - s))


def unpack(p, in_dim, width):
    in_pad = (in_dim + 31) // 32 * 32
    p = np.asarray(p, dtype=np.float64)
    sizes = [width * in_pad, width, width * width, width, width * width, width, width, 1]
    out, o = [], 0
    for s in sizes:
        out.append(p[o:o + s])
        o += s
    W1 = out[0].reshape(width, in_pad)
    W2 = out[2].reshape(width, width)
    W3 = out[4].reshape(width, width)
    return W1, out[1], W2, out[3], W3, out[5], out[6], out[7][0], in_pad


def forward(p, x, in_dim, width, emulate_bf16=True):
    r = (lambda a: bf16(a)) if emulate_bf16 else (lambda a: np.asarray(a, dtype=np.float64))
    W1, b1, W2, b2, W3, b3, w4, b4, in_pad = unpack(p, in_dim, width)
    X0 = np.zeros((x.shape[0], in_pad))
    X0[:, :in_dim] = x
    X0 = r(X0)
    Z1 = X0 @ r(W1).T + b1
    H1 = r(silu(Z1))
    Z2 = H1 @ r(W2).T + b2
    H2 = r(silu(Z2))
    Z3 = H2 @ r(W3).T + b3
    H3 = r(silu(Z3))
    out = H3 @ w4 + b4
    return out, (X0, Z1, H1, Z2, H2, Z3, H3)


def loss_and_grad(p, x, y, in_dim, width, emulate_bf16=True):
    r = (lambda a: bf16(a)) if emulate_bf16 else (lambda a: np.asarray(a, dtype=np.float64))
    W1, b1, W2, b2, W3, b3, w4, b4, in_pad = unpack(p, in_dim, width)
    out, (X0, Z1, H1, Z2, H2, Z3, H3) = forward(p, x, in_dim, width, emulate_bf16)
    B = x.shape[0]
    e = out - y
    loss = 0.5 * np.mean(e * e)
    dout = e / B
    dw4 = H3.T @ dout
    db4 = dout.sum()
    dZ3 = r(np.outer(dout, w4) * dsilu(r(Z3)))
    dW3 = dZ3.T @ H2
    db3 = dZ3.sum(0)
    dZ2 = r((dZ3 @ r(W3)) * dsilu(r(Z2)))
    dW2 = dZ2.T @ H1
    db2 = dZ2.sum(0)
    dZ1 = r((dZ2 @ r(W2)) * dsilu(r(Z1)))
    dW1 = dZ1.T @ X0
    db1 = dZ1.sum(0)
    g = np.concatenate([dW1.ravel(), db1, dW2.ravel(), db2, dW3.ravel(), db3, dw4, [db4]])
    return loss, g


def abs_scales(p, x, y, in_dim, width):
    """Scale of every output and gradient entry for element-wise comparisons:
    the same sums as ``forward`` / ``loss_and_grad`` taken over the absolute
    values of their terms (e.g. sum_r |dZ_ri| |H_rj| for dW_ij).  A GEMM that
    accumulates in FP32 errs by at most a small multiple of 2^-24 times this
    scale per entry, whatever cancellation the signed sum has."""
    W1, b1, W2, b2, W3, b3, w4, b4, in_pad = unpack(p, in_dim, width)
    out, (X0, Z1, H1, Z2, H2, Z3, H3) = forward(p, x, in_dim, width, True)
    B = x.shape[0]
    out_scale = np.abs(H3) @ np.abs(w4) + abs(b4)
    e = out - y
    dout = e / B
    dZ3 = bf16(np.outer(dout, w4) * dsilu(bf16(Z3)))
    dZ2 = bf16((dZ3 @ bf16(W3)) * dsilu(bf16(Z2)))
    dZ1 = bf16((dZ2 @ bf16(W2)) * dsilu(bf16(Z1)))
    a = np.abs
    g = np.concatenate([(a(dZ1).T @ a(X0)).ravel(), a(dZ1).sum(0),
                        (a(dZ2).T @ a(H1)).ravel(), a(dZ2).sum(0),
                        (a(dZ3).T @ a(H2)).ravel(), a(dZ3).sum(0),
                        a(H3).T @ a(dout), [a(dout).sum()]])
    return out_scale, g
