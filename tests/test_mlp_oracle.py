"""Pins of the MLP oracle: finite differences of the FP64 network, bfloat16
rounding against torch's conversion, and the zero-residual case."""
import numpy as np
import pytest

from oracle import mlp


def params(in_dim, width, seed):
    rng = np.random.default_rng(seed)
    in_pad = (in_dim + 31) // 32 * 32
    n = width * in_pad + width + 2 * (width * width + width) + width + 1
    p = rng.normal(0, 0.3, n)
    W1 = p[:width * in_pad].reshape(width, in_pad)
    W1[:, in_dim:] = 0.0
    return p


def test_bf16_rounding_matches_torch():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(0)
    a = np.concatenate([rng.normal(0, 1, 1000), rng.normal(0, 1e-3, 1000), [1.0, 1.0 + 2 ** -8,
                                                                           1.0 + 3 * 2 ** -9, -2.5]])
    ref = torch.tensor(a, dtype=torch.float32).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(mlp.bf16(a), ref)


@pytest.mark.parametrize("seed", [1, 2])
def test_gradient_matches_central_differences(seed):
    in_dim, width = 5, 16
    p = params(in_dim, width, seed)
    rng = np.random.default_rng(seed + 10)
    x = rng.normal(0, 1, (40, in_dim))
    y = rng.normal(0, 1, 40)
    _, g = mlp.loss_and_grad(p, x, y, in_dim, width, emulate_bf16=False)
    in_pad = 32
    live = np.ones_like(p, bool)
    live[:width * in_pad] = (np.arange(width * in_pad) % in_pad) < in_dim   # padded columns
    for _ in range(4):
        v = rng.normal(0, 1, p.shape) * live
        h = 1e-5
        lp, _ = mlp.loss_and_grad(p + h * v, x, y, in_dim, width, emulate_bf16=False)
        lm, _ = mlp.loss_and_grad(p - h * v, x, y, in_dim, width, emulate_bf16=False)
        assert abs((lp - lm) / (2 * h) - g @ v) <= 1e-7 * max(1.0, abs(g @ v))


def test_zero_residual_gives_zero_gradient():
    in_dim, width = 3, 8
    p = params(in_dim, width, 3)
    x = np.random.default_rng(4).normal(0, 1, (10, in_dim))
    y, _ = mlp.forward(p, x, in_dim, width, emulate_bf16=False)
    loss, g = mlp.loss_and_grad(p, x, y, in_dim, width, emulate_bf16=False)
    assert loss == 0.0 and np.all(g == 0.0)


def test_abs_scales_bound_the_signed_sums_and_equal_them_for_one_row():
    """abs_scales takes each gradient sum over |terms|: it bounds |grad| entry by
    entry, and with a single row every weight and bias gradient has one term,
    so the scale is exactly |grad| (a dropped or transposed factor would break
    either)."""
    in_dim, width = 5, 16
    p = params(in_dim, width, 5)
    rng = np.random.default_rng(6)
    x = rng.normal(0, 1, (30, in_dim))
    y = rng.normal(0, 1, 30)
    out, _ = mlp.forward(p, x, in_dim, width)
    _, g = mlp.loss_and_grad(p, x, y, in_dim, width)
    so, sg = mlp.abs_scales(p, x, y, in_dim, width)
    assert np.all(np.abs(g) <= sg * (1 + 1e-12))
    assert np.all(np.abs(out) <= so * (1 + 1e-12))
    assert np.sum(sg) > 1.5 * np.sum(np.abs(g))       # cancellation present with 30 rows
    _, g1 = mlp.loss_and_grad(p, x[:1], y[:1], in_dim, width)
    so1, sg1 = mlp.abs_scales(p, x[:1], y[:1], in_dim, width)
    assert np.allclose(sg1, np.abs(g1), rtol=1e-12, atol=0.0)
