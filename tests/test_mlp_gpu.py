"""The warm-start network's own kernels (BF16 tensor-core GEMMs, FP32
accumulation; every GEMM kernel: tcgen05 with the accumulator in tensor memory
and TMA or cp.async operand copies, and warp-level mma.sync) against the FP64
MLP oracle that rounds to bfloat16 where the kernels do."""
import numpy as np
import pytest

from oracle import mlp as omlp

pytestmark = pytest.mark.gpu


def rs():
    import paper_2507_23602_gb300 as m
    return m


def setup(in_dim, width, rows, seed, kind=0):
    net = rs().MLP(in_dim, width, seed=seed)
    net.set_gemm_kernel(kind)
    rng = np.random.default_rng(seed)
    x = rng.normal(0, 1, (rows, in_dim)).astype(np.float32)
    y = rng.normal(0, 1, rows).astype(np.float32)
    return net, x, y


KINDS = [0, 1, 2]   # GEMM_TCGEN05 (TMA), GEMM_MMA_SYNC, GEMM_TCGEN05_CPASYNC

# Element-wise bounds, per entry relative to its scale s (the same sum over the
# absolute values of its terms, oracle.mlp.abs_scales):
#  * FP32 accumulation of K <= 4096 products (tensor-core GEMMs, split-K sums):
#    at most about K 2^-24 s <= 2.5e-4 s;
#  * a bfloat16 operand (activation H or back-propagated dZ) rounded the other
#    way than in the FP64 oracle (its pre-rounding value within FP32 error of a
#    rounding boundary) moves its own term by one bf16 unit, 2^-8 of the term,
#    and the flipped terms of one sum are part of s: at most 2 x 2^-8 s;
# so |g - g_o| <= 1e-2 s for every entry.  Flips touch few terms of each sum:
# measured on GB300 over these shapes (all three GEMM kernels), err / s has a
# median below 1e-5 and a 99th percentile below 1.5e-4; the checks below leave
# a margin of ten and would fail for a wrong operand, index or dropped term,
# which put the error at the size of s itself.
REL_BOUND = 1e-2
REL_MEDIAN = 1e-4
REL_P99 = 2e-3


def elementwise(a, b, s):
    a = np.asarray(a, dtype=np.float64)
    err = np.abs(a - b)
    bad = err > REL_BOUND * s + 1e-12
    assert not np.any(bad), (np.flatnonzero(bad)[:8], err[bad][:8], s[bad][:8])
    r = err / np.maximum(s, 1e-30)
    q50, q99 = np.quantile(r, [0.5, 0.99])
    assert q50 <= REL_MEDIAN and q99 <= REL_P99, (q50, q99)


@pytest.mark.parametrize("kind", KINDS)
# (3, 64, 37): fewer rows than one TMA box; (5, 104, 300): K = 104, so the
# second K box is zero-filled past 40 of its 64 columns, and N = 104 < 128 rows;
# (6, 96, 500) and (4, 160, 333): the persistent kernel's last 64-column box
# half filled (N = 96, 160 are multiples of 32, not of 64); (40, 128, 700):
# in_pad 64, a full K box in the first layer and N = 64 in its weight
# gradient; (3, 32, 129): the narrowest persistent-kernel width, two row tiles
@pytest.mark.parametrize("in_dim,width,rows", [(18, 256, 1000), (18, 256, 4096), (5, 64, 300),
                                               (7, 200, 777), (3, 64, 37), (5, 104, 300),
                                               (6, 96, 500), (4, 160, 333), (40, 128, 700),
                                               (3, 32, 129)])
def test_forward_matches_oracle(in_dim, width, rows, kind):
    net, x, y = setup(in_dim, width, rows, 7, kind)
    try:
        out = net.forward(x)
        x64 = x.astype(np.float64)
        ref, _ = omlp.forward(net.params(), x64, in_dim, width)
        scale, _ = omlp.abs_scales(net.params(), x64, y.astype(np.float64), in_dim, width)
        elementwise(out, ref, scale)
    finally:
        net.close()


@pytest.mark.parametrize("kind", KINDS)
@pytest.mark.parametrize("in_dim,width,rows", [(18, 256, 2048), (5, 64, 300), (7, 200, 777),
                                               (5, 104, 300), (6, 96, 500), (4, 160, 333),
                                               (40, 128, 700), (3, 32, 129)])
def test_gradients_match_oracle(in_dim, width, rows, kind):
    net, x, y = setup(in_dim, width, rows, 11, kind)
    try:
        loss, g = net.gradients(x, y)
        x64, y64 = x.astype(np.float64), y.astype(np.float64)
        lo, go = omlp.loss_and_grad(net.params(), x64, y64, in_dim, width)
        assert abs(loss - lo) <= 1e-3 * abs(lo)
        _, scale = omlp.abs_scales(net.params(), x64, y64, in_dim, width)
        elementwise(g, go, scale)
    finally:
        net.close()


def test_training_reduces_the_loss():
    net = rs().MLP(2, 64, seed=3)
    rng = np.random.default_rng(5)
    x = rng.uniform(-1, 1, (4096, 2)).astype(np.float32)
    y = (np.sin(2 * x[:, 0]) * np.cos(x[:, 1])).astype(np.float32)
    try:
        l0, _ = net.gradients(x, y)
        for _ in range(300):
            idx = rng.integers(0, 4096, 512)
            net.train_step(x[idx], y[idx], 3e-3)
        l1, _ = net.gradients(x, y)
        assert l1 < 0.05 * l0, (l0, l1)
    finally:
        net.close()


def test_gemm_kernels_agree():
    """The tcgen05 and mma.sync GEMM kernels on the same network and batch:
    the same products summed in another order, so forward outputs and
    gradients agree to FP32 accumulation (plus the rare BF16 activation that
    rounds the other way)."""
    net, x, y = setup(18, 256, 5000, 13, 0)
    try:
        o0 = net.forward(x)
        l0, g0 = net.gradients(x, y)
        net.set_gemm_kernel(1)
        o1 = net.forward(x)
        l1, g1 = net.gradients(x, y)
        assert np.max(np.abs(o0 - o1)) <= 2e-3 * np.max(np.abs(o1)) + 1e-5
        assert abs(l0 - l1) <= 1e-3 * abs(l1)
        assert np.linalg.norm(g0 - g1) <= 1e-2 * np.linalg.norm(g1)
    finally:
        net.close()


@pytest.mark.parametrize("in_dim,width,rows", [(18, 256, 5000), (7, 200, 777), (3, 64, 37),
                                               (4, 160, 333), (40, 128, 700), (3, 32, 129)])
def test_tma_and_cp_async_copies_give_equal_results(in_dim, width, rows):
    """The default tcgen05 GEMMs (TMA operand copies into 128-byte swizzled
    tiles; the persistent kernel for the BF16 epilogues where N <= 256 is a
    multiple of 32) and the tcgen05 kernel with cp.async copies (unswizzled
    tiles): the same MMAs over the same K stages, so outputs, loss and
    gradients are bitwise equal."""
    net, x, y = setup(in_dim, width, rows, 17, rs().GEMM_TCGEN05)
    try:
        o0 = net.forward(x)
        l0, g0 = net.gradients(x, y)
        net.set_gemm_kernel(rs().GEMM_TCGEN05_CPASYNC)
        o2 = net.forward(x)
        l2, g2 = net.gradients(x, y)
        assert np.array_equal(o0, o2)
        assert l0 == l2
        assert np.array_equal(g0, g2)
    finally:
        net.close()


def test_gemm_kernel_kind_is_checked():
    net = rs().MLP(4, 64, seed=1)
    try:
        for bad in (3, -1):
            with pytest.raises(rs().RsotError):
                net.set_gemm_kernel(bad)
    finally:
        net.close()
