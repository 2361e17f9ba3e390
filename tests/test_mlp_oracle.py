"""Pins of the FP64 MLP oracle: GELU closed forms, the Gaussian NLL gradient, BF16 rounding, and
the full backward pass against central finite differences (exact FP64 mode)."""
import math

import numpy as np
import pytest

from oracle import mlp as M


def test_gelu_closed_forms():
    assert M.gelu(np.array([0.0]))[0] == 0.0
    assert M.gelu_grad(np.array([0.0]))[0] == pytest.approx(0.5)
    z = np.array([-3.0, -1.0, 0.5, 2.0])
    np.testing.assert_allclose(M.gelu(z), z * 0.5 * (1 + np.array([math.erf(t / math.sqrt(2)) for t in z])))
    h = 1e-6
    np.testing.assert_allclose(M.gelu_grad(z), (M.gelu(z + h) - M.gelu(z - h)) / (2 * h), rtol=1e-8)
    assert M.gelu(np.array([10.0]))[0] == pytest.approx(10.0)


def test_bf16_rounding():
    assert M.bf16(np.array([1.0]))[0] == 1.0
    assert M.bf16(np.array([1.0 + 2 ** -8]))[0] == 1.0            # tie to even (mantissa 7 bits)
    assert M.bf16(np.array([1.0 + 3 * 2 ** -8]))[0] == 1.0 + 2 ** -6
    assert M.bf16(np.array([3.0e38]))[0] > 3.0e38 * 0.99


def test_nll_gradient_closed_form():
    rng = np.random.default_rng(0)
    Y = rng.standard_normal((5, 8))
    a = rng.standard_normal((5, 4))
    L, dY = M.nll(Y, a)
    mu, s = Y[:, :4], Y[:, 4:]
    np.testing.assert_allclose(dY[:, :4], (mu - a) * np.exp(-2 * s) / 20)
    np.testing.assert_allclose(dY[:, 4:], (1 - (a - mu) ** 2 * np.exp(-2 * s)) / 20)
    assert L == pytest.approx(np.mean(0.5 * (a - mu) ** 2 * np.exp(-2 * s) + s))


def test_nll_clamps_the_log_std():
    """Outside [lo, hi] the log-std is clamped: the loss uses the bound and no gradient flows to
    that output."""
    Y = np.array([[0.3, -7.0], [-0.2, 3.5], [0.1, 0.4]])
    a = np.array([[0.5], [-1.0], [0.2]])
    L, dY = M.nll(Y, a, lo=-5.0, hi=2.0)
    s = np.array([-5.0, 2.0, 0.4])
    e = a[:, 0] - Y[:, 0]
    assert L == pytest.approx(np.mean(0.5 * e * e * np.exp(-2 * s) + s), rel=1e-14)
    assert dY[0, 1] == 0.0 and dY[1, 1] == 0.0 and dY[2, 1] != 0.0
    np.testing.assert_allclose(dY[:, 0], -e * np.exp(-2 * s) / 3, rtol=1e-14)


def _params(rng, fin, H, O, kin=64, scale=(0.3, 0.1, 0.1, 0.1, 0.05, 0.1)):
    shapes = [H * kin, H, H * H, H, O * H, O]
    return np.concatenate([rng.normal(0, sc, n) for sc, n in zip(scale, shapes)])


@pytest.mark.parametrize("sign", [1.0, -1.0])
def test_saturated_network_reduces_to_linear_algebra(sign):
    """GELU(z) = z Phi(z) equals z to within 1e-22 for z >= 10 and 0 to within 1e-22 for z <= -10.
    With every pre-activation beyond +10 the network is the affine chain
    W3 (W2 (W1 x + b1) + b2) + b3 (plain numpy products, x zero-padded to 64 columns); beyond -10
    it outputs b3 alone.  This fixes the layer order, each weight's orientation, each bias and the
    linear output layer."""
    fin, H, O = 5, 16, 8
    rng = np.random.default_rng(4)
    x = rng.uniform(0.5, 1.0, (3, fin))
    W1 = np.zeros((H, 64))
    W1[:, :fin] = sign * rng.uniform(20.0, 30.0, (H, fin))
    b1 = sign * rng.uniform(1.0, 2.0, H)
    W2 = rng.uniform(0.5, 1.0, (H, H))
    b2 = np.full(H, sign * 12.0)
    W3 = rng.standard_normal((O, H))
    b3 = rng.standard_normal(O)
    p = np.concatenate([W1.ravel(), b1, W2.ravel(), b2, W3.ravel(), b3])
    Y, _ = M.forward(p, x, fin, H, O, round_bf16=False)
    X0 = np.zeros((3, 64))
    X0[:, :fin] = x
    Z1 = X0 @ W1.T + b1
    if sign > 0:
        assert Z1.min() > 10 and (Z1 @ W2.T + b2).min() > 10
        np.testing.assert_allclose(Y, (Z1 @ W2.T + b2) @ W3.T + b3, rtol=1e-13)
    else:
        assert Z1.max() < -10
        np.testing.assert_allclose(Y, np.broadcast_to(b3, Y.shape), rtol=0, atol=1e-12)


def test_backward_matches_finite_differences():
    """Central differences of the exact (FP64) loss, on entries drawn from every parameter block
    (W1's input columns, b1, W2, b2, W3, b3); the padding columns of W1 see zero inputs, so their
    gradient is exactly zero."""
    fin, H, O = 5, 128, 256
    rng = np.random.default_rng(1)
    kin = 64
    p = _params(rng, fin, H, O, kin)
    x = rng.standard_normal((3, fin))
    a = rng.standard_normal((3, O // 2))
    L, g, _ = M.gradients(p, x, a, fin, H, O, round_bf16=False)
    starts = np.cumsum([0, H * kin, H, H * H, H, O * H, O])
    idx = [h * kin + c for h, c in zip(rng.integers(0, H, 8), rng.integers(0, fin, 8))]    # W1, real inputs
    for blk in range(1, 6):
        idx += list(rng.integers(starts[blk], starts[blk + 1], 8))
    for i in idx:
        e = np.zeros_like(p)
        e[i] = 1e-6
        Lp = M.nll(M.forward(p + e, x, fin, H, O, False)[0], a)[0]
        Lm = M.nll(M.forward(p - e, x, fin, H, O, False)[0], a)[0]
        assert g[i] == pytest.approx((Lp - Lm) / 2e-6, rel=1e-5, abs=1e-10)
    pad = g[:H * kin].reshape(H, kin)[:, fin:]
    assert np.all(pad == 0.0)
