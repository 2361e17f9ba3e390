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


def test_backward_matches_finite_differences():
    fin, H, O = 5, 128, 256
    rng = np.random.default_rng(1)
    kin = 64
    p = np.concatenate([rng.normal(0, 0.3, H * kin), rng.normal(0, 0.1, H), rng.normal(0, 0.1, H * H),
                        rng.normal(0, 0.1, H), rng.normal(0, 0.05, O * H), rng.normal(0, 0.1, O)])
    P, _ = M.unpack(p, fin, H, O)
    x = rng.standard_normal((3, fin))
    a = rng.standard_normal((3, O // 2))
    L, g, _ = M.gradients(p, x, a, fin, H, O, round_bf16=False)
    idx = rng.choice(len(p), 40, replace=False)
    # padding columns of W1 see zero inputs: their gradient is exactly zero
    for i in idx:
        e = np.zeros_like(p)
        e[i] = 1e-6
        Lp = M.nll(M.forward(p + e, x, fin, H, O, False)[0], a)[0]
        Lm = M.nll(M.forward(p - e, x, fin, H, O, False)[0], a)[0]
        assert g[i] == pytest.approx((Lp - Lm) / 2e-6, rel=1e-5, abs=1e-10)
