"""FP64 oracle of the learned proposal's MLP -- TEST INFRASTRUCTURE ONLY.

A plain forward/backward pass of in -> hidden -> hidden -> out with GELU (erf form) and the mean
Gaussian negative log-likelihood of target actions under (mean, clamped log-std) outputs, in
float64 numpy.  With ``bf16=True`` every operand the tensor-core path stores in BF16 (inputs,
weights, activations, pre-activations, back-propagated gradients) is rounded to BF16 at the same
points, so the comparison isolates accumulation order; with ``bf16=False`` it is the exact
function whose gradient the finite-difference pin checks.

Parity unpinned: where the BF16 rounding sits (which intermediates are rounded) mirrors what
the tensor-core kernels store; no CPU pin fixes it, only the GPU comparison does.  Everything
else (GELU and its derivative, the layers, the NLL and its clamp, every back-propagation step)
is pinned in tests/test_mlp_oracle.py, and tests/test_oracle_mutants.py checks that those pins
catch planted mistakes.
"""
import math

import numpy as np


def bf16(x):
    """Round float64 values to the nearest BF16 (ties to even), returned as float64."""
    f = np.asarray(x, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    u = (u + 0x7FFF + lsb) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


_erf = np.vectorize(math.erf)


def gelu(z):
    return 0.5 * z * (1.0 + _erf(z / math.sqrt(2.0)))


def gelu_grad(z):
    return 0.5 * (1.0 + _erf(z / math.sqrt(2.0))) + z * np.exp(-0.5 * z * z) / math.sqrt(2.0 * math.pi)


def unpack(params, fin, H, O):
    kin = (fin + 63) // 64 * 64
    p = np.asarray(params, np.float64)
    o = 0
    out = {}
    for name, shape in [("W1", (H, kin)), ("b1", (H,)), ("W2", (H, H)), ("b2", (H,)), ("W3", (O, H)), ("b3", (O,))]:
        n = int(np.prod(shape))
        out[name] = p[o:o + n].reshape(shape)
        o += n
    return out, kin


def forward(params, x, fin, H, O, round_bf16=True):
    r = bf16 if round_bf16 else (lambda a: np.asarray(a, np.float64))
    P, kin = unpack(params, fin, H, O)
    X0 = np.zeros((x.shape[0], kin))
    X0[:, :fin] = x
    X0 = r(X0)
    W1, W2, W3 = r(P["W1"]), r(P["W2"]), r(P["W3"])
    Z1 = X0 @ W1.T + P["b1"]
    H1 = r(gelu(Z1))
    Z2 = H1 @ W2.T + P["b2"]
    H2 = r(gelu(Z2))
    Y = H2 @ W3.T + P["b3"]
    return Y, dict(X0=X0, Z1=r(Z1), H1=H1, Z2=r(Z2), H2=H2, W1=W1, W2=W2, W3=W3)


def nll(Y, a, lo=-5.0, hi=2.0):
    """Mean over samples and action dims of (a - mu)^2 / (2 sigma^2) + log sigma, and dL/dY."""
    D = a.shape[1]
    mu, sr = Y[:, :D], Y[:, D:]
    s = np.clip(sr, lo, hi)
    e = a - mu
    iv = np.exp(-2.0 * s)
    n = a.shape[0] * D
    L = np.sum(0.5 * e * e * iv + s) / n
    dY = np.zeros_like(Y)
    dY[:, :D] = -e * iv / n
    dY[:, D:] = np.where((sr > lo) & (sr < hi), (1.0 - e * e * iv) / n, 0.0)
    return L, dY


def gradients(params, x, a, fin, H, O, lo=-5.0, hi=2.0, round_bf16=True):
    r = bf16 if round_bf16 else (lambda q: np.asarray(q, np.float64))
    Y, c = forward(params, x, fin, H, O, round_bf16)
    L, dY = nll(Y, a, lo, hi)
    dY = r(dY)
    g = {"W3": dY.T @ c["H2"], "b3": dY.sum(0)}
    dA2 = r((dY @ c["W3"]) * gelu_grad(c["Z2"]))
    g["W2"], g["b2"] = dA2.T @ c["H1"], dA2.sum(0)
    dA1 = r((dA2 @ c["W2"]) * gelu_grad(c["Z1"]))
    g["W1"], g["b1"] = dA1.T @ c["X0"], dA1.sum(0)
    flat = np.concatenate([g[k].reshape(-1) for k in ("W1", "b1", "W2", "b2", "W3", "b3")])
    return L, flat, Y
