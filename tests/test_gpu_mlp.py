"""The tensor-core MLP of the learned proposal against the FP64 oracle run on BF16-rounded
operands (forward outputs, NLL loss and every parameter gradient), and training progress."""
import numpy as np
import pytest
import torch

from oracle import mlp as M

pytestmark = pytest.mark.gpu

FIN, H, O = 49, 256, 1024


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2603_12185_gb300 import build
    build.build()


def _data(B, seed):
    rng = np.random.default_rng(seed)
    x = rng.standard_normal((B, FIN)).astype(np.float32)
    a = (0.05 * rng.standard_normal((B, O // 2))).astype(np.float32)
    return x, a


def _rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30)


@pytest.mark.parametrize("B", [1, 200, 4096])
def test_forward_matches_oracle(B):
    from paper_2603_12185_gb300 import comfree as CF
    net = CF.Mlp(FIN, H, O, max_batch=4096, seed=3)
    x, _ = _data(B, 4)
    y = net.forward(torch.from_numpy(x).cuda()).cpu().numpy()
    net.status()
    p = net.params().cpu().numpy()
    yo, _ = M.forward(p, x.astype(np.float64), FIN, H, O, round_bf16=True)
    assert np.abs(y - yo).max() <= 1e-2 * np.abs(yo).max() + 1e-4
    assert _rel(y, yo) < 5e-3


@pytest.mark.parametrize("B", [384, 300, 16384])
def test_gradients_match_oracle(B):
    """384 rows fill three 128-row tiles; 300 leave 84 zero-padded rows in the last (their
    gradient rows must be zero and add nothing to the weight and bias sums); 16384 is the
    benchmark's batch."""
    from paper_2603_12185_gb300 import comfree as CF
    net = CF.Mlp(FIN, H, O, max_batch=max(B, 512), seed=5)
    x, a = _data(B, 6)
    g, loss = net.gradients(torch.from_numpy(x).cuda(), torch.from_numpy(a).cuda())
    g = g.cpu().numpy()
    net.status()
    p = net.params().cpu().numpy()
    Lo, go, _ = M.gradients(p, x.astype(np.float64), a.astype(np.float64), FIN, H, O, round_bf16=True)
    assert loss.item() == pytest.approx(Lo, rel=2e-3)
    o = 0
    for name, shape in [("W1", (H, 64)), ("b1", (H,)), ("W2", (H, H)), ("b2", (H,)), ("W3", (O, H)), ("b3", (O,))]:
        n = int(np.prod(shape))
        assert _rel(g[o:o + n], go[o:o + n]) < 2e-2, name
        o += n


def test_training_reduces_the_loss():
    from paper_2603_12185_gb300 import comfree as CF
    net = CF.Mlp(FIN, H, O, max_batch=1024, seed=7)
    rng = np.random.default_rng(8)
    x = rng.standard_normal((1024, FIN)).astype(np.float32)
    Wt = rng.standard_normal((FIN, O // 2)).astype(np.float32) * 0.02
    a = np.tanh(x @ Wt).astype(np.float32)         # a learnable target map
    xt, at = torch.from_numpy(x).cuda(), torch.from_numpy(a).cuda()
    first = net.train_step(xt, at, lr=1e-3).item()
    for _ in range(200):
        last = net.train_step(xt, at, lr=1e-3).item()
    net.status()
    assert last < first - 0.5
