"""The hand-scene adjoint (cf_step_grad behind a torch.autograd.Function) against the oracle's
forward-mode reference gradient and FP64 central finite differences (h = 1e-6).

Loss of the cube (body 0) after T steps: |x_T - x*|^2 + (1 - (quat*^T quat_T)^2).  Each world is
checked along a seeded random direction in (initial joint velocities, per-step joint torques).
A world whose active set changes within +-h (oracle duals and oracle differences disagree) is
excluded and counted.
"""
import numpy as np
import pytest
import torch

import parity as PR
from oracle import oracle as O
from paper_2603_12185_gb300 import autograd as AG
from paper_2603_12185_gb300 import comfree as CF
from paper_2603_12185_gb300 import scenes as S

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2603_12185_gb300 import build
    build.build()
    O.build()


def _case(nworld, T, seed):
    sb = S.make_hand(nworld, seed=seed)
    rng = np.random.default_rng(seed + 100)
    tau = rng.normal(0, 0.05, (T, nworld, 16)).astype(np.float32)
    tp = np.array([0.0, 0.0, 0.05])
    tq = S.quat_about((0, 0, 1), 0.5)
    dirs_v = rng.standard_normal((nworld, 16))
    dirs_t = rng.standard_normal((T, nworld, 16))
    return sb, tau, tp, tq, dirs_v, dirs_t


def _gpu_grad(sb, tau, tp, tq, T, ckpt):
    _, b = CF.from_scenes(sb, max_ctrl_steps=T, grad_steps=T, grad_ckpt=ckpt)
    q0, v0 = CF.flatten_state(sb)
    q0 = torch.from_numpy(q0).cuda().requires_grad_(True)
    v0 = torch.from_numpy(v0).cuda().requires_grad_(True)
    tt = torch.from_numpy(tau.reshape(T, -1)).cuda().requires_grad_(True)
    qT, vT = AG.rollout(b, sb.dt, q0, v0, tt)
    W = sb.nworld
    qw = qT.view(W, 23)
    L = ((qw[:, :3] - torch.tensor(tp, device="cuda", dtype=torch.float32)) ** 2).sum(1) + \
        1 - (qw[:, 3:7] @ torch.tensor(tq, device="cuda", dtype=torch.float32)) ** 2
    L.sum().backward()
    return L.detach().cpu().numpy(), v0.grad.view(W, 22).cpu().numpy(), tt.grad.view(T, W, 16).cpu().numpy()


def _oracle(sb, w, tau_w, tp, tq, dv, dt_dir, h=1e-6):
    d = sb.world(w)
    T = tau_w.shape[0]
    tau_full = np.zeros((T, 22))
    tau_full[:, 6:] = tau_w
    dtau = np.zeros((T, 22))
    dtau[:, 6:] = dt_dir
    dv0 = np.zeros(22)
    dv0[6:] = dv
    q0 = PR.f32(sb.q0[w])
    v0 = PR.f32(sb.v0[w])
    L, dL = O.rollout_loss_dir(d, sb.params, sb.dt, q0, v0, tau_full, np.zeros(23), dv0, dtau, 0, tp, tq)
    Lp, _ = O.rollout_loss_dir(d, sb.params, sb.dt, q0, v0 + h * dv0, tau_full + h * dtau, np.zeros(23), dv0, dtau, 0,
                               tp, tq)
    Lm, _ = O.rollout_loss_dir(d, sb.params, sb.dt, q0, v0 - h * dv0, tau_full - h * dtau, np.zeros(23), dv0, dtau, 0,
                               tp, tq)
    return L, dL, (Lp - Lm) / (2 * h)


@pytest.mark.parametrize("T,ckpt,rtol", [(20, 5, 2e-3), (100, 10, 2e-2)])
def test_adjoint_matches_oracle_and_fd(T, ckpt, rtol):
    nworld = 16
    sb, tau, tp, tq, dirs_v, dirs_t = _case(nworld, T, seed=7)
    L, gv, gt = _gpu_grad(sb, tau, tp, tq, T, ckpt)
    checked, excluded = 0, 0
    for w in range(nworld):
        Lo, dLo, fd = _oracle(sb, w, tau[:, w].astype(np.float64), tp, tq, dirs_v[w], dirs_t[:, w])
        if abs(dLo - fd) > 1e-4 * max(abs(fd), 1e-6):
            excluded += 1        # the active set changes within +-h: not differentiable there
            continue
        g = float(gv[w, 6:] @ dirs_v[w] + np.sum(gt[:, w] * dirs_t[:, w]))
        assert L[w] == pytest.approx(Lo, rel=1e-3, abs=1e-6)
        assert g == pytest.approx(dLo, rel=rtol, abs=1e-6 * max(1.0, abs(dLo))), f"world {w}"
        checked += 1
    assert checked >= nworld // 2, f"only {checked} worlds checked ({excluded} excluded)"


def test_checkpoint_interval_does_not_change_the_gradient():
    T = 30
    sb, tau, tp, tq, _, _ = _case(4, T, seed=9)
    _, gv1, gt1 = _gpu_grad(sb, tau, tp, tq, T, 1)
    _, gv2, gt2 = _gpu_grad(sb, tau, tp, tq, T, 7)
    np.testing.assert_array_equal(gv1, gv2)
    np.testing.assert_array_equal(gt1, gt2)
