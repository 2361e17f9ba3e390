"""MPPI on the batched step: the kernels' update against its closed form, the fused cost against
a host recomputation, and an end-to-end control run that lowers the task cost."""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2603_12185_gb300 import build
    build.build()


def test_mppi_update_matches_closed_form():
    from paper_2603_12185_gb300 import comfree as CF
    N, H, nu, lam = 777, 5, 3, 0.3
    rng = np.random.default_rng(0)
    cost = rng.uniform(1, 5, N).astype(np.float32)
    U = rng.standard_normal((N, H, nu)).astype(np.float32)
    mean = torch.zeros(H * nu, device="cuda")
    stats = torch.zeros(3, device="cuda")
    c, u = torch.from_numpy(cost).cuda(), torch.from_numpy(U).cuda()
    CF.check(CF.lib().cf_mppi_update(N, H, nu, CF._ptr(c), CF._ptr(u), lam, CF._ptr(mean), CF._ptr(stats), CF._stream()))
    w = np.exp(-(cost.astype(np.float64) - cost.min()) / lam)
    ref = (w[:, None, None] * U).sum(0) / w.sum()
    np.testing.assert_allclose(mean.cpu().numpy().reshape(H, nu), ref, rtol=1e-4, atol=1e-5)
    st = stats.cpu().numpy()
    assert st[0] == pytest.approx(cost.min()) and st[1] == pytest.approx(cost.mean(), rel=1e-5)
    assert st[2] == pytest.approx(w.sum() ** 2 / (w * w).sum(), rel=1e-4)
    # with one sample (or lambda -> 0) the update is the argmin sample
    CF.check(CF.lib().cf_mppi_update(N, H, nu, CF._ptr(c), CF._ptr(u), 1e-6, CF._ptr(mean), None, CF._stream()))
    np.testing.assert_allclose(mean.cpu().numpy().reshape(H, nu), U[np.argmin(cost)], atol=1e-6)


def test_sampling_clips_and_mixes_the_proposal():
    from paper_2603_12185_gb300 import comfree as CF
    N, H, nu = 64, 4, 16
    mean = torch.full((H * nu,), 0.01, device="cuda")
    eps = torch.randn(N * H * nu, device="cuda")
    pm = torch.full((H * nu,), -0.02, device="cuda")
    pls = torch.full((H * nu,), -20.0, device="cuda")   # a near-deterministic proposal
    ctrl = torch.empty(H * N * nu, device="cuda")
    smp = torch.empty(N * H * nu, device="cuda")
    CF.check(CF.lib().cf_mppi_sample(N, H, nu, CF._ptr(mean), CF._ptr(eps), 0.5, 0.1, CF._ptr(pm), CF._ptr(pls), 16,
                                     CF._ptr(ctrl), CF._ptr(smp), CF._stream()))
    s = smp.cpu().numpy().reshape(N, H, nu)
    c = ctrl.cpu().numpy().reshape(H, N, nu)
    assert np.abs(s).max() <= 0.1 + 1e-7
    np.testing.assert_allclose(s[:16], -0.02, atol=1e-6)
    e = eps.cpu().numpy().reshape(N, H, nu)
    np.testing.assert_allclose(s[16:], np.clip(0.01 + 0.5 * e[16:], -0.1, 0.1), atol=1e-6)
    np.testing.assert_array_equal(c.transpose(1, 0, 2), s)


def test_fused_cost_matches_host_recomputation():
    """One-step rollouts: the running cost of the initial state plus the terminal cost of the final
    state, recomputed on the host from the oracle's kinematics."""
    from oracle import oracle as O
    from paper_2603_12185_gb300 import comfree as CF
    from paper_2603_12185_gb300 import mppi as MP
    from paper_2603_12185_gb300 import scenes as S
    sb = S.make_hand(6, seed=4)
    _, b = CF.from_scenes(sb)
    W = sb.nworld
    goals = torch.from_numpy(np.tile(np.array([0.01, -0.02, 0.04, 0.7071, 0, 0, 0.7071], np.float32), (W, 1))).cuda()
    q0, v0 = CF.flatten_state(sb)
    qref = torch.from_numpy(q0 + 0.05).cuda()
    costs = torch.zeros(W, device="cuda")
    cd = MP.default_cost()
    b.set_cost(cd, goals, qref, costs)
    b.step(sb.dt, 1)
    qT, _ = b.get_state()
    gpu = costs.cpu().numpy()
    qT = qT.cpu().numpy().reshape(W, 23)
    t = sb.templates[0]
    g = goals[0].cpu().numpy().astype(np.float64)
    for w in range(W):
        q = np.asarray(q0[w * 23:(w + 1) * 23], np.float64)
        _, _, poses = O.dynamics(sb.world(w), (0, 0, -9.81), q, np.zeros(22))
        dq = g[3:] @ q[3:7]
        c = cd.w_quat * (1 - dq * dq) + cd.w_pos * np.abs(q[:3] - g[:3]).sum()
        tips = 0.0
        for f in range(4):
            b_ = 1 + 4 * f + 3
            R = poses[b_, 3:12].reshape(3, 3)
            L = 2 * t.geom_size[2 + 4 * f + 3][1]
            tip = poses[b_, :3] + R @ np.array([0, 0, L])
            tips += np.sum((q[:3] - tip) ** 2)
        c += cd.w_contact * tips + cd.w_joint * np.sum((q[7:] - (q[7:] + 0.05)) ** 2)
        if np.hypot(*(q[:2] - g[:2])) > cd.fall_radius:
            c += cd.w_fallen
        qt = qT[w]
        dqt = g[3:] @ qt[3:7]
        c += cd.term_pos * np.sum((qt[:3] - g[:3]) ** 2) + cd.term_quat * (1 - dqt * dqt)
        assert gpu[w] == pytest.approx(c, rel=2e-4, abs=1e-5)


def test_mppi_lowers_the_task_cost():
    from paper_2603_12185_gb300 import mppi as MP
    from paper_2603_12185_gb300 import scenes as S
    sb = S.make_hand(2, seed=5)
    t = sb.templates[0]
    params = S.Params(**dict(S.HAND_PARAMS, d_user=0.002))
    ctl = MP.HandMPPI(t, params, N=512, seed=1)
    rng = np.random.default_rng(2)
    goal = MP.random_goal(sb.q0[0], rng)
    start = MP.task_cost(sb.q0[0], goal)
    final = MP.run_episode(ctl, sb.q0[0], sb.v0[0], goal, 60)
    assert np.isfinite(final)
    assert final < start
