"""MPPI on the batched step: the kernels' update against its closed form, the fused cost against
the oracle's MPC cost, and an end-to-end control run that lowers the task cost."""
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


def test_fused_cost_matches_the_oracle():
    """One-step rollouts: the running cost of the initial state plus the terminal cost of the final
    state (Sec. V, Eq. mpc), against the oracle's cost of the same states."""
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
    g = goals[0].cpu().numpy().astype(np.float64)
    qr = qref.cpu().numpy().astype(np.float64).reshape(W, 23)
    for w in range(W):
        q = np.asarray(q0[w * 23:(w + 1) * 23], np.float64)
        run, _ = O.mpc_cost(sb.world(w), q, g, qr[w], cd, cost_body=cd.body)
        _, term = O.mpc_cost(sb.world(w), qT[w].astype(np.float64), g, qr[w], cd, cost_body=cd.body)
        assert gpu[w] == pytest.approx(run + term, rel=2e-4, abs=1e-5)


def test_fused_cost_over_a_horizon_matches_the_oracle():
    """An 8-step controlled rollout: J = sum_t c(x_t) + V(x_8) on the GPU against the oracle's
    cost along the oracle's own trajectory (the states agree to the 1e-3 horizon tolerance, so
    the cost is compared at 1e-3)."""
    from oracle import oracle as O
    from paper_2603_12185_gb300 import comfree as CF
    from paper_2603_12185_gb300 import mppi as MP
    from paper_2603_12185_gb300 import scenes as S
    import parity as PT
    H = 8
    sb = S.make_hand(4, seed=9)
    rng = np.random.default_rng(3)
    nu = sb.templates[0].nu
    ctrl = [rng.normal(0.0, 0.05, (H, nu)).astype(np.float32) for _ in range(sb.nworld)]
    _, b = CF.from_scenes(sb, max_ctrl_steps=H)
    seq = np.concatenate([c for c in ctrl], axis=1)
    b.set_ctrl(torch.from_numpy(np.ascontiguousarray(seq)).cuda().reshape(-1))
    W = sb.nworld
    goal = np.array([0.0, 0.01, 0.04, 0.9238795, 0.0, 0.0, 0.3826834])
    goals = torch.from_numpy(np.tile(goal.astype(np.float32), (W, 1))).cuda()
    q0, _ = CF.flatten_state(sb)
    qref = torch.from_numpy(q0.copy()).cuda()
    costs = torch.zeros(W, device="cuda")
    cd = MP.default_cost()
    b.set_cost(cd, goals, qref, costs)
    b.step(sb.dt, H)
    gpu = costs.cpu().numpy()
    g = goals[0].cpu().numpy().astype(np.float64)
    for w in range(W):
        d = sb.world(w)
        q, v = PT.f32(sb.q0[w]), PT.f32(sb.v0[w])
        qr = PT.f32(q0[w * 23:(w + 1) * 23])
        J = 0.0
        for t in range(H):
            J += O.mpc_cost(d, q, g, qr, cd, cost_body=cd.body)[0]
            tau = PT.tau_full(sb, w, ctrl[w][t])[None]
            q, v, _ = O.step(d, sb.params, sb.dt, 1, q, v, tau)
        J += O.mpc_cost(d, q, g, qr, cd, cost_body=cd.body)[1]
        assert gpu[w] == pytest.approx(J, rel=1e-3)


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


def test_tick_graph_replays_the_eager_ticks():
    """A CUDA graph of one tick, replayed, gives the same plans and plant states as eager ticks
    from the same start and seed, bit for bit (the noise generator advances with each replay)."""
    from paper_2603_12185_gb300 import mppi as MP
    from paper_2603_12185_gb300 import scenes as S
    sb = S.make_hand(1, seed=8)
    t = sb.templates[0]
    params = S.Params(**dict(S.HAND_PARAMS, d_user=0.002))
    goal = MP.random_goal(sb.q0[0], np.random.default_rng(4))
    runs = []
    for graphed in (False, True):
        ctl = MP.HandMPPI(t, params, N=256, seed=3)
        ctl.reset(sb.q0[0], sb.v0[0], goal)
        plans, states = [], []
        if graphed:
            g = ctl.tick_graph()              # the first tick runs eagerly inside
            plans.append(ctl.mean.clone())
            states.append(torch.cat(ctl.plant.get_state()))
            for _ in range(4):
                g.replay()
                plans.append(ctl.mean.clone())
                states.append(torch.cat(ctl.plant.get_state()))
        else:
            for _ in range(5):
                ctl.tick()
                plans.append(ctl.mean.clone())
                states.append(torch.cat(ctl.plant.get_state()))
        torch.cuda.synchronize()
        runs.append((torch.stack(plans).cpu().numpy(), torch.stack(states).cpu().numpy()))
    (pe, se), (pg, sg) = runs
    assert np.array_equal(pe.view(np.uint32), pg.view(np.uint32))
    assert np.array_equal(se.view(np.uint32), sg.view(np.uint32))
    assert np.abs(se[-1] - se[0]).max() > 0   # the plant moved
