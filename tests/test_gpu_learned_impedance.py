"""The learned impedance (trace_mode 3; Sec. III-B's learning-based K(q), D(q)) on the GPU
against the FP64 oracle: single steps and short horizons with random networks (one shared set
and one set per world), the zero-output network against the heuristic kernel, the features and
regression targets the exact-mode step writes into its capture, the network's evaluation,
loss, gradient and Adam steps, and a fit that explains the exact impedance better than the best
constant and brings the step's impulses closer to the exact mode's."""
import dataclasses

import numpy as np
import pytest
import torch

import parity as PR
import test_gpu_parity as GP
from oracle import oracle as O
from paper_2603_12185_gb300 import comfree as CF
from paper_2603_12185_gb300 import impedance as IMP
from paper_2603_12185_gb300 import scenes as S

pytestmark = pytest.mark.gpu
NP = 49


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2603_12185_gb300 import build
    build.build()
    O.build()


def random_theta(seed, out_scale=0.3):
    """A network whose output spreads a few tenths around 0: impedances within ~e^+-1 of the
    heuristic, so the compared steps stay in the regime the parity tolerances were set for."""
    rng = np.random.default_rng(seed)
    th = np.zeros(NP)
    th[:32] = rng.normal(size=32)
    th[32:40] = rng.normal(scale=0.5, size=8)
    th[40:48] = rng.normal(scale=out_scale, size=8)
    th[48] = rng.normal(scale=0.2)
    return th.astype(np.float32)


def learned(sb):
    sb.params = dataclasses.replace(sb.params, trace_mode=3)
    return sb


def gpu_run(sb, thetas, nsteps=1, ctrl=None, capture=0):
    """thetas: one parameter vector for every world, or a list with one per world."""
    m, b = CF.from_scenes(sb, max_ctrl_steps=max(nsteps, 1), contact_capture=capture)
    per_world = isinstance(thetas, list)
    th = torch.from_numpy(np.stack(thetas) if per_world else np.asarray(thetas)[None]).float().cuda().contiguous()
    b.set_impedance_net(th, sb.nworld if per_world else 1)
    if ctrl is not None and b.total_nu:
        seq = np.concatenate([ctrl[w][:nsteps] for w in range(sb.nworld)], axis=1).astype(np.float32)
        b.set_ctrl(torch.from_numpy(seq.reshape(-1)).cuda())
    b.step(sb.dt, nsteps)
    q, v = b.get_state()
    torch.cuda.synchronize()
    q, v = q.cpu().numpy().astype(np.float64), v.cpu().numpy().astype(np.float64)
    out_q, out_v, qo, vo = [], [], 0, 0
    for w in range(sb.nworld):
        t = sb.template_of(w)
        out_q.append(q[qo:qo + t.nq])
        out_v.append(v[vo:vo + t.nv])
        qo += t.nq
        vo += t.nv
    return out_q, out_v, b


def oracle_run(sb, thetas, nsteps=1, ctrl=None):
    per_world = isinstance(thetas, list)
    qs, vs = [], []
    for w in range(sb.nworld):
        tau = None
        if ctrl is not None and sb.template_of(w).nu:
            tau = np.stack([PR.tau_full(sb, w, ctrl[w][s]) for s in range(nsteps)])
        th = np.asarray(thetas[w] if per_world else thetas, np.float64)
        q, v, _ = O.step(sb.world(w), sb.params, sb.dt, nsteps, sb.q0[w], sb.v0[w], tau, impnet=th)
        qs.append(q)
        vs.append(v)
    return qs, vs


def check(sb, thetas, nsteps, tol, ctrl=None, qatol=2e-6):
    qg, vg, _ = gpu_run(sb, thetas, nsteps, ctrl=ctrl)
    qo, vo = oracle_run(sb, thetas, nsteps, ctrl=ctrl)
    errs = [PR.vel_err(vg[w], vo[w], sb.dt) for w in range(sb.nworld)]
    assert max(errs) <= tol, f"worst world {int(np.argmax(errs))}: {max(errs):.3e}"
    for w in range(sb.nworld):
        np.testing.assert_allclose(qg[w], qo[w], rtol=0, atol=qatol)


def test_pile_single_step_shared_network():
    sb = learned(GP._advanced(S.make_pile(8, 16, seed=13), lambda w: 200 + 11 * w))
    check(sb, random_theta(1), 1, GP.TOL1)


def test_pile_per_world_networks_10_steps():
    sb = learned(GP._advanced(S.make_pile(6, 16, seed=14), lambda w: 220 + 7 * w))
    check(sb, [random_theta(10 + w) for w in range(6)], 10, GP.TOL50, qatol=2e-5)


def test_jammed_pile64_single_step():
    sb = learned(S.make_pile(4, 64, seed=7, jammed=True))
    check(sb, random_theta(2), 1, GP.TOL1)


def test_hand_single_step_and_10_steps():
    sb = S.make_hand(12, seed=3)
    ctrl = GP._hand_ctrl(sb, 300, seed=1)
    sb = learned(GP._advanced(sb, lambda w: 10 * w, ctrl=ctrl))
    c1 = GP._hand_ctrl(sb, 10, seed=2)
    check(sb, random_theta(3), 1, GP.TOL1, ctrl=c1)
    check(sb, [random_theta(30 + w) for w in range(12)], 10, GP.TOL50, ctrl=c1, qatol=2e-5)


def test_zero_output_network_matches_the_heuristic_kernel():
    """g = 0 reproduces mode 0, here through the two different kernel instantiations."""
    sb = GP._advanced(S.make_pile(4, 64, seed=15), lambda w: 300)
    th = random_theta(4)
    th[40:] = 0.0
    qg, vg, _ = PR.gpu_run(sb, 1)
    ql, vl, _ = gpu_run(learned(sb.subset(range(4))), th, 1)
    for w in range(4):
        assert PR.vel_err(vl[w], vg[w], sb.dt) <= 1e-5
        np.testing.assert_allclose(ql[w], qg[w], rtol=0, atol=1e-6)


@pytest.mark.parametrize("scene", ["pile", "hand"])
def test_exact_capture_features_and_targets(scene):
    """Every exact-mode contact record carries the features and ln(M_exact / M(phi)) of the
    oracle's same contact (M_exact the mean of the facets' exact impedances)."""
    if scene == "pile":
        sb = GP._advanced(S.make_pile(4, 64, seed=16), lambda w: 250 + 13 * w)
    else:
        sb = S.make_hand(8, seed=5)
        sb = GP._advanced(sb, lambda w: 12 * w, ctrl=GP._hand_ctrl(sb, 200, seed=3))
    se = IMP.with_mode(sb, 2)
    _, b = CF.from_scenes(se, contact_capture=4096)
    b.step(se.dt, 1)
    gpu = b.contacts()
    goff = PR.geom_offsets(se)
    n = 0
    for w in range(se.nworld):
        rec = O.step_record(se.world(w), se.params, se.dt, se.q0[w], se.v0[w])
        g0 = goff[int(se.world_scene[w])]
        og = {(c["geom_a"], c["geom_b"], c["sub"]): c for c in rec["contacts"]}
        for c in gpu[w]:
            k = (c["geom_a"] - g0, c["geom_b"] - g0, c["sub"])
            if k not in og:
                continue
            o = og[k]
            mh = o["r"] / (1 - o["r"]) / (o["trace_a"] + o["trace_b"])
            assert c["rho"] == pytest.approx(o["feat"][1], abs=2e-5)
            assert c["wn"] == pytest.approx(o["feat"][2], abs=2e-5)
            assert c["b_static"] == (o["feat"][3] == 1.0)
            assert c["target"] == pytest.approx(np.log(o["m_exact"] / mh), abs=2e-4)
            n += 1
    assert n > 20


def test_network_eval_loss_gradient_and_adam_match_the_oracle():
    rng = np.random.default_rng(7)
    th = rng.normal(scale=0.7, size=NP).astype(np.float32)
    x = rng.uniform(-1, 1, size=(5000, 4)).astype(np.float32)
    y = (rng.normal(size=5000) + 2.0).astype(np.float32)
    xt, yt = torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda()
    net = CF.ImpedanceNet(theta=th)
    np.testing.assert_allclose(net.eval(xt).cpu().numpy(), O.impnet_eval(th, x), rtol=1e-5, atol=2e-6)
    L, g = net.loss_grad(xt, yt)
    Lo, go = O.impnet_loss_grad(th, x, y)
    assert L.item() == pytest.approx(Lo, rel=1e-5)
    np.testing.assert_allclose(g.cpu().numpy(), go, rtol=1e-4, atol=1e-6 * np.abs(go).max())
    losses = net.fit(xt, yt, 20, lr=0.01).cpu().numpy()
    tho, lo = O.impnet_adam(th, x, y, 20, 0.01)
    np.testing.assert_allclose(losses, lo, rtol=1e-4)
    np.testing.assert_allclose(net.theta.cpu().numpy(), tho, rtol=0, atol=2e-4)
    # a continued fit carries Adam's step count and moments over
    more = net.fit(xt, yt, 10, lr=0.01).cpu().numpy()
    tho2, lo2 = O.impnet_adam(th, x, y, 30, 0.01)
    np.testing.assert_allclose(more, lo2[20:], rtol=1e-4)
    np.testing.assert_allclose(net.theta.cpu().numpy(), tho2, rtol=0, atol=3e-4)


def test_learned_step_without_network_is_refused():
    sb = learned(S.make_pile(2, 16, seed=1))
    _, b = CF.from_scenes(sb)
    with pytest.raises(CF.CfError, match="impedance network"):
        b.step(sb.dt, 1)
    with pytest.raises(CF.CfError):
        b.set_impedance_net(torch.zeros(3 * NP, device="cuda"), 3)


def test_fit_explains_the_exact_impedance_and_moves_impulses_toward_it():
    """Train on exact-mode contacts of settled and jammed piles, test on held-out worlds: the
    fitted network explains most of the target's spread that the best constant leaves, and a
    step with it lands closer to the exact step's contact impulses than the heuristic and the
    best constant rescaling do."""
    train = [IMP.advanced(S.make_pile(96, 64, seed=21), 300), S.make_pile(32, 64, seed=22, jammed=True)]
    test = [IMP.advanced(S.make_pile(16, 64, seed=23), 300), S.make_pile(8, 64, seed=24, jammed=True)]
    xs, ys = zip(*[IMP.exact_dataset(sb)[:2] for sb in train])
    x, y = torch.cat(xs), torch.cat(ys)
    net, losses = IMP.fit(x, y, iters=3000, lr=0.02)
    assert np.isfinite(losses).all() and losses[-1] < losses[0]
    const = IMP.constant_net(y)
    mean = float(y.mean())
    for sb in test:
        xt, yt, _ = IMP.exact_dataset(sb)
        r2, res, tot = IMP.r2(net, xt, yt, mean)
        print(f"held-out R^2 {r2:.3f} (residual {res:.4f}, constant {tot:.4f}, {len(yt)} contacts)")
        assert r2 > 0.9
        errs = IMP.impulse_errors(sb, {"learned": net, "constant": const})
        print("median relative impulse error vs exact:", errs)
        assert errs["learned"] < 0.5 * errs["constant"] and errs["learned"] < 0.5 * errs["heuristic"]


@pytest.mark.parametrize("mode", [2, 3])
def test_jammed_pile256_full_size_sampled(mode):
    """4096 worlds x 256 interpenetrating bodies, the bench's impedance-mode launch (one
    shared network for mode 3); one step compared with the oracle on sampled worlds.  The exact
    mode answers with velocities of tens of m/s, so positions get dt times the velocity
    tolerance on top of the usual 2e-6 m."""
    sb = S.make_pile(4096, 256, seed=5, jammed=True)
    sb.params = dataclasses.replace(sb.params, trace_mode=mode)
    th = random_theta(5)
    m, b = CF.from_scenes(sb)
    b.set_warps(0, 4)
    thd = torch.from_numpy(th[None]).cuda().contiguous()
    if mode == 3:
        b.set_impedance_net(thd, 1)
    b.step(sb.dt, 1)
    q, v = b.get_state()
    q, v = q.cpu().numpy().astype(np.float64), v.cpu().numpy().astype(np.float64)
    assert b.contact_counts().mean() > 300
    nq, nv = 7 * 256, 6 * 256
    for w in (0, 1234, 4095):
        sub = sb.subset([w])
        if mode == 3:
            qo, vo = oracle_run(sub, th, 1)
        else:
            qo, vo = PR.oracle_run(sub, nsteps=1)
        vg, qg = v[w * nv:(w + 1) * nv], q[w * nq:(w + 1) * nq]
        assert PR.vel_err(vg, vo[0], sb.dt) <= GP.TOL1
        np.testing.assert_allclose(qg, qo[0], rtol=0, atol=2e-6 + sb.dt * GP.TOL1 * np.abs(vo[0]).max())


def test_network_api_edges():
    """Empty evaluation, a misaligned input, a bad rate and a wrong number of sets are refused
    or handled without a launch; the library stays usable afterwards."""
    net = CF.ImpedanceNet(theta=random_theta(6))
    assert net.eval(torch.zeros(0, 4, device="cuda")).numel() == 0
    x = torch.zeros(33 * 4 + 1, device="cuda")
    with pytest.raises((CF.CfError, AssertionError)):
        net.eval(x[1:].view(33, 4))                       # 4-byte offset: not 16-byte aligned
    xt = torch.rand(100, 4, device="cuda")
    yt = torch.rand(100, device="cuda")
    with pytest.raises(CF.CfError):
        CF.check(CF.lib().cf_impnet_fit(CF._ptr(net.theta), CF._ptr(net.state), 0, CF._ptr(xt), CF._ptr(yt), 100, 1,
                                        0.0, None, None))
    sb = learned(S.make_pile(3, 16, seed=2))
    _, b = CF.from_scenes(sb)
    with pytest.raises(CF.CfError):
        b.set_impedance_net(torch.zeros(2 * NP, device="cuda"), 2)
    b.set_impedance_net(net.theta.view(1, -1), 1)
    b.step(sb.dt, 2)
    assert b.status()[0] == 0
    b.set_impedance_net(None)
    with pytest.raises(CF.CfError, match="impedance network"):
        b.step(sb.dt, 1)


def test_learned_steps_replay_from_a_cuda_graph():
    """A graph captured after the network is attached replays the learned step bit for bit,
    and picks up new parameter values written into the same buffer."""
    sb = learned(GP._advanced(S.make_pile(4, 16, seed=17), lambda w: 200))
    th = torch.from_numpy(random_theta(7)[None]).cuda().contiguous()
    _, ref = CF.from_scenes(sb)
    ref.set_impedance_net(th, 1)
    _, b = CF.from_scenes(sb)
    b.set_impedance_net(th, 1)
    g = b.graph(sb.dt, 1, repeat=3)          # one eager step, then three captured ones
    g.replay()
    for _ in range(4):
        ref.step(sb.dt, 1)
    torch.cuda.synchronize()
    q1, v1 = b.get_state()
    q2, v2 = ref.get_state()
    assert torch.equal(q1, q2) and torch.equal(v1, v2)
    th.mul_(0.5)                             # new values in the same buffer
    g.replay()
    for _ in range(3):
        ref.step(sb.dt, 1)
    torch.cuda.synchronize()
    assert torch.equal(b.get_state()[1], ref.get_state()[1])
