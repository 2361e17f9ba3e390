"""The hand-scene adjoint (cf_step_grad behind a torch.autograd.Function) against the oracle's
forward-mode reference gradient and FP64 central finite differences (h = 1e-6).

Loss of the cube (body 0) after T steps: |x_T - x*|^2 + (1 - (quat*^T quat_T)^2).  Each world is
checked along a seeded random direction in (initial joint velocities, per-step joint torques).
A world whose active set changes within +-h (oracle duals and oracle differences disagree) is
excluded and counted.
"""
import dataclasses

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


def _case(nworld, T, seed, limited=False):
    sb = S.make_hand(nworld, seed=seed)
    if limited:
        # tight limits (abduction +-0.03 rad, flexion [0, 0.3] rad) and dry friction 0.005 N m on
        # every hinge: limits and friction are active from the first steps
        sb.templates[0] = S.with_joint_limits(sb.templates[0], abduction=(-0.03, 0.03), flexion=(0.0, 0.3),
                                              frictionloss=0.005)
    rng = np.random.default_rng(seed + 100)
    tau = rng.normal(0, 0.05, (T, nworld, 16)).astype(np.float32)
    tp = np.array([0.0, 0.0, 0.05])
    tq = S.quat_about((0, 0, 1), 0.5)
    dirs_v = rng.standard_normal((nworld, 16))
    dirs_t = rng.standard_normal((T, nworld, 16))
    return sb, tau, tp, tq, dirs_v, dirs_t


def _gpu_grad(sb, tau, tp, tq, T, ckpt, net=None):
    _, b = CF.from_scenes(sb, max_ctrl_steps=T, grad_steps=T, grad_ckpt=ckpt)
    if net is not None:
        b.set_impedance_net(torch.tensor(net, dtype=torch.float32, device="cuda").view(1, -1), 1)
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


def _oracle(sb, w, tau_w, tp, tq, dv, dt_dir, h=1e-6, net=None):
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
    L, dL = O.rollout_loss_dir(d, sb.params, sb.dt, q0, v0, tau_full, np.zeros(23), dv0, dtau, 0, tp, tq, impnet=net)
    Lp, _ = O.rollout_loss_dir(d, sb.params, sb.dt, q0, v0 + h * dv0, tau_full + h * dtau, np.zeros(23), dv0, dtau, 0,
                               tp, tq, impnet=net)
    Lm, _ = O.rollout_loss_dir(d, sb.params, sb.dt, q0, v0 - h * dv0, tau_full - h * dtau, np.zeros(23), dv0, dtau, 0,
                               tp, tq, impnet=net)
    return L, dL, (Lp - Lm) / (2 * h)


def _dual(sb, w, tau_w, tp, tq, coord, net=None):
    """The oracle's forward-mode derivative of the loss along one unit direction: ("v", k) the
    k-th hinge rate of v0, ("tau", s, k) the k-th torque at step s."""
    T = tau_w.shape[0]
    tau_full = np.zeros((T, 22))
    tau_full[:, 6:] = tau_w
    dv0, dtau = np.zeros(22), np.zeros((T, 22))
    if coord[0] == "v":
        dv0[6 + coord[1]] = 1.0
    else:
        dtau[coord[1], 6 + coord[2]] = 1.0
    return O.rollout_loss_dir(sb.world(w), sb.params, sb.dt, PR.f32(sb.q0[w]), PR.f32(sb.v0[w]), tau_full,
                              np.zeros(23), dv0, dtau, 0, tp, tq, impnet=net)[1]


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


def test_adjoint_element_by_element():
    """Every coordinate of dL/dv0 (the 16 hinge rates) and of dL/dtau at steps 0, 5 and 19 (16
    torques each) at T = 20, each against the oracle's forward-mode dual along that unit
    direction: 64 derivatives per world.  A coordinate passes within 1e-3 of its own size, with
    an absolute floor of 1e-3 of the world's largest derivative (coordinates of fingers that do
    not touch the cube are ~0 and carry only FP32 round-off).  A world is used only where the
    oracle's dual agrees with its FP64 central difference along a random direction (the active
    set does not change within +-h)."""
    T, nworld, steps = 20, 10, (0, 5, 19)
    sb, tau, tp, tq, dirs_v, dirs_t = _case(nworld, T, seed=13)
    _, gv, gt = _gpu_grad(sb, tau, tp, tq, T, 5)
    checked = uncoupled = 0
    for w in range(nworld):
        tw = tau[:, w].astype(np.float64)
        _, dLo, fd = _oracle(sb, w, tw, tp, tq, dirs_v[w], dirs_t[:, w])
        if abs(dLo - fd) > 1e-4 * max(abs(fd), 1e-6):
            continue
        ref, gpu = [], []
        for k in range(16):
            ref.append(_dual(sb, w, tw, tp, tq, ("v", k)))
            gpu.append(gv[w, 6 + k])
        for s_ in steps:
            for k in range(16):
                ref.append(_dual(sb, w, tw, tp, tq, ("tau", s_, k)))
                gpu.append(gt[s_, w, k])
        ref, gpu = np.array(ref), np.array(gpu)
        scale = np.abs(ref).max()
        if scale == 0.0:
            # no finger reaches the cube within T steps: the loss does not depend on the hand
            assert np.abs(gpu).max() == 0.0, f"world {w}: uncoupled, gpu {np.abs(gpu).max():.3e}"
            uncoupled += 1
            continue
        bad = np.abs(gpu - ref) > 1e-3 * (np.abs(ref) + 1e-3 * scale)
        assert not bad.any(), f"world {w}: coordinates {np.flatnonzero(bad)} gpu {gpu[bad]} oracle {ref[bad]}"
        checked += 1
    assert checked >= 4, f"only {checked} of {nworld} worlds checked ({uncoupled} uncoupled)"


def test_adjoint_with_joint_limits_and_dry_friction():
    """Hands whose hinges are limited and carry dry friction (the per-hinge constraint impulses
    of the step): every coordinate of dL/dv0 and of dL/dtau at steps 0 and 9 at T = 10 against
    the oracle's duals (1e-3 of the coordinate, floor 1e-3 of the world's largest), and the
    random-direction derivative against FP64 central differences (worlds whose active set
    changes within +-h excluded and counted)."""
    T, nworld = 10, 8
    sb, tau, tp, tq, dirs_v, dirs_t = _case(nworld, T, seed=17, limited=True)
    assert sb.templates[0].body_frictionloss.max() > 0
    _, gv, gt = _gpu_grad(sb, tau, tp, tq, T, 5)
    checked = 0
    for w in range(nworld):
        tw = tau[:, w].astype(np.float64)
        _, dLo, fd = _oracle(sb, w, tw, tp, tq, dirs_v[w], dirs_t[:, w])
        if abs(dLo - fd) > 1e-4 * max(abs(fd), 1e-6):
            continue
        g = float(gv[w, 6:] @ dirs_v[w] + np.sum(gt[:, w] * dirs_t[:, w]))
        assert g == pytest.approx(dLo, rel=2e-3, abs=1e-6 * max(1.0, abs(dLo))), f"world {w}"
        ref = [_dual(sb, w, tw, tp, tq, ("v", k)) for k in range(16)]
        gpu = list(gv[w, 6:])
        for s_ in (0, T - 1):
            ref += [_dual(sb, w, tw, tp, tq, ("tau", s_, k)) for k in range(16)]
            gpu += list(gt[s_, w])
        ref, gpu = np.array(ref), np.array(gpu)
        scale = np.abs(ref).max()
        bad = np.abs(gpu - ref) > 1e-3 * (np.abs(ref) + 1e-3 * scale)
        assert not bad.any(), f"world {w}: coordinates {np.flatnonzero(bad)} gpu {gpu[bad]} oracle {ref[bad]}"
        checked += 1
    assert checked >= nworld // 2, f"only {checked} of {nworld} worlds checked"


@pytest.mark.parametrize("mode", [2, 3])
def test_adjoint_in_the_exact_and_learned_impedance_modes(mode):
    """The impedance modes of Sec. III-B through the adjoint.
    - trace_mode 2: the exact diagonal impedance, M_j = 1 / ((k dt + d) J~_j M~^-1 J~_j^T) per
      facet from the contact's Gram blocks, and its one-row form at joint limits.
    - trace_mode 3: the learned one, M(phi) times exp(clamp(g(x))) of a seeded network (FP32
      values, as the GPU holds them).
    As with joint limits, every coordinate of dL/dv0 and of dL/dtau at steps 0 and 9 at
    T = 10 is checked against the oracle's duals, and the random-direction derivative against
    FP64 central differences."""
    T, nworld = 10, 8
    sb, tau, tp, tq, dirs_v, dirs_t = _case(nworld, T, seed=19, limited=True)
    sb.params = dataclasses.replace(sb.params, trace_mode=mode)
    net = None
    if mode == 3:
        net = np.random.default_rng(3).normal(0.0, 0.4, O.impnet_params()).astype(np.float32).astype(np.float64)
    _, gv, gt = _gpu_grad(sb, tau, tp, tq, T, 5, net=net)
    checked = 0
    for w in range(nworld):
        tw = tau[:, w].astype(np.float64)
        _, dLo, fd = _oracle(sb, w, tw, tp, tq, dirs_v[w], dirs_t[:, w], net=net)
        if abs(dLo - fd) > 1e-4 * max(abs(fd), 1e-6):
            continue
        g = float(gv[w, 6:] @ dirs_v[w] + np.sum(gt[:, w] * dirs_t[:, w]))
        assert g == pytest.approx(dLo, rel=2e-3, abs=1e-6 * max(1.0, abs(dLo))), f"world {w}"
        ref = [_dual(sb, w, tw, tp, tq, ("v", k), net=net) for k in range(16)]
        gpu = list(gv[w, 6:])
        for s_ in (0, T - 1):
            ref += [_dual(sb, w, tw, tp, tq, ("tau", s_, k), net=net) for k in range(16)]
            gpu += list(gt[s_, w])
        ref, gpu = np.array(ref), np.array(gpu)
        scale = np.abs(ref).max()
        bad = np.abs(gpu - ref) > 1e-3 * (np.abs(ref) + 1e-3 * scale)
        assert not bad.any(), f"world {w}: coordinates {np.flatnonzero(bad)} gpu {gpu[bad]} oracle {ref[bad]}"
        checked += 1
    assert checked >= nworld // 2, f"only {checked} of {nworld} worlds checked"


def test_checkpoint_interval_does_not_change_the_gradient():
    T = 30
    sb, tau, tp, tq, _, _ = _case(4, T, seed=9)
    _, gv1, gt1 = _gpu_grad(sb, tau, tp, tq, T, 1)
    _, gv2, gt2 = _gpu_grad(sb, tau, tp, tq, T, 7)
    np.testing.assert_array_equal(gv1, gv2)
    np.testing.assert_array_equal(gt1, gt2)


def _geo_scene(nworld, seed):
    """Two stacked free boxes (box-box contacts), a free cylinder (standing or lying), a free
    ellipsoid and a hinged sphere arm over the cylinder, on a plane; friction (0.8, 0.005, 0.005)
    so that every facet subspace acts.  Returns the batch; q per world: 4 free bodies x 7, then
    the hinge."""
    import worlds as Wd
    mu = (0.8, 0.005, 0.005)
    cyl = S.cylinder_mass_inertia(0.03, 0.04, 1000.0)
    ell = S.ellipsoid_mass_inertia((0.04, 0.03, 0.02), 1000.0)
    d = Wd.world([dict(mass=0.2, inertia=S.box_mass_inertia((0.03, 0.03, 0.02), 0.2)[1]),
                  dict(mass=0.3, inertia=S.box_mass_inertia((0.04, 0.04, 0.02), 0.3)[1]),
                  dict(mass=cyl[0], inertia=cyl[1]), dict(mass=ell[0], inertia=ell[1]),
                  dict(parent=-1, jnt=S.HINGE, pos=(0.15, 0.0, 0.1635), axis=(0, 1, 0), ipos=(0, 0, -0.06),
                       mass=0.1, inertia=(1e-4, 1e-4, 1e-4), damping=0.02)],
                 [dict(type=S.PLANE, body=-1, mu=mu),
                  dict(type=S.BOX, body=0, size=(0.03, 0.03, 0.02), mu=mu),
                  dict(type=S.BOX, body=1, size=(0.04, 0.04, 0.02), mu=mu),
                  dict(type=S.CYLINDER, body=2, size=(0.03, 0.04, 0), mu=mu),
                  dict(type=S.ELLIPSOID, body=3, size=(0.04, 0.03, 0.02), mu=mu),
                  dict(type=S.SPHERE, body=4, pos=(0, 0, -0.06), size=(0.025, 0, 0), mu=mu)])
    t = S.Template(name="geo", pile=False, **{k: np.asarray(v) for k, v in d.items()})
    rng = np.random.default_rng(seed)
    q0, v0 = [], []
    for w in range(nworld):
        qb = np.concatenate([[0.0, 0.0, 0.0195], S.quat_about((0, 0, 1), rng.uniform(-0.3, 0.3))])
        qa = np.concatenate([rng.uniform(-0.005, 0.005, 2), [0.0595 - rng.uniform(0, 0.001)],
                             S.quat_about((0, 0, 1), rng.uniform(-0.5, 0.5))])
        if w % 2:   # the cylinder lying on its side
            qc = np.concatenate([[0.15, 0.0, 0.0295], S.quat_about((1, 0, 0), np.pi / 2)])
        else:
            qc = np.concatenate([[0.15, 0.0, 0.0395], S.quat_about((0, 0, 1), rng.uniform(0, 1))])
        qe = np.concatenate([[-0.15, 0.0, 0.0195], S.quat_about((0, 0, 1), rng.uniform(0, 1))])
        q0.append(np.concatenate([qa, qb, qc, qe, [rng.uniform(-0.05, 0.05)]]))
        v0.append(np.concatenate([rng.normal(0, 0.05, 24), [rng.normal(0, 0.3)]]))
    return S.Batch([t], S.Params(**S.PILE_PARAMS), np.zeros(nworld, np.int32), [None] * nworld, q0, v0, 0.002, 100,
                   {"workload": "geo"})


def test_adjoint_through_box_box_cylinder_and_ellipsoid_contacts():
    """Box-box (clipped face vertices), cylinder-plane (rim points), ellipsoid-plane (support
    point) and sphere-cylinder contacts through the adjoint.  The pose loss of the top box, of
    the cylinder and of the ellipsoid after T = 10 steps: every coordinate of dL/dv0 (25) and
    dL/dtau of the hinge at steps 0 and 9 against the oracle's duals (1e-3 of the coordinate,
    floor 1e-3 of the largest), the random-direction derivative against FP64 central
    differences (worlds whose active set changes within +-h excluded and counted)."""
    T, nworld = 10, 8
    sb = _geo_scene(nworld, seed=23)
    nq, nv = 29, 25
    rng = np.random.default_rng(29)
    tau = rng.normal(0, 0.005, (T, nworld, 1)).astype(np.float32)
    tp = np.array([0.01, -0.01, 0.05])
    tq = S.quat_about((0, 0, 1), 0.3)
    checked = {}
    for body in (0, 2, 3):
        _, b = CF.from_scenes(sb, max_ctrl_steps=T, grad_steps=T, grad_ckpt=5)
        q0, v0 = CF.flatten_state(sb)
        q0 = torch.from_numpy(q0).cuda().requires_grad_(True)
        v0 = torch.from_numpy(v0).cuda().requires_grad_(True)
        tt = torch.from_numpy(tau.reshape(T, -1)).cuda().requires_grad_(True)
        qT, vT = AG.rollout(b, sb.dt, q0, v0, tt)
        qw = qT.view(nworld, nq)[:, 7 * body:7 * body + 7]
        L = ((qw[:, :3] - torch.tensor(tp, device="cuda", dtype=torch.float32)) ** 2).sum(1) + \
            1 - (qw[:, 3:7] @ torch.tensor(tq, device="cuda", dtype=torch.float32)) ** 2
        L.sum().backward()
        gv = v0.grad.view(nworld, nv).cpu().numpy()
        gt = tt.grad.view(T, nworld).cpu().numpy()
        checked[body] = 0
        for w in range(nworld):
            d = sb.world(w)
            qw0, vw0 = PR.f32(sb.q0[w]), PR.f32(sb.v0[w])
            tau_full = np.zeros((T, nv))
            tau_full[:, nv - 1] = tau[:, w, 0]

            def dual(dv, dtau):
                return O.rollout_loss_dir(d, sb.params, sb.dt, qw0, vw0, tau_full, np.zeros(nq), dv, dtau, body, tp,
                                          tq)

            dv_r = rng.standard_normal(nv)
            dt_r = np.zeros((T, nv))
            dt_r[:, nv - 1] = rng.standard_normal(T)
            _, dLo = dual(dv_r, dt_r)
            h = 1e-6
            Lp = O.rollout_loss_dir(d, sb.params, sb.dt, qw0, vw0 + h * dv_r, tau_full + h * dt_r, np.zeros(nq),
                                    dv_r, dt_r, body, tp, tq)[0]
            Lm = O.rollout_loss_dir(d, sb.params, sb.dt, qw0, vw0 - h * dv_r, tau_full - h * dt_r, np.zeros(nq),
                                    dv_r, dt_r, body, tp, tq)[0]
            fd = (Lp - Lm) / (2 * h)
            if abs(dLo - fd) > 1e-4 * max(abs(fd), 1e-6):
                continue
            g = float(gv[w] @ dv_r + gt[:, w] @ dt_r[:, nv - 1])
            assert g == pytest.approx(dLo, rel=2e-3, abs=1e-6 * max(1.0, abs(dLo))), f"body {body} world {w}"
            ref, gpu = [], []
            for k in range(nv):
                e = np.zeros(nv)
                e[k] = 1.0
                ref.append(dual(e, np.zeros((T, nv)))[1])
                gpu.append(gv[w, k])
            for s_ in (0, T - 1):
                e = np.zeros((T, nv))
                e[s_, nv - 1] = 1.0
                ref.append(dual(np.zeros(nv), e)[1])
                gpu.append(gt[s_, w])
            ref, gpu = np.array(ref), np.array(gpu)
            scale = np.abs(ref).max()
            bad = np.abs(gpu - ref) > 1e-3 * (np.abs(ref) + 1e-3 * scale)
            assert not bad.any(), f"body {body} world {w}: {np.flatnonzero(bad)} gpu {gpu[bad]} oracle {ref[bad]}"
            checked[body] += 1
    assert all(c >= nworld // 2 for c in checked.values()), checked
