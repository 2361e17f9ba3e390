"""Joint limits and dry joint friction (Sec. III-A's system model; readings in the oracle) on the
GPU against the FP64 oracle: closed forms on a single hinge, and single steps, contact sets and
50-step horizons of hands whose hinges are limited and frictional."""
import numpy as np
import pytest
import torch

import parity as PR
import test_gpu_parity as GP
import worlds as Wd
from paper_2603_12185_gb300 import comfree as CF
from paper_2603_12185_gb300 import scenes as S

pytestmark = pytest.mark.gpu
DT = 0.002


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2603_12185_gb300 import build
    build.build()
    from oracle import oracle as O
    O.build()


def _hinge_batch(axis, ipos, rng=(0.0, 0.0), fl=0.0, q0=0.0):
    d = Wd.world([dict(parent=-1, jnt=S.HINGE, pos=(0, 0, 1.0), axis=axis, ipos=ipos, mass=1.0,
                       inertia=(1e-3, 1e-3, 2e-3), range=rng, frictionloss=fl)],
                 [dict(type=S.PLANE, body=-1)])
    t = S.Template(name="hinge", pile=False, **{k: np.asarray(v) for k, v in d.items()})
    m = CF.Model([t], S.Params())
    b = CF.Batch(m, np.zeros(1, np.int32))
    b.set_state(torch.tensor([q0], dtype=torch.float32, device="cuda"), torch.zeros(1, device="cuda"))
    return b


@pytest.mark.parametrize("q0,v_exp", [(-0.51, 0.019), (0.51, -0.019), (0.2, 0.0)])
def test_joint_limit_closed_form(q0, v_exp):
    b = _hinge_batch((0, 0, 1), (0, 0, 0), rng=(-0.5, 0.5), q0=q0)
    b.step(DT, 1)
    _, v = b.get_state()
    assert float(v[0]) == pytest.approx(v_exp, rel=1e-5, abs=1e-7)


def test_dry_friction_holds_and_slips():
    b = _hinge_batch((0, 1, 0), (0.1, 0, 0), fl=2.0)
    b.step(DT, 100)
    q, v = b.get_state()
    assert abs(float(v[0])) < 1e-6 and abs(float(q[0])) < 1e-6
    b = _hinge_batch((0, 1, 0), (0.1, 0, 0), fl=0.5)
    b.step(DT, 1)
    _, v = b.get_state()
    assert float(v[0]) == pytest.approx((0.981 - 0.5) * DT / 0.011, rel=1e-4)


def _limited_hand(nworld, seed):
    sb = S.make_hand(nworld, seed=seed)
    sb.templates[0] = S.with_joint_limits(sb.templates[0], abduction=(-0.03, 0.03), flexion=(0.0, 0.3),
                                          frictionloss=0.005)
    return sb


@pytest.fixture(scope="module")
def limited_hand_states():
    sb = _limited_hand(16, seed=8)
    ctrl = GP._hand_ctrl(sb, 300, seed=9)
    return GP._advanced(sb, lambda w: 15 * w, ctrl=ctrl)


def test_limited_hand_single_step(limited_hand_states):
    ctrl = GP._hand_ctrl(limited_hand_states, 1, seed=10)
    GP._check_single_step(limited_hand_states, ctrl=ctrl)


def test_limited_hand_contact_sets(limited_hand_states):
    assert GP._check_contact_sets(limited_hand_states) > 5


def test_limited_hand_50_step_horizon(limited_hand_states):
    sb = limited_hand_states
    ctrl = GP._hand_ctrl(sb, 50, seed=11)
    qg, vg, _ = PR.gpu_run(sb, 50, ctrl=ctrl)
    qo, vo = PR.oracle_run(sb, nsteps=50, ctrl=ctrl)
    errs = [PR.vel_err(vg[w], vo[w], sb.dt) for w in range(sb.nworld)]
    assert max(errs) <= GP.TOL50, f"worst {max(errs):.3e}"


def test_limits_hold_the_fingers_back():
    """The same random torques for 300 steps on the hand with and without limits: the limits
    (soft like the contacts, k = 0.1) cut the mean excursion beyond the range by more than half."""
    def excess(sb, qs):
        rng = sb.templates[0].body_range[1:]
        e = []
        for q in qs:
            ang = np.asarray(q)[7:]
            e.append(np.maximum(ang - rng[:, 1], 0) + np.maximum(rng[:, 0] - ang, 0))
        return float(np.mean(e))
    lim = _limited_hand(64, seed=12)
    free = S.make_hand(64, seed=12)
    ctrl = [np.random.default_rng(w).normal(0, 0.05, (300, 16)) for w in range(64)]
    ql, _, bl = PR.gpu_run(lim, 300, ctrl=ctrl)
    qf, _, _ = PR.gpu_run(free, 300, ctrl=ctrl)
    assert bl.status()[0] == 0
    e_lim, e_free = excess(lim, ql), excess(lim, qf)
    assert e_free > 0.01 and e_lim < 0.5 * e_free, (e_lim, e_free)


def test_adjoint_runs_on_joint_constraints():
    """The adjoint covers limited hinges and dry friction (gradients are checked against the
    oracle in test_gpu_adjoint.py); here: it runs on limited hands and returns finite values."""
    sb = _limited_hand(2, seed=1)
    _, b = CF.from_scenes(sb, max_ctrl_steps=4, grad_steps=4, grad_ckpt=2)
    gq = torch.ones(b.total_nq, device="cuda")
    gv = torch.zeros(b.total_nv, device="cuda")
    dq0, dv0, dtau = b.step_grad(4, sb.dt, gq, gv)
    assert torch.isfinite(dq0).all() and torch.isfinite(dv0).all() and torch.isfinite(dtau).all()
