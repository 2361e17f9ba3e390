"""The exact diagonal impedance of Sec. III-B (trace_mode 2) on the GPU against the FP64 oracle:
single steps from oracle states (<= 1e-4 relative velocity error), contact sets and facet
impulse sums, for spheres on a plane, piles (free bodies, 18-facet cone) and hands (hinge
chains through the trees' M~^-1, a free cube)."""
import dataclasses

import numpy as np
import pytest

import parity as PR
import test_gpu_parity as GP
from paper_2603_12185_gb300 import scenes as S

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2603_12185_gb300 import build
    build.build()
    from oracle import oracle as O
    O.build()


def exact(sb):
    sb.params = dataclasses.replace(sb.params, trace_mode=2)
    return sb


def heuristic_then_exact(sb, steps_of, ctrl=None):
    """States advanced by the oracle with the (stable) heuristic impedance, then switched to the
    exact mode for the compared step: the per-facet diagonal overshoots where many facets and
    contacts share a normal, and dense piles diverge under it within a few hundred steps."""
    sb = GP._advanced(sb, steps_of, ctrl=ctrl)
    return exact(sb)


def test_spheres_exact_single_step_and_contacts():
    sb = exact(S.make_spheres_on_plane(32, 8, seed=1))
    GP._check_single_step(GP._advanced(sb, lambda w: 150 + 5 * w))
    # every sphere 2 mm into the plane, sliding (the facets of each contact differ)
    rng = np.random.default_rng(2)
    for w in range(sb.nworld):
        q = sb.q0[w].reshape(-1, 7).copy()
        v = sb.v0[w].reshape(-1, 6).copy()
        q[:, 2] = 0.048
        v[:, :2] = rng.normal(0, 0.2, (len(v), 2))
        v[:, 3:] = rng.normal(0, 2.0, (len(v), 3))
        sb.q0[w], sb.v0[w] = q.reshape(-1), v.reshape(-1)
    GP._check_single_step(sb)
    assert GP._check_contact_sets(sb) >= 32 * 8   # every sphere-plane contact (and some sphere pairs)


def test_pile_exact_single_step_and_contacts():
    sb = heuristic_then_exact(S.make_pile(8, 16, seed=13), lambda w: 200 + 11 * w)
    GP._check_single_step(sb)
    assert GP._check_contact_sets(sb) > 8


def test_jammed_pile_exact_single_step():
    """Interpenetrating starts: the exact mode answers with velocities of tens of m/s, so the
    position check allows dt times the velocity tolerance on top of the usual 2e-6 m."""
    sb = exact(S.make_pile(4, 64, seed=7, jammed=True))
    qg, vg, _ = PR.gpu_run(sb, 1)
    qo, vo = PR.oracle_run(sb, nsteps=1)
    for w in range(sb.nworld):
        assert PR.vel_err(vg[w], vo[w], sb.dt) <= GP.TOL1
        atol = 2e-6 + sb.dt * GP.TOL1 * np.abs(vo[w]).max()
        np.testing.assert_allclose(qg[w], qo[w], rtol=0, atol=atol)


def test_hand_exact_single_step_and_contacts():
    sb = S.make_hand(16, seed=4)
    ctrl = GP._hand_ctrl(sb, 300, seed=5)
    sb = heuristic_then_exact(sb, lambda w: 12 * w, ctrl=ctrl)
    ctrl1 = GP._hand_ctrl(sb, 1, seed=6)
    GP._check_single_step(sb, ctrl=ctrl1)
    assert GP._check_contact_sets(sb) > 5   # the oracle record step runs without controls


def test_exact_mode_adjoint_runs_and_pile_adjoint_is_refused():
    """cf_step_grad covers the exact impedance (its gradients are checked against the oracle's
    duals in test_gpu_adjoint.py) and still refuses pile scenes."""
    import torch
    from paper_2603_12185_gb300 import comfree as CF
    sb = exact(S.make_hand(2, seed=4))
    _, b = CF.from_scenes(sb, max_ctrl_steps=4, grad_steps=4, grad_ckpt=2)
    gq = torch.zeros(b.total_nq, device="cuda")
    gv = torch.zeros(b.total_nv, device="cuda")
    out = b.step_grad(4, sb.dt, gq, gv)
    torch.cuda.synchronize()
    assert all(torch.isfinite(t).all() for t in out if t is not None)
    sp = exact(S.make_pile(2, 16))
    _, bp = CF.from_scenes(sp, max_ctrl_steps=4, grad_steps=4, grad_ckpt=2)
    with pytest.raises(CF.CfError, match="pile"):
        bp.step_grad(4, sp.dt, torch.zeros(bp.total_nq, device="cuda"), torch.zeros(bp.total_nv, device="cuda"))
