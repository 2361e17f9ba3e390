"""GPU (FP32, through the C ABI) against the FP64 oracle, element by element on seeded inputs.

Tolerances: single steps from oracle states <= 1e-4 relative velocity error, 50-step horizons
<= 1e-3 (error measure in tests/parity.py); contact sets identical except pairs whose gap is
within 1e-6 m of the margin.
"""
import numpy as np
import pytest

import parity as PR
from paper_2603_12185_gb300 import scenes as S

pytestmark = pytest.mark.gpu

TOL1, TOL50 = 1e-4, 1e-3


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2603_12185_gb300 import build
    build.build()
    from oracle import oracle as O
    O.build()


def _advanced(sb, steps_of, ctrl=None):
    """Oracle-advance world w by steps_of(w) steps; returns a batch holding the (FP32-rounded)
    oracle states."""
    qs, vs = [], []
    for w in range(sb.nworld):
        n = steps_of(w)
        if n:
            sub = sb.subset([w])
            cc = None if ctrl is None or ctrl[w] is None else [ctrl[w][:n]]
            q, v = PR.oracle_run(sub, nsteps=n, ctrl=cc)
            qs.append(q[0])
            vs.append(v[0])
        else:
            qs.append(sb.q0[w])
            vs.append(sb.v0[w])
    return PR.with_states(sb, qs, vs)


def _check_single_step(sb, ctrl=None, tol=TOL1):
    qg, vg, _ = PR.gpu_run(sb, 1, ctrl=ctrl)
    qo, vo = PR.oracle_run(sb, nsteps=1, ctrl=ctrl)
    errs = [PR.vel_err(vg[w], vo[w], sb.dt) for w in range(sb.nworld)]
    assert max(errs) <= tol, f"worst world {int(np.argmax(errs))}: {max(errs):.3e}"
    for w in range(sb.nworld):
        np.testing.assert_allclose(qg[w], qo[w], rtol=0, atol=2e-6)
    return errs


def _check_contact_sets(sb, ctrl=None, cap=4096):
    _, _, b = PR.gpu_run(sb, 1, ctrl=ctrl, capture=cap)
    gpu = b.contacts()
    goff = PR.geom_offsets(sb)
    from oracle import oracle as O
    margin = sb.params.margin
    total = 0
    for w in range(sb.nworld):
        rec = O.step_record(sb.world(w), sb.params, sb.dt, sb.q0[w], sb.v0[w])
        g0 = goff[int(sb.world_scene[w])]
        og = {(c["geom_a"], c["geom_b"], c["sub"]): c for c in rec["contacts"]}
        gg = {(c["geom_a"] - g0, c["geom_b"] - g0, c["sub"]): c for c in gpu[w]}
        for k in set(og) ^ set(gg):
            c = og.get(k) or gg.get(k)
            assert abs(c["phi"] - margin) < 1e-6, f"world {w}: contact {k} only on one side (phi={c['phi']})"
        for k in set(og) & set(gg):
            assert gg[k]["phi"] == pytest.approx(og[k]["phi"], abs=2e-6)
            np.testing.assert_allclose(gg[k]["normal"], og[k]["normal"], atol=2e-4)
            np.testing.assert_allclose(gg[k]["pos"], og[k]["pos"], atol=2e-6)
            # impulses carry k M(phi) times the FP32 rounding of phi (~1e-8 m): absolute floor 1e-7 N s
            assert gg[k]["lam_sum"] == pytest.approx(og[k]["lam_sum"], rel=2e-3, abs=1e-7)
            total += 1
    return total


# ------------------------------------------------------------------------------------------
# spheres on a plane (64 worlds x 8 spheres, 4-facet cone)
# ------------------------------------------------------------------------------------------
@pytest.fixture(scope="module")
def spheres_states():
    sb = S.make_spheres_on_plane(64, 8, seed=0)
    return _advanced(sb, lambda w: 150 + 6 * w)


def test_spheres_single_step(spheres_states):
    errs = _check_single_step(spheres_states)
    assert np.mean(errs) < TOL1


def test_spheres_contact_sets(spheres_states):
    assert _check_contact_sets(spheres_states) > 50


def test_spheres_50_step_horizon(spheres_states):
    sb = spheres_states
    qg, vg, _ = PR.gpu_run(sb, 50)
    qo, vo = PR.oracle_run(sb, nsteps=50)
    errs = [PR.vel_err(vg[w], vo[w], sb.dt) for w in range(sb.nworld)]
    assert max(errs) <= TOL50, f"worst {max(errs):.3e}"


# ------------------------------------------------------------------------------------------
# walled piles of spheres and capsules (18-facet 6D cone)
# ------------------------------------------------------------------------------------------
@pytest.mark.parametrize("n,worlds,settle", [(16, 16, 300), (64, 6, 250)])
def test_pile_single_step_and_contacts(n, worlds, settle):
    sb = S.make_pile(worlds, n, seed=11)
    sb = _advanced(sb, lambda w: settle + 7 * w)
    _check_single_step(sb)
    assert _check_contact_sets(sb) > worlds


def test_pile_50_step_horizon():
    sb = _advanced(S.make_pile(8, 16, seed=12), lambda w: 250 + 9 * w)
    qg, vg, _ = PR.gpu_run(sb, 50)
    qo, vo = PR.oracle_run(sb, nsteps=50)
    errs = [PR.vel_err(vg[w], vo[w], sb.dt) for w in range(sb.nworld)]
    assert max(errs) <= TOL50, f"worst {max(errs):.3e}"


def test_jammed_pile256_full_size_sampled():
    """4096 worlds x 256 interpenetrating bodies, the bench's launch shape; one step compared on
    sampled worlds (each with ~1000 contacts)."""
    sb = S.make_pile(4096, 256, seed=5, jammed=True)
    qg, vg, b = PR.gpu_run(sb, 1)
    counts = b.contact_counts()
    assert counts.mean() > 300
    for w in (0, 1234, 4095):
        qo, vo = PR.oracle_run(sb, worlds=[w], nsteps=1)
        assert PR.vel_err(vg[w], vo[0], sb.dt) <= TOL1
        np.testing.assert_allclose(qg[w], qo[0], rtol=0, atol=2e-6)


def test_jammed_pile_contact_sets():
    sb = S.make_pile(3, 64, seed=6, jammed=True)
    assert _check_contact_sets(sb) > 100


# ------------------------------------------------------------------------------------------
# the hand with a free cube (hinge trees, capsule/box/plane contacts, torques)
# ------------------------------------------------------------------------------------------
def _hand_ctrl(sb, T, seed=0):
    rng = np.random.default_rng(seed)
    return [rng.normal(0, 0.05, (T, 16)) for _ in range(sb.nworld)]


@pytest.fixture(scope="module")
def hand_states():
    sb = S.make_hand(24, seed=3)
    ctrl = _hand_ctrl(sb, 400, seed=1)
    return _advanced(sb, lambda w: 10 * w, ctrl=ctrl)


def test_hand_single_step(hand_states):
    ctrl = _hand_ctrl(hand_states, 1, seed=2)
    _check_single_step(hand_states, ctrl=ctrl)


def test_hand_contact_sets(hand_states):
    assert _check_contact_sets(hand_states) > 10


def test_hand_50_step_horizon(hand_states):
    sb = hand_states
    ctrl = _hand_ctrl(sb, 50, seed=3)
    qg, vg, _ = PR.gpu_run(sb, 50, ctrl=ctrl)
    qo, vo = PR.oracle_run(sb, nsteps=50, ctrl=ctrl)
    errs = [PR.vel_err(vg[w], vo[w], sb.dt) for w in range(sb.nworld)]
    assert max(errs) <= TOL50, f"worst {max(errs):.3e}"


# ------------------------------------------------------------------------------------------
# uneven worlds in one persistent launch
# ------------------------------------------------------------------------------------------
def test_mixed_batch_single_step():
    sb = S.make_mixed(12, seed=2)
    ctrl = [np.random.default_rng(w).normal(0, 0.05, (400, 16)) if sb.world_scene[w] == 3 else None
            for w in range(sb.nworld)]
    sb = _advanced(sb, lambda w: 0 if sb.world_scene[w] == 2 else 200 + 5 * w, ctrl=ctrl)
    ctrl1 = [c[:1] if c is not None else None for c in ctrl]
    _check_single_step(sb, ctrl=ctrl1)
