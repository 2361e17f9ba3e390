"""Box-box contacts (corner rule) on the GPU against the FP64 oracle: piles with boxes among the
spheres and capsules (the pile path), two free boxes and a hinge in an articulated scene, and
stacked cubes resting over many steps."""
import numpy as np
import pytest
import torch

import parity as PR
import test_gpu_parity as GP
import worlds as Wd
from paper_2603_12185_gb300 import comfree as CF
from paper_2603_12185_gb300 import scenes as S

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2603_12185_gb300 import build
    build.build()
    from oracle import oracle as O
    O.build()


def _box_pairs(sb):
    n = 0
    for w in range(sb.nworld):
        t = sb.world_param[w][:, 4]
        n += int((t == S.BOX).sum())
    return n


def test_box_pile_single_step_and_contacts():
    sb = S.make_pile(8, 24, seed=31, box_frac=0.5)
    assert _box_pairs(sb) > 40
    sb = GP._advanced(sb, lambda w: 200 + 13 * w)
    GP._check_single_step(sb)
    assert GP._check_contact_sets(sb) > 16


def _capsules_to_spheres(sb):
    """Deep capsule-box overlaps put the capsule's deepest axis point on the box's medial plane,
    where two faces are equally deep by construction (the face, hence the normal, is then a tie
    that FP32 and FP64 may break differently); jammed starts use boxes and spheres only."""
    for blk in sb.world_param:
        caps = blk[:, 4] == S.CAPSULE
        for i in np.nonzero(caps)[0]:
            m, inertia = S.sphere_mass_inertia(blk[i, 5], 1000.0)
            blk[i, 0], blk[i, 1:4], blk[i, 4], blk[i, 6] = m, inertia, S.SPHERE, 0.0
    return sb


def test_jammed_box_pile_contact_sets():
    sb = _capsules_to_spheres(S.make_pile(3, 48, seed=32, jammed=True, box_frac=0.7))
    total = GP._check_contact_sets(sb)
    assert total > 50
    GP._check_single_step(sb)


def test_box_pile_50_step_horizon():
    sb = GP._advanced(S.make_pile(6, 16, seed=33, box_frac=0.5), lambda w: 250 + 9 * w)
    qg, vg, _ = PR.gpu_run(sb, 50)
    qo, vo = PR.oracle_run(sb, nsteps=50)
    errs = [PR.vel_err(vg[w], vo[w], sb.dt) for w in range(sb.nworld)]
    assert max(errs) <= GP.TOL50, f"worst {max(errs):.3e}"


def _artic_boxes():
    """Two free boxes and a hinged capsule arm over a plane: an articulated (non-pile) scene."""
    d = Wd.world([dict(mass=0.3, inertia=S.box_mass_inertia((0.04, 0.03, 0.02), 0.3)[1]),
                  dict(mass=0.2, inertia=S.box_mass_inertia((0.03, 0.03, 0.03), 0.2)[1]),
                  dict(parent=-1, jnt=S.HINGE, pos=(0.1, 0, 0.12), axis=(0, 1, 0), ipos=(0, 0, 0.04), mass=0.05,
                       inertia=(3e-5, 3e-5, 1e-5), damping=0.05)],
                 [dict(type=S.PLANE, body=-1),
                  dict(type=S.BOX, body=0, size=(0.04, 0.03, 0.02)),
                  dict(type=S.BOX, body=1, size=(0.03, 0.03, 0.03)),
                  dict(type=S.CAPSULE, body=2, pos=(0, 0, 0.04), size=(0.01, 0.04, 0))])
    return S.Template(name="boxes", pile=False, **{k: np.asarray(v) for k, v in d.items()})


def test_articulated_box_box_single_steps():
    t = _artic_boxes()
    rng = np.random.default_rng(34)
    nw = 16
    q0, v0 = [], []
    for w in range(nw):
        qa = np.array([0, 0, 0.0195, 1, 0, 0, 0], float)   # 0.5 mm into the floor
        qb = np.concatenate([rng.uniform(-0.02, 0.02, 2), [0.0695 - rng.uniform(0, 0.004)],
                             S.random_quats(rng, 1)[0] if w % 2 else [1, 0, 0, 0]])
        q0.append(np.concatenate([qa, qb, [rng.uniform(-0.5, 0.5)]]))
        v0.append(np.concatenate([np.zeros(6), rng.normal(0, 0.1, 6), [0.0]]))
    sb = S.Batch([t], S.Params(**S.PILE_PARAMS), np.zeros(nw, np.int32), [None] * nw, q0, v0, 0.002, 100,
                 {"workload": "boxes"})
    assert GP._check_contact_sets(sb) >= nw
    GP._check_single_step(sb)
    sb2 = GP._advanced(sb, lambda w: 40 + 5 * w)
    GP._check_single_step(sb2)


def test_stacked_cubes_hold():
    """Three 10 cm cubes stacked on the floor hold for 0.4 s on the GPU, and match the oracle's
    trajectory (k = 1, d = 0.01, 4 facets; the same case the oracle pins)."""
    d = Wd.world([dict(mass=1.0, inertia=S.box_mass_inertia((0.05,) * 3, 1.0)[1]) for _ in range(3)],
                 [dict(type=S.PLANE, body=-1)] + [dict(type=S.BOX, body=i, size=(0.05, 0.05, 0.05)) for i in range(3)])
    t = S.Template(name="stack", pile=False, **{k: np.asarray(v) for k, v in d.items()})
    p = S.Params(n_t=4, k_user=1.0, d_user=0.01)
    q = np.array([0, 0, 0.05, 1, 0, 0, 0, 0.005, 0, 0.151, 1, 0, 0, 0, -0.004, 0.003, 0.252, 1, 0, 0, 0], float)
    sb = S.Batch([t], p, np.zeros(1, np.int32), [None], [q], [np.zeros(18)], 0.002, 200, {"workload": "stack"})
    qg, vg, b = PR.gpu_run(sb, 200)
    assert b.status()[0] == 0
    qf = np.asarray(qg[0]).reshape(3, 7)
    assert np.abs(vg[0]).max() < 0.1
    for i in range(3):
        assert abs(qf[i, 2] - (0.05 + 0.1 * i)) < 0.012
        assert np.hypot(*(qf[i, :2] - q.reshape(3, 7)[i, :2])) < 0.005
    qo, vo = PR.oracle_run(sb, nsteps=200)
    np.testing.assert_allclose(qg[0], qo[0], atol=2e-4)
