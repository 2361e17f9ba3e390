"""Cylinders and ellipsoids (ellipsoid-plane by the support point, cylinder-plane by three rim
points per cap, sphere-cylinder by the closest point of the solid) on the GPU against the FP64 oracle: piles where they
replace part of the spheres and capsules (plane and sphere-cylinder contacts), and an
articulated scene with a free cylinder, a free ellipsoid and a hinged sphere."""
import numpy as np
import pytest
import torch

import parity as PR
import test_gpu_parity as GP
import worlds as Wd
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


def _kinds(sb):
    t = np.concatenate([blk[:, 4] for blk in sb.world_param])
    return int((t == S.CYLINDER).sum()), int((t == S.ELLIPSOID).sum())


def test_round_pile_single_step_and_contacts():
    sb = S.make_pile(8, 24, seed=51, round_frac=0.6)
    nc, ne = _kinds(sb)
    assert nc > 20 and ne > 20
    sb = GP._advanced(sb, lambda w: 220 + 13 * w)
    GP._check_single_step(sb)
    assert GP._check_contact_sets(sb) > 16


def test_jammed_round_pile_single_step():
    sb = S.make_pile(3, 48, seed=52, jammed=True, round_frac=0.6)
    GP._check_single_step(sb)
    GP._check_contact_sets(sb)


def test_round_pile_50_step_horizon():
    sb = GP._advanced(S.make_pile(6, 16, seed=53, round_frac=0.6), lambda w: 250 + 9 * w)
    qg, vg, _ = PR.gpu_run(sb, 50)
    qo, vo = PR.oracle_run(sb, nsteps=50)
    errs = [PR.vel_err(vg[w], vo[w], sb.dt) for w in range(sb.nworld)]
    assert max(errs) <= GP.TOL50, f"worst {max(errs):.3e}"


def test_articulated_cylinder_ellipsoid_scene():
    cyl = S.cylinder_mass_inertia(0.03, 0.04, 1000.0)
    ell = S.ellipsoid_mass_inertia((0.04, 0.03, 0.02), 1000.0)
    d = Wd.world([dict(mass=cyl[0], inertia=cyl[1]), dict(mass=ell[0], inertia=ell[1]),
                  dict(parent=-1, jnt=S.HINGE, pos=(0.0, 0.0, 0.15), axis=(0, 1, 0), ipos=(0, 0, -0.06), mass=0.1,
                       inertia=(1e-4, 1e-4, 1e-4), damping=0.02)],
                 [dict(type=S.PLANE, body=-1), dict(type=S.CYLINDER, body=0, size=(0.03, 0.04, 0)),
                  dict(type=S.ELLIPSOID, body=1, size=(0.04, 0.03, 0.02)),
                  dict(type=S.SPHERE, body=2, pos=(0, 0, -0.06), size=(0.025, 0, 0))])
    t = S.Template(name="rounds", pile=False, **{k: np.asarray(v) for k, v in d.items()})
    rng = np.random.default_rng(54)
    q0, v0 = [], []
    for w in range(12):
        qc = np.concatenate([rng.uniform(-0.03, 0.03, 2), [0.06], S.random_quats(rng, 1)[0]])
        qe = np.concatenate([rng.uniform(0.06, 0.1, 1), rng.uniform(-0.03, 0.03, 1), [0.05], S.random_quats(rng, 1)[0]])
        q0.append(np.concatenate([qc, qe, [rng.uniform(-0.6, 0.6)]]))
        v0.append(np.concatenate([rng.normal(0, 0.2, 6), rng.normal(0, 0.2, 6), [rng.normal(0, 1.0)]]))
    sb = S.Batch([t], S.Params(**S.PILE_PARAMS), np.zeros(12, np.int32), [None] * 12, q0, v0, 0.002, 100,
                 {"workload": "rounds"})
    sb = GP._advanced(sb, lambda w: 30 + 10 * w)
    GP._check_single_step(sb)
    assert GP._check_contact_sets(sb) >= 12
