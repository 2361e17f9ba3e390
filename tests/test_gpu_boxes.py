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


def _face_normal(q, body, n):
    """True when n is, to 2e-4, plus or minus a face normal (a column of R) of the box `body`."""
    w, x, y, z = q[7 * body + 3:7 * body + 7] / np.linalg.norm(q[7 * body + 3:7 * body + 7])
    R = np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)],
                  [2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)],
                  [2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)]])
    return np.abs(np.abs(R.T @ np.asarray(n)).max() - 1.0) < 2e-4


def test_jammed_box_pile_with_capsules():
    """Jammed piles of boxes, capsules and spheres.  A capsule whose axis runs deep inside a box
    meets the box's signed distance at its minimum along the axis, where two face distances are
    equal (the minimiser sits on a kink of the piecewise-linear distance): the contact's face,
    hence its normal and point, is then a tie that FP32 and FP64 may break differently, with
    the same gap.  Contact sets are compared key by key; a key whose normals differ passes only
    as such a tie: both normals are faces of the box and the gaps agree within 1e-6 m (plus the
    2e-6 m FP32 rounding of the gap).  Because contacts decouple (each contact's impulse depends
    on its own bodies only), a tie changes the velocities of its two bodies alone: the single
    step is compared on every other body."""
    from oracle import oracle as O
    sb = S.make_pile(3, 48, seed=32, jammed=True, box_frac=0.7)
    qg, vg, b = PR.gpu_run(sb, 1, capture=4096)
    gpu = b.contacts()
    margin = sb.params.margin
    ties, total, compared = 0, 0, 0
    for w in range(sb.nworld):
        types = sb.world_param[w][:, 4]
        q = PR.f32(sb.q0[w])
        rec = O.step_record(sb.world(w), sb.params, sb.dt, q, PR.f32(sb.v0[w]))
        og = {(c["geom_a"], c["geom_b"], c["sub"]): c for c in rec["contacts"]}
        gg = {(c["geom_a"], c["geom_b"], c["sub"]): c for c in gpu[w]}
        for k in set(og) ^ set(gg):
            c = og.get(k) or gg.get(k)
            assert abs(c["phi"] - margin) < 1e-6, f"world {w}: contact {k} only on one side (phi={c['phi']})"
        tied = set()
        for k in set(og) & set(gg):
            o, g = og[k], gg[k]
            assert g["phi"] == pytest.approx(o["phi"], abs=3e-6)
            total += 1
            if np.abs(np.asarray(g["normal"]) - o["normal"]).max() > 2e-4:
                a, bb = k[0], k[1]
                box = a if types[a] == S.BOX else bb
                other = bb if box == a else a
                assert bb < len(types) and types[box] == S.BOX and types[other] == S.CAPSULE, \
                    f"world {w}: normals differ on {k}, not a capsule-box pair"
                assert _face_normal(q, box, g["normal"]) and _face_normal(q, box, o["normal"]), \
                    f"world {w}: {k} normals are not box faces"
                tied |= {a, bb}
                ties += 1
                continue
            np.testing.assert_allclose(g["pos"], o["pos"], atol=2e-6)
            assert g["lam_sum"] == pytest.approx(o["lam_sum"], rel=2e-3, abs=1e-7)
        keep = np.array([i for i in range(len(types)) if i not in tied], int)
        idx = (6 * keep[:, None] + np.arange(6)).ravel()
        vo = rec["v"]
        err = np.abs(vg[w][idx] - vo[idx]).max() / (np.abs(vo).max() + 9.81 * sb.dt)
        assert err <= GP.TOL1, f"world {w}: {err:.3e} on the untied bodies"
        compared += len(keep)
    assert total > 50 and compared > 100
    print(f"{total} common contacts, {ties} capsule-box ties")


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
    """Three 10 cm cubes stacked on the floor hold for 0.4 s on the GPU (k = 1, d = 0.01, 4 facets;
    the same case the oracle pins), and match the oracle over a 50-step horizon at the horizon
    tolerance: velocities within 1e-3 of the world's scale max|v| + g dt, and positions within
    the bound that tolerance implies for their integral, 50 dt 1e-3 (max|v| + g dt)."""
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
    q50, v50, _ = PR.gpu_run(sb, 50)
    qo, vo = PR.oracle_run(sb, nsteps=50)
    assert PR.vel_err(v50[0], vo[0], sb.dt) <= GP.TOL50
    vmax = max(np.abs(PR.oracle_run(sb, nsteps=n)[1][0]).max() for n in (10, 20, 30, 40, 50))
    bound = 50 * sb.dt * GP.TOL50 * (vmax + 9.81 * sb.dt)
    np.testing.assert_allclose(q50[0][[0, 1, 2, 7, 8, 9, 14, 15, 16]], qo[0][[0, 1, 2, 7, 8, 9, 14, 15, 16]],
                               rtol=0, atol=bound)
