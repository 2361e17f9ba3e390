"""Edge cases on the GPU: empty and single-body inputs, the largest pile that fits one world's
shared memory and the first that does not, and the degenerate coincident-centre contact."""
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


def test_empty_world_list_is_a_no_op():
    sb = S.make_pile(4, 16, seed=41)
    _, b = CF.from_scenes(sb)
    q0, v0 = [t.clone() for t in b.get_state()]
    b.step(sb.dt, 3, worlds=[])
    q1, v1 = b.get_state()
    assert torch.equal(q0, q1) and torch.equal(v0, v1)


def test_zero_worlds_are_rejected():
    m = CF.Model([S.make_pile(1, 16, seed=1).templates[0]], S.Params())
    with pytest.raises(CF.CfError) as e:
        CF.Batch(m, np.zeros(0, np.int32))
    assert e.value.status == 1


def test_single_body_worlds():
    sb = GP._advanced(S.make_pile(6, 1, seed=42), lambda w: 40 * w)
    GP._check_single_step(sb)
    qg, vg, _ = PR.gpu_run(sb, 50)
    qo, vo = PR.oracle_run(sb, nsteps=50)
    assert max(PR.vel_err(vg[w], vo[w], sb.dt) for w in range(sb.nworld)) <= GP.TOL50


def test_largest_pile_world_matches_the_oracle():
    """1024 interpenetrating bodies in one world (about 209 KB of shared memory with 8 warps):
    one step against the oracle."""
    sb = S.make_pile(2, 1024, seed=43, jammed=True)
    qg, vg, b = PR.gpu_run(sb, 1)
    assert b.contact_counts().min() > 1000
    qo, vo = PR.oracle_run(sb, nsteps=1)
    for w in range(sb.nworld):
        assert PR.vel_err(vg[w], vo[w], sb.dt) <= GP.TOL1
        atol = 2e-6 + sb.dt * GP.TOL1 * np.abs(vo[w]).max()
        np.testing.assert_allclose(qg[w], qo[w], rtol=0, atol=atol)


def test_pile_too_large_for_shared_memory_is_refused():
    sb = S.make_pile(1, 1400, seed=44)
    with pytest.raises(CF.CfError) as e:
        CF.from_scenes(sb)
    assert e.value.status == 7


def test_coincident_sphere_centres():
    """Two spheres at one point: the normal is +z by convention (both sides), so the step is
    defined and matches the oracle."""
    d = Wd.world([dict(mass=1.0, inertia=(4e-4,) * 3), dict(mass=2.0, inertia=(8e-4,) * 3)],
                 [dict(type=S.PLANE, body=-1), dict(type=S.SPHERE, body=0, size=(0.03, 0, 0)),
                  dict(type=S.SPHERE, body=1, size=(0.04, 0, 0))])
    t = S.Template(name="twins", pile=False, **{k: np.asarray(v) for k, v in d.items()})
    q = np.array([0.1, 0.2, 0.5, 1, 0, 0, 0, 0.1, 0.2, 0.5, 1, 0, 0, 0], float)
    v = np.array([0.1, 0, 0, 0, 0, 0, -0.1, 0, 0, 0, 0, 0], float)
    sb = S.Batch([t], S.Params(n_t=8, n_tor=2, n_rol=8), np.zeros(1, np.int32), [None], [q], [v], 0.002, 1,
                 {"workload": "twins"})
    GP._check_single_step(sb)
    _, _, b = PR.gpu_run(sb, 1, capture=8)
    c = b.contacts()[0]
    assert len(c) == 1 and np.allclose(c[0]["normal"], [0, 0, 1])
