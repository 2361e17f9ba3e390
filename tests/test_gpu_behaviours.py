"""The paper's qualitative behaviours on the CUDA path (Sec. IV-A..C):
torsional friction decays a spin about the normal, faster for a larger coefficient; rolling
friction decays a rolling capsule, faster for a larger coefficient; a cube thrown onto a plane
slides to rest without drift or growth, also at dt = 0.02 s; rest penetration shrinks as k_user
grows."""
import numpy as np
import pytest
import torch

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


def template(d, name="t"):
    return S.Template(name=name, pile=False, **{k: np.asarray(v) for k, v in d.items()})


def run(d, params, q0, v0, dt, steps, every):
    m = CF.Model([template(d)], params)
    b = CF.Batch(m, np.zeros(1, np.int32))
    b.set_state(np.asarray(q0, np.float32), np.asarray(v0, np.float32))
    out = []
    for _ in range(steps // every):
        b.step(dt, every)
        q, v = b.get_state()
        out.append((q.cpu().numpy().astype(np.float64), v.cpu().numpy().astype(np.float64)))
    st, _ = b.status()
    assert st == 0
    return out


def test_torsional_friction_decays_spin_monotonically():
    """A sphere on a vertical hinge, pressed 2 mm into the floor, spinning about the normal.
    The contact point lies on the hinge axis, so no DoF moves it translationally and the
    translational point-Jacobian trace tr(J M~^-1 J^T) that M(phi) divides by is zero; the test uses the per-body 1/m impedance (trace_mode 1)."""
    finals = {}
    for mu_tor in (0.002, 0.01):
        d = Wd.world([dict(parent=-1, jnt=S.HINGE, pos=(0, 0, 0.048), axis=(0, 0, 1), mass=1.0,
                           inertia=(1e-3, 1e-3, 1e-3))],
                     [dict(type=S.PLANE, body=-1, mu=(0.5, mu_tor, 0.0)),
                      dict(type=S.SPHERE, body=0, size=(0.05, 0, 0), mu=(0.5, mu_tor, 0.0))])
        p = S.Params(n_t=4, n_tor=2, n_rol=0, trace_mode=1)
        tr = run(d, p, [0.0], [10.0], 0.002, 500, 25)
        w = np.array([v[0] for _, v in tr])
        assert np.all(np.diff(w) <= 1e-6) and w[-1] < 10.0
        finals[mu_tor] = w[-1]
    assert finals[0.01] < finals[0.002]


def test_rolling_friction_decays_a_rolling_capsule():
    finals = {}
    for mu_rol in (0.002, 0.01):
        d = Wd.world([dict(mass=1.0, inertia=(2e-3, 2e-3, 5e-4))],
                     [dict(type=S.PLANE, body=-1, mu=(0.8, 0.0, mu_rol)),
                      dict(type=S.CAPSULE, body=0, size=(0.03, 0.05, 0), mu=(0.8, 0.0, mu_rol))])
        p = S.Params(n_t=8, n_tor=2, n_rol=8)
        # axis along y, rolling along +x: omega_y = v / r
        qa = S.quat_about((1, 0, 0), np.pi / 2)
        q0 = [0, 0, 0.028, *qa]
        R = np.array([[1, 0, 0], [0, 0, -1], [0, 1, 0]], float)
        v0 = [0.5, 0, 0, *(R.T @ np.array([0, 0.5 / 0.03, 0]))]
        tr = run(d, p, q0, v0, 0.002, 1000, 50)
        vx = np.array([v[0] for _, v in tr])
        assert np.all(np.diff(vx[2:]) <= 1e-5)
        finals[mu_rol] = vx[-1]
    assert finals[0.01] < finals[0.002]


@pytest.mark.parametrize("dt", [0.002, 0.02])
def test_thrown_cube_slides_to_rest_without_drift(dt):
    d = Wd.world([dict(mass=1.0, inertia=S.box_mass_inertia([0.05] * 3, 1.0)[1])],
                 [dict(type=S.PLANE, body=-1, mu=(0.5, 0, 0)), dict(type=S.BOX, body=0, size=(0.05, 0.05, 0.05),
                                                                       mu=(0.5, 0, 0))])
    p = S.Params(n_t=4, k_user=0.3, d_user=0.005)
    steps = int(round(3.0 / dt))
    tr = run(d, p, [0, 0, 0.2, 1, 0, 0, 0], [2.0, 0, 0, 0.1, 0.1, 0.1], dt, steps, max(1, steps // 60))
    speed = np.array([np.hypot(v[0], v[1]) for _, v in tr])
    z = np.array([q[2] for q, _ in tr])
    assert np.all(np.isfinite(speed)) and np.all(np.isfinite(z))
    assert speed[-1] < 0.05 * 2.0                      # at rest
    land = int(np.argmax(z < 0.06))
    assert np.all(np.diff(speed[land + 1:]) <= 1e-3)   # no growth once sliding
    assert abs(z[-1] - z[-5]) < 1e-3 and 0.03 < z[-1] < 0.06


def test_rest_penetration_shrinks_with_k_user():
    depth = {}
    for k in (0.1, 0.3, 0.5):
        d = Wd.sphere_on_plane()
        p = S.Params(n_t=4, k_user=k, d_user=0.001)
        tr = run(d, p, [0, 0, 0.05, 1, 0, 0, 0], [0] * 6, 0.002, 3000, 3000)
        depth[k] = 0.05 - tr[-1][0][2]
    assert depth[0.1] > depth[0.3] > depth[0.5] > 0
