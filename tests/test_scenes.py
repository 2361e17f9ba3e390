"""The seeded synthetic inputs hold to the recipe they state: the walled-bin piles (a 50/50
sphere/capsule mix with the stated size ranges, density and masses, deposited without
overlapping bounding spheres inside the 0.6 m bin, unit quaternions, at rest), seeded
reproducibility, the interpenetrating start of the jammed variant, the hand's sizes, and the
solid-body inertias against numerical integration."""
import numpy as np
import pytest

from paper_2603_12185_gb300 import scenes as S


def _pile_arrays(sb):
    blk = np.stack(sb.world_param)                                # [W, n, 8]: m, I, type, r, h, -
    q = np.stack([np.asarray(x).reshape(-1, 7) for x in sb.q0])   # [W, n, 7]
    return blk, q


def test_pile_is_seeded():
    a, b, c = S.make_pile(8, 64, seed=3), S.make_pile(8, 64, seed=3), S.make_pile(8, 64, seed=4)
    for x, y in zip(a.q0, b.q0):
        assert np.array_equal(x, y)
    for x, y in zip(a.world_param, b.world_param):
        assert np.array_equal(x, y)
    assert not np.array_equal(a.q0[0], c.q0[0])


def test_pile_follows_its_recipe():
    sb = S.make_pile(64, 64, seed=1)
    blk, q = _pile_arrays(sb)
    m, inert, typ, r, h = blk[..., 0], blk[..., 1:4], blk[..., 4], blk[..., 5], blk[..., 6]
    caps, sph = typ == S.CAPSULE, typ == S.SPHERE
    assert np.all(caps | sph)
    assert abs(caps.mean() - 0.5) < 0.05                           # 4096 fair draws
    assert np.all((r[sph] >= 0.03) & (r[sph] <= 0.06)) and np.all(h[sph] == 0.0)
    assert np.all(r[caps] == 0.03) and np.all((h[caps] >= 0.03) & (h[caps] <= 0.08))
    vol = 4.0 / 3.0 * np.pi * r ** 3 + np.pi * r * r * 2.0 * h   # caps: a cylinder of length 2h
    np.testing.assert_allclose(m, 1000.0 * vol, rtol=1e-12)
    assert np.all(inert > 0)
    # placement: inside the walls (+-0.3 m) and above the floor, no bounding spheres overlapping
    bound = r + h
    p = q[..., :3]
    assert np.all(np.abs(p[..., :2]) <= 0.3 - bound[..., None] + 1e-12)
    assert np.all(p[..., 2] >= bound - 1e-12)
    d = np.linalg.norm(p[:, :, None, :] - p[:, None, :, :], axis=-1)
    lim = bound[:, :, None] + bound[:, None, :]
    off = ~np.eye(64, dtype=bool)[None]
    assert np.all((d >= lim * (1 - 1e-9))[np.broadcast_to(off, d.shape)])
    np.testing.assert_allclose(np.linalg.norm(q[..., 3:], axis=-1), 1.0, atol=1e-12)
    assert all(np.all(v == 0.0) for v in sb.v0)
    assert sb.params.n_t == 8 and sb.params.n_tor == 2 and sb.params.n_rol == 8


def test_jammed_pile_starts_interpenetrating():
    blk, q = _pile_arrays(S.make_pile(4, 64, seed=2, jammed=True))
    bound = blk[..., 5] + blk[..., 6]
    p = q[..., :3]
    d = np.linalg.norm(p[:, :, None, :] - p[:, None, :, :], axis=-1)
    lim = bound[:, :, None] + bound[:, None, :]
    overlaps = ((d < lim) & ~np.eye(64, dtype=bool)[None]).sum() // 2
    assert overlaps > 4 * 20


def test_hand_sizes():
    sb = S.make_hand(2, seed=0)
    t = sb.templates[0]
    assert len(t.body_parent) == 17 and int((t.body_jnt == S.HINGE).sum()) == 16
    assert len(sb.q0[0]) == 23 and len(sb.v0[0]) == 22


def _grid_inertia(inside, ext, n=161):
    """Volume and principal moments of a unit-density solid within the box +-ext by midpoint
    integration on an n^3 grid."""
    gx, gy, gz = [(np.arange(n) + 0.5) / n * 2 * e - e for e in ext]
    x, y, z = np.meshgrid(gx, gy, gz, indexing="ij")
    mask = inside(x, y, z)
    dv = 8 * ext[0] * ext[1] * ext[2] / n ** 3
    vol = mask.sum() * dv
    ixx = ((y * y + z * z) * mask).sum() * dv
    izz = ((x * x + y * y) * mask).sum() * dv
    return vol, ixx, izz


@pytest.mark.parametrize("r,h", [(0.03, 0.05), (0.02, 0.08)])
def test_capsule_inertia_against_integration(r, h):
    """The capsule's closed form (a cylinder of length 2h plus two hemispherical caps, each cap
    moved to its end by the parallel-axis theorem) against a grid integration of the solid."""
    inside = lambda x, y, z: x * x + y * y + (z - np.clip(z, -h, h)) ** 2 <= r * r
    vol, ixx, izz = _grid_inertia(inside, (r, r, h + r))
    m, (ix, _, iz) = S.capsule_mass_inertia(r, h, 1.0)
    assert m == pytest.approx(vol, rel=1e-2)
    assert ix == pytest.approx(ixx, rel=1e-2) and iz == pytest.approx(izz, rel=1e-2)


def test_sphere_and_box_inertia_against_integration():
    vol, ixx, izz = _grid_inertia(lambda x, y, z: x * x + y * y + z * z <= 0.04 ** 2, (0.04, 0.04, 0.04))
    m, i = S.sphere_mass_inertia(0.04, 1.0)
    assert m == pytest.approx(vol, rel=2e-2) and i[0] == pytest.approx(ixx, rel=2e-2)
    hs = (0.02, 0.03, 0.045)
    vol, ixx, izz = _grid_inertia(lambda x, y, z: np.ones_like(x, dtype=bool), hs)
    m, i = S.box_mass_inertia(np.array(hs), 8.0 * np.prod(hs))
    assert m == pytest.approx(vol, rel=1e-12)
    assert i[0] == pytest.approx(ixx, rel=1e-3) and i[2] == pytest.approx(izz, rel=1e-3)


def test_cylinder_and_ellipsoid_inertia_against_integration():
    r, h = 0.03, 0.05                                  # radius, half length along z
    vol, ixx, izz = _grid_inertia(lambda x, y, z: x * x + y * y <= r * r, (r, r, h))
    m, i = S.cylinder_mass_inertia(r, h, 1.0)
    assert m == pytest.approx(vol, rel=1e-2)
    assert i[0] == pytest.approx(ixx, rel=1e-2) and i[2] == pytest.approx(izz, rel=1e-2)
    e = np.array([0.05, 0.03, 0.02])
    inside = lambda x, y, z: (x / e[0]) ** 2 + (y / e[1]) ** 2 + (z / e[2]) ** 2 <= 1.0
    vol, ixx, izz = _grid_inertia(inside, tuple(e))
    m, i = S.ellipsoid_mass_inertia(e, 1.0)
    assert m == pytest.approx(vol, rel=1e-2)
    assert i[0] == pytest.approx(ixx, rel=1e-2) and i[2] == pytest.approx(izz, rel=1e-2)


def test_hand_geometry_by_forward_kinematics():
    """The hand as its generator describes it, read back through the oracle's (separately pinned)
    forward kinematics: finger f's base at radius 6.5 cm, azimuth pi/4 + f pi/2, height 1.5 cm;
    its first joint about the vertical, the other three about the horizontal flexion axis, and a
    positive flexion curls the finger toward the centre; links stacked end to end."""
    from oracle import oracle as O
    sb = S.make_hand(1, seed=0)
    d = sb.world(0)
    q = np.array(sb.q0[0], float)
    nq = len(q)
    q[7:] = 0.0
    _, _, P = O.dynamics(d, (0, 0, -9.81), q, np.zeros(len(sb.v0[0])))
    for f in range(4):
        a = np.pi / 4 + f * np.pi / 2
        er = np.array([np.cos(a), np.sin(a), 0.0])
        b0 = 1 + 4 * f
        np.testing.assert_allclose(P[b0, :3], 0.065 * er + [0, 0, 0.015], atol=1e-12)
        R0 = P[b0, 3:12].reshape(3, 3)
        np.testing.assert_allclose(R0 @ d["body_axis"][b0], [0, 0, 1], atol=1e-12)   # abduction: vertical
        for j in range(1, 4):
            b = b0 + j
            R = P[b, 3:12].reshape(3, 3)
            ax = R @ d["body_axis"][b]
            assert abs(ax[2]) < 1e-12                                                  # flexion: horizontal
            L = d["body_pos"][b][2]
            assert 0.03 <= L <= 0.05
            np.testing.assert_allclose(P[b, :3], P[b - 1, :3] + P[b - 1, 3:12].reshape(3, 3) @ [0, 0, L], atol=1e-12)
        tip = lambda PP: PP[b0 + 3, :3] + PP[b0 + 3, 3:12].reshape(3, 3) @ [0, 0, 0.04]
        qc = q.copy()
        qc[7 + 4 * f + 1] = 0.5                                                        # flex the second joint
        _, _, Pc = O.dynamics(d, (0, 0, -9.81), qc, np.zeros(len(sb.v0[0])))
        assert np.hypot(*tip(Pc)[:2]) < np.hypot(*tip(P)[:2]) - 0.01
    assert nq == 23
