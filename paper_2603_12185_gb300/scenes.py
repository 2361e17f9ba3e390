"""Seeded synthetic scene generators shared by the CUDA path, the oracle tests and the bench.

This module holds input data only: body/geom descriptions, masses and inertias computed
from density, and seeded initial states.  None of the contact method's arithmetic (the
smooth prediction, narrowphase, dual-cone facets, impulses, correction or integration)
lives here.

Data model (all arrays are numpy):

* ``Template`` -- one scene layout: a kinematic forest of bodies (free bodies, or fixed-base
  chains/trees of hinge joints) plus primitive geoms.  Body ``b``'s joint frame is placed at
  ``body_pos/body_quat`` in its parent's frame (hinge bodies; ignored for free bodies whose
  pose lives in ``q``).  ``body_ipos`` is the centre of mass in the body frame and
  ``body_inertia`` the principal inertia about it, with the principal axes equal to the body
  axes.  Free bodies must have ``body_ipos == 0`` (body frame at the centre of mass).
  Geom types: 0 plane (static only, normal = local +z), 1 sphere (size[0]=r), 2 capsule
  (size[0]=r, size[1]=half length along local z), 3 box (size = half extents).
* ``pile`` templates are the special case "every body is free and carries exactly one geom at
  its origin (geom i on body i), remaining geoms are static planes"; only they accept the
  per-world override block ``[mass, I1, I2, I3, geom_type, s0, s1, s2]`` per body.
* ``Batch`` -- W worlds, each naming a template, with optional per-world overrides and the
  initial state.  State per world: q = per body (free: x y z qw qx qy qz | hinge: angle),
  v = per body (free: world linear velocity, body-frame angular velocity | hinge: rate).

Generators:

* ``make_spheres_on_plane``  -- worlds of identical spheres on a ground plane, 4-facet cone.
* ``make_pile``              -- walled bins with a seeded sphere/capsule mix, 18-facet 6D cone.
* ``make_hand``              -- a 16-DoF four-finger hand on a static palm around a free cube.
* ``make_mixed``             -- interleaves pile16 / pile64 / pile256 / hand worlds.
"""
from __future__ import annotations

import dataclasses
from dataclasses import dataclass, field
import numpy as np

PLANE, SPHERE, CAPSULE, BOX, CYLINDER, ELLIPSOID = 0, 1, 2, 3, 4, 5
FREE, HINGE = 0, 1
PARAM_STRIDE = 8  # per-body override block: mass, I1, I2, I3, type, s0, s1, s2


# ----------------------------------------------------------------------------------------
# plain rigid-body input data (mass properties from density, quaternions for poses)
# ----------------------------------------------------------------------------------------
def sphere_mass_inertia(r, rho):
    m = rho * 4.0 / 3.0 * np.pi * r ** 3
    i = 0.4 * m * r * r
    return m, np.array([i, i, i])


def capsule_mass_inertia(r, h, rho):
    """Solid capsule along local z: cylinder of length 2h plus two hemispherical caps."""
    mc = rho * np.pi * r * r * 2.0 * h
    ms = rho * 4.0 / 3.0 * np.pi * r ** 3
    izz = mc * r * r / 2.0 + ms * 2.0 * r * r / 5.0
    ixx = mc * ((2.0 * h) ** 2 / 12.0 + r * r / 4.0) + ms * (83.0 / 320.0 * r * r + (h + 3.0 * r / 8.0) ** 2)
    return mc + ms, np.array([ixx, ixx, izz])


def box_mass_inertia(half, m):
    a, b, c = 2.0 * np.asarray(half, dtype=np.float64)
    return m, np.array([m * (b * b + c * c) / 12.0, m * (a * a + c * c) / 12.0, m * (a * a + b * b) / 12.0])


def cylinder_mass_inertia(r, h, rho):
    """Solid cylinder of radius r, half length h along z."""
    m = rho * np.pi * r * r * 2.0 * h
    return m, np.array([m * (3 * r * r + 4 * h * h) / 12.0, m * (3 * r * r + 4 * h * h) / 12.0, 0.5 * m * r * r])


def ellipsoid_mass_inertia(e, rho):
    """Solid ellipsoid with semi-axes e = (a, b, c)."""
    a, b, c = np.asarray(e, dtype=np.float64)
    m = rho * 4.0 / 3.0 * np.pi * a * b * c
    return m, np.array([m * (b * b + c * c) / 5.0, m * (a * a + c * c) / 5.0, m * (a * a + b * b) / 5.0])


def random_quats(rng, n):
    """Uniformly distributed unit quaternions (w, x, y, z), Shoemake's subgroup algorithm."""
    u1, u2, u3 = rng.random(n), rng.random(n), rng.random(n)
    a, b = np.sqrt(1.0 - u1), np.sqrt(u1)
    qx, qy = a * np.sin(2 * np.pi * u2), a * np.cos(2 * np.pi * u2)
    qz, qw = b * np.sin(2 * np.pi * u3), b * np.cos(2 * np.pi * u3)
    q = np.stack([qw, qx, qy, qz], axis=-1)
    q[q[:, 0] < 0] *= -1.0
    return q


def quat_about(axis, angle):
    axis = np.asarray(axis, dtype=np.float64)
    axis = axis / np.linalg.norm(axis)
    return np.concatenate([[np.cos(angle / 2)], np.sin(angle / 2) * axis])


def _quat_rotate(q, v):
    w, x, y, z = q
    r = np.array([
        [1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)],
        [2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)],
        [2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)],
    ])
    return r @ v


# ----------------------------------------------------------------------------------------
@dataclass
class Params:
    gravity: tuple = (0.0, 0.0, -9.81)
    k_user: float = 0.1
    d_user: float = 0.001
    solimp: tuple = (0.9, 0.95, 0.001, 0.5, 2.0)
    margin: float = 0.0
    n_t: int = 4
    n_tor: int = 0
    n_rol: int = 0
    trace_mode: int = 0  # 0: translational point-Jacobian trace, 1: sum of 1/m of the bodies,
    #                      2: exact diagonal impedance per facet (Sec. III-B),
    #                      3: mode 0 scaled by the learned impedance network (Sec. III-B)


@dataclass
class Template:
    name: str
    body_parent: np.ndarray
    body_jnt: np.ndarray
    body_pos: np.ndarray
    body_quat: np.ndarray
    body_axis: np.ndarray
    body_ipos: np.ndarray
    body_mass: np.ndarray
    body_inertia: np.ndarray
    body_damping: np.ndarray
    geom_type: np.ndarray
    geom_body: np.ndarray
    geom_pos: np.ndarray
    geom_quat: np.ndarray
    geom_size: np.ndarray
    geom_mu: np.ndarray
    pile: bool = False
    body_range: np.ndarray = None         # [nbody, 2] hinge limits (lower < upper limits), or None
    body_frictionloss: np.ndarray = None  # [nbody] hinge dry friction (N m), or None

    @property
    def nbody(self):
        return len(self.body_parent)

    @property
    def ngeom(self):
        return len(self.geom_type)

    @property
    def nq(self):
        return int(sum(7 if j == FREE else 1 for j in self.body_jnt))

    @property
    def nv(self):
        return int(sum(6 if j == FREE else 1 for j in self.body_jnt))

    @property
    def nu(self):
        """Actuated DoFs: every hinge joint takes a torque; free bodies are unactuated."""
        return int(sum(1 for j in self.body_jnt if j == HINGE))


@dataclass
class Batch:
    templates: list
    params: Params
    world_scene: np.ndarray            # int32 [W]
    world_param: list                  # per world: float64 [nbody, 8] override block or None
    q0: list                           # per world float64 [nq]
    v0: list                           # per world float64 [nv]
    dt: float = 0.002
    nsteps: int = 1
    meta: dict = field(default_factory=dict)

    @property
    def nworld(self):
        return len(self.world_scene)

    def template_of(self, w):
        return self.templates[int(self.world_scene[w])]

    def world(self, w):
        """Full description of world ``w`` with its overrides merged into the template arrays."""
        t = self.template_of(w)
        d = {k: np.array(getattr(t, k)) for k in (
            "body_parent", "body_jnt", "body_pos", "body_quat", "body_axis", "body_ipos", "body_mass",
            "body_inertia", "body_damping", "geom_type", "geom_body", "geom_pos", "geom_quat", "geom_size",
            "geom_mu")}
        for k in ("body_range", "body_frictionloss"):
            if getattr(t, k) is not None:
                d[k] = np.array(getattr(t, k), dtype=np.float64)
        p = self.world_param[w]
        if p is not None:
            nb = t.nbody
            d["body_mass"] = p[:, 0].astype(np.float64).copy()
            d["body_inertia"] = p[:, 1:4].astype(np.float64).copy()
            d["geom_type"][:nb] = p[:, 4].astype(np.int32)
            d["geom_size"][:nb] = p[:, 5:8].astype(np.float64)
        return d

    def subset(self, worlds):
        worlds = [int(w) for w in worlds]
        return Batch(self.templates, self.params, self.world_scene[worlds].copy(),
                     [self.world_param[w] for w in worlds], [self.q0[w].copy() for w in worlds],
                     [self.v0[w].copy() for w in worlds], self.dt, self.nsteps, dict(self.meta))


def _planes(walls: bool, half: float = 0.3):
    """Static planes: the floor z=0 and, for a bin, four inward-facing walls at +-half."""
    pos = [[0, 0, 0]]
    quat = [[1, 0, 0, 0]]
    if walls:
        s = np.sqrt(0.5)
        pos += [[-half, 0, 0], [half, 0, 0], [0, -half, 0], [0, half, 0]]
        # local +z mapped to +x, -x, +y, -y respectively
        quat += [[s, 0, s, 0], [s, 0, -s, 0], [s, -s, 0, 0], [s, s, 0, 0]]
    return np.array(pos, dtype=np.float64), np.array(quat, dtype=np.float64)


def _pile_template(name, n, plane_pos, plane_quat, mu):
    nplane = len(plane_pos)
    ng = n + nplane
    gt = np.full(ng, SPHERE, np.int32)
    gt[n:] = PLANE
    gb = np.concatenate([np.arange(n, dtype=np.int32), np.full(nplane, -1, np.int32)])
    gpos = np.zeros((ng, 3))
    gpos[n:] = plane_pos
    gquat = np.zeros((ng, 4))
    gquat[:, 0] = 1.0
    gquat[n:] = plane_quat
    gsize = np.zeros((ng, 3))
    gsize[:n, 0] = 0.05
    gmu = np.tile(np.asarray(mu, dtype=np.float64), (ng, 1))
    return Template(
        name=name,
        body_parent=np.full(n, -1, np.int32), body_jnt=np.full(n, FREE, np.int32),
        body_pos=np.zeros((n, 3)), body_quat=np.tile([1.0, 0, 0, 0], (n, 1)),
        body_axis=np.tile([0, 0, 1.0], (n, 1)), body_ipos=np.zeros((n, 3)),
        body_mass=np.ones(n), body_inertia=np.full((n, 3), 1e-3), body_damping=np.zeros(n),
        geom_type=gt, geom_body=gb, geom_pos=gpos, geom_quat=gquat, geom_size=gsize, geom_mu=gmu, pile=True)


def make_spheres_on_plane(nworld=64, nbody=8, seed=0, radius=0.05, mass=1.0, mu=0.5, dt=0.002, nsteps=500):
    """Worlds of identical solid spheres dropped on a ground plane (4-facet pyramidal cone).

    Initial xy ~ U[-0.5, 0.5] m, z ~ U[0.1, 1.0] m, zero velocity, identity orientation."""
    rng = np.random.default_rng(seed)
    pp, pq = _planes(False)
    t = _pile_template(f"spheres{nbody}", nbody, pp, pq, (mu, 0.0, 0.0))
    m, inertia = mass, np.full(3, 0.4 * mass * radius * radius)
    blk = np.zeros((nbody, PARAM_STRIDE))
    blk[:, 0] = m
    blk[:, 1:4] = inertia
    blk[:, 4] = SPHERE
    blk[:, 5] = radius
    q0, v0 = [], []
    for _ in range(nworld):
        q = np.zeros((nbody, 7))
        q[:, 0:2] = rng.uniform(-0.5, 0.5, size=(nbody, 2))
        q[:, 2] = rng.uniform(0.1, 1.0, size=nbody)
        q[:, 3] = 1.0
        q0.append(q.reshape(-1))
        v0.append(np.zeros(nbody * 6))
    params = Params(k_user=0.1, d_user=0.001, n_t=4, n_tor=0, n_rol=0)
    return Batch([t], params, np.zeros(nworld, np.int32), [blk.copy() for _ in range(nworld)], q0, v0, dt, nsteps,
                 {"workload": f"spheres_on_plane_{nworld}x{nbody}"})


def _pile_worlds(rng, nworld, n, rho=1000.0, half=0.3, box_h=0.6, jammed=False, box_frac=0.0, round_frac=0.0):
    """Per-world sphere/capsule mixes placed without overlap of their bounding spheres.

    Random sequential deposition, vectorised across worlds: body k draws x, y uniformly inside
    the bin and a drop height z ~ U[b, 0.6 - b] (b = bounding radius).  If a body already placed
    overlaps it there, it is raised to the lowest height that clears every placed body whose
    footprint overlaps its own.  Sparse worlds start scattered through the 0.6 m cube; dense
    ones start as a loose column that rises well above it and collapses into the bin."""
    is_caps = rng.random((nworld, n)) < 0.5
    r = np.where(is_caps, 0.03, rng.uniform(0.03, 0.06, size=(nworld, n)))
    h = np.where(is_caps, rng.uniform(0.03, 0.08, size=(nworld, n)), 0.0)
    bound = r + h
    is_box = np.zeros((nworld, n), bool)
    hs = np.zeros((nworld, n, 3))
    if box_frac > 0.0:  # boxes with half extents U[0.02, 0.045] m replace a fraction of the bodies
        is_box = rng.random((nworld, n)) < box_frac
        hs = rng.uniform(0.02, 0.045, size=(nworld, n, 3))
        is_caps = is_caps & ~is_box
        bound = np.where(is_box, np.linalg.norm(hs, axis=2), bound)
    kind = np.zeros((nworld, n), np.int32)    # 1: cylinder, 2: ellipsoid (replacing spheres/capsules)
    ext = np.zeros((nworld, n, 3))
    if round_frac > 0.0:  # cylinders r U[0.02, 0.04], h U[0.02, 0.05]; ellipsoids semi-axes U[0.02, 0.05]
        pick = (rng.random((nworld, n)) < round_frac) & ~is_box
        kind = np.where(pick, 1 + (rng.random((nworld, n)) < 0.5), 0)
        cyl = np.stack([rng.uniform(0.02, 0.04, (nworld, n)), rng.uniform(0.02, 0.05, (nworld, n)),
                        np.zeros((nworld, n))], axis=2)
        ell = rng.uniform(0.02, 0.05, size=(nworld, n, 3))
        ext = np.where((kind == 1)[..., None], cyl, ell)
        is_caps = is_caps & (kind == 0)
        bound = np.where(kind == 1, np.hypot(cyl[..., 0], cyl[..., 1]),
                         np.where(kind == 2, ell.max(axis=2), bound))
    pos = np.zeros((nworld, n, 3))
    for k in range(n):
        bk = bound[:, k]
        pos[:, k, 0] = -half + bk + 2 * (half - bk) * rng.random(nworld)
        pos[:, k, 1] = -half + bk + 2 * (half - bk) * rng.random(nworld)
        z = bk + np.maximum(box_h - 2 * bk, 0.0) * rng.random(nworld)
        if k and not jammed:
            dxy2 = ((pos[:, :k, :2] - pos[:, k:k + 1, :2]) ** 2).sum(-1)
            lim = bound[:, :k] + bk[:, None]
            dz = np.sqrt(np.maximum(lim * lim - dxy2, 0.0))
            hit = dxy2 < lim * lim
            over = hit & (np.abs(z[:, None] - pos[:, :k, 2]) < dz)
            zreq = np.where(hit, pos[:, :k, 2] + dz, -np.inf).max(axis=1)
            z = np.where(over.any(axis=1), np.maximum(z, zreq), z)
        pos[:, k, 2] = z
    quat = random_quats(rng, nworld * n).reshape(nworld, n, 4)
    blocks = []
    for w in range(nworld):
        blk = np.zeros((n, PARAM_STRIDE))
        for i in range(n):
            if kind[w, i]:
                if kind[w, i] == 1:
                    m, inertia = cylinder_mass_inertia(ext[w, i, 0], ext[w, i, 1], rho)
                    blk[i, 4] = CYLINDER
                else:
                    m, inertia = ellipsoid_mass_inertia(ext[w, i], rho)
                    blk[i, 4] = ELLIPSOID
                blk[i, 0] = m
                blk[i, 1:4] = inertia
                blk[i, 5:8] = ext[w, i]
                continue
            if is_box[w, i]:
                m, inertia = box_mass_inertia(hs[w, i], rho * 8.0 * float(np.prod(hs[w, i])))
                blk[i, 0] = m
                blk[i, 1:4] = inertia
                blk[i, 4] = BOX
                blk[i, 5:8] = hs[w, i]
                continue
            if is_caps[w, i]:
                m, inertia = capsule_mass_inertia(r[w, i], h[w, i], rho)
                blk[i, 4] = CAPSULE
            else:
                m, inertia = sphere_mass_inertia(r[w, i], rho)
                blk[i, 4] = SPHERE
            blk[i, 0] = m
            blk[i, 1:4] = inertia
            blk[i, 5] = r[w, i]
            blk[i, 6] = h[w, i]
        blocks.append(blk)
    q0 = [np.concatenate([pos[w], quat[w]], axis=1).reshape(-1) for w in range(nworld)]
    v0 = [np.zeros(6 * n) for _ in range(nworld)]
    return blocks, q0, v0


PILE_PARAMS = dict(k_user=0.1, d_user=0.001, n_t=8, n_tor=2, n_rol=8)
PILE_MU = (0.8, 0.005, 0.005)


def make_pile(nworld=4096, nbody=16, seed=0, dt=0.002, nsteps=1000, jammed=False, box_frac=0.0, round_frac=0.0):
    """Walled bins (floor + 4 walls at +-0.3 m) with a seeded 50/50 sphere/capsule mix.

    Spheres r ~ U[0.03, 0.06] m; capsules r = 0.03 m, half length ~ U[0.03, 0.08] m; density
    1000 kg/m^3; uniform random orientations; zero velocity; 6D cone with 8 tangential,
    2 torsional and 8 rolling facets, mu = 0.8, torsional/rolling coefficients 0.005 m.

    jammed=True skips the overlap rejection: bodies start interpenetrating anywhere in the
    0.6 m cube, so the very first step already resolves thousands of contacts per world (a
    contact-rich input for single-step checks at full size)."""
    rng = np.random.default_rng(seed)
    pp, pq = _planes(True)
    t = _pile_template(f"pile{nbody}", nbody, pp, pq, PILE_MU)
    blocks, q0, v0 = _pile_worlds(rng, nworld, nbody, jammed=jammed, box_frac=box_frac, round_frac=round_frac)
    return Batch([t], Params(**PILE_PARAMS), np.zeros(nworld, np.int32), blocks, q0, v0, dt, nsteps,
                 {"workload": f"pile_{nworld}x{nbody}" + ("_jammed" if jammed else "") +
                  (f"_boxes{box_frac:g}" if box_frac > 0 else "") +
                  (f"_cylell{round_frac:g}" if round_frac > 0 else "")})


# ----------------------------------------------------------------------------------------
# four-finger hand around a free cube
# ----------------------------------------------------------------------------------------
HAND_LINK_R = 0.01
HAND_CUBE_HALF = 0.03
HAND_CUBE_MASS = 0.1


def hand_template(seed=0, rho=1000.0, damping=0.1, mu=PILE_MU):
    """A static palm plane (z = 0, normal +z), a free 6 cm / 0.1 kg cube (body 0) and four
    fingers of four hinge joints each (bodies 1..16).  Finger f stands at radius 6.5 cm,
    azimuth pi/4 + f pi/2, base height 1.5 cm.  Its first joint turns about the vertical
    (abduction), the next three about the horizontal axis that curls the finger toward the
    cube (positive angle = inward).  Each body carries one capsule link (r = 1 cm) of seeded
    length U[0.03, 0.05] m along its local +z; joint damping 0.1."""
    rng = np.random.default_rng(seed)
    lengths = rng.uniform(0.03, 0.05, size=(4, 4))
    nb = 1 + 16
    parent = np.full(nb, -1, np.int32)
    jnt = np.full(nb, HINGE, np.int32)
    jnt[0] = FREE
    bpos = np.zeros((nb, 3))
    bquat = np.tile([1.0, 0, 0, 0], (nb, 1))
    baxis = np.tile([1.0, 0, 0], (nb, 1))
    bipos = np.zeros((nb, 3))
    bmass = np.zeros(nb)
    binert = np.zeros((nb, 3))
    bdamp = np.full(nb, damping)
    bdamp[0] = 0.0
    bmass[0], binert[0] = box_mass_inertia([HAND_CUBE_HALF] * 3, HAND_CUBE_MASS)
    gtype = [PLANE, BOX]
    gbody = [-1, 0]
    gpos = [[0, 0, 0], [0, 0, 0]]
    gquat = [[1, 0, 0, 0], [1, 0, 0, 0]]
    gsize = [[0, 0, 0], [HAND_CUBE_HALF] * 3]
    for f in range(4):
        a = np.pi / 4 + f * np.pi / 2
        er = np.array([np.cos(a), np.sin(a), 0.0])
        et = np.array([-np.sin(a), np.cos(a), 0.0])
        # base frame: x = flexion axis (-e_t), y = e_r, z = up
        rot = np.stack([-et, er, [0, 0, 1.0]], axis=1)
        w = np.sqrt(max(0.0, 1 + rot[0, 0] + rot[1, 1] + rot[2, 2])) / 2
        qb = np.array([w, (rot[2, 1] - rot[1, 2]) / (4 * w), (rot[0, 2] - rot[2, 0]) / (4 * w),
                       (rot[1, 0] - rot[0, 1]) / (4 * w)])
        for j in range(4):
            b = 1 + 4 * f + j
            L = lengths[f, j]
            if j == 0:
                parent[b] = -1
                bpos[b] = 0.065 * er + np.array([0, 0, 0.015])
                bquat[b] = qb
                baxis[b] = [0, 0, 1.0]
            else:
                parent[b] = b - 1
                bpos[b] = [0, 0, lengths[f, j - 1]]
                baxis[b] = [1.0, 0, 0]
            bipos[b] = [0, 0, L / 2]
            bmass[b], binert[b] = capsule_mass_inertia(HAND_LINK_R, L / 2, rho)
            gtype.append(CAPSULE)
            gbody.append(b)
            gpos.append([0, 0, L / 2])
            gquat.append([1, 0, 0, 0])
            gsize.append([HAND_LINK_R, L / 2, 0])
    ng = len(gtype)
    return Template(
        name="hand", body_parent=parent, body_jnt=jnt, body_pos=bpos, body_quat=bquat, body_axis=baxis,
        body_ipos=bipos, body_mass=bmass, body_inertia=binert, body_damping=bdamp,
        geom_type=np.array(gtype, np.int32), geom_body=np.array(gbody, np.int32),
        geom_pos=np.array(gpos, np.float64), geom_quat=np.array(gquat, np.float64),
        geom_size=np.array(gsize, np.float64), geom_mu=np.tile(np.asarray(mu, np.float64), (ng, 1)), pile=False)


def _cube_lowest(q):
    c = np.array([[sx, sy, sz] for sx in (-1, 1) for sy in (-1, 1) for sz in (-1, 1)]) * HAND_CUBE_HALF
    return min(_quat_rotate(q, ci)[2] for ci in c)


def hand_states(rng, nworld):
    """Seeded cube poses (position jitter, uniform orientation, lowest corner 0.5-15 mm above the
    palm) and finger joint angles (abduction U[-0.1, 0.1], flexion U[0.1, 0.45] rad)."""
    q0, v0 = [], []
    quats = random_quats(rng, nworld)
    for w in range(nworld):
        qc = quats[w]
        z = -_cube_lowest(qc) + rng.uniform(0.0005, 0.015)
        cube = np.concatenate([[rng.uniform(-0.01, 0.01), rng.uniform(-0.01, 0.01), z], qc])
        fing = np.zeros(16)
        for f in range(4):
            fing[4 * f] = rng.uniform(-0.1, 0.1)
            fing[4 * f + 1:4 * f + 4] = rng.uniform(0.1, 0.45, size=3)
        q0.append(np.concatenate([cube, fing]))
        v0.append(np.zeros(6 + 16))
    return q0, v0


HAND_PARAMS = dict(k_user=0.1, d_user=0.002, n_t=8, n_tor=2, n_rol=8)


def with_joint_limits(t, abduction=(-0.35, 0.35), flexion=(-0.2, 1.3), frictionloss=0.0):
    """Copy of a hand template whose hinges are limited (the first joint of each finger to
    `abduction`, the three flexion joints to `flexion`, radians) and carry dry friction."""
    rng_ = np.zeros((t.nbody, 2))
    fl = np.zeros(t.nbody)
    for b in range(t.nbody):
        if t.body_jnt[b] != HINGE:
            continue
        first = t.body_parent[b] < 0 or t.body_jnt[t.body_parent[b]] != HINGE
        rng_[b] = abduction if first else flexion
        fl[b] = frictionloss
    return dataclasses.replace(t, name=t.name + "_limited", body_range=rng_, body_frictionloss=fl)


def make_hand(nworld=1024, seed=0, dt=0.002, nsteps=100, d_user=0.002, joint_limits=False, frictionloss=0.0):
    rng = np.random.default_rng(seed)
    t = hand_template(seed)
    if joint_limits or frictionloss > 0.0:
        t = with_joint_limits(t, frictionloss=frictionloss)
    q0, v0 = hand_states(rng, nworld)
    p = dict(HAND_PARAMS)
    p["d_user"] = d_user
    return Batch([t], Params(**p), np.zeros(nworld, np.int32), [None] * nworld, q0, v0, dt, nsteps,
                 {"workload": f"hand_{nworld}"})


def make_mixed(nworld=8192, seed=0, dt=0.002, nsteps=1):
    """World i uses scene (i mod 4) in {pile16, pile64, pile256, hand}."""
    rng = np.random.default_rng(seed)
    pp, pq = _planes(True)
    sizes = (16, 64, 256)
    temps = [_pile_template(f"pile{n}", n, pp, pq, PILE_MU) for n in sizes] + [hand_template(seed)]
    counts = [len(range(s, nworld, 4)) for s in range(4)]
    per = []
    for s, n in enumerate(sizes):
        per.append(_pile_worlds(rng, counts[s], n))
    hq, hv = hand_states(rng, counts[3])
    per.append(([None] * counts[3], hq, hv))
    scene = np.arange(nworld, dtype=np.int32) % 4
    idx = [0, 0, 0, 0]
    blocks, q0, v0 = [], [], []
    for w in range(nworld):
        s = int(scene[w])
        blocks.append(per[s][0][idx[s]])
        q0.append(per[s][1][idx[s]])
        v0.append(per[s][2][idx[s]])
        idx[s] += 1
    return Batch(temps, Params(k_user=0.1, d_user=0.001, n_t=8, n_tor=2, n_rol=8), scene, blocks, q0, v0, dt,
                 nsteps, {"workload": f"mixed_{nworld}"})
