"""Tiny hand-built world descriptions for tests (same dict layout as scenes.Batch.world())."""
import numpy as np

from paper_2603_12185_gb300 import scenes as S


def world(bodies, geoms):
    """bodies: list of dicts(parent, jnt, pos, quat, axis, ipos, mass, inertia, damping);
    geoms: list of dicts(type, body, pos, quat, size, mu)."""
    nb = len(bodies)
    d = {
        "body_parent": np.array([b.get("parent", -1) for b in bodies], np.int32).reshape(nb),
        "body_jnt": np.array([b.get("jnt", S.FREE) for b in bodies], np.int32).reshape(nb),
        "body_pos": np.array([b.get("pos", (0, 0, 0)) for b in bodies], float).reshape(nb, 3),
        "body_quat": np.array([b.get("quat", (1, 0, 0, 0)) for b in bodies], float).reshape(nb, 4),
        "body_axis": np.array([b.get("axis", (0, 0, 1)) for b in bodies], float).reshape(nb, 3),
        "body_ipos": np.array([b.get("ipos", (0, 0, 0)) for b in bodies], float).reshape(nb, 3),
        "body_mass": np.array([b.get("mass", 1.0) for b in bodies], float).reshape(nb),
        "body_inertia": np.array([b.get("inertia", (1e-3, 1e-3, 1e-3)) for b in bodies], float).reshape(nb, 3),
        "body_damping": np.array([b.get("damping", 0.0) for b in bodies], float).reshape(nb),
        "geom_type": np.array([g["type"] for g in geoms], np.int32),
        "geom_body": np.array([g.get("body", -1) for g in geoms], np.int32),
        "geom_pos": np.array([g.get("pos", (0, 0, 0)) for g in geoms], float).reshape(-1, 3),
        "geom_quat": np.array([g.get("quat", (1, 0, 0, 0)) for g in geoms], float).reshape(-1, 4),
        "geom_size": np.array([g.get("size", (0, 0, 0)) for g in geoms], float).reshape(-1, 3),
        "geom_mu": np.array([g.get("mu", (0.5, 0.0, 0.0)) for g in geoms], float).reshape(-1, 3),
        "body_range": np.array([b.get("range", (0.0, 0.0)) for b in bodies], float).reshape(nb, 2),
        "body_frictionloss": np.array([b.get("frictionloss", 0.0) for b in bodies], float).reshape(nb),
    }
    return d


def sphere_on_plane(r=0.05, m=1.0, inertia=1e-3, mu=(0.5, 0.0, 0.0), plane_quat=(1, 0, 0, 0)):
    return world([dict(mass=m, inertia=(inertia,) * 3)],
                 [dict(type=S.PLANE, body=-1, quat=plane_quat, mu=mu), dict(type=S.SPHERE, body=0, size=(r, 0, 0), mu=mu)])


def free_state(pos, quat=(1, 0, 0, 0), lin=(0, 0, 0), ang=(0, 0, 0)):
    return np.array(list(pos) + list(quat), float), np.array(list(lin) + list(ang), float)


def params(**kw):
    p = S.Params()
    for k, v in kw.items():
        setattr(p, k, v)
    return p
