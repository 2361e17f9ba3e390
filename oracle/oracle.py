"""ctypes wrapper of the FP64 ComFree step oracle (oracle/oracle.cpp).

TEST INFRASTRUCTURE ONLY: tests/, __graft_entry__.smoke() and bench.py's cpu_baseline leg are
the only callers.  The product path never imports this module.

A world description is any mapping with the numpy arrays produced by
``paper_2603_12185_gb300.scenes.Batch.world(w)``: body_parent, body_jnt, body_pos, body_quat,
body_axis, body_ipos, body_mass, body_inertia, body_damping, geom_type, geom_body, geom_pos,
geom_quat, geom_size, geom_mu.  Parameters are any object with the attributes of
``scenes.Params``.  The wrapper itself imports nothing from the package.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.cpp")
_LIB = os.path.join(_HERE, "_build", "liboracle.so")
_lock = threading.Lock()
_lib = None


def compile_source(src: str, out: str, opt: str = "-O2") -> str:
    """Compile an oracle source file into the shared library `out` (g++ -fopenmp)."""
    cmd = ["g++", opt, "-std=c++17", "-fopenmp", "-fPIC", "-shared", src, "-o", out + ".tmp"]
    subprocess.run(cmd, check=True)
    os.replace(out + ".tmp", out)
    return out


def build(force: bool = False) -> str:
    """Compile oracle.cpp into oracle/_build/liboracle.so (g++ -O2 -fopenmp)."""
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        compile_source(_SRC, _LIB)
    return _LIB


class OWorld(C.Structure):
    _fields_ = [("nbody", C.c_int), ("ngeom", C.c_int)] + [
        (n, C.c_void_p) for n in ("body_parent", "body_jnt", "body_pos", "body_quat", "body_axis", "body_ipos",
                                  "body_mass", "body_inertia", "body_damping", "geom_type", "geom_body",
                                  "geom_pos", "geom_quat", "geom_size", "geom_mu", "body_range",
                                  "body_frictionloss")]


class OParams(C.Structure):
    _fields_ = [("gravity", C.c_double * 3), ("k_user", C.c_double), ("d_user", C.c_double),
                ("solimp", C.c_double * 5), ("margin", C.c_double), ("n_t", C.c_int), ("n_tor", C.c_int),
                ("n_rol", C.c_int), ("trace_mode", C.c_int), ("impnet", C.c_void_p)]


class OContact(C.Structure):
    _fields_ = [("geom_a", C.c_int), ("geom_b", C.c_int), ("body_a", C.c_int), ("body_b", C.c_int),
                ("sub", C.c_int), ("phi", C.c_double), ("pos", C.c_double * 3), ("normal", C.c_double * 3),
                ("t1", C.c_double * 3), ("t2", C.c_double * 3), ("trace_a", C.c_double),
                ("trace_b", C.c_double), ("r", C.c_double), ("mphi", C.c_double), ("lam_sum", C.c_double),
                ("wrench", C.c_double * 6), ("nfacet", C.c_int), ("nactive", C.c_int), ("feat", C.c_double * 4),
                ("m_exact", C.c_double)]


def load(path: str):
    """The oracle library at `path` with its entry points' argument types declared."""
    L = C.CDLL(path)
    P = C.POINTER
    L.ow_sizes.argtypes = [P(OWorld), P(C.c_int), P(C.c_int)]
    L.ow_step.argtypes = [P(OWorld), P(OParams), C.c_double, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p,
                          P(C.c_int)]
    L.ow_step_batch.argtypes = [C.c_int, C.c_void_p, P(OParams), C.c_double, C.c_int, C.c_void_p,
                                C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int]
    L.ow_step_record.argtypes = [P(OWorld), P(OParams), C.c_double, C.c_void_p, C.c_void_p, C.c_void_p,
                                 C.c_void_p, C.c_void_p, C.c_void_p, P(OContact), C.c_int, P(C.c_int)]
    L.ow_dynamics.argtypes = [P(OWorld), C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                              C.c_void_p]
    L.ow_cholesky.argtypes = [C.c_void_p, C.c_int]
    L.ow_capsule_box_param.argtypes = [C.c_void_p, C.c_void_p, C.c_double, C.c_void_p]
    L.ow_capsule_box_param.restype = C.c_double
    L.ow_solimp_r.argtypes = [C.c_double, C.c_void_p]
    L.ow_solimp_r.restype = C.c_double
    L.ow_rollout_loss_dir.argtypes = [P(OWorld), P(OParams), C.c_double, C.c_int] + [C.c_void_p] * 6 + [
        C.c_int, C.c_void_p, C.c_void_p, P(C.c_double), P(C.c_double)]
    L.ow_max_threads.restype = C.c_int
    L.ow_impnet_params.restype = C.c_int
    L.ow_impnet_eval.argtypes = [C.c_void_p, C.c_void_p, C.c_int, C.c_void_p]
    L.ow_impnet_loss_grad.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int, C.c_void_p]
    L.ow_impnet_loss_grad.restype = C.c_double
    L.ow_mpc_cost.argtypes = [P(OWorld), C.c_int] + [C.c_void_p] * 4 + [P(C.c_double), P(C.c_double)]
    return L


def lib():
    global _lib
    with _lock:
        if _lib is None:
            _lib = load(build())
    return _lib


def _p(a):
    return a.ctypes.data_as(C.c_void_p)


class World:
    """Owns contiguous copies of one world's description and the ctypes struct pointing at them."""

    _INT = ("body_parent", "body_jnt", "geom_type", "geom_body")

    # optional per-body arrays: absent means no joint limits and no joint friction
    _OPTIONAL = {"body_range": 2, "body_frictionloss": 1}

    def __init__(self, desc):
        self.arrays = {}
        nb = len(desc["body_parent"])
        for k in OWorld._fields_[2:]:
            name = k[0]
            dt = np.int32 if name in self._INT else np.float64
            val = desc.get(name)
            if val is None:
                val = np.zeros(nb * self._OPTIONAL[name])
            self.arrays[name] = np.ascontiguousarray(np.asarray(val, dtype=dt).reshape(-1))
        self.s = OWorld(len(self.arrays["body_parent"]), len(self.arrays["geom_type"]),
                        *[_p(self.arrays[k[0]]) for k in OWorld._fields_[2:]])
        nq, nv = C.c_int(), C.c_int()
        if lib().ow_sizes(C.byref(self.s), C.byref(nq), C.byref(nv)):
            raise ValueError("unsupported world structure")
        self.nq, self.nv = nq.value, nv.value


class _ParamsStruct(OParams):
    """OParams that also keeps the learned impedance's parameter array alive."""


def params_struct(p, impnet=None):
    """impnet: the learned impedance's parameters (trace_mode 3), else None."""
    s = _ParamsStruct()
    s.gravity[:] = list(p.gravity)
    s.k_user, s.d_user = p.k_user, p.d_user
    s.solimp[:] = list(p.solimp)
    s.margin = p.margin
    s.n_t, s.n_tor, s.n_rol, s.trace_mode = p.n_t, p.n_tor, p.n_rol, p.trace_mode
    if p.trace_mode == 3:
        if impnet is None:
            raise ValueError("trace_mode 3 needs the impedance network's parameters")
        s._theta = np.ascontiguousarray(impnet, np.float64).reshape(-1)
        if s._theta.size != impnet_params():
            raise ValueError("wrong number of impedance network parameters")
        s.impnet = s._theta.ctypes.data
    return s


def step(desc, params, dt, nsteps, q, v, tau=None, impnet=None):
    """Advance one world; returns (q, v, total contacts over the steps).  tau: [nsteps, nv] or None;
    impnet: the learned impedance's parameters when params.trace_mode == 3."""
    w = desc if isinstance(desc, World) else World(desc)
    q = np.array(q, dtype=np.float64).copy()
    v = np.array(v, dtype=np.float64).copy()
    t = None if tau is None else np.ascontiguousarray(np.asarray(tau, np.float64).reshape(nsteps, w.nv))
    nc = C.c_int()
    ps = params_struct(params, impnet)
    rc = lib().ow_step(C.byref(w.s), C.byref(ps), dt, nsteps, _p(q), _p(v), None if t is None else _p(t),
                       C.byref(nc))
    if rc:
        raise RuntimeError("oracle step failed (mass matrix not positive definite?)")
    return q, v, nc.value


def step_record(desc, params, dt, q, v, tau=None, cap=20000, impnet=None):
    """One step with its intermediates: dict(q, v, vs, p, c, contacts=[dict]).  Each contact also
    carries the learned impedance's inputs `feat` and the mean exact facet impedance `m_exact`."""
    w = desc if isinstance(desc, World) else World(desc)
    q = np.array(q, dtype=np.float64).copy()
    v = np.array(v, dtype=np.float64).copy()
    vs, pg, cb = np.zeros(w.nv), np.zeros(w.nv), np.zeros(w.nv)
    cs = (OContact * cap)()
    n = C.c_int()
    t = None if tau is None else np.ascontiguousarray(np.asarray(tau, np.float64))
    ps = params_struct(params, impnet)
    rc = lib().ow_step_record(C.byref(w.s), C.byref(ps), dt, _p(q), _p(v), None if t is None else _p(t), _p(vs),
                              _p(pg), _p(cb), cs, cap, C.byref(n))
    if rc:
        raise RuntimeError("oracle step failed")
    contacts = []
    for i in range(min(n.value, cap)):
        k = cs[i]
        contacts.append(dict(geom_a=k.geom_a, geom_b=k.geom_b, body_a=k.body_a, body_b=k.body_b, sub=k.sub, phi=k.phi,
                             pos=np.array(k.pos[:]), normal=np.array(k.normal[:]), t1=np.array(k.t1[:]),
                             t2=np.array(k.t2[:]), trace_a=k.trace_a, trace_b=k.trace_b, r=k.r, mphi=k.mphi,
                             lam_sum=k.lam_sum, wrench=np.array(k.wrench[:]), nfacet=k.nfacet,
                             nactive=k.nactive, feat=np.array(k.feat[:]), m_exact=k.m_exact))
    return dict(q=q, v=v, vs=vs, p=pg, c=cb, contacts=contacts)


def dynamics(desc, gravity, q, v):
    """(M dense [nv, nv], c [nv], poses [nbody, 15] = x, R row-major, com)."""
    w = desc if isinstance(desc, World) else World(desc)
    q = np.ascontiguousarray(q, dtype=np.float64)
    v = np.ascontiguousarray(v, dtype=np.float64)
    M = np.zeros((w.nv, w.nv))
    c = np.zeros(w.nv)
    poses = np.zeros((len(w.arrays["body_parent"]), 15))
    g = np.ascontiguousarray(gravity, dtype=np.float64)
    if lib().ow_dynamics(C.byref(w.s), _p(g), _p(q), _p(v), _p(M), _p(c), _p(poses)):
        raise RuntimeError("oracle dynamics failed")
    return M, c, poses


def cholesky(A):
    a = np.ascontiguousarray(A, dtype=np.float64).copy()
    if lib().ow_cholesky(_p(a), a.shape[0]):
        raise np.linalg.LinAlgError("not positive definite")
    return a


def capsule_box_param(x0, w, h, half):
    x0 = np.ascontiguousarray(x0, np.float64)
    w = np.ascontiguousarray(w, np.float64)
    half = np.ascontiguousarray(half, np.float64)
    return lib().ow_capsule_box_param(_p(x0), _p(w), float(h), _p(half))


def solimp_r(aphi, solimp):
    s = np.ascontiguousarray(solimp, np.float64)
    return lib().ow_solimp_r(float(aphi), _p(s))


def rollout_loss_dir(desc, params, dt, q0, v0, tau, dq0, dv0, dtau, body, target_pos, target_quat, impnet=None):
    """(L, dL/d(direction)) for the free body `body` after len(tau) steps (forward-mode duals);
    impnet: the learned impedance's parameters when params.trace_mode == 3."""
    w = desc if isinstance(desc, World) else World(desc)
    T = len(tau)
    arr = [np.ascontiguousarray(a, np.float64) for a in (q0, v0, tau, dq0, dv0, dtau, target_pos, target_quat)]
    L, dL = C.c_double(), C.c_double()
    ps = params_struct(params, impnet)
    rc = lib().ow_rollout_loss_dir(C.byref(w.s), C.byref(ps), dt, T, _p(arr[0]), _p(arr[1]), _p(arr[2]),
                                   _p(arr[3]), _p(arr[4]), _p(arr[5]), body, _p(arr[6]), _p(arr[7]), C.byref(L),
                                   C.byref(dL))
    if rc:
        raise RuntimeError("oracle rollout failed")
    return L.value, dL.value


MPC_WEIGHTS = ("w_quat", "w_pos", "w_contact", "w_joint", "w_fallen", "fall_radius", "term_pos", "term_quat")


def mpc_cost(desc, q, goal, qref, weights, cost_body=0):
    """(running, terminal) MPC cost of state q (Sec. V, Eq. mpc): goal = target position and
    quaternion of the free body `cost_body`, qref = home pose (hinge entries), weights = any
    object with the attributes in MPC_WEIGHTS."""
    w = desc if isinstance(desc, World) else World(desc)
    q = np.ascontiguousarray(q, np.float64)
    g = np.ascontiguousarray(goal, np.float64)
    r = np.ascontiguousarray(qref, np.float64)
    wt = np.array([float(getattr(weights, k)) for k in MPC_WEIGHTS], np.float64)
    run, term = C.c_double(), C.c_double()
    if lib().ow_mpc_cost(C.byref(w.s), cost_body, _p(q), _p(g), _p(r), _p(wt), C.byref(run), C.byref(term)):
        raise RuntimeError("oracle mpc cost failed")
    return run.value, term.value


class BatchRunner:
    """Steps many worlds in parallel with OpenMP (the timed CPU baseline)."""

    def __init__(self, descs, params, impnet=None):
        self.worlds = [d if isinstance(d, World) else World(d) for d in descs]
        self.ptrs = (C.c_void_p * len(self.worlds))(*[C.cast(C.pointer(w.s), C.c_void_p) for w in self.worlds])
        self.params = params_struct(params, impnet)
        self.qadr = np.cumsum([0] + [w.nq for w in self.worlds[:-1]]).astype(np.int64)
        self.vadr = np.cumsum([0] + [w.nv for w in self.worlds[:-1]]).astype(np.int64)

    def run(self, q, v, dt, nsteps, nthreads=0):
        contacts = np.zeros(len(self.worlds), np.int64)
        fails = lib().ow_step_batch(len(self.worlds), self.ptrs, C.byref(self.params), dt, nsteps, _p(q),
                                    _p(self.qadr), _p(v), _p(self.vadr), _p(contacts), nthreads)
        if fails:
            raise RuntimeError(f"{fails} oracle worlds failed")
        return contacts


def max_threads():
    return lib().ow_max_threads()


# ---------------------------------------------------------------------------------------------
# learned impedance (Sec. III-B): the network, its loss and the optimiser that fits it
# ---------------------------------------------------------------------------------------------
def impnet_params():
    """Number of parameters of the learned impedance network."""
    return lib().ow_impnet_params()


def impnet_eval(theta, x):
    """g(x) for x[n, 4] (unclamped)."""
    th = np.ascontiguousarray(theta, np.float64)
    x = np.ascontiguousarray(x, np.float64).reshape(-1, 4)
    out = np.zeros(len(x))
    lib().ow_impnet_eval(_p(th), _p(x), len(x), _p(out))
    return out


def impnet_loss_grad(theta, x, y):
    """(L, dL/dtheta) of the mean squared error (1/n) sum (g(x_i) - y_i)^2."""
    th = np.ascontiguousarray(theta, np.float64)
    x = np.ascontiguousarray(x, np.float64).reshape(-1, 4)
    y = np.ascontiguousarray(y, np.float64)
    g = np.zeros(th.size)
    L = lib().ow_impnet_loss_grad(_p(th), _p(x), _p(y), len(x), _p(g))
    return L, g


def impnet_adam(theta, x, y, iters, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """Full-batch Adam (Kingma and Ba, ICLR 2015, Algorithm 1, with the bias corrections
    applied to the moments) on the mean squared error; returns (theta, losses before each
    update)."""
    th = np.array(theta, np.float64)
    m = np.zeros_like(th)
    v = np.zeros_like(th)
    losses = []
    for t in range(1, iters + 1):
        L, g = impnet_loss_grad(th, x, y)
        losses.append(L)
        m = beta1 * m + (1 - beta1) * g
        v = beta2 * v + (1 - beta2) * g * g
        mh = m / (1 - beta1 ** t)
        vh = v / (1 - beta2 ** t)
        th = th - lr * mh / (np.sqrt(vh) + eps)
    return th, np.array(losses)
