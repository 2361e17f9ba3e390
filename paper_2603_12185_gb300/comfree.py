"""Thin Python binding of libcomfree (include/comfree.h): argument marshalling only.

Every step of the simulation runs in the library's CUDA kernels; PyTorch provides the device
memory (the batch workspace and state tensors) and the stream.  There is no CPU fallback:
loading fails loudly when libcomfree.so has not been built.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np
import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libcomfree.so")

CF_OK = 0
STATUS = {0: "CF_OK", 1: "CF_ERR_INVALID_ARGUMENT", 2: "CF_ERR_OUT_OF_MEMORY", 3: "CF_ERR_CUDA",
          4: "CF_ERR_CONTACT_OVERFLOW", 5: "CF_ERR_NONFINITE", 6: "CF_ERR_TIMEOUT", 7: "CF_ERR_UNSUPPORTED"}


class CfError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class SceneDesc(C.Structure):
    _fields_ = [("nbody", C.c_int32), ("ngeom", C.c_int32)] + [
        (n, C.c_void_p) for n in ("body_parent", "body_jnt", "body_pos", "body_quat", "body_axis", "body_ipos",
                                  "body_mass", "body_inertia", "body_damping", "geom_type", "geom_body", "geom_pos",
                                  "geom_quat", "geom_size", "geom_mu")] + [("pile", C.c_int32)] + [
        (n, C.c_void_p) for n in ("body_range", "body_frictionloss")]


class ModelDesc(C.Structure):
    _fields_ = [("nscene", C.c_int32), ("scenes", C.POINTER(SceneDesc)), ("gravity", C.c_double * 3),
                ("k_user", C.c_double), ("d_user", C.c_double), ("solimp", C.c_double * 5), ("margin", C.c_double),
                ("n_t", C.c_int32), ("n_tor", C.c_int32), ("n_rol", C.c_int32), ("trace_mode", C.c_int32)]


class BatchOpts(C.Structure):
    _fields_ = [("max_ctrl_steps", C.c_int32), ("contact_capture", C.c_int32), ("grad_steps", C.c_int32),
                ("grad_ckpt", C.c_int32)]


class Contact(C.Structure):
    _fields_ = [("geom_a", C.c_int32), ("geom_b", C.c_int32), ("sub", C.c_int32), ("flags", C.c_int32),
                ("phi", C.c_float), ("pos", C.c_float * 3), ("normal", C.c_float * 3), ("lam_sum", C.c_float),
                ("mphi", C.c_float), ("rho", C.c_float), ("wn", C.c_float), ("target", C.c_float)]


CONTACT_DTYPE = np.dtype([("geom_a", np.int32), ("geom_b", np.int32), ("sub", np.int32), ("flags", np.int32),
                          ("phi", np.float32), ("pos", np.float32, 3), ("normal", np.float32, 3),
                          ("lam_sum", np.float32), ("mphi", np.float32), ("rho", np.float32),
                          ("wn", np.float32), ("target", np.float32)])
CONTACT_B_STATIC = 1


class CostDesc(C.Structure):
    _fields_ = [("body", C.c_int32), ("w_quat", C.c_float), ("w_pos", C.c_float), ("w_contact", C.c_float),
                ("w_joint", C.c_float), ("w_fallen", C.c_float), ("fall_radius", C.c_float), ("term_pos", C.c_float),
                ("term_quat", C.c_float)]


EXPORTS = ("cf_model_create", "cf_model_destroy", "cf_scene_sizes", "cf_batch_workspace_bytes", "cf_batch_create",
           "cf_batch_destroy", "cf_batch_sizes", "cf_set_state", "cf_get_state", "cf_set_ctrl", "cf_step", "cf_step_host",
           "cf_get_contact_counts", "cf_get_contacts", "cf_batch_status", "cf_batch_autotune", "cf_batch_set_warps",
           "cf_step_grad", "cf_step_noalloc", "cf_status_string", "cf_last_error", "cf_mlp_workspace_bytes",
           "cf_mlp_create", "cf_mlp_destroy", "cf_mlp_param_count", "cf_mlp_forward", "cf_mlp_gradients",
           "cf_mlp_train_step", "cf_mlp_get_params", "cf_mlp_status", "cf_set_cost", "cf_mppi_sample",
           "cf_mppi_update", "cf_mppi_shift", "cf_mppi_blend", "cf_broadcast_state", "cf_mppi_features",
           "cf_batch_set_impedance_net", "cf_impnet_eval", "cf_impnet_state_floats", "cf_impnet_loss_grad",
           "cf_impnet_fit")

_lib = None


def lib():
    """Load libcomfree.so (raises if it has not been built: there is no fallback path)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: build it with `python -m paper_2603_12185_gb300.build`")
    L = C.CDLL(LIB_PATH)
    P, V, I32, I64 = C.POINTER, C.c_void_p, C.c_int32, C.c_int64
    L.cf_model_create.argtypes = [P(ModelDesc), P(V)]
    L.cf_model_destroy.argtypes = [V]
    L.cf_model_destroy.restype = None
    L.cf_scene_sizes.argtypes = [V, I32, P(I32)]
    L.cf_batch_workspace_bytes.argtypes = [V, I32, V, P(BatchOpts), P(C.c_size_t)]
    L.cf_batch_create.argtypes = [V, I32, V, V, P(BatchOpts), V, C.c_size_t, V, P(V)]
    L.cf_batch_destroy.argtypes = [V]
    L.cf_batch_destroy.restype = None
    L.cf_batch_sizes.argtypes = [V, P(I64), P(I64), P(I64)]
    L.cf_set_state.argtypes = [V, V, V, I32, V]
    L.cf_get_state.argtypes = [V, V, V, I32, V]
    L.cf_set_ctrl.argtypes = [V, V, I32, I32, V]
    L.cf_step.argtypes = [V, V, I32, C.c_float, I32, V]
    L.cf_step_host.argtypes = [V, V, V, C.c_float, I32, V]
    L.cf_get_contact_counts.argtypes = [V, V, I32, V]
    L.cf_get_contacts.argtypes = [V, V, V, V]
    L.cf_batch_status.argtypes = [V, V, I32, V]
    L.cf_batch_autotune.argtypes = [V, C.c_float, V, V]
    L.cf_batch_set_warps.argtypes = [V, I32, I32]
    L.cf_step_grad.argtypes = [V, I32, C.c_float, V, V, V, V, V, V]
    L.cf_step_noalloc.argtypes = [V, I32, I32, V, V, V, C.c_float, I32, V, V]
    L.cf_mlp_workspace_bytes.argtypes = [I32, I32, I32, I32, P(C.c_size_t)]
    L.cf_mlp_create.argtypes = [I32, I32, I32, I32, V, V, C.c_size_t, V, P(V)]
    L.cf_mlp_destroy.argtypes = [V]
    L.cf_mlp_destroy.restype = None
    L.cf_mlp_param_count.argtypes = [V, P(I64)]
    L.cf_mlp_forward.argtypes = [V, V, I32, V, V]
    L.cf_mlp_gradients.argtypes = [V, V, V, I32, C.c_float, C.c_float, V, V, V]
    L.cf_mlp_train_step.argtypes = [V, V, V, I32, C.c_float, C.c_float, C.c_float, V, V]
    L.cf_mlp_get_params.argtypes = [V, V, V]
    L.cf_mlp_status.argtypes = [V, V]
    L.cf_set_cost.argtypes = [V, P(CostDesc), V, V, V]
    L.cf_mppi_sample.argtypes = [I32, I32, I32, V, V, C.c_float, C.c_float, V, V, I32, V, V, V]
    L.cf_mppi_update.argtypes = [I32, I32, I32, V, V, C.c_float, V, V, V]
    L.cf_mppi_shift.argtypes = [I32, I32, V, V]
    L.cf_mppi_blend.argtypes = [I32, V, V, C.c_float, V, V]
    L.cf_broadcast_state.argtypes = [V, V, I32, I32, I32, V, V, V]
    L.cf_mppi_features.argtypes = [V, I32, V, I32, C.c_float, V, I32, C.c_float, V, V]
    L.cf_batch_set_impedance_net.argtypes = [V, V, I32]
    L.cf_impnet_eval.argtypes = [V, V, I32, V, V]
    L.cf_impnet_state_floats.argtypes = []
    L.cf_impnet_state_floats.restype = C.c_size_t
    L.cf_impnet_loss_grad.argtypes = [V, V, V, I32, V, V, V, V]
    L.cf_impnet_fit.argtypes = [V, V, I32, V, V, I32, I32, C.c_float, V, V]
    L.cf_status_string.argtypes = [I32]
    L.cf_status_string.restype = C.c_char_p
    L.cf_last_error.argtypes = []
    L.cf_last_error.restype = C.c_char_p
    _lib = L
    return L


def check(status):
    if status != CF_OK:
        raise CfError(status, lib().cf_last_error().decode())


def _stream(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


def _ptr(t):
    if t is None:
        return None
    if isinstance(t, torch.Tensor):
        return C.c_void_p(t.data_ptr())
    return t.ctypes.data_as(C.c_void_p)


class Model:
    """A validated model built from scene templates (scenes.Template) and parameters (scenes.Params)."""

    _INT = ("body_parent", "body_jnt", "geom_type", "geom_body")

    def __init__(self, templates, params):
        keep = []
        descs = (SceneDesc * len(templates))()
        required = [n for n, _ in SceneDesc._fields_[2:17]]
        optional = ("body_range", "body_frictionloss")
        for i, t in enumerate(templates):
            arrs = {}
            for name in required + list(optional):
                val = getattr(t, name, None)
                if val is None:
                    arrs[name] = None
                    continue
                a = np.ascontiguousarray(val, dtype=np.int32 if name in self._INT else np.float64)
                arrs[name] = a
                keep.append(a)
            descs[i] = SceneDesc(len(t.body_parent), len(t.geom_type), *[_ptr(arrs[n]) for n in required],
                                 int(bool(t.pile)), *[_ptr(arrs[n]) for n in optional])
        d = ModelDesc()
        d.nscene = len(templates)
        d.scenes = descs
        d.gravity[:] = list(params.gravity)
        d.k_user, d.d_user = params.k_user, params.d_user
        d.solimp[:] = list(params.solimp)
        d.margin = params.margin
        d.n_t, d.n_tor, d.n_rol, d.trace_mode = params.n_t, params.n_tor, params.n_rol, params.trace_mode
        h = C.c_void_p()
        check(lib().cf_model_create(C.byref(d), C.byref(h)))
        self.h = h
        self.templates = templates
        self.params = params

    def scene_sizes(self, scene):
        s = (C.c_int32 * 5)()
        check(lib().cf_scene_sizes(self.h, scene, s))
        return dict(nq=s[0], nv=s[1], nu=s[2], nbody=s[3], ngeom=s[4])

    def __del__(self):
        if getattr(self, "h", None) and _lib is not None:
            _lib.cf_model_destroy(self.h)
            self.h = None


class Batch:
    """W worlds stepped on the GPU inside a caller-owned (torch) device workspace."""

    def __init__(self, model, scene_of_world, world_params=None, max_ctrl_steps=1, contact_capture=0, grad_steps=0,
                 grad_ckpt=10, device="cuda", stream=None):
        self.model = model
        self.scene_of_world = np.ascontiguousarray(scene_of_world, dtype=np.int32)
        self.W = len(self.scene_of_world)
        self.opts = BatchOpts(max_ctrl_steps, contact_capture, grad_steps, grad_ckpt)
        nbytes = C.c_size_t()
        check(lib().cf_batch_workspace_bytes(model.h, self.W, _ptr(self.scene_of_world), C.byref(self.opts),
                                             C.byref(nbytes)))
        self.workspace = torch.empty(nbytes.value + 256, dtype=torch.uint8, device=device)
        off = (-self.workspace.data_ptr()) % 256
        self.ws_ptr = self.workspace.data_ptr() + off
        wp = None if world_params is None else np.ascontiguousarray(world_params, dtype=np.float32)
        h = C.c_void_p()
        check(lib().cf_batch_create(model.h, self.W, _ptr(self.scene_of_world), _ptr(wp), C.byref(self.opts),
                                    C.c_void_p(self.ws_ptr), nbytes.value, _stream(stream), C.byref(h)))
        self.h = h
        nq, nv, nu = C.c_int64(), C.c_int64(), C.c_int64()
        check(lib().cf_batch_sizes(h, C.byref(nq), C.byref(nv), C.byref(nu)))
        self.total_nq, self.total_nv, self.total_nu = nq.value, nv.value, nu.value
        self.device = device

    def __del__(self):
        if getattr(self, "h", None) and _lib is not None:
            _lib.cf_batch_destroy(self.h)
            self.h = None

    # ---- state ----
    def set_state_async(self, q, v, stream=None):
        """Enqueue the copy of pinned host tensors q, v on `stream` and return (cf_set_state mode 2)."""
        assert q.is_pinned() and v.is_pinned() and q.numel() == self.total_nq and v.numel() == self.total_nv
        check(lib().cf_set_state(self.h, _ptr(q), _ptr(v), 2, _stream(stream)))

    def get_state_async(self, q, v, stream=None):
        """Enqueue the copy of the state into pinned host tensors q, v on `stream` and return."""
        assert q.is_pinned() and v.is_pinned() and q.numel() == self.total_nq and v.numel() == self.total_nv
        check(lib().cf_get_state(self.h, _ptr(q), _ptr(v), 2, _stream(stream)))

    def set_state(self, q, v, stream=None):
        on_dev = isinstance(q, torch.Tensor) and q.is_cuda
        if on_dev:
            q = q.contiguous().float()
            v = v.contiguous().float()
        else:
            q = np.ascontiguousarray(q, dtype=np.float32)
            v = np.ascontiguousarray(v, dtype=np.float32)
        assert (q.numel() if on_dev else q.size) == self.total_nq
        check(lib().cf_set_state(self.h, _ptr(q), _ptr(v), int(on_dev), _stream(stream)))

    def get_state(self, out_q=None, out_v=None, stream=None):
        """Device tensors by default; host numpy arrays when the outputs given are numpy/pinned CPU."""
        if out_q is None:
            out_q = torch.empty(self.total_nq, dtype=torch.float32, device=self.device)
            out_v = torch.empty(self.total_nv, dtype=torch.float32, device=self.device)
        on_dev = isinstance(out_q, torch.Tensor) and out_q.is_cuda
        check(lib().cf_get_state(self.h, _ptr(out_q), _ptr(out_v), int(on_dev), _stream(stream)))
        return out_q, out_v

    def set_ctrl(self, tau, stream=None):
        on_dev = isinstance(tau, torch.Tensor) and tau.is_cuda
        if on_dev:
            tau = tau.contiguous().float()
            T = tau.numel() // max(self.total_nu, 1)
        else:
            tau = np.ascontiguousarray(tau, dtype=np.float32)
            T = tau.size // max(self.total_nu, 1)
        check(lib().cf_set_ctrl(self.h, _ptr(tau), T, int(on_dev), _stream(stream)))

    def step(self, dt, nsteps=1, worlds=None, stream=None):
        wl = None if worlds is None else np.ascontiguousarray(worlds, dtype=np.int32)
        check(lib().cf_step(self.h, _ptr(wl), 0 if wl is None else len(wl), float(dt), int(nsteps), _stream(stream)))

    def step_host(self, q, v, dt, nsteps=1, stream=None):
        """Step every world with the state in pinned host tensors q[total_nq], v[total_nv]: the
        step kernel reads them and writes the new state back in place (cf_step_host); the
        batch's own device state is untouched.  Asynchronous on `stream`."""
        assert q.is_pinned() and v.is_pinned() and q.dtype == torch.float32 and v.dtype == torch.float32
        assert q.is_contiguous() and v.is_contiguous() and q.numel() == self.total_nq and v.numel() == self.total_nv
        check(lib().cf_step_host(self.h, _ptr(q), _ptr(v), float(dt), int(nsteps), _stream(stream)))

    def graph(self, dt, nsteps=1, repeat=1):
        """A CUDA graph of `repeat` all-world cf_step launches (dt, nsteps each); replay() runs
        them again on the current stream.  One eager step first sets the kernel attributes, so
        the batch advances by nsteps here."""
        self.step(dt, nsteps)
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            for _ in range(repeat):
                self.step(dt, nsteps)
        return g

    def contact_counts(self, stream=None):
        out = np.zeros(self.W, np.int32)
        check(lib().cf_get_contact_counts(self.h, _ptr(out), 0, _stream(stream)))
        return out

    def contact_counts_device(self, out, stream=None):
        check(lib().cf_get_contact_counts(self.h, _ptr(out), 1, _stream(stream)))
        return out

    def set_impedance_net(self, theta, n_sets=1):
        """Learned impedance of trace_mode 3 (cf_batch_set_impedance_net): theta is a device
        tensor [n_sets, 49] (n_sets 1 or the number of worlds), kept referenced here; None
        detaches it."""
        if theta is None:
            self._impnet = None
            check(lib().cf_batch_set_impedance_net(self.h, None, 0))
            return
        assert theta.is_cuda and theta.dtype == torch.float32 and theta.is_contiguous()
        assert theta.numel() == n_sets * IMPNET_PARAMS
        self._impnet = theta
        check(lib().cf_batch_set_impedance_net(self.h, _ptr(theta), int(n_sets)))

    def contacts_array(self, stream=None):
        """The captured contacts as one numpy record array (CONTACT_DTYPE) and the per-world
        counts (needs contact_capture > 0)."""
        cap = self.opts.contact_capture
        buf = np.zeros(self.W * cap, CONTACT_DTYPE)
        counts = np.zeros(self.W, np.int32)
        check(lib().cf_get_contacts(self.h, buf.ctypes.data_as(C.c_void_p), _ptr(counts), _stream(stream)))
        keep = (np.arange(cap)[None, :] < np.minimum(counts, cap)[:, None]).reshape(-1)
        return buf[keep], counts

    def contacts(self, stream=None):
        """List (per world) of captured contacts as dicts (needs contact_capture > 0)."""
        cap = self.opts.contact_capture
        buf = (Contact * (self.W * cap))()
        counts = np.zeros(self.W, np.int32)
        check(lib().cf_get_contacts(self.h, buf, _ptr(counts), _stream(stream)))
        out = []
        for w in range(self.W):
            lst = []
            for i in range(counts[w]):
                c = buf[w * cap + i]
                lst.append(dict(geom_a=c.geom_a, geom_b=c.geom_b, sub=c.sub, phi=c.phi, pos=np.array(c.pos[:]),
                                normal=np.array(c.normal[:]), lam_sum=c.lam_sum, mphi=c.mphi, rho=c.rho,
                                wn=c.wn, target=c.target, b_static=bool(c.flags & CONTACT_B_STATIC)))
            out.append(lst)
        return out

    def status(self, clear=False, stream=None):
        flags = np.zeros(self.W, np.int32)
        st = lib().cf_batch_status(self.h, _ptr(flags), int(clear), _stream(stream))
        return st, flags

    def autotune(self, dt, stream=None):
        chosen = np.zeros(len(self.model.templates), np.int32)
        check(lib().cf_batch_autotune(self.h, float(dt), _stream(stream), _ptr(chosen)))
        return chosen

    def set_warps(self, scene, warps):
        check(lib().cf_batch_set_warps(self.h, int(scene), int(warps)))

    def set_cost(self, desc, goals, qref, costs):
        """Fused MPC cost (CostDesc or None to switch off); goals [W, 7], qref [total_nq], costs [W] on device."""
        self._cost_refs = (goals, qref, costs)
        if desc is None:
            check(lib().cf_set_cost(self.h, None, None, None, None))
        else:
            check(lib().cf_set_cost(self.h, C.byref(desc), _ptr(goals), _ptr(qref), _ptr(costs)))

    def step_grad(self, T, dt, dqT, dvT, stream=None):
        dq0 = torch.empty(self.total_nq, dtype=torch.float32, device=self.device)
        dv0 = torch.empty(self.total_nv, dtype=torch.float32, device=self.device)
        dtau = torch.zeros(max(T * self.total_nu, 1), dtype=torch.float32, device=self.device)
        check(lib().cf_step_grad(self.h, int(T), float(dt), _ptr(dqT.contiguous()), _ptr(dvT.contiguous()), _ptr(dq0),
                                 _ptr(dv0), _ptr(dtau), _stream(stream)))
        return dq0, dv0, dtau[:T * self.total_nu].view(T, self.total_nu) if self.total_nu else dtau[:0]


class Pipeline:
    """Steps blocks of worlds (one Batch per block) from and back to pinned host state, each
    block on its own stream, so that one block's host-to-device copy, step and device-to-host
    copy overlap the others'.  step() returns when every block's new state is in host memory."""

    def __init__(self, batches):
        self.batches = list(batches)
        self.streams = [torch.cuda.Stream() for _ in self.batches]

    def step(self, host_q, host_v, dt, nsteps=1):
        """host_q, host_v: per-block pinned CPU tensors, read and then overwritten in place."""
        for b, s, q, v in zip(self.batches, self.streams, host_q, host_v):
            b.set_state_async(q, v, stream=s)
            b.step(dt, nsteps, stream=s)
            b.get_state_async(q, v, stream=s)
        for s in self.streams:
            s.synchronize()

    def status(self):
        return [b.status() for b in self.batches]


def step_noalloc(model, scene, n_worlds, q, v, world_params, dt, nsteps, contacts=None, stream=None):
    """cf_step_noalloc on device tensors (q, v updated in place); no allocation by the library."""
    check(lib().cf_step_noalloc(model.h, int(scene), int(n_worlds), _ptr(q), _ptr(v), _ptr(world_params), float(dt),
                                int(nsteps), _ptr(contacts), _stream(stream)))


def flatten_state(sb):
    """Concatenated (q, v) of a scenes.Batch in world order (float32)."""
    return (np.concatenate([np.asarray(q, np.float32) for q in sb.q0]),
            np.concatenate([np.asarray(v, np.float32) for v in sb.v0]))


def flatten_params(sb):
    blocks = [p for p in sb.world_param if p is not None]
    if not blocks:
        return None
    return np.concatenate([np.asarray(p, np.float32).reshape(-1) for p in blocks])


def from_scenes(sb, **opts):
    """(Model, Batch) for a scenes.Batch with its initial state uploaded."""
    m = Model(sb.templates, sb.params)
    b = Batch(m, sb.world_scene, flatten_params(sb), **opts)
    q, v = flatten_state(sb)
    b.set_state(torch.from_numpy(q).cuda(), torch.from_numpy(v).cuda())
    return m, b


def mlp_param_shapes(fin, hidden, fout):
    kin = (fin + 63) // 64 * 64
    return [("W1", (hidden, kin)), ("b1", (hidden,)), ("W2", (hidden, hidden)), ("b2", (hidden,)),
            ("W3", (fout, hidden)), ("b3", (fout,))]


def mlp_init(fin, hidden, fout, seed=0, out_scale=0.1):
    """Seeded uniform fan-in initialisation (flat FP32, the library's parameter layout); the padding
    columns of W1 are zero and the output layer starts small."""
    rng = np.random.default_rng(seed)
    parts = []
    fans = {"W1": fin, "W2": hidden, "W3": hidden}
    for name, shape in mlp_param_shapes(fin, hidden, fout):
        if name.startswith("W"):
            lim = np.sqrt(6.0 / fans[name]) * (out_scale if name == "W3" else 1.0)
            w = rng.uniform(-lim, lim, shape)
            if name == "W1":
                w[:, fin:] = 0.0
            parts.append(w.reshape(-1))
        else:
            parts.append(np.zeros(shape))
    return np.concatenate(parts).astype(np.float32)


IMPNET_PARAMS = 49
IMPNET_INPUTS = 4


def impnet_init(seed=0, scale=0.5):
    """Initial learned-impedance parameters: first-layer weights ~ N(0, scale^2) (seeded),
    biases and output layer 0, so g = 0 (the heuristic) until it is fitted."""
    th = np.zeros(IMPNET_PARAMS, np.float32)
    th[:32] = np.random.default_rng(seed).normal(scale=scale, size=32)
    return th


def impedance_features(rec, solimp_width):
    """Inputs x[n, 4] of the learned impedance from captured contact records (CONTACT_DTYPE),
    the same features the step kernel forms: clamp(phi / width, -1, 1), the trace's rotational
    share rho, the free-body normal row over the trace wn, side B static."""
    x = np.empty((len(rec), IMPNET_INPUTS), np.float32)
    x[:, 0] = np.clip(rec["phi"] / np.float32(solimp_width), -1.0, 1.0)
    x[:, 1] = rec["rho"]
    x[:, 2] = rec["wn"]
    x[:, 3] = (rec["flags"] & CONTACT_B_STATIC) != 0
    return x


class ImpedanceNet:
    """Parameters of the learned impedance (trace_mode 3) on the device, with its Adam state
    (cf_impnet_*)."""

    def __init__(self, theta=None, seed=0, device="cuda"):
        th = impnet_init(seed) if theta is None else np.asarray(theta, np.float32).reshape(IMPNET_PARAMS)
        self.theta = torch.from_numpy(np.ascontiguousarray(th)).to(device)
        self.state = torch.zeros(int(lib().cf_impnet_state_floats()), dtype=torch.float32, device=device)
        self.steps = 0
        self.device = device

    @staticmethod
    def _x(x):
        x = x.contiguous().float()
        assert x.dim() == 2 and x.shape[1] == IMPNET_INPUTS and x.data_ptr() % 16 == 0
        return x

    def eval(self, x, stream=None):
        """g(x) (unclamped) at device inputs x[n, 4]."""
        x = self._x(x)
        g = torch.empty(x.shape[0], dtype=torch.float32, device=self.device)
        check(lib().cf_impnet_eval(_ptr(self.theta), _ptr(x), x.shape[0], _ptr(g), _stream(stream)))
        return g

    def loss_grad(self, x, y, stream=None):
        x = self._x(x)
        y = y.contiguous().float()
        g = torch.empty(IMPNET_PARAMS, dtype=torch.float32, device=self.device)
        L = torch.empty(1, dtype=torch.float32, device=self.device)
        check(lib().cf_impnet_loss_grad(_ptr(self.theta), _ptr(x), _ptr(y), x.shape[0], _ptr(self.state), _ptr(g),
                                        _ptr(L), _stream(stream)))
        return L, g

    def fit(self, x, y, iters, lr=0.02, stream=None):
        """iters full-batch Adam steps on the mean squared error; returns the losses (device)."""
        x = self._x(x)
        y = y.contiguous().float()
        losses = torch.empty(max(iters, 1), dtype=torch.float32, device=self.device)
        check(lib().cf_impnet_fit(_ptr(self.theta), _ptr(self.state), self.steps, _ptr(x), _ptr(y), x.shape[0],
                                  int(iters), float(lr), _ptr(losses), _stream(stream)))
        self.steps += iters
        return losses[:iters]


class Mlp:
    """The BF16 tensor-core MLP of the learned proposal (cf_mlp_*)."""

    def __init__(self, fin=49, hidden=256, fout=1024, max_batch=4096, params=None, seed=0, device="cuda", stream=None):
        self.fin, self.hidden, self.fout, self.max_batch = fin, hidden, fout, max_batch
        n = C.c_size_t()
        check(lib().cf_mlp_workspace_bytes(fin, hidden, fout, max_batch, C.byref(n)))
        self.workspace = torch.empty(n.value + 256, dtype=torch.uint8, device=device)
        off = (-self.workspace.data_ptr()) % 256
        p = mlp_init(fin, hidden, fout, seed) if params is None else np.asarray(params, np.float32)
        pt = torch.from_numpy(np.ascontiguousarray(p)).to(device)
        h = C.c_void_p()
        check(lib().cf_mlp_create(fin, hidden, fout, max_batch, _ptr(pt), C.c_void_p(self.workspace.data_ptr() + off),
                                  n.value, _stream(stream), C.byref(h)))
        self.h = h
        k = C.c_int64()
        check(lib().cf_mlp_param_count(h, C.byref(k)))
        self.nparam = k.value
        self.device = device
        self.loss = torch.zeros(1, dtype=torch.float32, device=device)

    def __del__(self):
        if getattr(self, "h", None) and _lib is not None:
            _lib.cf_mlp_destroy(self.h)
            self.h = None

    def forward(self, x, out=None, stream=None):
        x = x.contiguous().float()
        B = x.shape[0]
        out = torch.empty(B, self.fout, dtype=torch.float32, device=self.device) if out is None else out
        check(lib().cf_mlp_forward(self.h, _ptr(x), B, _ptr(out), _stream(stream)))
        return out

    def gradients(self, x, target, lo=-5.0, hi=2.0, stream=None):
        x = x.contiguous().float()
        target = target.contiguous().float()
        g = torch.empty(self.nparam, dtype=torch.float32, device=self.device)
        check(lib().cf_mlp_gradients(self.h, _ptr(x), _ptr(target), x.shape[0], lo, hi, _ptr(g), _ptr(self.loss),
                                     _stream(stream)))
        return g, self.loss

    def train_step(self, x, target, lr=1e-3, lo=-5.0, hi=2.0, stream=None):
        x = x.contiguous().float()
        target = target.contiguous().float()
        check(lib().cf_mlp_train_step(self.h, _ptr(x), _ptr(target), x.shape[0], lr, lo, hi, _ptr(self.loss),
                                      _stream(stream)))
        return self.loss

    def params(self, stream=None):
        p = torch.empty(self.nparam, dtype=torch.float32, device=self.device)
        check(lib().cf_mlp_get_params(self.h, _ptr(p), _stream(stream)))
        return p

    def status(self, stream=None):
        check(lib().cf_mlp_status(self.h, _stream(stream)))
