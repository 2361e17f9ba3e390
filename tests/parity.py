"""Helpers shared by the GPU parity tests: oracle-advanced states, GPU runs through the C ABI,
and the error measures the tolerances are stated in.

Relative velocity error of a world: max_i |v_gpu,i - v_oracle,i| / (max_i |v_oracle,i| + g dt),
over all velocity coordinates of the world (the floor g dt is the velocity change gravity makes
in one step, so resting worlds are not measured against round-off).
"""
import numpy as np
import torch

from oracle import oracle as O
from paper_2603_12185_gb300 import comfree as CF
from paper_2603_12185_gb300 import scenes as S

G = 9.81


def f32(x):
    return np.asarray(x, np.float32).astype(np.float64)


def with_states(sb, qs, vs):
    out = sb.subset(range(sb.nworld))
    out.q0 = [f32(q) for q in qs]
    out.v0 = [f32(v) for v in vs]
    return out


def tau_full(sb, w, tau_u):
    """Generalised force vector of world w from its actuated-hinge controls."""
    t = sb.template_of(w)
    full = np.zeros(t.nv)
    k = 0
    off = 0
    for b in range(t.nbody):
        if t.body_jnt[b] == S.HINGE:
            full[off] = tau_u[k]
            k += 1
            off += 1
        else:
            off += 6
    return full


def oracle_run(sb, worlds=None, nsteps=1, ctrl=None):
    """Advance worlds with the oracle from sb's states; ctrl: per world [nsteps, nu] or None."""
    worlds = range(sb.nworld) if worlds is None else worlds
    qs, vs = [], []
    for w in worlds:
        d = sb.world(w)
        tau = None
        if ctrl is not None and ctrl[w] is not None and sb.template_of(w).nu:
            tau = np.stack([tau_full(sb, w, ctrl[w][s]) for s in range(nsteps)])
        q, v, _ = O.step(d, sb.params, sb.dt, nsteps, sb.q0[w], sb.v0[w], tau)
        qs.append(q)
        vs.append(v)
    return qs, vs


def gpu_run(sb, nsteps=1, ctrl=None, capture=0, warps=None, calls=1):
    """Run `calls` launches of `nsteps` steps on the GPU; returns per-world (q, v) and the batch."""
    T = nsteps
    m, b = CF.from_scenes(sb, max_ctrl_steps=max(T, 1), contact_capture=capture)
    if warps:
        for s, wp in warps.items():
            b.set_warps(s, wp)
    if ctrl is not None and b.total_nu:
        seq = np.zeros((T, b.total_nu), np.float32)
        off = 0
        for w in range(sb.nworld):
            nu = sb.template_of(w).nu
            if nu:
                seq[:, off:off + nu] = ctrl[w][:T]
            off += nu
        b.set_ctrl(torch.from_numpy(seq.reshape(-1)).cuda())
    for _ in range(calls):
        b.step(sb.dt, nsteps)
    q, v = b.get_state()
    torch.cuda.synchronize()
    q, v = q.cpu().numpy().astype(np.float64), v.cpu().numpy().astype(np.float64)
    qs, vs = [], []
    qo = vo = 0
    for w in range(sb.nworld):
        t = sb.template_of(w)
        qs.append(q[qo:qo + t.nq])
        vs.append(v[vo:vo + t.nv])
        qo += t.nq
        vo += t.nv
    return qs, vs, b


def vel_err(vg, vo, dt):
    return np.abs(vg - vo).max() / (np.abs(vo).max() + G * dt)


def geom_offsets(sb):
    off, acc = [], 0
    for t in sb.templates:
        off.append(acc)
        acc += t.ngeom
    return off


def oracle_fp32_state(sb, nsteps, snapshots):
    """The FP64 oracle stepped one step at a time with its state rounded to FP32 after every step
    (as the GPU stores it in HBM between steps), worlds spread over the host cores.  Returns
    {step: (qs, vs)} at the requested snapshot steps, plus the same for the plain FP64 oracle:
    (fp32_state, fp64).  Where the two part by more than the comparison's tolerance, the
    dynamics themselves amplify FP32 rounding of the state past it, and no FP32 implementation
    can be held to that tolerance there."""
    runner = O.BatchRunner([sb.world(w) for w in range(sb.nworld)], sb.params)
    nq, nv = len(sb.q0[0]), len(sb.v0[0])
    q32 = np.concatenate([f32(x) for x in sb.q0])
    v32 = np.concatenate([f32(x) for x in sb.v0])
    q64, v64 = q32.copy(), v32.copy()
    out32, out64 = {}, {}
    done = 0
    for s in sorted(snapshots):
        runner.run(q64, v64, sb.dt, s - done)
        for _ in range(s - done):
            runner.run(q32, v32, sb.dt, 1)
            q32[:] = q32.astype(np.float32)
            v32[:] = v32.astype(np.float32)
        done = s
        split = lambda a, n: [a[i * n:(i + 1) * n].copy() for i in range(sb.nworld)]
        out32[s] = (split(q32, nq), split(v32, nv))
        out64[s] = (split(q64, nq), split(v64, nv))
    return out32, out64
