"""Learned impedance K(q), D(q) (Sec. III-B allows them to be learned instead of set by the
heuristic): data from the exact diagonal impedance, the fit, and its evaluation.

The paper names the exact form K dt + D = (1/dt) (J~ M^-1 J~^T)^-1 (diagonal) as what the
heuristic approximates, and calls it expensive.  Here a small network learns, per contact and
from four configuration features, the log ratio between the exact impedance (the mean over the
contact's facets of M_j = 1 / ((k dt + d) J~_j M~^-1 J~_j^T)) and the heuristic M(phi); the
step then uses M(phi) exp(g(x)) at about the heuristic's cost (trace_mode 3).

1. `exact_dataset`: one exact-mode step (trace_mode 2) of some worlds with contact capture;
   the step kernel writes every contact's features and target into its capture record.
2. `fit`: full-batch Adam on the mean squared error (cf_impnet_fit).
3. `r2` and `impulse_errors`: how much of the target's spread the network explains, and how
   close the learned step's contact impulses come to the exact step's.
"""
from __future__ import annotations

import dataclasses

import numpy as np
import torch

from . import comfree as CF


def with_mode(sb, mode):
    """A copy of the scenes.Batch sb whose model uses impedance mode `mode`."""
    out = sb.subset(range(sb.nworld))
    out.params = dataclasses.replace(sb.params, trace_mode=mode)
    return out


def exact_dataset(sb, capture=4096):
    """(x [n, 4], y [n]) on the device, and the capture records, from one exact-mode step of
    every world of sb from its initial state.  Contacts whose target is not finite (a facet
    with no inverse mass) are dropped."""
    se = with_mode(sb, 2)
    _, b = CF.from_scenes(se, contact_capture=capture)
    b.step(se.dt, 1)
    rec, counts = b.contacts_array()
    if (counts > capture).any():
        raise RuntimeError(f"contact capture overflow: {int(counts.max())} > {capture}")
    keep = np.isfinite(rec["target"])
    rec = rec[keep]
    x = CF.impedance_features(rec, se.params.solimp[2])
    dev = b.device
    return torch.from_numpy(x).to(dev), torch.from_numpy(rec["target"].astype(np.float32)).to(dev), rec


def fit(x, y, iters=3000, lr=0.02, seed=0, net=None):
    """Fit (or continue fitting) a learned impedance network; returns (net, losses on host)."""
    net = net or CF.ImpedanceNet(seed=seed, device=x.device)
    losses = net.fit(x, y, iters, lr)
    return net, losses.cpu().numpy()


def constant_net(y, device="cuda"):
    """The best constant rescaling of the heuristic (g = mean target): the 'one-size-fits-most'
    global parameter, fitted to the same data."""
    th = np.zeros(CF.IMPNET_PARAMS, np.float32)
    th[-1] = float(y.mean())
    return CF.ImpedanceNet(theta=th, device=device)


def r2(net, x, y, mean_train):
    """Coefficient of determination of the network on (x, y) against the constant mean_train."""
    g = net.eval(x)
    res = torch.mean((g - y) ** 2).item()
    tot = torch.mean((y - mean_train) ** 2).item()
    return 1.0 - res / tot, res, tot


def step_impulses(sb, mode, net=None, capture=4096):
    """Per-contact summed normal impulses of one step of sb's worlds from their initial states
    in impedance mode `mode`, keyed by (world, geom_a, geom_b, sub)."""
    sm = with_mode(sb, mode)
    _, b = CF.from_scenes(sm, contact_capture=capture)
    if mode == 3:
        b.set_impedance_net(net.theta.view(1, -1), 1)
    b.step(sm.dt, 1)
    rec, counts = b.contacts_array()
    world = np.repeat(np.arange(sb.nworld), np.minimum(counts, capture))
    return {(int(w), int(a), int(g), int(s)): float(l)
            for w, a, g, s, l in zip(world, rec["geom_a"], rec["geom_b"], rec["sub"], rec["lam_sum"])}


def impulse_errors(sb, nets, capture=4096):
    """Median relative error of the per-contact normal impulse of one step against the exact
    mode's, over contacts the exact step pushes (lambda > 0): for the heuristic (mode 0) and
    for every named network in `nets` (mode 3)."""
    ref = step_impulses(sb, 2, capture=capture)
    keys = [k for k, v in ref.items() if v > 0]
    r = np.array([ref[k] for k in keys])
    out = {}
    runs = {"heuristic": step_impulses(sb, 0, capture=capture)}
    for name, net in nets.items():
        runs[name] = step_impulses(sb, 3, net, capture=capture)
    for name, got in runs.items():
        g = np.array([got.get(k, 0.0) for k in keys])
        out[name] = float(np.median(np.abs(g - r) / r))
    out["contacts"] = len(keys)
    return out


def advanced(sb, nsteps):
    """A copy of sb whose worlds start from the state after nsteps heuristic (mode 0) steps on
    the GPU."""
    s0 = with_mode(sb, 0)
    _, b = CF.from_scenes(s0)
    b.step(s0.dt, nsteps)
    q, v = b.get_state()
    q, v = q.cpu().numpy().astype(np.float64), v.cpu().numpy().astype(np.float64)
    out = sb.subset(range(sb.nworld))
    qo = vo = 0
    for w in range(sb.nworld):
        t = sb.template_of(w)
        out.q0[w], out.v0[w] = q[qo:qo + t.nq].copy(), v[vo:vo + t.nv].copy()
        qo += t.nq
        vo += t.nv
    return out
