"""Sampling MPC (MPPI) for in-hand cube reorientation on the batched ComFree step, with an
optional learned proposal (the tensor-core MLP) mixed into the sampling distribution.

Per control tick (all on the GPU, one rollout launch):
  1. broadcast the plant state to the N rollout worlds (cf_broadcast_state);
  2. draw standard normals (caller-side random numbers are inputs to the sampler);
  3. proposal: features = (q, v, goal quaternion) -> MLP -> Gaussian over the H x nu plan;
  4. sample N control sequences (cf_mppi_sample): n_prop from the proposal, the rest around the
     warm-started mean, clipped to the torque limit;
  5. roll all N worlds H steps with the fused running/terminal cost (cf_set_cost, cf_step);
  6. MPPI update of the mean (cf_mppi_update); apply its first action to the plant; shift.
The engine simulates and scores every rollout: the network only proposes.
"""
from __future__ import annotations

import ctypes as C

import numpy as np
import torch

from . import comfree as CF
from . import scenes as S

NU, NQ, NV = 16, 23, 22
V_SCALE, F_CLAMP = 0.1, 10.0   # proposal inputs: velocities x 0.1, every feature clamped to +-10


def default_cost():
    return CF.CostDesc(body=0, w_quat=2.0, w_pos=2.0, w_contact=10.0, w_joint=0.05, w_fallen=5.0, fall_radius=0.08,
                       term_pos=50.0, term_quat=20.0)


def quat_mul(a, b):
    w1, x1, y1, z1 = a
    w2, x2, y2, z2 = b
    return np.array([w1 * w2 - x1 * x2 - y1 * y2 - z1 * z2, w1 * x2 + x1 * w2 + y1 * z2 - z1 * y2,
                     w1 * y2 - x1 * z2 + y1 * w2 + z1 * x2, w1 * z2 + x1 * y2 - y1 * x2 + z1 * w2])


def task_cost(q, goal):
    """Evaluation cost of a plant state: |p - p*|^2 + (1 - (q*^T q)^2) of the cube."""
    p, qu = q[:3], q[3:7]
    return float(np.sum((p - goal[:3]) ** 2) + 1.0 - np.dot(goal[3:], qu) ** 2)


class HandMPPI:
    def __init__(self, template, params, N=1024, H=32, dt=0.005, sigma=1.0, lam=0.1, limit=2.0, mlp=None,
                 n_prop=0, seed=0, cost=None, device="cuda", warps=2):
        self.N, self.H, self.dt, self.sigma, self.lam, self.limit = N, H, dt, sigma, lam, limit
        self.mlp, self.n_prop = mlp, (n_prop if mlp is not None else 0)
        self.model = CF.Model([template], params)
        self.rollouts = CF.Batch(self.model, np.zeros(N, np.int32), max_ctrl_steps=H)
        self.rollouts.set_warps(0, warps)  # warps per rollout world (2: the fastest for 1024 hands)
        self.plant = CF.Batch(self.model, np.zeros(1, np.int32), max_ctrl_steps=1)
        dev = device
        self.goals = torch.zeros(N, 7, device=dev)
        self.qref = torch.zeros(N * NQ, device=dev)
        self.costs = torch.zeros(N, device=dev)
        self.cost_desc = cost or default_cost()
        self.rollouts.set_cost(self.cost_desc, self.goals, self.qref, self.costs)
        self.mean = torch.zeros(H * NU, device=dev)
        self.ctrl = torch.empty(H * N * NU, device=dev)
        self.samples = torch.empty(N * H * NU, device=dev)
        self.noise = torch.empty(N * H * NU, device=dev)
        self.stats = torch.zeros(3, device=dev)
        self.qall = torch.empty(N * NQ, device=dev)
        self.vall = torch.empty(N * NV, device=dev)
        self.feat = torch.empty(1, NQ + NV + 4, device=dev)
        self.gen = torch.Generator(device=dev)
        self.gen.manual_seed(seed)
        self.goal = None

    def reset(self, q0, v0, goal):
        q0 = torch.as_tensor(np.asarray(q0, np.float32), device=self.mean.device)
        v0 = torch.as_tensor(np.asarray(v0, np.float32), device=self.mean.device)
        self.plant.set_state(q0, v0)
        self.goal = np.asarray(goal, np.float64)
        g = torch.as_tensor(self.goal.astype(np.float32), device=self.mean.device)
        self.goals.copy_(g.expand(self.N, 7))
        s = CF._stream()
        CF.check(CF.lib().cf_broadcast_state(CF._ptr(q0), CF._ptr(v0), NQ, NV, self.N, CF._ptr(self.qref),
                                             CF._ptr(self.vall), s))
        self.mean.zero_()

    def features(self, qp, vp):
        g = self.goals[0, 3:7].contiguous()
        CF.check(CF.lib().cf_mppi_features(CF._ptr(qp), NQ, CF._ptr(vp), NV, V_SCALE, CF._ptr(g), 4, F_CLAMP,
                                           CF._ptr(self.feat), CF._stream()))
        return self.feat

    def tick(self):
        s = CF._stream()
        qp, vp = self.plant.get_state()
        CF.check(CF.lib().cf_broadcast_state(CF._ptr(qp), CF._ptr(vp), NQ, NV, self.N, CF._ptr(self.qall),
                                             CF._ptr(self.vall), s))
        self.rollouts.set_state(self.qall, self.vall)
        self.costs.zero_()
        torch.randn(self.noise.shape, generator=self.gen, device=self.noise.device, out=self.noise)
        pm = pls = None
        if self.n_prop:
            y = self.mlp.forward(self.features(qp, vp))
            half = y.shape[1] // 2
            pm, pls = y[0, :half].contiguous(), y[0, half:].clamp(-5.0, 2.0).contiguous()
        CF.check(CF.lib().cf_mppi_sample(self.N, self.H, NU, CF._ptr(self.mean), CF._ptr(self.noise), self.sigma,
                                         self.limit, CF._ptr(pm), CF._ptr(pls), self.n_prop, CF._ptr(self.ctrl),
                                         CF._ptr(self.samples), s))
        self.rollouts.set_ctrl(self.ctrl)
        self.rollouts.step(self.dt, self.H)
        CF.check(CF.lib().cf_mppi_update(self.N, self.H, NU, CF._ptr(self.costs), CF._ptr(self.samples), self.lam,
                                         CF._ptr(self.mean), CF._ptr(self.stats), s))
        plan = self.mean.clone()
        self.plant.set_ctrl(self.mean[:NU])
        self.plant.step(self.dt, 1)
        CF.check(CF.lib().cf_mppi_shift(self.H, NU, CF._ptr(self.mean), s))
        return plan

    def plant_state(self):
        q, v = self.plant.get_state()
        return q.cpu().numpy().astype(np.float64), v.cpu().numpy().astype(np.float64)


def random_goal(q0, rng):
    """Target: the initial position with the orientation turned about the vertical by +-(30..90) deg."""
    ang = rng.uniform(np.pi / 6, np.pi / 2) * rng.choice([-1.0, 1.0])
    qt = quat_mul(S.quat_about((0, 0, 1), ang), q0[3:7])
    return np.concatenate([q0[:3], qt])


def run_episode(ctl, q0, v0, goal, ticks, record=None):
    ctl.reset(q0, v0, goal)
    for _ in range(ticks):
        if record is not None:
            qp, vp = ctl.plant.get_state()
            feat = ctl.features(qp, vp)[0].clone()
        plan = ctl.tick()
        if record is not None:
            record.append((feat, plan))
    q, _ = ctl.plant_state()
    return task_cost(q, goal)


def collect_and_train(template, params, episodes=32, ticks=60, N=1024, seed=0, epochs=300, mlp=None, lr=1e-3,
                      log=None):
    """Plain-MPPI episodes on seeded random goals; each tick's updated plan is an elite target for
    the proposal; then Adam epochs of the Gaussian NLL on the tensor-core MLP."""
    rng = np.random.default_rng(seed)
    sb = S.make_hand(episodes, seed=seed + 1)
    ctl = HandMPPI(template, params, N=N, seed=seed)
    rec = []
    finals = []
    for e in range(episodes):
        goal = random_goal(sb.q0[e], rng)
        finals.append(run_episode(ctl, sb.q0[e], sb.v0[e], goal, ticks, rec))
    X = torch.stack([r[0] for r in rec])
    Y = torch.stack([r[1] for r in rec])
    keep = torch.isfinite(X).all(1) & torch.isfinite(Y).all(1)
    X, Y = X[keep].contiguous(), Y[keep].contiguous()
    mlp = mlp or CF.Mlp(NQ + NV + 4, 256, 2 * 32 * NU, max_batch=max(len(rec), 128), seed=seed)
    losses = []
    for ep in range(epochs):
        losses.append(mlp.train_step(X, Y, lr=lr).item())
    mlp.status()
    if log is not None:
        log.update(samples=len(rec), plain_final=float(np.mean(finals)), loss_first=losses[0], loss_last=losses[-1])
    return mlp, float(np.mean(finals))


def cold_start_costs(template, params, N, mlp=None, n_prop=0, goals_seed=77, episodes=16, seed=5):
    """Best rollout cost of the first control tick from a cold start (zero warm-start mean) on
    seeded held-out starts and goals: how good a plan N rollouts find with and without the
    proposal before any warm start helps.  Returns the per-goal costs."""
    rng = np.random.default_rng(goals_seed)
    sb = S.make_hand(episodes, seed=goals_seed + 1)
    goals = [random_goal(sb.q0[e], rng) for e in range(episodes)]
    ctl = HandMPPI(template, params, N=N, seed=seed, mlp=mlp, n_prop=n_prop)
    out = []
    for e in range(episodes):
        ctl.reset(sb.q0[e], sb.v0[e], goals[e])
        ctl.tick()
        out.append(float(ctl.stats[0].item()))
    return np.array(out)


def compare(template, params, mlp, goals_seed=123, episodes=8, ticks=60, plain_N=1024, learned_N=(128, 256, 512),
            n_prop_frac=0.5):
    """Final task cost of plain MPPI (plain_N rollouts) against MPPI with the proposal at fewer rollouts,
    on the same seeded held-out goals and starts."""
    rng = np.random.default_rng(goals_seed)
    sb = S.make_hand(episodes, seed=goals_seed + 1)
    goals = [random_goal(sb.q0[e], rng) for e in range(episodes)]
    out = {}
    ctl = HandMPPI(template, params, N=plain_N, seed=goals_seed)
    out[f"plain_{plain_N}"] = float(np.mean([run_episode(ctl, sb.q0[e], sb.v0[e], goals[e], ticks)
                                             for e in range(episodes)]))
    for n in learned_N:
        ctl = HandMPPI(template, params, N=n, mlp=mlp, n_prop=int(n * n_prop_frac), seed=goals_seed)
        out[f"learned_{n}"] = float(np.mean([run_episode(ctl, sb.q0[e], sb.v0[e], goals[e], ticks)
                                             for e in range(episodes)]))
        ctl = HandMPPI(template, params, N=n, seed=goals_seed)
        out[f"plain_{n}"] = float(np.mean([run_episode(ctl, sb.q0[e], sb.v0[e], goals[e], ticks)
                                           for e in range(episodes)]))
    return out
