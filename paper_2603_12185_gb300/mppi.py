"""Sampling MPC (MPPI) for in-hand cube reorientation on the batched ComFree step, with an
optional learned proposal (the tensor-core MLP) mixed into the sampling distribution.

Per control tick (all on the GPU, one rollout launch):
  1. broadcast the plant state to the N rollout worlds (cf_broadcast_state);
  2. draw standard normals (caller-side random numbers are inputs to the sampler);
  3. proposal, one of two modes:
     - "mix": features = (q, v, goal quaternion) -> MLP -> Gaussian over the H x nu plan, and
       n_prop of the N samples are drawn from it;
     - "warm" (the learned warm start): features = (q, v, goal quaternion, the first steps of the
       warm-start plan m) -> MLP -> a correction D of the plan, and the samples are drawn around
       m + D with MPPI's own sigma (all N, or n_prop of them with the rest around m; D = 0 is
       plain MPPI);
  4. sample N control sequences (cf_mppi_sample), clipped to the torque limit;
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
PLAN_IN = 8 * NU               # the learned warm start also sees the first 8 steps of the plan


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
                 n_prop=0, seed=0, cost=None, device="cuda", warps=2, mode="mix"):
        self.N, self.H, self.dt, self.sigma, self.lam, self.limit = N, H, dt, sigma, lam, limit
        self.mode = mode
        self.mlp = mlp
        # "warm": n_prop of the N samples (all when n_prop = 0) around the corrected plan, the
        # rest around the warm start itself
        self.n_prop = (n_prop if mlp is not None else 0) if mode == "mix" else ((n_prop or N) if mlp is not None else 0)
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
        self.feat = torch.empty(1, NQ + NV + 4 + (PLAN_IN if mode == "warm" else 0), device=dev)
        if mode == "warm":
            self.prop_mean = torch.empty(H * NU, device=dev)
            self.prop_logstd = torch.full((H * NU,), float(np.log(sigma)), device=dev)
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
        """The network's input: (q, 0.1 v, goal quaternion), and in "warm" mode the first 8 steps of
        the current warm-start plan, each clamped to +-10."""
        g = self.goals[0, 3:7].contiguous()
        s = CF._stream()
        CF.check(CF.lib().cf_mppi_features(CF._ptr(qp), NQ, CF._ptr(vp), NV, V_SCALE, CF._ptr(g), 4, F_CLAMP,
                                           CF._ptr(self.feat), s))
        if self.mode == "warm":
            tail = self.feat[0, NQ + NV + 4:]
            CF.check(CF.lib().cf_mppi_features(CF._ptr(self.mean), PLAN_IN, CF._ptr(self.mean), 0, 1.0, None, 0,
                                               F_CLAMP, CF._ptr(tail), s))
        return self.feat

    def tick(self, apply=True):
        """One control tick; returns the updated plan.  apply=False leaves the plant and the warm
        start unshifted (the plan a teacher computes for a given state and warm start)."""
        s = CF._stream()
        qp, vp = self.plant.get_state()
        CF.check(CF.lib().cf_broadcast_state(CF._ptr(qp), CF._ptr(vp), NQ, NV, self.N, CF._ptr(self.qall),
                                             CF._ptr(self.vall), s))
        self.rollouts.set_state(self.qall, self.vall)
        self.costs.zero_()
        torch.randn(self.noise.shape, generator=self.gen, device=self.noise.device, out=self.noise)
        pm = pls = None
        if self.n_prop and self.mode == "mix":
            y = self.mlp.forward(self.features(qp, vp))
            half = y.shape[1] // 2
            pm, pls = y[0, :half].contiguous(), y[0, half:].clamp(-5.0, 2.0).contiguous()
        elif self.n_prop:
            y = self.mlp.forward(self.features(qp, vp))
            CF.check(CF.lib().cf_mppi_blend(self.H * NU, CF._ptr(self.mean), CF._ptr(y[0, :self.H * NU]), 1.0,
                                            CF._ptr(self.prop_mean), s))
            pm, pls = self.prop_mean, self.prop_logstd
        CF.check(CF.lib().cf_mppi_sample(self.N, self.H, NU, CF._ptr(self.mean), CF._ptr(self.noise), self.sigma,
                                         self.limit, CF._ptr(pm), CF._ptr(pls), self.n_prop, CF._ptr(self.ctrl),
                                         CF._ptr(self.samples), s))
        self.rollouts.set_ctrl(self.ctrl)
        self.rollouts.step(self.dt, self.H)
        CF.check(CF.lib().cf_mppi_update(self.N, self.H, NU, CF._ptr(self.costs), CF._ptr(self.samples), self.lam,
                                         CF._ptr(self.mean), CF._ptr(self.stats), s))
        plan = self.mean.clone()
        if apply:
            self.plant.set_ctrl(self.mean[:NU])
            self.plant.step(self.dt, 1)
            CF.check(CF.lib().cf_mppi_shift(self.H, NU, CF._ptr(self.mean), s))
        return plan

    def tick_graph(self):
        """A CUDA graph of one control tick (apply=True): each replay() runs the next tick on the
        current stream with the same buffers, its plan left in self.mean, and draws fresh noise
        (the controller's generator is registered with the graph), so replays reproduce the
        eager ticks bit for bit.  One eager tick runs first (kernel attributes), so the plant
        advances by one tick here.  A tick is a dozen small launches around the rollout; the
        graph removes their host launch overhead."""
        self.tick()
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        g.register_generator_state(self.gen)
        with torch.cuda.graph(g):
            self.tick()
        return g

    def plan_from(self, qp, vp, mean):
        """The plan one tick computes from plant state (qp, vp) and warm start `mean` (device),
        without stepping this controller's plant."""
        self.plant.set_state(qp, vp)
        self.mean.copy_(mean)
        return self.tick(apply=False)

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


def dagger_warm_start(template, params, iters=3, episodes=24, ticks=60, N=256, N_teacher=1024, epochs=600,
                      lr=1e-3, seed=0, log=None):
    """Train the learned warm start by dataset aggregation (DAgger, Ross et al., AISTATS 2011):
    iteration 0 runs plain MPPI with N rollouts, later iterations the learned controller with
    the current network; at every tick visited, a teacher tick with N_teacher rollouts from the
    same state and the same warm start m gives the label, and the network learns the correction
    (teacher plan - m) by the Gaussian NLL on the tensor-core MLP, over all ticks collected so
    far.  Returns the network."""
    rng = np.random.default_rng(seed)
    sb = S.make_hand(episodes, seed=seed + 1)
    goals = [random_goal(sb.q0[e], rng) for e in range(episodes)]
    teacher = HandMPPI(template, params, N=N_teacher, seed=seed + 7)
    mlp = CF.Mlp(NQ + NV + 4 + PLAN_IN, 256, 2 * 32 * NU, max_batch=max(iters * episodes * ticks, 128), seed=seed)
    X, Y, stats = [], [], []
    for it in range(iters):
        student = HandMPPI(template, params, N=N, seed=seed + 11 + it, mlp=mlp if it else None, mode="warm")
        finals = []
        for e in range(episodes):
            student.reset(sb.q0[e], sb.v0[e], goals[e])
            teacher.reset(sb.q0[e], sb.v0[e], goals[e])
            for _ in range(ticks):
                qp, vp = student.plant.get_state()
                m = student.mean.clone()
                label = teacher.plan_from(qp, vp, m)
                X.append(student.features(qp, vp)[0].clone())
                Y.append(label - m)
                student.tick()
            finals.append(task_cost(student.plant_state()[0], goals[e]))
        Xt, Yt = torch.stack(X), torch.stack(Y)
        keep = torch.isfinite(Xt).all(1) & torch.isfinite(Yt).all(1)
        Xt, Yt = Xt[keep].contiguous(), Yt[keep].contiguous()
        losses = [mlp.train_step(Xt, Yt, lr=lr).item() for _ in range(epochs)]
        stats.append({"iteration": it, "samples": int(len(Yt)), "student_final_cost": float(np.mean(finals)),
                      "nll_first": losses[0], "nll_last": losses[-1]})
    mlp.status()
    if log is not None:
        log["dagger"] = stats
    return mlp


def final_costs(template, params, arms, goals_seed=123, episodes=48, ticks=60):
    """Final task cost of each arm over the same seeded held-out starts and goals.  arms: name ->
    dict(N, mlp=None, mode="warm", n_prop=0).  Returns name -> per-goal final costs (numpy) and
    name -> CUDA-event milliseconds per tick."""
    rng = np.random.default_rng(goals_seed)
    sb = S.make_hand(episodes, seed=goals_seed + 1)
    goals = [random_goal(sb.q0[e], rng) for e in range(episodes)]
    costs, tick_ms = {}, {}
    for name, a in arms.items():
        ctl = HandMPPI(template, params, N=a["N"], mlp=a.get("mlp"), mode=a.get("mode", "warm"),
                       n_prop=a.get("n_prop", 0), seed=goals_seed)
        out = []
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ms = 0.0
        for e in range(episodes):
            ctl.reset(sb.q0[e], sb.v0[e], goals[e])
            torch.cuda.synchronize()
            e0.record()
            for _ in range(ticks):
                ctl.tick()
            e1.record()
            torch.cuda.synchronize()
            ms += e0.elapsed_time(e1)
            out.append(task_cost(ctl.plant_state()[0], goals[e]))
        costs[name] = np.array(out)
        tick_ms[name] = ms / (episodes * ticks)
    return costs, tick_ms
