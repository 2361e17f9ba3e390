"""Benchmark of the batched ComFree step on GB300.

Workload (dense-contact scaling): 4096 walled bins, each with 256 free bodies (seeded 50/50
sphere/capsule mix, density 1000), 6D cone with 8 tangential + 2 torsional + 8 rolling facets,
mu = 0.8, dt = 2 ms, a 1000-step drop episode.  One bench "step" is one simulation step of all
4096 worlds (one launch of the fused step kernel).  The timed K steps are the last K steps of
the episode (the settled, densest part); the steps before them run untimed.  The same run also
measures 16- and 64-body bins (4096 worlds each) for the contacts/world sweep.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Prints one JSON line (rank 0).  Under torchrun each rank simulates its own 4096 worlds (weak
scaling, no collective on the data path; the timing barrier and max use torch.distributed).
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2603_12185_gb300 import replicas as R  # noqa: E402

EPISODE = 1000
WORLDS = 4096
BODIES = 256
SWEEP = (16, 64)
BYTES_PER_BODY = (7 + 6) * 4 * 2 + 8 * 4   # q, v read + written, 8-float parameter block read
METRIC = "world-steps/s & contacts resolved/s vs contacts/world at 1 GB300; % of HBM roofline"
# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) of one step-kernel launch of the
# 4096 x 256 pile workload late in the episode (step_kernel<0, 2, 0>, 4 warps per world, the
# shape the autotuner picks), from one ncu capture of the kernel sources whose digest is given;
# reported as null once the sources differ from the ones measured.
STEP_SOURCES = ("cf_step.cu", "cf_device_math.cuh", "cf_internal.cuh")
TRAFFIC = {"digest": "16e2000bbbeae51a", "bytes": 93.12e6}
# warp instructions executed (smsp__inst_executed.sum) by one such launch, same capture rules:
# the step's issue-rate bound is this count over the issue ceiling (SMs x 4 schedulers x 1
# warp instruction per cycle x the SM clock sampled during the timed region)
INSTRUCTIONS = {"digest": "16e2000bbbeae51a", "warp_instructions": 331.6e6}


def step_digest():
    """Digest of the step kernel's code: the sources with comments and whitespace removed, so
    that an edit of a comment keeps the counters measured on the code."""
    import hashlib
    import re
    h = hashlib.sha256()
    for f in STEP_SOURCES:
        with open(os.path.join(ROOT, "paper_2603_12185_gb300", "csrc", f)) as fh:
            src = fh.read()
        src = re.sub(r"/\*.*?\*/", " ", src, flags=re.S)
        src = re.sub(r"//[^\n]*", " ", src)
        h.update(" ".join(src.split()).encode())
    return h.hexdigest()[:16]


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--worlds", type=int, default=WORLDS)
    ap.add_argument("--bodies", type=int, default=BODIES)
    ap.add_argument("--no-sweep", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--e2e-steps", type=int, default=100, help="end-to-end steps (0: skip, for profiles)")
    ap.add_argument("--no-extras", action="store_true")
    ap.add_argument("--e2e-blocks", type=int, default=8, help="blocks of worlds of the end-to-end pipeline")
    ap.add_argument("--episode", type=int, default=EPISODE, help="episode length (the timed steps are its last)")
    ap.add_argument("--warps", type=int, default=0,
                    help="warps per world (0: autotune); a fixed shape makes profiles comparable")
    ap.add_argument("--jammed", action="store_true",
                    help="start from interpenetrating bodies (contact-rich first steps; for short profiles)")
    ap.add_argument("--mlp-only", action="store_true",
                    help="time only the proposal MLP's tensor-core training step and forward pass (for profiles)")
    ap.add_argument("--proposal-size", default=None, help="iters,episodes,goals of --only proposal (default 3,24,48)")
    ap.add_argument("--only", default=None, choices=sorted(ONLY),
                    help="run one of the other workloads alone and print its JSON (for profiles)")
    ap.add_argument("--impedance", default="heuristic", choices=sorted(IMPEDANCE_MODES),
                    help="impedance mode of the headline workload (the exact and learned forms of Sec. III-B; "
                         "for profiles)")
    return ap.parse_args()


def peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


class Clocks:
    """nvidia-smi sampling during the timed region (SM clock, max clock, throttle reasons)."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.rows = []
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                                          "-lms", "200", "-i", str(self.index)], stdout=subprocess.PIPE,
                                         stderr=subprocess.DEVNULL, text=True)
            threading.Thread(target=self._read, daemon=True).start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([x.strip() for x in line.split(",")])

    def stop(self):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(2)
            except Exception:
                self.proc.kill()
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in self.rows:
            try:
                sm.append(float(r[1]))
                mx = max(mx, float(r[2]))
                for n, val in zip(names, r[5:9]):
                    if val.strip().lower() == "active":
                        reasons.add(n)
            except Exception:
                pass
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": mx or None,
                "reasons": sorted(reasons), "samples": len(sm)}


def dist_setup():
    import torch
    n = int(os.environ.get("WORLD_SIZE", "1"))
    if n > 1:
        import torch.distributed as dist
        local = int(os.environ.get("LOCAL_RANK", "0"))
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
        return dist.get_rank(), n, local
    return 0, 1, 0


def barrier_max(x, world):
    """Max over the replicas (after a barrier): the whole job is as slow as its slowest rank."""
    if world == 1:
        return x
    import torch.distributed as dist
    from paper_2603_12185_gb300 import replicas as R
    dist.barrier()
    return R.reduce_scalar(x, "max")


def barrier_sum(x, world):
    if world == 1:
        return x
    from paper_2603_12185_gb300 import replicas as R
    return R.reduce_scalar(x, "sum")


IMPEDANCE_MODES = {"heuristic": 0, "exact": 2, "learned": 3}


def learned_impedance(rank, evaluate=False):
    """A learned impedance network (trace_mode 3) fitted to exact-mode contacts of 96 settled
    pile64 worlds and 32 jammed pile256 worlds: (net, fit statistics); evaluate=True adds the
    held-out R^2 and impulse errors on 8 other jammed pile256 worlds."""
    import torch
    from paper_2603_12185_gb300 import impedance as IMP
    from paper_2603_12185_gb300 import scenes as S
    train = [IMP.advanced(S.make_pile(96, 64, seed=R.rank_seed(1960, rank)), 300),
             S.make_pile(32, 256, seed=R.rank_seed(1961, rank), jammed=True)]
    xs, ys = zip(*[IMP.exact_dataset(t)[:2] for t in train])
    x, y = torch.cat(xs), torch.cat(ys)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    net, losses = IMP.fit(x, y, iters=3000, lr=0.02)
    fit = {"train_contacts": int(len(y)), "adam_steps": 3000, "fit_s": time.perf_counter() - t0,
           "loss_first": float(losses[0]), "loss_last": float(losses[-1])}
    if evaluate:
        held = S.make_pile(8, 256, seed=R.rank_seed(1962, rank), jammed=True)
        xh, yh, _ = IMP.exact_dataset(held)
        fit["held_out_r2"] = IMP.r2(net, xh, yh, float(y.mean()))[0]
        fit["median_rel_impulse_err_vs_exact"] = IMP.impulse_errors(
            held, {"learned": net, "constant": IMP.constant_net(y)})
    return net, fit


def run_pile(nbody, nworld, steps, warmup, rank, flush=None, episode=EPISODE, jammed=False, warps=0,
             impedance="heuristic"):
    """Simulate the episode; time the last `steps` steps with CUDA events on the launch stream,
    flushing L2 (256 MB write) between timed steps outside the timed intervals.  The autotuner
    runs half way through the untimed part, on a state like the timed one (it restores it).
    impedance: the impedance mode of the whole run (the learned one is fitted first)."""
    import dataclasses
    import torch
    from paper_2603_12185_gb300 import comfree as CF
    from paper_2603_12185_gb300 import scenes as S
    sb = S.make_pile(nworld, nbody, seed=R.rank_seed(1000, rank), jammed=jammed)
    sb.params = dataclasses.replace(sb.params, trace_mode=IMPEDANCE_MODES[impedance])
    net = learned_impedance(rank)[0] if impedance == "learned" else None
    model, b = CF.from_scenes(sb)
    if net is not None:
        b.set_impedance_net(net.theta.view(1, -1), 1)
    stream = torch.cuda.current_stream()
    preroll = max(warmup, episode - steps)
    if warps > 0:
        b.set_warps(0, warps)
    for i in range(preroll):
        if i == preroll // 2 and warps <= 0:
            b.autotune(sb.dt)
        b.step(sb.dt, 1)
    torch.cuda.synchronize()
    counts = torch.zeros(nworld, dtype=torch.int32, device="cuda")
    contact_sum = torch.zeros(nworld, dtype=torch.int64, device="cuda")
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    for i in range(steps):
        if flush is not None:
            flush.add_(1.0)
        ev[i][0].record(stream)
        b.step(sb.dt, 1)
        ev[i][1].record(stream)
        b.contact_counts_device(counts)
        contact_sum += counts
    torch.cuda.synchronize()
    times = [a.elapsed_time(c) for a, c in ev]
    st, _ = b.status()
    if st != 0:
        raise RuntimeError(f"device status {st} after the episode")
    return dict(ms=float(np.sum(times)), per_launch_ms=float(np.mean(times)), steps=steps, preroll=preroll,
                contacts=int(contact_sum.sum().item()), worlds=nworld, bodies=nbody, sb=sb, batch=b, model=model,
                net=net)


def run_e2e(res, steps, blocks=8):
    """Same workload through the public API with the state in pinned host memory: every step
    moves q, v host -> device, steps, and moves the new state device -> host, the host waiting
    for it.  Measured three ways:
    - serially on one batch (copy in, step, copy out);
    - with comfree.Pipeline, which splits the worlds into `blocks` batches on their own streams
      so that one block's copies overlap another's step;
    - in place (Batch.step_host): the step kernel reads the host state and writes it back itself.
    The reported value is the faster of the last two."""
    import torch
    from paper_2603_12185_gb300 import comfree as CF
    b = res["batch"]
    sb = res["sb"]
    dt = sb.dt
    q, v = b.get_state()
    nbytes = (b.total_nq + b.total_nv) * 4
    # serial: one batch, synchronous host copies
    hq = torch.empty(b.total_nq, dtype=torch.float32, pin_memory=True)
    hv = torch.empty(b.total_nv, dtype=torch.float32, pin_memory=True)
    hq.copy_(q.cpu())
    hv.copy_(v.cpu())
    b.set_state(hq, hv)
    b.step(dt, 1)
    b.get_state(hq, hv)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(steps):
        b.set_state(hq, hv)          # host -> device (synchronous copy of pinned buffers)
        b.step(dt, 1)
        b.get_state(hq, hv)          # device -> host, synchronises and checks device status
    torch.cuda.synchronize()
    serial = res["worlds"] * steps / (time.perf_counter() - t0)
    # pipelined: blocks of worlds on their own streams
    W = res["worlds"]
    edges = [W * k // blocks for k in range(blocks + 1)]
    batches, bq, bv = [], [], []
    qo = vo = 0
    for k in range(blocks):
        _, bk = CF.from_scenes(sb.subset(range(edges[k], edges[k + 1])))
        if res["net"] is not None:
            bk.set_impedance_net(res["net"].theta.view(1, -1), 1)
        bk.autotune(dt)
        batches.append(bk)
        bq.append(q[qo:qo + bk.total_nq].cpu().pin_memory())
        bv.append(v[vo:vo + bk.total_nv].cpu().pin_memory())
        qo += bk.total_nq
        vo += bk.total_nv
    pipe = CF.Pipeline(batches)
    pipe.step(bq, bv, dt)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(steps):
        pipe.step(bq, bv, dt)
    torch.cuda.synchronize()
    sec = time.perf_counter() - t0
    for st, _ in pipe.status():
        if st != 0:
            raise RuntimeError(f"device status {st} in the pipelined run")
    pipelined = W * steps / sec
    # in place: the step kernel reads the pinned host state and writes the new state back itself
    # (cf_step_host; the transfers run over the host link while other worlds compute), and every
    # step ends with the host synchronised on it, the new state in host memory
    b.step_host(hq, hv, dt)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(steps):
        b.step_host(hq, hv, dt)
        torch.cuda.synchronize()
    in_place = W * steps / (time.perf_counter() - t0)
    st, _ = b.status()
    if st != 0:
        raise RuntimeError(f"device status {st} in the in-place run")
    best = "in_place" if in_place >= pipelined else "pipelined"
    return dict(value=max(in_place, pipelined), serial=serial, pipelined=pipelined, in_place=in_place,
                blocks=blocks, h2d=nbytes, d2h=nbytes,
                api="Batch.step_host (cf_step_host) on pinned host state" if best == "in_place"
                else f"comfree.Pipeline, {blocks} blocks")


def mlp_throughput(batch=16384, reps=20):
    """The learned MPPI proposal's MLP (49 -> 256 -> 256 -> 1024, GELU; BF16 operands on the
    tcgen05 tensor cores, FP32 accumulation): CUDA-event time of a forward pass and of one
    training step (forward, backward, Adam) at `batch` rows, with the dense FLOPs of the GEMMs
    (the first layer's K padded to 64) and their fraction of the measured bf16 peak."""
    import torch
    from paper_2603_12185_gb300 import comfree as CF
    fin, H, O = 49, 256, 1024
    kin = (fin + 63) // 64 * 64
    mlp = CF.Mlp(fin, H, O, max_batch=batch, seed=0)
    g = torch.Generator(device="cuda")
    g.manual_seed(0)
    x = torch.randn(batch, fin, device="cuda", generator=g)
    y = 0.1 * torch.randn(batch, O // 2, device="cuda", generator=g)
    out = torch.empty(batch, O, device="cuda")

    def timed(fn):
        for _ in range(3):
            fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            fn()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps

    ms_f = timed(lambda: mlp.forward(x, out))
    ms_t = timed(lambda: mlp.train_step(x, y, lr=1e-5))
    mlp.status()
    flop_f = 2.0 * batch * (kin * H + H * H + H * O)
    flop_t = flop_f + 2.0 * batch * (kin * H + 2 * H * H + 2 * H * O)   # weight and activation gradients
    pk, src = peaks()
    tf_f, tf_t = flop_f / ms_f / 1e9, flop_t / ms_t / 1e9
    return {"batch": batch, "forward_ms": ms_f, "forward_tflops": tf_f, "train_step_ms": ms_t, "train_tflops": tf_t,
            "frac_of_bf16_peak": {"forward": tf_f / pk["bf16_tflops"], "train": tf_t / pk["bf16_tflops"]},
            "peak_source": src}


def _timed(fn, reps):
    import torch
    fn()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        fn()
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps


def extra_spheres(rank):
    """Small case: 64 worlds x 8 spheres on a plane, 500 steps, one launch per step, one launch
    for all 500 steps (the kernel keeps the worlds in shared memory across steps), and 100
    one-step launches replayed from one CUDA graph."""
    from paper_2603_12185_gb300 import comfree as CF
    from paper_2603_12185_gb300 import scenes as S
    sb = S.make_spheres_on_plane(64, seed=R.rank_seed(1900, rank))
    _, b = CF.from_scenes(sb)
    ms1 = _timed(lambda: b.step(sb.dt, 1), 500)
    ms500 = _timed(lambda: b.step(sb.dt, 500), 3)
    g = b.graph(sb.dt, 1, repeat=100)
    ms_graph = _timed(g.replay, 5) / 100
    return {"world_steps_per_s": 64 / (ms1 / 1e3), "ms_per_step": ms1,
            "world_steps_per_s_graph": 64 / (ms_graph / 1e3), "ms_per_step_graph": ms_graph,
            "world_steps_per_s_500_steps_per_launch": 64 * 500 / (ms500 / 1e3)}


def algorithmic_bytes_per_step(sb, controls=False):
    """Algorithmic HBM bytes of one step of every world of a scene batch (the roofline's
    numerator): a pile world moves BYTES_PER_BODY per body (q and v read and written, its
    8-float parameter block read); an articulated world reads and writes its q and v and, when
    controls are set, reads one torque per hinge."""
    from paper_2603_12185_gb300 import scenes as S
    total = 0
    for w in range(sb.nworld):
        t = sb.template_of(w)
        if t.pile:
            total += BYTES_PER_BODY * len(t.body_parent)
        else:
            total += 8 * (len(sb.q0[w]) + len(sb.v0[w]))
            if controls:
                total += 4 * int((np.asarray(t.body_jnt) == S.HINGE).sum())
    return total


def extra_mixed(rank):
    """Uneven worlds: 8192 worlds interleaving pile16/pile64/pile256/hand, one launch per step,
    eager and from a CUDA graph of ten launches."""
    from paper_2603_12185_gb300 import comfree as CF
    from paper_2603_12185_gb300 import scenes as S
    sb = S.make_mixed(8192, seed=R.rank_seed(2000, rank))
    _, b = CF.from_scenes(sb)
    chosen = b.autotune(sb.dt)
    for _ in range(300):
        b.step(sb.dt, 1)
    ms = _timed(lambda: b.step(sb.dt, 1), 20)
    c = b.contact_counts()
    g = b.graph(sb.dt, 1, repeat=10)
    ms_graph = _timed(g.replay, 5) / 10
    by = algorithmic_bytes_per_step(sb)
    pk, src = peaks()
    gbs = by / (ms / 1e3) / 1e9
    return {"world_steps_per_s": 8192 / (ms / 1e3), "ms_per_step": ms,
            "world_steps_per_s_graph": 8192 / (ms_graph / 1e3), "ms_per_step_graph": ms_graph,
            "contacts_per_world": float(c.mean()), "warps_per_world": [int(x) for x in chosen],
            "bytes_per_step": by, "hbm_gbs": gbs, "hbm_frac": gbs / pk["hbm_gbs"], "peak_source": src}


def extra_impedance(rank):
    """The exact diagonal impedance (trace_mode 2) and the learned impedance (trace_mode 3,
    fitted here to exact-mode contacts of other piles) against the heuristic: one step of the
    jammed 4096 x 256 pile from the same state (events around the step only)."""
    import dataclasses
    import torch
    from paper_2603_12185_gb300 import comfree as CF
    from paper_2603_12185_gb300 import scenes as S
    net, fit = learned_impedance(rank, evaluate=True)
    sbj = S.make_pile(4096, 256, seed=R.rank_seed(1950, rank), jammed=True)
    res = {"learned_fit": fit}
    for mode in (0, 2, 3):
        sbj.params = dataclasses.replace(sbj.params, trace_mode=mode)
        _, bj = CF.from_scenes(sbj)
        bj.set_warps(0, 4)
        if mode == 3:
            bj.set_impedance_net(net.theta.view(1, -1), 1)
        q0, v0 = bj.get_state()
        q0, v0 = q0.clone(), v0.clone()
        ts = []
        for i in range(6):
            bj.set_state(q0, v0)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            bj.step(sbj.dt, 1)
            e1.record()
            torch.cuda.synchronize()
            if i:
                ts.append(e0.elapsed_time(e1))
        res[{0: "heuristic", 2: "exact", 3: "learned"}[mode]] = {
            "ms_per_step": float(np.mean(ts)), "contacts_per_world": float(bj.contact_counts().mean())}
        del bj
    return res


HAND_BYTES = (23 + 22) * 4 * 2 + 16 * 4   # q, v read + written, 16 torques read, per world-step


def extra_adjoint(rank, reps=3):
    """The hand adjoint: 1024 worlds, 100 steps, checkpoints every 10 (forward + reverse)."""
    import torch
    from paper_2603_12185_gb300 import comfree as CF
    from paper_2603_12185_gb300 import scenes as S
    T = 100
    sb = S.make_hand(1024, seed=R.rank_seed(2100, rank))
    _, b = CF.from_scenes(sb, max_ctrl_steps=T, grad_steps=T, grad_ckpt=10)
    q0, v0 = CF.flatten_state(sb)
    q0, v0 = torch.from_numpy(q0).cuda(), torch.from_numpy(v0).cuda()
    tau = torch.randn(T, b.total_nu, device="cuda") * 0.05
    gq = torch.randn(b.total_nq, device="cuda")
    gv = torch.zeros(b.total_nv, device="cuda")

    def grad_once():
        b.set_state(q0, v0)
        b.set_ctrl(tau.reshape(-1))
        b.step_grad(T, sb.dt, gq, gv)

    ms = _timed(grad_once, reps)
    return {"ms": ms, "world_steps_per_s": 1024 * T / (ms / 1e3)}


def extra_hand_rollout(rank, reps=10):
    """Forward hand rollouts alone (the MPPI tick's simulation): 1024 hand worlds x 32 steps of
    5 ms in one launch with the fused cost, 2 warps per world; world-steps/s and the fraction of
    HBM bandwidth at (23 + 22) floats of state read and written plus 16 torques per world-step."""
    import torch
    from paper_2603_12185_gb300 import comfree as CF
    from paper_2603_12185_gb300 import mppi as MP
    from paper_2603_12185_gb300 import scenes as S
    t = S.hand_template(0)
    params = S.Params(**dict(S.HAND_PARAMS, d_user=0.002))
    ctl = MP.HandMPPI(t, params, N=1024)
    sbh = S.make_hand(1, seed=R.rank_seed(2200, rank))
    ctl.reset(sbh.q0[0], sbh.v0[0], MP.random_goal(sbh.q0[0], np.random.default_rng(rank)))
    ctl.tick()
    ctl.rollouts.set_ctrl(torch.randn(32 * 1024 * 16, device="cuda") * 0.3)
    q, v = ctl.rollouts.get_state()
    q, v = q.clone(), v.clone()

    def roll():
        ctl.rollouts.set_state(q, v)
        ctl.rollouts.step(0.005, 32)

    ms = _timed(roll, reps)
    ws = 1024 * 32 / (ms / 1e3)
    pk, src = peaks()
    gbs = ws * HAND_BYTES / 1e9
    return {"ms_per_launch": ms, "world_steps_per_s": ws, "bytes_per_world_step": HAND_BYTES,
            "hbm_gbs": gbs, "hbm_frac": gbs / pk["hbm_gbs"], "peak_source": src}


def extra_mppi(rank, reps=10):
    """One MPPI control tick: 1024 rollouts x 32 steps of 5 ms with the fused cost and the update,
    eagerly and replayed from a CUDA graph of the tick."""
    from paper_2603_12185_gb300 import mppi as MP
    from paper_2603_12185_gb300 import scenes as S
    t = S.hand_template(0)
    params = S.Params(**dict(S.HAND_PARAMS, d_user=0.002))
    ctl = MP.HandMPPI(t, params, N=1024)
    sbh = S.make_hand(1, seed=R.rank_seed(2200, rank))
    ctl.reset(sbh.q0[0], sbh.v0[0], MP.random_goal(sbh.q0[0], np.random.default_rng(rank)))
    ms = _timed(ctl.tick, reps)
    g = ctl.tick_graph()
    ms_graph = _timed(g.replay, reps)
    return {"ms": ms, "rollout_world_steps_per_s": 1024 * 32 / (ms / 1e3), "ms_graph": ms_graph,
            "rollout_world_steps_per_s_graph": 1024 * 32 / (ms_graph / 1e3)}


def extra_proposal(rank, iters=None, episodes=None, goals=None, ticks=60):
    """The learned warm start for sampling MPC (Sec. V's MPPI with a learned proposal added):
    trained by DAgger against 1024-rollout teacher ticks on seeded goals, then the final task
    cost over `goals` held-out starts and goals (paired: the same starts and goals in every arm)
    for plain MPPI at 1024, 512 and 256 rollouts and the learned warm start at 512, 256 and 128
    rollouts (and at 256 with half the rollouts around the uncorrected warm start), with each
    arm's CUDA-event time per tick (MLP inference included)."""
    from paper_2603_12185_gb300 import mppi as MP
    from paper_2603_12185_gb300 import scenes as S
    iters = iters or PROPOSAL["iters"]
    episodes = episodes or PROPOSAL["episodes"]
    goals = goals or PROPOSAL["goals"]
    t = S.hand_template(0)
    params = S.Params(**dict(S.HAND_PARAMS, d_user=0.002))
    log = {}
    import time as _t
    t0 = _t.perf_counter()
    mlp = MP.dagger_warm_start(t, params, iters=iters, episodes=episodes, seed=R.rank_seed(2300, rank), log=log)
    train_s = _t.perf_counter() - t0
    arms = {"plain_1024": dict(N=1024), "plain_512": dict(N=512), "plain_256": dict(N=256),
            "learned_512": dict(N=512, mlp=mlp), "learned_256": dict(N=256, mlp=mlp),
            "hedged_256": dict(N=256, mlp=mlp, n_prop=128), "learned_128": dict(N=128, mlp=mlp)}
    costs, tick_ms = MP.final_costs(t, params, arms, goals_seed=R.rank_seed(2400, rank), episodes=goals, ticks=ticks)
    out = {"train_s": train_s, "dagger": log["dagger"], "goals": goals, "ticks": ticks,
           "dagger_episodes": episodes, "dagger_iterations": iters}

    def paired(a, b):
        d = costs[a] - costs[b]
        return [float(d.mean()), float(d.std(ddof=1) / np.sqrt(len(d)))]

    for k, c in costs.items():
        out[k] = {"final_cost_mean": float(c.mean()), "final_cost_se": float(c.std(ddof=1) / np.sqrt(len(c))),
                  "paired_diff_vs_plain_1024": paired(k, "plain_1024"), "ms_per_tick": tick_ms[k]}
    out["learned_256"]["paired_diff_vs_plain_256"] = paired("learned_256", "plain_256")
    out["hedged_256"]["paired_diff_vs_plain_256"] = paired("hedged_256", "plain_256")
    out["learned_512"]["paired_diff_vs_plain_512"] = paired("learned_512", "plain_512")
    return out


PROPOSAL = {"iters": 3, "episodes": 24, "goals": 48}


EXTRAS = {"spheres_64x8": extra_spheres, "mixed_8192": extra_mixed,
          "impedance_modes_jammed_pile_4096x256": extra_impedance, "adjoint_hand_1024x100": extra_adjoint,
          "hand_rollout_1024x32": extra_hand_rollout, "mppi_tick_1024x32": extra_mppi,
          "proposal_mlp_49x256x1024": lambda rank: mlp_throughput()}
ONLY_ALONE = {"proposal_warm_start_hand": extra_proposal}   # minutes: only with --only
ONLY = {"proposal": "proposal_warm_start_hand", "spheres": "spheres_64x8", "mixed": "mixed_8192", "impedance": "impedance_modes_jammed_pile_4096x256",
        "adjoint": "adjoint_hand_1024x100", "hand": "hand_rollout_1024x32", "mppi": "mppi_tick_1024x32",
        "mlp": "proposal_mlp_49x256x1024"}


def run_extras(rank):
    """The other workloads, each timed with CUDA events after warm-up (reported beside the headline):
    the small case, mixed batches of uneven worlds in one persistent launch, the impedance modes,
    the hand adjoint, hand rollouts, an MPPI tick and the proposal MLP."""
    return {k: fn(rank) for k, fn in EXTRAS.items()}


def _oracle_sample(nbody, rank):
    """The bounded sample of the headline workload that the oracle steps: for 256 bodies the 16
    sampled worlds (0, 256, ..., 3840) of the seeded 4096-world batch at step 800 of the episode,
    where the GPU's timed window starts (advanced there by the oracle alone,
    oracle/late_states.py); other body counts, 16 worlds of the same workload from the initial
    state.  Returns (scene batch, its step, a description, q, v in FP64)."""
    from paper_2603_12185_gb300 import scenes as S
    late = None
    if nbody == 256 and rank == 0:
        from oracle import late_states as LS
        if os.path.exists(LS.PATH):
            late = LS
    if late is not None:
        sb, _ = late.load()
        start = late.STEPS
        where = (f"worlds {late.WORLDS[0]}, {late.WORLDS[1]}, ..., {late.WORLDS[-1]} of the seeded 4096 x {nbody} "
                 f"batch from their step-{start} state (the start of the GPU's timed window; oracle-advanced)")
    else:
        sb = S.make_pile(16, nbody, seed=R.rank_seed(1000, rank))
        start = 0
        where = f"16 worlds x {nbody} bodies of the same seeded workload from the initial state"
    q = np.concatenate([np.asarray(x, np.float32).astype(np.float64) for x in sb.q0])
    v = np.concatenate([np.asarray(x, np.float32).astype(np.float64) for x in sb.v0])
    return sb, start, where, q, v


def cpu_baseline(nbody, rank, budget_s=40.0, min_steps=100):
    """The FP64 oracle as it stands, OpenMP over the host cores, on the bounded sample of
    `_oracle_sample`, stepped for at least min_steps steps or until the budget is spent."""
    from oracle import oracle as O
    sb, start, where, q, v = _oracle_sample(nbody, rank)
    nw = sb.nworld
    runner = O.BatchRunner([sb.world(w) for w in range(nw)], sb.params)
    cores = O.max_threads()
    chunk, done, t_total, contacts = 5, 0, 0.0, 0
    while done < min_steps or t_total < budget_s / 4:
        t0 = time.perf_counter()
        c = runner.run(q, v, sb.dt, chunk)
        t_total += time.perf_counter() - t0
        done += chunk
        contacts += int(c.sum())
        if t_total > budget_s:
            break
    ws = nw * done / t_total
    return dict(value=ws, unit="world-steps/s", cores=cores, kind="oracle",
                sample=f"{where}, steps {start + 1}..{start + done} (FP64, {cores} OpenMP threads, {t_total:.1f} s)",
                contacts_per_s=contacts / t_total, contacts_per_world=contacts / (nw * done), seconds=t_total,
                steps=done)


def reference_arm(args, budget_s=240.0):
    """The reference arm: the FP64 oracle as it stands, OpenMP over the host cores, timed over
    exactly `args.steps` steps after `args.warmup` untimed ones.  Each step is one oracle step of
    a bounded sample of the workload: for the 256-body headline the 16 sampled worlds of the
    seeded 4096-world batch, continuing from their step-800 state (where the GPU's timed window
    starts; oracle-advanced), otherwise 16 worlds of the same batch from the initial state.  One
    more untimed step measures the step time; if K + W steps of all 16 worlds would exceed
    `budget_s`, each step takes fewer worlds (never fewer than the host's threads)."""
    from oracle import oracle as O
    nbody = args.bodies
    sb, start, where, q, v = _oracle_sample(nbody, 0)
    cores = O.max_threads()
    runner = O.BatchRunner([sb.world(w) for w in range(sb.nworld)], sb.params)
    t0 = time.perf_counter()
    runner.run(q, v, sb.dt, 1)
    t_all = time.perf_counter() - t0
    n = sb.nworld
    if (args.steps + args.warmup) * t_all > budget_s:
        n = max(min(cores, sb.nworld), 1)
        runner = O.BatchRunner([sb.world(w) for w in range(n)], sb.params)
    nq, nv = sum(len(x) for x in sb.q0[:n]), sum(len(x) for x in sb.v0[:n])
    qs, vs = q[:nq].copy(), v[:nv].copy()
    for _ in range(args.warmup):
        runner.run(qs, vs, sb.dt, 1)
    contacts = 0
    t0 = time.perf_counter()
    for _ in range(args.steps):
        contacts += int(runner.run(qs, vs, sb.dt, 1).sum())
    seconds = time.perf_counter() - t0
    ws = n * args.steps / seconds
    first = start + 2 + args.warmup
    sample = (f"{where}; {n} of them per step, one oracle step each, steps {first}..{first + args.steps - 1} timed "
              f"after {args.warmup + 1} untimed (FP64, {cores} OpenMP threads, {seconds:.1f} s)")
    return {"impl": "reference", "metric": METRIC, "value": ws, "unit": "world-steps/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * seconds / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"pile_{args.worlds}x{nbody}", "worlds_sampled": n, "bodies_per_world": nbody},
            "contacts_per_s": contacts / seconds, "contacts_per_world": contacts / (n * args.steps),
            "cpu_baseline": {"value": ws, "unit": "world-steps/s", "cores": cores, "kind": "oracle",
                             "sample": sample, "contacts_per_s": contacts / seconds},
            "e2e": {"value": ws, "unit": "world-steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main():
    args = parse()
    if args.mlp_only:
        print(json.dumps({"proposal_mlp_49x256x1024": mlp_throughput()}), flush=True)
        return
    if args.proposal_size:
        PROPOSAL.update(zip(("iters", "episodes", "goals"), (int(x) for x in args.proposal_size.split(","))))
    if args.only:
        import torch
        from paper_2603_12185_gb300 import build
        build.build()
        torch.cuda.set_device(0)
        name = ONLY[args.only]
        fn = EXTRAS.get(name) or ONLY_ALONE[name]
        print(json.dumps({name: fn(0)}), flush=True)
        return
    if args.impl == "reference":
        if int(os.environ.get("RANK", "0")) == 0:
            print(json.dumps(reference_arm(args)), flush=True)
        return

    import torch
    rank, world, local = dist_setup()
    torch.cuda.set_device(local)
    from paper_2603_12185_gb300 import build
    if rank == 0:
        build.build()
    if world > 1:
        torch.distributed.barrier()
    build.build()
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")  # 256 MB > 129 MB L2

    # sweep: smaller bins first (each also a warm-up of the library)
    sweep = {}
    if not args.no_sweep:
        for n in SWEEP:
            r = run_pile(n, args.worlds, min(args.steps, 100), args.warmup, rank, flush=flush, episode=args.episode,
                         jammed=args.jammed)
            sec = barrier_max(r["ms"] / 1e3, world)
            sweep[str(n)] = {"world_steps_per_s": world * r["worlds"] * r["steps"] / sec,
                             "contacts_per_s": barrier_sum(r["contacts"], world) / sec,
                             "contacts_per_world": r["contacts"] / (r["worlds"] * r["steps"]),
                             "ms_per_step": 1e3 * sec / r["steps"]}
            del r

    clocks = Clocks(local)
    clocks.start()
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    res = run_pile(args.bodies, args.worlds, args.steps, args.warmup, rank, flush=flush, episode=args.episode,
                   jammed=args.jammed, warps=args.warps, impedance=args.impedance)
    torch.cuda.synchronize()
    clk = clocks.stop()
    sec = barrier_max(res["ms"] / 1e3, world)
    total_contacts = barrier_sum(res["contacts"], world)
    value = world * res["worlds"] * res["steps"] / sec
    e2e = run_e2e(res, args.e2e_steps, blocks=args.e2e_blocks) if args.e2e_steps > 0 else None
    if e2e is not None:
        e2e_v = barrier_sum(e2e["value"], world) if world > 1 else e2e["value"]

    pk, src = peaks()
    launch_s = res["per_launch_ms"] / 1e3
    alg_bytes = res["worlds"] * res["bodies"] * BYTES_PER_BODY
    achieved = alg_bytes / launch_s / 1e9
    issue = None
    if INSTRUCTIONS["digest"] == step_digest() and args.impedance == "heuristic":
        sms = torch.cuda.get_device_properties(local).multi_processor_count
        mhz = clk["sm_mhz"] or pk.get("sm_max_mhz", 2070.0)
        ceiling = sms * 4 * mhz * 1e6
        issue = {"warp_instructions_per_launch": INSTRUCTIONS["warp_instructions"],
                 "ceiling_warp_instructions_per_s": ceiling, "sm_mhz": mhz,
                 "frac": INSTRUCTIONS["warp_instructions"] / (ceiling * launch_s)}
    roofline = {"bound": "hbm", "achieved": achieved, "peak": pk["hbm_gbs"], "unit": "GB/s",
                "frac": achieved / pk["hbm_gbs"], "issue": issue,
                "traffic": (TRAFFIC["bytes"] if TRAFFIC["digest"] == step_digest() and args.impedance == "heuristic"
                            else None),
                "kernel_digest": step_digest(), "peak_source": src,
                "kernel": "cf::step_kernel", "algorithmic_bytes_per_launch": alg_bytes}
    line = {"metric": METRIC, "value": value, "unit": "world-steps/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * sec / res["steps"], "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"pile_{res['worlds']}x{res['bodies']}" + ("_jammed" if args.jammed else "") +
                       ("" if args.impedance == "heuristic" else f"_{args.impedance}_impedance"),
                       "worlds_per_gpu": res["worlds"],
                       "bodies_per_world": res["bodies"], "facets_per_contact": 18, "dt": 0.002,
                       "episode_steps": args.episode, "timed_steps": f"last {res['steps']} of the episode",
                       "preroll_untimed": res["preroll"], "l2": "flushed (256 MB write) between timed steps",
                       "parallelism": f"replicas x{world}"},
            "contacts_per_s": total_contacts / sec,
            "contacts_per_world": res["contacts"] / (res["worlds"] * res["steps"]),
            "sweep_bodies": sweep,
            "roofline": roofline,
            "e2e": None if e2e is None else {
                "value": e2e_v, "unit": "world-steps/s", "h2d_bytes_per_step": e2e["h2d"],
                "d2h_bytes_per_step": e2e["d2h"], "api": e2e["api"], "serial_value": e2e["serial"],
                "pipelined_value": e2e["pipelined"], "in_place_value": e2e["in_place"]},
            "gpu_launches": res["steps"],
            "clocks": clk}
    if not args.no_extras:
        line["other_workloads"] = run_extras(rank)
    if rank == 0 and world == 1 and not args.no_cpu:
        cb = cpu_baseline(args.bodies, rank)
        line["cpu_baseline"] = {k: cb[k] for k in ("value", "unit", "cores", "kind", "sample", "contacts_per_s",
                                                    "contacts_per_world")}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.barrier()
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
