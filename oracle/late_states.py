"""Late-episode states of the dense-contact workload, advanced by the FP64 oracle alone.

TEST INFRASTRUCTURE ONLY, like the rest of oracle/: the GPU parity tests on the settled
256-body pile and the timed CPU baseline of bench.py start from these states.  Nothing here
touches the CUDA path: the states come from the seeded generator and the oracle's own steps.

Workload: the walled-bin batch of 4096 worlds x 256 bodies with the seed of the benchmark's
first replica (1000); the 16 worlds 0, 256, ..., 3840 are advanced STEPS steps (dt = 2 ms) from
their initial states, which are the same FP32-rounded values the GPU starts from.  The
benchmark times steps STEPS+1.. of the same episode on the GPU, so these are the same worlds at
the same point of the episode (on the oracle's own trajectory).  Saved as float32, the
precision both sides take their inputs in, to late_states_pile256.npz beside this file.

    python -m oracle.late_states          # a few minutes on 8 host cores
"""
from __future__ import annotations

import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from oracle import oracle as O  # noqa: E402
from paper_2603_12185_gb300 import scenes as S  # noqa: E402

PATH = os.path.join(HERE, "late_states_pile256.npz")
SEED, NWORLD, NBODY = 1000, 4096, 256
WORLDS = tuple(range(0, NWORLD, 256))
STEPS = 800


def batch():
    """The sampled worlds (a scenes.Batch) with their initial states."""
    return S.make_pile(NWORLD, NBODY, seed=SEED).subset(WORLDS)


def load():
    """(scenes.Batch of the sampled worlds holding their step-STEPS states, contacts per world at
    the last step).  The states are FP32 values widened to FP64."""
    z = np.load(PATH)
    sb = batch()
    nq, nv = 7 * NBODY, 6 * NBODY
    sb.q0 = [z["q"][i * nq:(i + 1) * nq].astype(np.float64) for i in range(len(WORLDS))]
    sb.v0 = [z["v"][i * nv:(i + 1) * nv].astype(np.float64) for i in range(len(WORLDS))]
    return sb, z["contacts"]


def main():
    sb = batch()
    runner = O.BatchRunner([sb.world(w) for w in range(sb.nworld)], sb.params)
    q = np.concatenate([np.asarray(x, np.float32).astype(np.float64) for x in sb.q0])
    v = np.concatenate([np.asarray(x, np.float32).astype(np.float64) for x in sb.v0])
    t0 = time.perf_counter()
    contacts = None
    for done in range(0, STEPS, 100):
        n = min(100, STEPS - done)
        runner.run(q, v, sb.dt, n - 1)
        contacts = runner.run(q, v, sb.dt, 1)
        print(f"step {done + n}: {contacts.mean():.0f} contacts per world, {time.perf_counter() - t0:.0f} s",
              flush=True)
    np.savez_compressed(PATH, q=q.astype(np.float32), v=v.astype(np.float32), contacts=contacts,
                        worlds=np.array(WORLDS), steps=STEPS, seed=SEED)
    print("wrote", PATH)


if __name__ == "__main__":
    main()
