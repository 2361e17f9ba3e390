"""The multi-GPU path of the bench is replicas only: every rank owns distinct worlds, and only
timings/counts are reduced.  Checked with two gloo ranks on the CPU."""
import os
import socket

import pytest
import torch.multiprocessing as mp

from paper_2603_12185_gb300 import replicas as R


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    import numpy as np
    import torch.distributed as dist
    from paper_2603_12185_gb300 import scenes as S
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    sb = S.make_pile(4, 16, seed=R.rank_seed(7, rank))
    ms = 10.0 + rank                     # this rank's measured time
    contacts = 100 * (rank + 1)
    out[rank] = dict(q0=np.concatenate(sb.q0)[:8].tolist(), tmax=R.reduce_scalar(ms, "max"),
                     csum=R.reduce_scalar(contacts, "sum"))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_own_distinct_worlds_and_reduce_timings():
    port = _free_port()
    with mp.get_context("spawn").Manager() as m:  # no fork of a process that may hold OpenMP threads
        out = m.dict()
        mp.spawn(_worker, args=(2, port, out), nprocs=2, join=True)
        res = dict(out)
    assert res[0]["q0"] != res[1]["q0"]               # distinct seeded worlds per rank
    assert res[0]["tmax"] == res[1]["tmax"] == 11.0   # max over ranks
    assert res[0]["csum"] == res[1]["csum"] == 300.0  # whole-job sum


@pytest.mark.parametrize("total,world", [(4096, 1), (4096, 2), (10, 3), (8192, 8)])
def test_world_blocks_partition(total, world):
    blocks = [R.world_block(total, r, world) for r in range(world)]
    assert blocks[0][0] == 0 and blocks[-1][1] == total
    assert all(blocks[i][1] == blocks[i + 1][0] for i in range(world - 1))
    assert max(b - a for a, b in blocks) - min(b - a for a, b in blocks) <= 1
