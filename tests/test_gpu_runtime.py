"""GPU runtime properties of the C ABI: determinism across launch shapes, fused multi-step
equals repeated steps, state round trips, subsets, error reporting."""
import numpy as np
import pytest
import torch

import parity as PR
from paper_2603_12185_gb300 import comfree as CF
from paper_2603_12185_gb300 import scenes as S

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2603_12185_gb300 import build
    build.build()


def _state(b):
    q, v = b.get_state()
    torch.cuda.synchronize()
    return q.cpu().numpy(), v.cpu().numpy()


def test_results_do_not_depend_on_warps_per_world():
    """Impulses accumulate in fixed point, so the sum is order independent: every launch shape
    gives bitwise the same state."""
    sb = S.make_pile(16, 64, seed=3, jammed=True)
    ref = None
    for wp in (1, 2, 4, 8):
        _, b = CF.from_scenes(sb)
        b.set_warps(0, wp)
        for _ in range(5):
            b.step(sb.dt, 1)
        st = _state(b)
        if ref is None:
            ref = st
        else:
            assert np.array_equal(st[0], ref[0]) and np.array_equal(st[1], ref[1]), f"warps={wp}"


def test_fused_steps_equal_repeated_steps():
    sb = S.make_mixed(16, seed=4)
    _, b1 = CF.from_scenes(sb)
    _, b2 = CF.from_scenes(sb)
    b1.step(sb.dt, 20)
    for _ in range(20):
        b2.step(sb.dt, 1)
    s1, s2 = _state(b1), _state(b2)
    assert np.array_equal(s1[0], s2[0]) and np.array_equal(s1[1], s2[1])


def test_graph_replay_equals_eager_steps():
    """The all-world step captured in a CUDA graph (mixed piles and hands, one launch per
    step) replays bit-identically to eager launches from the same state."""
    sb = S.make_mixed(64, seed=11)
    _, b = CF.from_scenes(sb)
    b.step(sb.dt, 2)
    q0, v0 = _state(b)
    b.set_state(torch.from_numpy(q0).cuda(), torch.from_numpy(v0).cuda())
    for _ in range(6):
        b.step(sb.dt, 1)
    qe, ve = _state(b)
    ce = b.contact_counts()
    b.set_state(torch.from_numpy(q0).cuda(), torch.from_numpy(v0).cuda())
    g = b.graph(sb.dt, 1, repeat=3)          # one eager step, then three captured ones
    b.set_state(torch.from_numpy(q0).cuda(), torch.from_numpy(v0).cuda())
    g.replay()
    g.replay()
    qg, vg = _state(b)
    assert np.array_equal(qg, qe) and np.array_equal(vg, ve)
    assert np.array_equal(b.contact_counts(), ce)
    st, _ = b.status()
    assert st == 0


def test_pipeline_matches_one_batch():
    """comfree.Pipeline (blocks of worlds on their own streams, state in pinned host memory)
    gives bit-identical states to stepping all worlds in one batch."""
    sb = S.make_pile(8, 16, seed=21)
    _, full = CF.from_scenes(sb)
    full.step(sb.dt, 20)
    q0, v0 = _state(full)
    blocks, hq, hv = [], [], []
    qo = vo = 0
    for lo, hi in ((0, 3), (3, 8)):
        _, bk = CF.from_scenes(sb.subset(range(lo, hi)))
        blocks.append(bk)
        hq.append(torch.from_numpy(q0[qo:qo + bk.total_nq].copy()).pin_memory())
        hv.append(torch.from_numpy(v0[vo:vo + bk.total_nv].copy()).pin_memory())
        qo += bk.total_nq
        vo += bk.total_nv
    pipe = CF.Pipeline(blocks)
    for _ in range(3):
        pipe.step(hq, hv, sb.dt)
    for _ in range(3):
        full.step(sb.dt, 1)
    q1, v1 = _state(full)
    assert np.array_equal(np.concatenate([t.numpy() for t in hq]), q1)
    assert np.array_equal(np.concatenate([t.numpy() for t in hv]), v1)
    assert all(st == 0 for st, _ in pipe.status())


@pytest.mark.parametrize("kind", ["pile", "mixed"])
def test_step_host_matches_device_steps(kind):
    """cf_step_host (the kernel reads and writes the state in pinned host memory) gives states
    bit-identical to device steps of the same batch, leaves the batch's device state alone, and
    refuses pageable host memory."""
    sb = S.make_pile(8, 64, seed=23) if kind == "pile" else S.make_mixed(8, seed=23)
    _, b = CF.from_scenes(sb)
    b.step(sb.dt, 30)
    q0, v0 = _state(b)
    hq = torch.from_numpy(q0.copy()).pin_memory()
    hv = torch.from_numpy(v0.copy()).pin_memory()
    for _ in range(4):
        b.step_host(hq, hv, sb.dt)
    torch.cuda.synchronize()
    qd, vd = _state(b)
    assert np.array_equal(qd, q0) and np.array_equal(vd, v0)   # the device state untouched
    for _ in range(4):
        b.step(sb.dt, 1)
    q1, v1 = _state(b)
    assert np.array_equal(hq.numpy().view(np.uint32), q1.view(np.uint32))
    assert np.array_equal(hv.numpy().view(np.uint32), v1.view(np.uint32))
    assert b.status()[0] == 0
    pq = torch.from_numpy(q0.copy())
    pv = torch.from_numpy(v0.copy())
    with pytest.raises(CF.CfError, match="page-locked"):
        CF.check(CF.lib().cf_step_host(b.h, CF._ptr(pq), CF._ptr(pv), float(sb.dt), 1, CF._stream()))


def test_state_round_trip_host_and_device():
    sb = S.make_mixed(8, seed=5)
    _, b = CF.from_scenes(sb)
    q, v = PR.f32(np.concatenate(sb.q0)).astype(np.float32), PR.f32(np.concatenate(sb.v0)).astype(np.float32)
    v = v + np.float32(0.25)
    b.set_state(q, v)                      # host pointers
    qo = np.empty_like(q)
    vo = np.empty_like(v)
    b.get_state(qo, vo)                    # host pointers
    assert np.array_equal(qo, q) and np.array_equal(vo, v)
    qd, vd = b.get_state()
    assert np.array_equal(qd.cpu().numpy(), q)


def test_subset_step_leaves_other_worlds_alone():
    sb = S.make_pile(10, 16, seed=6, jammed=True)
    _, b = CF.from_scenes(sb)
    q0, v0 = _state(b)
    b.step(sb.dt, 3, worlds=[1, 4, 7])
    q1, v1 = _state(b)
    nq, nv = 7 * 16, 6 * 16
    for w in range(10):
        same = np.array_equal(q1[w * nq:(w + 1) * nq], q0[w * nq:(w + 1) * nq])
        assert same == (w not in (1, 4, 7))
    _, b2 = CF.from_scenes(sb.subset([4]))
    b2.step(sb.dt, 3)
    q2, _ = _state(b2)
    assert np.array_equal(q2, q1[4 * nq:5 * nq])


def test_nonfinite_state_is_reported():
    sb = S.make_pile(4, 16, seed=7)
    _, b = CF.from_scenes(sb)
    q, v = _state(b)
    v[6 * 16 + 3] = np.nan          # world 1, body 0, angular velocity
    b.set_state(torch.from_numpy(q).cuda(), torch.from_numpy(v).cuda())
    b.step(sb.dt, 1)
    st, flags = b.status()
    assert st == 5 and flags[1] & 1 and not flags[0] & 1
    st, _ = b.status(clear=True)
    st, flags = b.status()
    assert st == 0 and not flags.any()


def test_velocity_change_out_of_range_is_reported():
    """Two overlapping spheres closing at 1e6 m/s: the contact's velocity change exceeds the
    pile scatter's range, which raises CF_FLAG_RANGE (8) and CF_ERR_NONFINITE (5) instead of
    wrapping the fixed-point words."""
    sb = S.make_pile(2, 16, seed=7)
    _, b = CF.from_scenes(sb)
    q, v = _state(b)
    nq, nv = 7 * 16, 6 * 16
    q[nq:nq + 3] = [0.0, 0.0, 0.2]                  # world 1: body 0 and body 1 overlap
    q[nq + 7:nq + 10] = [0.0, 0.0, 0.2 + 0.01]
    v[nv + 2] = 1e6
    v[nv + 6 + 2] = -1e6
    b.set_state(torch.from_numpy(q).cuda(), torch.from_numpy(v).cuda())
    b.step(sb.dt, 1)
    st, flags = b.status()
    assert st == 5 and flags[1] & 8 and not flags[0] & 8
    b.status(clear=True)


def test_invalid_arguments_are_rejected():
    sb = S.make_pile(2, 16, seed=8)
    _, b = CF.from_scenes(sb)
    with pytest.raises(CF.CfError) as e:
        b.step(-1.0, 1)
    assert e.value.status == 1
    with pytest.raises(CF.CfError):
        b.step(sb.dt, 1, worlds=[0, 0])
    with pytest.raises(CF.CfError):
        b.step(sb.dt, 1, worlds=[5])
    with pytest.raises(CF.CfError) as e:
        b.contacts()
    assert e.value.status == 7


def test_contact_capture_overflow_is_reported():
    sb = S.make_pile(2, 64, seed=9, jammed=True)
    _, b = CF.from_scenes(sb, contact_capture=4)
    b.step(sb.dt, 1)
    with pytest.raises(CF.CfError) as e:
        b.contacts()
    assert e.value.status == 4


def test_autotune_keeps_state_and_results():
    sb = S.make_mixed(16, seed=10)
    _, b1 = CF.from_scenes(sb)
    chosen = b1.autotune(sb.dt)
    assert all(c in (1, 2, 4, 8) for c in chosen)
    _, b2 = CF.from_scenes(sb)
    b1.step(sb.dt, 4)
    b2.step(sb.dt, 4)
    s1, s2 = _state(b1), _state(b2)
    assert np.array_equal(s1[0], s2[0]) and np.array_equal(s1[1], s2[1])
