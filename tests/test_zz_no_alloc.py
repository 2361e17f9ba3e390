"""cf_step_noalloc: the entry point for callers that cannot allocate device memory (its scratch
is a static device array).  Checked against the regular batch path (cf_step) through the C ABI
on two calls in a row.  Collected last on purpose (file name), and independent of the other
tests: it builds everything it needs in its own process state."""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2603_12185_gb300 import build
    build.build()


def _template_blocks(sb):
    """sb with every world's parameter block set to the template's own bodies and geoms, so the
    batch path (which always reads blocks for piles) computes what a call without blocks does."""
    from paper_2603_12185_gb300 import scenes as S
    t = sb.templates[0]
    nb = t.nbody
    blk = np.zeros((nb, 8))
    blk[:, 0] = t.body_mass
    blk[:, 1:4] = t.body_inertia
    blk[:, 4] = t.geom_type[:nb]
    blk[:, 5:8] = t.geom_size[:nb]
    out = sb.subset(range(sb.nworld))
    out.world_param = [blk.copy() for _ in range(sb.nworld)]
    assert (t.geom_type[:nb] == S.SPHERE).all()
    return out


def _reference(sb, nsteps, calls):
    from paper_2603_12185_gb300 import comfree as CF
    _, b = CF.from_scenes(sb)
    out = []
    for _ in range(calls):
        b.step(sb.dt, nsteps)
        q, v = b.get_state()
        torch.cuda.synchronize()
        out.append((q.cpu().numpy(), v.cpu().numpy(), b.contact_counts()))
    return out


@pytest.mark.parametrize("maker", ["pile", "hand"])
def test_noalloc_matches_batch_step_on_two_calls(maker):
    from paper_2603_12185_gb300 import comfree as CF
    from paper_2603_12185_gb300 import scenes as S
    sb = S.make_pile(24, 64, seed=21, jammed=True) if maker == "pile" else S.make_hand(16, seed=22)
    ref = _reference(sb, 3, 2)
    model = CF.Model(sb.templates, sb.params)
    q0, v0 = CF.flatten_state(sb)
    q = torch.from_numpy(q0).cuda()
    v = torch.from_numpy(v0).cuda()
    wp = CF.flatten_params(sb)
    wp = None if wp is None else torch.from_numpy(wp).cuda()
    counts = torch.zeros(sb.nworld, dtype=torch.int32, device="cuda")
    for call in range(2):
        CF.step_noalloc(model, 0, sb.nworld, q, v, wp, sb.dt, 3, counts)
        torch.cuda.synchronize()
        rq, rv, rc = ref[call]
        qn, vn = q.cpu().numpy(), v.cpu().numpy()
        np.testing.assert_allclose(qn, rq, rtol=0, atol=2e-6)
        err = np.abs(vn - rv).max() / (np.abs(rv).max() + 9.81 * sb.dt)
        assert err <= 1e-4
        assert np.array_equal(counts.cpu().numpy(), rc)


def test_noalloc_template_pile_on_a_side_stream():
    """A pile call without parameter blocks (the scene's own bodies and geoms) and without a
    contact-count output, enqueued on a non-default stream, against the batch path."""
    from paper_2603_12185_gb300 import comfree as CF
    from paper_2603_12185_gb300 import scenes as S
    sb = _template_blocks(S.make_pile(12, 64, seed=24, jammed=True))
    ref = _reference(sb, 2, 2)
    model = CF.Model(sb.templates, sb.params)
    q0, v0 = CF.flatten_state(sb)
    q = torch.from_numpy(q0).cuda()
    v = torch.from_numpy(v0).cuda()
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    for call in range(2):
        with torch.cuda.stream(side):
            CF.step_noalloc(model, 0, sb.nworld, q, v, None, sb.dt, 2, None, stream=side)
        side.synchronize()
        rq, rv, _ = ref[call]
        np.testing.assert_allclose(q.cpu().numpy(), rq, rtol=0, atol=2e-6)
        vn = v.cpu().numpy()
        assert np.abs(vn - rv).max() / (np.abs(rv).max() + 9.81 * sb.dt) <= 1e-4


def test_noalloc_rejects_misaligned_parameter_blocks():
    """The kernel reads the blocks as float4: a pointer off a 16-byte boundary is refused on the
    host, before any launch, and the state is left as it was."""
    from paper_2603_12185_gb300 import comfree as CF
    from paper_2603_12185_gb300 import scenes as S
    sb = S.make_pile(4, 16, seed=25, jammed=True)
    model = CF.Model(sb.templates, sb.params)
    q0, v0 = CF.flatten_state(sb)
    q = torch.from_numpy(q0).cuda()
    v = torch.from_numpy(v0).cuda()
    wp = torch.from_numpy(CF.flatten_params(sb)).cuda()
    shifted = torch.zeros(wp.numel() + 4, device="cuda")
    shifted[1:1 + wp.numel()] = wp
    with pytest.raises(CF.CfError) as e:
        CF.step_noalloc(model, 0, sb.nworld, q, v, shifted[1:], sb.dt, 1)
    assert e.value.status == 1
    torch.cuda.synchronize()
    assert np.array_equal(q.cpu().numpy(), q0) and np.array_equal(v.cpu().numpy(), v0)


def test_noalloc_rejects_oversized_calls():
    from paper_2603_12185_gb300 import comfree as CF
    from paper_2603_12185_gb300 import scenes as S
    sb = S.make_pile(1, 16, seed=23)
    model = CF.Model(sb.templates, sb.params)
    q = torch.zeros(16385 * 112, device="cuda")
    v = torch.zeros(16385 * 96, device="cuda")
    with pytest.raises(CF.CfError) as e:
        CF.step_noalloc(model, 0, 16385, q, v, None, sb.dt, 1)
    assert e.value.status == 1
