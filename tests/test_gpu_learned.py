"""What the learned proposal gains in sampling MPC (the hand application of Sec. V, with a
learned sampling distribution added to it).

Plain MPPI (1024 rollouts) runs seeded training episodes; every tick's updated plan is an
elite target; the tensor-core MLP is trained on them by the library's own kernels.  Then, on
held-out starts and goals, the best rollout cost of the first tick from a cold start is
compared: 64 rollouts with half drawn from the proposal against plain sampling with 64 and
with 256 rollouts.  Every rollout is simulated and scored by the engine in both arms."""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def trained():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2603_12185_gb300 import build
    build.build()
    from paper_2603_12185_gb300 import mppi as MP
    from paper_2603_12185_gb300 import scenes as S
    tpl = S.hand_template(0)
    params = S.Params(**dict(S.HAND_PARAMS, d_user=0.002))
    log = {}
    mlp, _ = MP.collect_and_train(tpl, params, episodes=24, ticks=80, N=1024, seed=0, epochs=800, log=log)
    return MP, tpl, params, mlp, log


def test_training_lowers_the_nll(trained):
    _, _, _, _, log = trained
    assert log["samples"] >= 1500
    assert log["loss_last"] < 0.6 * log["loss_first"]


def test_proposal_finds_better_cold_start_plans_with_fewer_rollouts(trained):
    MP, tpl, params, mlp, _ = trained
    plain64 = MP.cold_start_costs(tpl, params, 64)
    learned64 = MP.cold_start_costs(tpl, params, 64, mlp=mlp, n_prop=32)
    plain256 = MP.cold_start_costs(tpl, params, 256)
    assert np.all(np.isfinite(learned64))
    print("cold-start best rollout cost: plain64 %.3f learned64 %.3f plain256 %.3f"
          % (plain64.mean(), learned64.mean(), plain256.mean()))
    assert learned64.mean() < plain64.mean()
    assert learned64.mean() < plain256.mean()


def test_learned_warm_start_with_zero_output_is_plain_mppi():
    """The learned warm start samples around m + D, D the network's correction of the plan: a
    network whose output is exactly zero (all parameters zero: GELU(0) = 0) must reproduce plain
    MPPI bit for bit, plans and plant states alike."""
    from paper_2603_12185_gb300 import build
    build.build()
    from paper_2603_12185_gb300 import comfree as CF
    from paper_2603_12185_gb300 import mppi as MP
    from paper_2603_12185_gb300 import scenes as S
    tpl = S.hand_template(0)
    params = S.Params(**dict(S.HAND_PARAMS, d_user=0.002))
    fin = MP.NQ + MP.NV + 4 + MP.PLAN_IN
    probe = CF.Mlp(fin, 256, 2 * 32 * MP.NU, max_batch=4, seed=0)
    zero = CF.Mlp(fin, 256, 2 * 32 * MP.NU, max_batch=4, params=np.zeros(probe.nparam, np.float32))
    sb = S.make_hand(1, seed=31)
    goal = MP.random_goal(sb.q0[0], np.random.default_rng(3))
    plans = []
    for mlp in (None, zero):
        ctl = MP.HandMPPI(tpl, params, N=128, seed=5, mlp=mlp, mode="warm")
        ctl.reset(sb.q0[0], sb.v0[0], goal)
        plans.append([ctl.tick().cpu().numpy() for _ in range(5)] + [ctl.plant_state()[0]])
    for a, b in zip(*plans):
        np.testing.assert_array_equal(a, b)


def test_dagger_training_lowers_the_nll():
    """Two DAgger iterations of the learned warm start on a few episodes: the labels (1024-rollout
    teacher plans minus the warm start) are finite and each iteration's training lowers the NLL."""
    from paper_2603_12185_gb300 import build
    build.build()
    from paper_2603_12185_gb300 import mppi as MP
    from paper_2603_12185_gb300 import scenes as S
    tpl = S.hand_template(0)
    params = S.Params(**dict(S.HAND_PARAMS, d_user=0.002))
    log = {}
    MP.dagger_warm_start(tpl, params, iters=2, episodes=4, ticks=20, N=128, N_teacher=512, epochs=200, seed=1,
                         log=log)
    st = log["dagger"]
    assert [s["samples"] for s in st] == [80, 160]
    for s in st:
        assert np.isfinite(s["nll_last"]) and s["nll_last"] < s["nll_first"]
