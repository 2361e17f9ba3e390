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
