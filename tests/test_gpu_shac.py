"""Learner on the GPU (Sec. 3.2, Algorithm 1): the TD-lambda target kernel
against the oracle's term-by-term Eq. td-lambda, and short training runs of
the short-horizon actor-critic learner through the simulator."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2204_07137_gb300 import build
    build.build()


@pytest.mark.parametrize("h,N,p_done,lam", [(32, 1001, 0.05, 0.95), (7, 37, 0.0, 0.95), (5, 300, 0.3, 0.0),
                                            (9, 64, 0.1, 1.0), (1, 10, 0.5, 0.95)])
def test_td_lambda_kernel_matches_oracle(oracle_mod, h, N, p_done, lam):
    from paper_2204_07137_gb300.shac import td_lambda
    rng = np.random.default_rng(h * 1000 + N)
    r = rng.normal(size=(h, N)).astype(np.float32)
    v = rng.normal(scale=10.0, size=(h + 1, N)).astype(np.float32)
    d = (rng.random((h, N)) < p_done).astype(np.uint8)
    got = td_lambda(torch.from_numpy(r).cuda(), torch.from_numpy(v).cuda(),
                    torch.from_numpy(d).cuda() if p_done > 0 else None, 0.99, lam)
    torch.cuda.synchronize()
    ref = oracle_mod.td_lambda(r, v, d if p_done > 0 else None, 0.99, lam)
    # FP32: a target sums at most h terms of size |r| + |V|
    np.testing.assert_allclose(got.cpu().numpy(), ref, rtol=1e-5, atol=2e-6 * h * (1 + np.abs(v).max()))


def test_shac_learns_on_the_cartpole():
    """Algorithm 1 end to end with the cart-pole hyperparameters of the
    appendix table (N = 64, h = 32): the untrained deterministic policy lets
    the pole fall and spin (mean reward over the 240-step task horizon far
    below -20; a pole hanging still scores about -pi^2), and within 120
    learning episodes (learning-rate schedule over 200; evaluated every 20) the
    learned policy removes at least 90 % of that cost, and the training reward
    of the last 20 episodes beats that of the first 20.  A single fixed-seed
    run's evaluation is chaotic in the FP32 rounding of the simulator (a
    240-step rollout of a falling pole), so the test asks for the improvement,
    not for a fixed reward level."""
    from paper_2204_07137_gb300 import inputs as I
    from paper_2204_07137_gb300.shac import SHAC
    agent = SHAC(I.cartpole(), n_envs=64, h=32, episodes=200, seed=0)
    before = agent.evaluate(240, 0)
    evals, hist = [], []
    for k in range(120):
        hist.append(agent.episode())
        if (k + 1) % 20 == 0:
            evals.append(agent.evaluate(240, 0))
    for s in hist:
        assert np.isfinite([s["policy_loss"], s["critic_loss"], s["mean_reward"]]).all()
    first = np.mean([s["mean_reward"] for s in hist[:20]])
    last = np.mean([s["mean_reward"] for s in hist[-20:]])
    assert before < -20.0 and max(evals) > 0.1 * before and last > first, (before, evals, first, last)
    assert agent.sim.status() == 0


def test_shac_episode_on_a_free_root_model_with_early_termination():
    """Ant-like model: episodes with height terminations run, reset and keep
    every loss finite (the reset cuts the gradient)."""
    from paper_2204_07137_gb300 import inputs as I
    from paper_2204_07137_gb300.shac import SHAC
    agent = SHAC(I.ant(), n_envs=32, h=8, episodes=4, seed=1)
    for _ in range(3):
        s = agent.episode()
        assert np.isfinite([s["policy_loss"], s["critic_loss"], s["mean_reward"]]).all()
    assert all(torch.isfinite(p.grad).all() for p in agent.actor.parameters() if p.grad is not None)
