"""The learner's data-parallel update (Algorithm 1 over environments split
across ranks): two gloo ranks of N/2 environments each apply, after every
learning episode, the update one process over all N environments applies.
CPU only: the simulator is replaced by a small differentiable stand-in (a
damped cart with a pendulum-like coordinate, written in PyTorch) and the
TD-lambda targets by the oracle's term-by-term definition; the learner's own
logic (sharded rollouts, sliced noise and minibatches, gradient and statistics
all-reduce) is what runs."""
import os
import socket
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

N, H, EPISODES = 8, 4, 2


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _dynamics(q, qd, a):
    """Stand-in for the simulator on cart-pole-shaped state blocks (q, qd
    [2][n], a [1][n]): a semi-implicit step of a linear damped system driven
    by the action, reward -(theta^2 + 0.1 x^2)."""
    n = a.numel()
    q2, qd2 = q.view(2, n), qd.view(2, n)
    dt = 1.0 / 60.0
    acc = torch.stack([2.0 * a.view(n) - 0.5 * q2[0] - 0.1 * qd2[0],
                       9.81 * q2[1] - 3.0 * a.view(n) - 0.2 * qd2[1]])
    qdn = qd2 + dt * acc
    qn = q2 + dt * qdn
    r = -(qn[1] ** 2 + 0.1 * qn[0] ** 2)
    return qn.reshape(-1), qdn.reshape(-1), r


def _targets(reward, value, done, gamma, lam):
    from oracle import oracle
    t = oracle.td_lambda(reward.double().numpy(), value.double().numpy(), done.numpy().astype(bool), gamma, lam)
    return torch.from_numpy(np.asarray(t, np.float32))


def _run(group):
    sys.path.insert(0, ROOT)
    from paper_2204_07137_gb300 import inputs as I
    from paper_2204_07137_gb300.shac import SHAC
    agent = SHAC(I.cartpole(), n_envs=N, h=H, episodes=10, seed=3, critic_iters=2, group=group,
                 dynamics=_dynamics, targets=_targets, device="cpu")
    init = [p.detach().clone().numpy() for p in list(agent.actor.parameters()) + list(agent.critic.parameters())]
    stats = [agent.episode()]
    grads = [p.grad.detach().clone().numpy() for p in agent.actor.parameters()]   # all-reduced, episode 1
    stats += [agent.episode() for _ in range(EPISODES - 1)]
    params = [p.detach().clone().numpy() for p in list(agent.actor.parameters()) + list(agent.critic.parameters())]
    return init, grads, params, stats, agent.norm.mean.numpy().copy()


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    torch.set_num_threads(1)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        out[rank] = _run(dist)
    finally:
        dist.destroy_process_group()


def test_two_ranks_of_half_the_environments_apply_the_single_rank_update():
    torch.set_num_threads(1)
    init, ref_grads, ref_params, ref_stats, ref_mean = _run(None)
    port = _free_port()
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_worker, args=(2, port, out), nprocs=2, join=True)
    _, g0, p0, s0, m0 = out[0]
    _, g1, p1, s1, m1 = out[1]
    for a, b in zip(p0, p1):          # every rank holds the same networks
        np.testing.assert_array_equal(a, b)
    # the summed actor gradient of the first episode is the single process's
    # (up to FP32 reassociation of the sum over environments)
    for a, b in zip(g0, ref_grads):
        np.testing.assert_allclose(a, b, rtol=1e-5, atol=1e-6 * np.abs(b).max())
    # after the episodes' Adam steps: Adam divides each gradient component by
    # its own magnitude, so a component that is zero up to rounding moves by a
    # rounding-dependent step; the parameters agree to a small fraction of the
    # update each tensor received
    for a, b, c in zip(p0, ref_params, init):
        step = np.abs(b - c).max()
        np.testing.assert_allclose(a, b, rtol=0, atol=max(2e-3 * step, 1e-7))
    # observation statistics: the second episode runs on networks that differ at rounding level
    np.testing.assert_allclose(m0, ref_mean, rtol=1e-6, atol=1e-9)
    for a, b in zip(s0, ref_stats):
        np.testing.assert_allclose(a["policy_loss"], b["policy_loss"], rtol=1e-5)
        np.testing.assert_allclose(a["mean_reward"], b["mean_reward"], rtol=1e-5)
        np.testing.assert_allclose(a["critic_loss"], b["critic_loss"], rtol=1e-4)
    # the update is not trivially zero
    assert any(np.abs(a).sum() > 0 for a in ref_params)


def test_environment_count_must_split_over_the_ranks():
    class FakeGroup:
        def get_world_size(self):
            return 3

        def get_rank(self):
            return 0
    sys.path.insert(0, ROOT)
    from paper_2204_07137_gb300 import inputs as I
    from paper_2204_07137_gb300.shac import SHAC
    with pytest.raises(ValueError):
        SHAC(I.cartpole(), n_envs=8, h=H, group=FakeGroup(), dynamics=_dynamics, targets=_targets, device="cpu")
