"""Policy in the loop (muscle-actuated lower body, config 5): the actor
gradient dL/dtheta of an h-step window, computed by PyTorch autograd through
the library's step adjoint, against the appendix A.1 recursion evaluated with
the FP64 oracle's step adjoints and a float64 CPU copy of the policy at the
GPU's states and actions; and CUDA-graph capture of forward + backward."""
import copy

import numpy as np
import pytest

from helpers import assert_grad_close
from paper_2204_07137_gb300 import inputs as I

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2204_07137_gb300 import build
    build.build()


def T(x):
    return torch.from_numpy(np.ascontiguousarray(np.asarray(x, np.float32).reshape(-1))).cuda()


def _setup(N, h, seed=0):
    from paper_2204_07137_gb300.policy import PolicyMLP, observation_size
    from paper_2204_07137_gb300.sim import Simulator
    m = I.mtu()
    sim = Simulator([(m, N)], form="batched", h_max=1)
    g = torch.Generator().manual_seed(seed)
    pol = PolicyMLP(observation_size(m), m.na, generator=g).cuda()
    q0, qd0 = I.initial_state(m, N, seed)
    return m, sim, pol, T(q0), T(qd0)


def test_policy_window_gradient_matches_oracle_recursion(oracle_mod):
    from paper_2204_07137_gb300.policy import free_root_observation, policy_window_loss
    N, h = 2, 3
    m, sim, pol, q0, qd0 = _setup(N, h)
    keep = []
    loss = policy_window_loss(sim, pol, q0, qd0, h, keep)
    loss.backward()
    g_gpu = torch.cat([p.grad.reshape(-1) for p in pol.parameters()]).cpu().numpy()
    assert np.isfinite(g_gpu).all() and np.abs(g_gpu).max() > 0

    o = oracle_mod.Oracle(m)
    pol64 = copy.deepcopy(pol).double().cpu()
    params = list(pol64.parameters())
    theta_bar = [torch.zeros_like(p) for p in params]
    qbar = np.zeros((N, m.nq))
    qdbar = np.zeros((N, m.nv))
    rbar = np.full(N, -1.0 / (N * h))
    for t in range(h - 1, -1, -1):
        q, qd, a = (x.detach().cpu().numpy().astype(np.float64) for x in keep[t])
        q, qd, a = q.reshape(m.nq, N), qd.reshape(m.nv, N), a.reshape(m.na, N)
        sq, sqd, sa = o.step_vjp(q.T, qd.T, a.T, qbar, qdbar, rbar)
        qt = torch.tensor(q, requires_grad=True)
        qdt = torch.tensor(qd, requires_grad=True)
        a64 = pol64(free_root_observation(qt, qdt))
        grads = torch.autograd.grad(a64, [qt, qdt] + params, grad_outputs=torch.tensor(sa))
        for k, gk in enumerate(grads[2:]):
            theta_bar[k] += gk
        qbar = sq + grads[0].numpy().T
        qdbar = sqd + grads[1].numpy().T
    g_ref = torch.cat([x.reshape(-1) for x in theta_bar]).numpy()
    assert_grad_close(g_gpu[:, None], g_ref[:, None], "policy window dL/dtheta", axis_env=-1)


def test_policy_window_graph_capture_replays_forward_and_backward():
    """The whole window - observation, policy, simulator steps, and the actor
    gradient through the step adjoints - captured in one CUDA graph; replays
    reproduce the eager loss and gradient."""
    from paper_2204_07137_gb300.policy import policy_window_loss
    N, h = 4, 3
    m, sim, pol, q0, qd0 = _setup(N, h, seed=1)
    params = list(pol.parameters())
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):   # eager reference and warm-up on a side stream, never the legacy one
        loss_ref = policy_window_loss(sim, pol, q0, qd0, h)
        g_ref = torch.autograd.grad(loss_ref, params)
        for _ in range(2):
            torch.autograd.grad(policy_window_loss(sim, pol, q0, qd0, h), params)
    torch.cuda.current_stream().wait_stream(s)
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        loss_g = policy_window_loss(sim, pol, q0, qd0, h)
        g_g = torch.autograd.grad(loss_g, params)
    for _ in range(2):
        graph.replay()
        torch.cuda.synchronize()
        assert torch.allclose(loss_g, loss_ref, rtol=1e-6, atol=0)
        for a, b in zip(g_g, g_ref):
            assert torch.allclose(a, b, rtol=1e-5, atol=1e-9)


def test_full_size_policy_window_gradient_on_sampled_environments(oracle_mod):
    """512 environments, h = 8, the loss restricted to 4 sampled environments
    by its per-environment weights (environments are independent, so dL/dtheta
    is exactly their contribution): GPU autograd through the step adjoints
    against the appendix A.1 recursion over the sampled environments."""
    from paper_2204_07137_gb300.policy import free_root_observation, policy_window_loss
    N, h = 512, 8
    m, sim, pol, q0, qd0 = _setup(N, h, seed=2)
    envs = np.sort(np.random.default_rng(5).choice(N, size=4, replace=False))
    w = torch.zeros(N, device="cuda")
    w[torch.from_numpy(envs).cuda()] = 1.0
    keep = []
    loss = policy_window_loss(sim, pol, q0, qd0, h, keep, env_weight=w)
    loss.backward()
    g_gpu = torch.cat([p.grad.reshape(-1) for p in pol.parameters()]).cpu().numpy()
    assert np.isfinite(g_gpu).all() and np.abs(g_gpu).max() > 0
    o = oracle_mod.Oracle(m)
    pol64 = copy.deepcopy(pol).double().cpu()
    params = list(pol64.parameters())
    theta_bar = [torch.zeros_like(p) for p in params]
    ne = len(envs)
    qbar, qdbar = np.zeros((ne, m.nq)), np.zeros((ne, m.nv))
    rbar = np.full(ne, -1.0 / (N * h))
    for t in range(h - 1, -1, -1):
        q, qd, a = (x.detach().cpu().numpy().astype(np.float64) for x in keep[t])
        q, qd, a = q.reshape(m.nq, N)[:, envs], qd.reshape(m.nv, N)[:, envs], a.reshape(m.na, N)[:, envs]
        sq, sqd, sa = o.step_vjp(q.T, qd.T, a.T, qbar, qdbar, rbar)
        qt = torch.tensor(q, requires_grad=True)
        qdt = torch.tensor(qd, requires_grad=True)
        a64 = pol64(free_root_observation(qt, qdt))
        grads = torch.autograd.grad(a64, [qt, qdt] + params, grad_outputs=torch.tensor(sa))
        for k, gk in enumerate(grads[2:]):
            theta_bar[k] += gk
        qbar = sq + grads[0].numpy().T
        qdbar = sqd + grads[1].numpy().T
    g_ref = torch.cat([x.reshape(-1) for x in theta_bar]).numpy()
    assert_grad_close(g_gpu[:, None], g_ref[:, None], "policy window dL/dtheta, 512 envs, 4 sampled", axis_env=-1)
