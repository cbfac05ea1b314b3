"""Short-horizon actor-critic learner on the GB300 simulator (Sec. 3.2,
Algorithm 1, appendix A.1 and the hyperparameter tables of the appendix).

One learning episode:
  1. roll out N trajectories of h steps with the stochastic policy, each
     continuing where the last episode's trajectory stopped (Sec. 3.2:
     gradients are cut between learning episodes), each step through ``SimStep`` (the library's step, its
     backward the library's step adjoint); an environment whose task ends
     (root below the task height, or the task horizon) restarts from a fresh
     seeded initial state, which cuts the gradient there;
  2. policy loss, Eq. policy_loss: -1/(N h) sum_i [sum_t gamma^(t - t0) r_t +
     gamma^(h - t0) V_target(s_h)], the discount restarting at every reset;
  3. one Adam step of the actor on the analytic gradient;
  4. critic targets by TD-lambda (Eq. td-lambda) with the target critic,
     computed by the library's ``shac_td_lambda`` kernel;
  5. critic fit on the window's states (Eq. critic_loss), several iterations
     over minibatches;
  6. soft update of the target critic, V' <- alpha V' + (1 - alpha) V;
  7. running observation normalisation updated with the window's observations.

The networks are ordinary PyTorch modules (dense layers through cuBLAS); the
simulator, its adjoint and the targets run in the library's kernels.

Data-parallel over GPUs: with a process group, the N environments are split
into contiguous slices, one per rank; each rank rolls out its slice, and the
actor gradient, the critic gradients and the observation statistics are summed
over ranks (all-reduce), so every rank applies the same update, the one a
single process over all N environments would apply.  Initial states, the
policy noise and the critic minibatches are drawn for all N environments with
the same seed on every rank and sliced, so the result does not depend on the
number of ranks beyond floating-point reassociation of the sums.
"""
from __future__ import annotations

import ctypes
import math
import time
from typing import Dict

import numpy as np
import torch
from torch import nn

from . import _lib, inputs as I
from .policy import free_root_observation
from .sim import SimStep, Simulator

# Appendix hyperparameter tables (optimal settings per task; the general
# setting for the tasks the tables do not list).
PAPER_HPARAMS = {
    "cartpole": dict(actor_lr=1e-2, critic_lr=1e-3, alpha=0.2, episodes=500),
    "ant": dict(actor_lr=2e-3, critic_lr=2e-3, alpha=0.2, episodes=2000),
    "humanoid": dict(actor_lr=2e-3, critic_lr=5e-4, alpha=0.995, episodes=2000),
    "mtu": dict(actor_lr=2e-3, critic_lr=5e-4, alpha=0.995, episodes=2000),
}
# The general table gives no episode count; 2000 is what the optimal table
# uses for every task but cart-pole.
GENERAL_HPARAMS = dict(actor_lr=2e-3, critic_lr=5e-4, alpha=0.995, episodes=2000)


def td_lambda(reward: torch.Tensor, value: torch.Tensor, done: torch.Tensor | None, gamma: float,
              lam: float, stream=None) -> torch.Tensor:
    """TD-lambda critic targets (Eq. td-lambda) by the library kernel:
    reward [h, N], value [h+1, N] float32, done [h, N] uint8 or None -> [h, N]."""
    h, N = reward.shape
    for name, t, shape in (("reward", reward, (h, N)), ("value", value, (h + 1, N))):
        if not (t.is_cuda and t.dtype == torch.float32 and t.is_contiguous() and tuple(t.shape) == shape):
            raise ValueError(f"{name}: expected contiguous float32 CUDA tensor of shape {shape}")
    if done is not None and not (done.is_cuda and done.dtype == torch.uint8 and done.is_contiguous()
                                 and tuple(done.shape) == (h, N)):
        raise ValueError(f"done: expected contiguous uint8 CUDA tensor of shape {(h, N)}")
    out = torch.empty(h, N, device=reward.device)
    s = torch.cuda.current_stream(reward.device) if stream is None else stream
    _lib.check(_lib.load().shac_td_lambda(ctypes.c_void_p(s.cuda_stream), h, N, ctypes.c_void_p(reward.data_ptr()),
                                          ctypes.c_void_p(value.data_ptr()),
                                          ctypes.c_void_p(0 if done is None else done.data_ptr()),
                                          float(gamma), float(lam), ctypes.c_void_p(out.data_ptr())),
               "shac_td_lambda")
    return out


class RunningNorm:
    """Running mean and variance of observations (parallel-update form),
    normalising by the statistics of previous learning episodes."""

    def __init__(self, dim: int, device, eps: float = 1e-5, clip: float = 5.0):
        self.mean = torch.zeros(dim, dtype=torch.float64, device=device)
        self.var = torch.ones(dim, dtype=torch.float64, device=device)
        self.count = eps
        self.eps = eps
        self.clip = clip

    def __call__(self, x: torch.Tensor) -> torch.Tensor:
        y = (x - self.mean.float()) / torch.sqrt(self.var.float() + self.eps)
        return y.clamp(-self.clip, self.clip)

    def update(self, x: torch.Tensor, group=None):
        """Fold a batch of observations in; with a process group, the batch is
        the union of every rank's x (count, sum and sum of squares summed in
        float64 over ranks)."""
        x = x.detach().reshape(-1, x.shape[-1]).double()
        stats = torch.cat([torch.tensor([float(x.shape[0])], dtype=torch.float64, device=x.device), x.sum(0),
                           (x * x).sum(0)])
        if group is not None:
            group.all_reduce(stats)
        d_ = x.shape[1]
        n = float(stats[0])
        m = stats[1:1 + d_] / n
        v = torch.clamp(stats[1 + d_:] / n - m * m, min=0.0)
        tot = self.count + n
        d = m - self.mean
        self.mean = self.mean + d * (n / tot)
        self.var = (self.var * self.count + v * n + d * d * (self.count * n / tot)) / tot
        self.count = tot


# Policy and value network hidden sizes per task (appendix table of network
# settings); tasks it does not list take the ant's setting.
PAPER_NETWORKS = {
    "cartpole": ((64, 64), (64, 64)),
    "ant": ((128, 64, 32), (64, 64)),
    "humanoid": ((256, 128), (128, 128)),
    "mtu": ((512, 256), (256, 256)),
}
GENERAL_NETWORKS = PAPER_NETWORKS["ant"]


def mlp(sizes, out_scale: float = 1.0):
    """Linear layers with an ELU and a layer normalisation after every hidden
    layer (appendix: ELU hidden activations, each hidden layer normalised)."""
    layers = []
    for k, (a, b) in enumerate(zip(sizes[:-1], sizes[1:])):
        lin = nn.Linear(a, b)
        if k == len(sizes) - 2:
            with torch.no_grad():
                lin.weight.mul_(out_scale)
                lin.bias.zero_()
        layers.append(lin)
        if k < len(sizes) - 2:
            layers.append(nn.ELU())
            layers.append(nn.LayerNorm(b))
    return nn.Sequential(*layers)


class GaussianPolicy(nn.Module):
    """a = tanh(mu_theta(o) + sigma_theta * eps), eps ~ N(0, I) given
    (reparameterisation, Sec. 3.2); sigma a learned per-action scale."""

    def __init__(self, n_obs: int, n_act: int, hidden=(64, 64), log_std0: float = -1.0):
        super().__init__()
        self.mu = mlp([n_obs, *hidden, n_act], out_scale=0.1)
        self.log_std = nn.Parameter(torch.full((n_act,), float(log_std0)))

    def forward(self, obs: torch.Tensor, eps: torch.Tensor) -> torch.Tensor:
        return torch.tanh(self.mu(obs) + torch.exp(self.log_std) * eps)


def observation(model, q: torch.Tensor, qd: torch.Tensor, a_prev: torch.Tensor | None = None) -> torch.Tensor:
    """Observation of a single-group state block (q [nq, N], qd [nv, N]) ->
    [N, n_obs], as the appendix A.3 observation tables list it: free-root
    models the root height, quaternion, world linear and angular velocity,
    joint angles and velocities, up and heading projections
    (``policy.free_root_observation``), and for torque-actuated ones the
    previous step's actions a_prev [N, na]; planar models everything but the
    forward position (height, pitch, joints and all velocities); the cart-pole
    x, x_dot, sin theta, cos theta, theta_dot."""
    N = q.shape[1]
    if int(model.joint_type[0]) == I.FREE:
        o = free_root_observation(q, qd)
        if len(model.muscle_fmax) == 0:   # torque actuation: the last actions are observed
            if a_prev is None:
                a_prev = torch.zeros(N, model.na, device=q.device, dtype=q.dtype)
            o = torch.cat([o, a_prev], dim=1)
        return o
    if model.name == "cartpole":
        return torch.stack([q[0], qd[0], torch.sin(q[1]), torch.cos(q[1]), qd[1]], dim=0).transpose(0, 1)
    return torch.cat([q[1:], qd], dim=0).transpose(0, 1)


class SHAC:
    """Algorithm 1 on one articulation model with N environments.

    group: an initialised torch.distributed module (or None): the N
    environments are split over its ranks (N divisible by the world size) and
    the gradients and observation statistics are all-reduced.
    dynamics: (q, qd, a) -> (q_next, qd_next, reward), differentiable, on
    structure-of-arrays blocks of this rank's environments; default the
    library's step (``SimStep``, its backward the step adjoint).
    targets: (reward, value, done, gamma, lam) -> TD-lambda targets; default the
    library's kernel (``td_lambda``)."""

    def __init__(self, model, n_envs: int = 64, h: int = 32, gamma: float = 0.99, lam: float = 0.95,
                 actor_lr: float | None = None, critic_lr: float | None = None, alpha: float | None = None,
                 betas=(0.7, 0.95), critic_iters: int = 16, critic_minibatches: int = 4, episodes: int | None = None,
                 seed: int = 0, device=None, grad_clip: float | None = None, group=None, dynamics=None,
                 targets=None):
        hp = dict(PAPER_HPARAMS.get(model.name, GENERAL_HPARAMS))
        for k, v in (("actor_lr", actor_lr), ("critic_lr", critic_lr), ("alpha", alpha), ("episodes", episodes)):
            if v is not None:
                hp[k] = v
        self.group = group
        self.world = group.get_world_size() if group is not None else 1
        self.rank = group.get_rank() if group is not None else 0
        if int(n_envs) % self.world:
            raise ValueError(f"n_envs = {n_envs} is not divisible by the world size {self.world}")
        self.N_global = int(n_envs)
        self.model, self.N, self.h, self.gamma, self.lam = model, self.N_global // self.world, int(h), gamma, lam
        self.env0 = self.rank * self.N                      # first global environment of this rank
        self.alpha, self.critic_iters, self.critic_minibatches = hp["alpha"], critic_iters, critic_minibatches
        self.episodes = max(1, int(hp["episodes"]))   # length of the linear learning-rate decay
        self.grad_clip = grad_clip
        if dynamics is None:
            self.sim = Simulator([(model, self.N)], form="batched", h_max=1, device=device)
            dev = self.sim.device
            self.dynamics = lambda q, qd, a: SimStep.apply(self.sim, q, qd, a)
        else:
            self.sim = None
            dev = torch.device("cpu" if device is None else device)
            self.dynamics = dynamics
        self.targets = td_lambda if targets is None else targets
        self.device = dev
        self.term_height, self.horizon = I.episode_rule(model)
        self.height_q = 2 if int(model.joint_type[0]) == I.FREE else int(model.height_q)
        torch.manual_seed(seed)   # network initialisation
        self.seed = seed
        q, qd = self._initial(0)
        self.q, self.qd = q, qd
        e0 = np.random.default_rng(seed).integers(0, self.horizon, self.N_global)[self.env0:self.env0 + self.N]
        self.e = torch.from_numpy(e0).to(dev)
        self.a_prev = torch.zeros(self.N, model.na, device=dev)   # last actions (observed by torque models)
        n_obs = self._obs(q, qd, self.a_prev).shape[1]
        pol_hidden, val_hidden = PAPER_NETWORKS.get(model.name, GENERAL_NETWORKS)
        self.actor = GaussianPolicy(n_obs, model.na, hidden=pol_hidden).to(dev)
        self.critic = mlp([n_obs, *val_hidden, 1]).to(dev)
        self.target = mlp([n_obs, *val_hidden, 1]).to(dev)
        self.target.load_state_dict(self.critic.state_dict())
        for p in self.target.parameters():
            p.requires_grad_(False)
        self.actor_opt = torch.optim.Adam(self.actor.parameters(), lr=hp["actor_lr"], betas=betas)
        self.critic_opt = torch.optim.Adam(self.critic.parameters(), lr=hp["critic_lr"], betas=betas)
        self.lr0 = (hp["actor_lr"], hp["critic_lr"])
        self.norm = RunningNorm(n_obs, dev)
        self.rng = torch.Generator(device=dev).manual_seed(seed + 1)
        self.episode_index = 0

    def _initial(self, k: int):
        """Seeded initial states of this rank's slice of the N environments."""
        q, qd = I.initial_state(self.model, self.N_global, self.seed * 1000 + k)
        sl = slice(self.env0, self.env0 + self.N)
        return (torch.from_numpy(np.ascontiguousarray(q[:, sl]).reshape(-1)).to(self.device),
                torch.from_numpy(np.ascontiguousarray(qd[:, sl]).reshape(-1)).to(self.device))

    def _allreduce_grads(self, params):
        """Sum the gradients of params over the ranks (one flat buffer)."""
        if self.group is None:
            return
        params = [p for p in params if p.grad is not None]
        flat = torch.cat([p.grad.reshape(-1) for p in params])
        self.group.all_reduce(flat)
        off = 0
        for p in params:
            n = p.grad.numel()
            p.grad.copy_(flat[off:off + n].view_as(p.grad))
            off += n

    def _obs(self, q, qd, a_prev):
        return observation(self.model, q.view(self.model.nq, self.N), qd.view(self.model.nv, self.N), a_prev)

    @torch.no_grad()
    def evaluate(self, steps: int, seed: int) -> float:
        """Mean reward of the deterministic policy (eps = 0) over `steps` steps
        from fresh seeded initial states (a separate batch; no learning)."""
        m, N = self.model, self.N
        q, qd = (torch.from_numpy(np.ascontiguousarray(x[:, self.env0:self.env0 + N]).reshape(-1)).to(self.device)
                 for x in I.initial_state(m, self.N_global, 10_000 + seed))
        zero = torch.zeros(N, m.na, device=self.device)
        a = zero
        tot = 0.0
        for _ in range(steps):
            a = self.actor(self.norm(self._obs(q, qd, a)), zero)
            q, qd, r = self.dynamics(q, qd, a.transpose(0, 1).contiguous().view(-1))
            tot += float(r.mean())
        return tot / steps

    def episode(self) -> Dict[str, float]:
        """One learning episode; returns its losses, mean reward and the
        forward / backward / critic times in seconds (CUDA events)."""
        m, N, h, gamma = self.model, self.N, self.h, self.gamma
        NG, sl = self.N_global, slice(self.env0, self.env0 + self.N)
        cuda = self.device.type == "cuda"
        ev = [torch.cuda.Event(enable_timing=True) if cuda else None for _ in range(4)]
        wall = [0.0] * 4

        def mark(k):
            if cuda:
                ev[k].record()
            else:
                wall[k] = time.perf_counter()
        frac = 1.0 - self.episode_index / self.episodes          # linear learning-rate decay
        for opt, lr0 in ((self.actor_opt, self.lr0[0]), (self.critic_opt, self.lr0[1])):
            for grp in opt.param_groups:
                grp["lr"] = lr0 * max(frac, 0.0)
        mark(0)
        # 1-2. rollout through the differentiable simulator and the policy loss
        q, qd = self.q, self.qd                                  # detached: cut between episodes
        a_prev = self.a_prev
        q_reset, qd_reset = self._initial(1 + self.episode_index)
        disc = torch.ones(N, device=self.device)
        total = torch.zeros(N, device=self.device)
        obs_raw, rews, dones = [], [], []
        for t in range(h):
            o = self._obs(q, qd, a_prev)
            obs_raw.append(o.detach())
            eps = torch.randn(NG, m.na, device=self.device, generator=self.rng)[sl]   # drawn for all N
            a = self.actor(self.norm(o), eps)
            qn, qdn, r = self.dynamics(q, qd, a.transpose(0, 1).contiguous().view(-1))
            total = total + disc * r
            self.e = self.e + 1
            d = self.e >= self.horizon
            if self.height_q >= 0 and self.term_height > -math.inf:
                d = d | (qn.view(m.nq, N)[self.height_q] < self.term_height)
            self.e = torch.where(d, torch.zeros_like(self.e), self.e)
            disc = torch.where(d, torch.ones_like(disc), disc * gamma)
            # an ended episode restarts from a reset state: a constant, so no gradient crosses it
            dq = d.repeat(m.nq)
            dqd = d.repeat(m.nv)
            q = torch.where(dq, q_reset, qn)
            qd = torch.where(dqd, qd_reset, qdn)
            a_prev = torch.where(d[:, None], torch.zeros_like(a), a)   # a new episode starts with no action
            rews.append(r.detach())
            dones.append(d)
        o_end = self._obs(q, qd, a_prev)
        obs_raw.append(o_end.detach())
        v_end = self.target(self.norm(o_end)).squeeze(-1)
        total = total + disc * v_end
        loss = -total.sum() / (NG * h)          # this rank's share of the loss over all N environments
        mark(1)
        # 3. actor update on the analytic gradient, summed over the ranks
        self.actor_opt.zero_grad(set_to_none=True)
        loss.backward()
        self._allreduce_grads(self.actor.parameters())
        if self.grad_clip is not None:
            nn.utils.clip_grad_norm_(self.actor.parameters(), self.grad_clip)
        self.actor_opt.step()
        self.q, self.qd, self.a_prev = q.detach(), qd.detach(), a_prev.detach()
        mark(2)
        # 4-6. critic: TD-lambda targets with the target critic, fit, soft update
        with torch.no_grad():
            obs_all = torch.stack(obs_raw)                       # [h+1, N, n_obs]
            on = self.norm(obs_all)
            values = self.target(on).squeeze(-1).contiguous()   # [h+1, N]
            reward = torch.stack(rews).contiguous()
            done = torch.stack(dones).to(torch.uint8).contiguous()
            tgt = self.targets(reward, values, done, gamma, self.lam)
        x = on[:h].reshape(h * N, -1)
        y = tgt.reshape(h * N)
        c_loss = 0.0
        for _ in range(self.critic_iters):
            # minibatches over the samples (t, environment) of all N environments;
            # this rank fits the ones of its slice, the squared errors summed
            # over ranks and divided by the whole minibatch's size
            perm = torch.randperm(h * NG, device=self.device, generator=self.rng)
            for b in perm.chunk(self.critic_minibatches):
                t_, e_ = b // NG, b % NG
                mine = (e_ >= self.env0) & (e_ < self.env0 + N)
                idx = t_[mine] * N + (e_[mine] - self.env0)
                pred = self.critic(x[idx]).squeeze(-1)
                l = ((pred - y[idx]) ** 2).sum() / b.numel()
                self.critic_opt.zero_grad(set_to_none=True)
                l.backward()
                self._allreduce_grads(self.critic.parameters())
                self.critic_opt.step()
                lsum = l.detach().reshape(1)
                if self.group is not None:
                    self.group.all_reduce(lsum)
                c_loss = float(lsum)
        with torch.no_grad():
            for pt, pc in zip(self.target.parameters(), self.critic.parameters()):
                pt.mul_(self.alpha).add_(pc, alpha=1.0 - self.alpha)
        # 7. observation statistics of this episode (all ranks), used from the next one on
        self.norm.update(obs_all[:h], self.group)
        mark(3)
        if cuda:
            torch.cuda.synchronize()
            t = [ev[0].elapsed_time(ev[k]) * 1e-3 for k in range(4)]
        else:
            t = [wall[k] - wall[0] for k in range(4)]
        self.episode_index += 1
        summ = torch.tensor([float(loss.detach()), float(reward.sum()), float(done.sum())], dtype=torch.float64,
                            device=self.device)
        if self.group is not None:
            self.group.all_reduce(summ)
        return {"policy_loss": float(summ[0]), "critic_loss": c_loss,
                "mean_reward": float(summ[1]) / (h * NG), "resets": int(summ[2]),
                "t_forward": t[1] - t[0], "t_backward": t[2] - t[1], "t_critic": t[3] - t[2]}
