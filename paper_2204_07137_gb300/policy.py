"""Policy-in-the-loop short-horizon window (appendix A.1, Eq. policy_loss).

The actor loss over an h-step window backpropagates through the simulator into
the policy parameters: every step is  obs = o(s_t),  a_t = pi_theta(obs),
s_{t+1}, r_t = F(s_t, a_t)  with F the library's step (``SimStep``, whose
backward is the library's step adjoint), and the loss is the negative mean
reward, -1/(N h) sum_t sum_i r_t^i (the critic term is not part of this path).
Observation and MLP are ordinary PyTorch ops, so autograd produces the
appendix A.1 recursion: s_bar_t = dR/ds + s_bar_{t+1} (dF/ds + dF/da dpi/ds),
theta_bar = sum_t a_bar_t dpi/dtheta.

Observation of a free-root model (appendix A.3 observation tables):
[root height, root quaternion (4), root linear velocity (world, 3), root
angular velocity (world, 3), joint angles, joint velocities, up and heading
projections (2)].
"""
from __future__ import annotations

from typing import List

import torch
from torch import nn

from .sim import SimStep, Simulator


def quat_rotation(qx, qy, qz, qw):
    """Rows of the rotation matrix of unit quaternions (x, y, z, w), batched."""
    r00 = 1 - 2 * (qy * qy + qz * qz); r01 = 2 * (qx * qy - qz * qw); r02 = 2 * (qx * qz + qy * qw)
    r10 = 2 * (qx * qy + qz * qw); r11 = 1 - 2 * (qx * qx + qz * qz); r12 = 2 * (qy * qz - qx * qw)
    r20 = 2 * (qx * qz - qy * qw); r21 = 2 * (qy * qz + qx * qw); r22 = 1 - 2 * (qx * qx + qy * qy)
    return (r00, r01, r02), (r10, r11, r12), (r20, r21, r22)


def free_root_observation(q: torch.Tensor, qd: torch.Tensor) -> torch.Tensor:
    """q [nq, N], qd [nv, N] (one group, structure of arrays) -> obs [N, 13 + 2 (nq - 7)... ]."""
    quat = q[3:7]
    R = quat_rotation(quat[0], quat[1], quat[2], quat[3])
    wb, vb = qd[0:3], qd[3:6]
    v = torch.stack([R[k][0] * vb[0] + R[k][1] * vb[1] + R[k][2] * vb[2] for k in range(3)])
    w = torch.stack([R[k][0] * wb[0] + R[k][1] * wb[1] + R[k][2] * wb[2] for k in range(3)])
    up = R[2][2].unsqueeze(0)
    heading = R[0][0].unsqueeze(0)
    obs = torch.cat([q[2:3], quat, v, w, q[7:], qd[6:], up, heading], dim=0)
    return obs.transpose(0, 1)


def observation_size(model) -> int:
    return 1 + 4 + 3 + 3 + (model.nq - 7) + (model.nv - 6) + 2


class PolicyMLP(nn.Module):
    """obs -> 256 -> 128 -> n_act, ELU hidden activations, weights ~ N(0, std);
    a sigmoid maps the output to muscle activations in [0, 1] (torque models:
    tanh to [-1, 1])."""

    def __init__(self, n_obs: int, n_act: int, hidden=(256, 128), std: float = 0.05, muscles: bool = True,
                 generator=None):
        super().__init__()
        dims = [n_obs, *hidden, n_act]
        self.layers = nn.ModuleList(nn.Linear(a, b) for a, b in zip(dims[:-1], dims[1:]))
        with torch.no_grad():
            for lin in self.layers:
                lin.weight.normal_(0.0, std, generator=generator)
                lin.bias.normal_(0.0, std, generator=generator)
        self.muscles = muscles

    def forward(self, x):
        for k, lin in enumerate(self.layers):
            x = lin(x)
            if k + 1 < len(self.layers):
                x = torch.nn.functional.elu(x)
        return torch.sigmoid(x) if self.muscles else torch.tanh(x)


def policy_window_loss(sim: Simulator, policy: nn.Module, q0: torch.Tensor, qd0: torch.Tensor, h: int,
                       keep: List | None = None, env_weight: torch.Tensor | None = None,
                       actions: torch.Tensor | None = None) -> torch.Tensor:
    """Negative mean reward of an h-step window with the policy in the loop
    (single-group simulator).  If ``keep`` is a list, the per-step states and
    actions are appended to it (for checks).  env_weight [N]: per-environment
    weights of the rewards (default all ones).  actions [h, n_act * N]: given
    open-loop actions instead of the policy's (the same step loop without the
    network)."""
    assert len(sim.groups) == 1
    model, N = sim.groups[0]
    q, qd = q0, qd0
    total = q0.new_zeros(())
    for t in range(h):
        if actions is None:
            obs = free_root_observation(q.view(model.nq, N), qd.view(model.nv, N))
            a = policy(obs)                                   # [N, n_act]
            a_soa = a.transpose(0, 1).contiguous().view(-1)   # [n_act * N]
        else:
            a_soa = actions[t]
        if keep is not None:
            keep.append((q, qd, a_soa))
        q, qd, r = SimStep.apply(sim, q, qd, a_soa)
        total = total + (r.sum() if env_weight is None else (env_weight * r).sum())
    if keep is not None:
        keep.append((q, qd, None))
    return -total / (N * h)
