"""Small, self-contained workload runs for profiler captures (ncu).

    python -m paper_2204_07137_gb300.profile_case --workload ant --envs 2048 --form batched --h 32 --reps 2

Runs `reps` window forward + window adjoint passes of one workload through
the public API and exits 0; no timing, no checks.  Used by the ncu commands
recorded under profiles/ (launch lists, counter captures, FP32 op counts of the
plain form).
"""
from __future__ import annotations

import argparse

import numpy as np
import torch

from . import build, inputs as I
from .sim import Simulator


def main():
    p = argparse.ArgumentParser()
    p.add_argument("--workload", default="ant", choices=["cartpole", "ant", "humanoid", "mtu", "hetero"])
    p.add_argument("--envs", type=int, default=2048)
    p.add_argument("--form", default="batched", choices=["batched", "plain"])
    p.add_argument("--h", type=int, default=32)
    p.add_argument("--reps", type=int, default=1)
    p.add_argument("--lanes", type=int, default=0)
    p.add_argument("--warps", type=int, default=0)
    p.add_argument("--tape", type=int, default=1, help="window tape (batched form): 1 keep, 0 recompute")
    a = p.parse_args()
    build.build()
    if a.workload == "hetero":
        groups = [(I.cartpole(), 2 * a.envs), (I.ant(), a.envs), (I.humanoid(), a.envs // 2)]
    else:
        groups = [({"cartpole": I.cartpole, "ant": I.ant, "humanoid": I.humanoid, "mtu": I.mtu}[a.workload](),
                   a.envs)]
    sim = Simulator(groups, form=a.form, h_max=a.h)
    if a.lanes or a.warps:
        sim.set_launch(-1, a.lanes, a.warps)
    if a.form == "batched" and a.tape:
        sim.set_window_tape(True)
    dev = sim.device
    q0 = sim.pack([I.initial_state(m, n, 0)[0] for m, n in groups], "q")
    qd0 = sim.pack([I.initial_state(m, n, 0)[1] for m, n in groups], "qd")
    act = torch.cat([torch.from_numpy(I.window_actions(m, n, a.h, 0).reshape(a.h, -1)) for m, n in groups],
                    dim=1).to(dev).contiguous()
    rb = torch.ones(a.h, sim.n_envs, device=dev)
    zq = torch.zeros(a.h + 1, sim.q_size, device=dev)
    zqd = torch.zeros(a.h + 1, sim.qd_size, device=dev)
    for _ in range(a.reps):
        f = sim.window_forward(q0, qd0, act)
        sim.window_adjoint(f[0], f[1], act, rb, zq, zqd)
    torch.cuda.synchronize()
    assert np.isfinite(f[0].cpu().numpy()).all()


if __name__ == "__main__":
    main()
