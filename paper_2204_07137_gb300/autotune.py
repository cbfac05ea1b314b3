"""Launch-shape autotuner for the batched form.

Chooses, by measurement, the environment-to-warp packing (lanes per
environment, i.e. environments per warp, for each articulation group) and the
CTA size (warps per CTA) of the persistent forward and adjoint kernels.
Coordinate descent: each group's team size in turn (the others fixed), then
the warps per CTA; every candidate is timed as a short window forward +
adjoint with CUDA events after a warm-up.  Results never change beyond FP32
reassociation inside a team (the parity tests run every team size).
"""
from __future__ import annotations

import json
import os
from typing import Dict, List, Optional

import torch

from . import _lib, inputs as I
from .sim import Simulator

LANES = (1, 2, 4, 8, 16, 32)
WARPS = (1, 2, 4, 8)


class _Inputs:
    def __init__(self, sim: Simulator, h: int):
        dev = sim.device
        self.q0 = sim.pack([I.initial_state(m, n, 0)[0] for m, n in sim.groups], "q")
        self.qd0 = sim.pack([I.initial_state(m, n, 0)[1] for m, n in sim.groups], "qd")
        self.act = torch.cat([torch.from_numpy(I.window_actions(m, n, h, 0).reshape(h, -1)) for m, n in sim.groups],
                             dim=1).to(dev).contiguous()
        self.rb = torch.ones(h, sim.n_envs, device=dev)
        self.zq = torch.zeros(h + 1, sim.q_size, device=dev)
        self.zqd = torch.zeros(h + 1, sim.qd_size, device=dev)


def time_window(sim: Simulator, x: _Inputs, reps: int = 3) -> float:
    """ms per window forward + adjoint (median of reps after one warm-up)."""
    f = sim.window_forward(x.q0, x.qd0, x.act)
    a = sim.window_adjoint(f[0], f[1], x.act, x.rb, x.zq, x.zqd)
    torch.cuda.synchronize()
    ts = []
    for _ in range(reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        sim.window_forward(x.q0, x.qd0, x.act, out=f)
        sim.window_adjoint(f[0], f[1], x.act, x.rb, x.zq, x.zqd, out=a)
        e1.record()
        e1.synchronize()
        ts.append(e0.elapsed_time(e1))
    ts.sort()
    return ts[len(ts) // 2]


def autotune(sim: Simulator, h: int = 4, reps: int = 3, verbose: bool = False) -> Dict:
    """Tune sim in place (batched form); returns the chosen shape and the timings."""
    if sim.form != "batched":
        return {}
    x = _Inputs(sim, h)
    log: List = []
    lanes = [sim.get_launch(g)[0] for g in range(len(sim.groups))]
    warps = sim.get_launch(0)[1]

    def apply(ls, w):
        for g, l in enumerate(ls):
            sim.set_launch(g, l, w)

    def measure(ls, w):
        try:   # shapes whose scratch does not fit in shared memory are rejected by the library
            apply(ls, w)
            t = time_window(sim, x, reps)
        except _lib.ShacError:
            t = float("inf")
        log.append({"lanes": list(ls), "warps": w, "ms": t})
        if verbose:
            print(f"  lanes {ls} warps {w}: {t:.3f} ms", flush=True)
        return t

    best = measure(lanes, warps)
    for g in range(len(sim.groups)):
        for l in LANES:
            if l == lanes[g]:
                continue
            trial = list(lanes)
            trial[g] = l
            t = measure(trial, warps)
            if t < best:
                best, lanes = t, trial
    for w in WARPS:
        if w == warps:
            continue
        t = measure(lanes, w)
        if t < best:
            best, warps = t, w
    apply(lanes, warps)
    return {"lanes": lanes, "warps": warps, "ms_window_h": best, "h": h, "log": log}


def save(result: Dict, path: str, key: str) -> None:
    data = {}
    if os.path.exists(path):
        with open(path) as f:
            data = json.load(f)
    data[key] = {k: v for k, v in result.items() if k != "log"}
    with open(path, "w") as f:
        json.dump(data, f, indent=1)


def load(path: str, key: str) -> Optional[Dict]:
    if not os.path.exists(path):
        return None
    with open(path) as f:
        return json.load(f).get(key)


if __name__ == "__main__":
    import argparse
    from . import build
    p = argparse.ArgumentParser()
    p.add_argument("--workload", default="ant-2048")
    p.add_argument("--h", type=int, default=4)
    a = p.parse_args()
    build.build()
    wl = I.workload(a.workload)
    s = Simulator(wl.groups, form="batched", h_max=a.h)
    r = autotune(s, h=a.h, verbose=True)
    print(json.dumps({k: v for k, v in r.items() if k != "log"}))
