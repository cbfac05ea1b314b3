"""Benchmark: env-steps/s of the forward + adjoint window (h = 32) of the
differentiable simulator on the 2048-environment ant-like workload.

One bench "step" is one pass of the whole hot path over one batch: the
window forward (32 control steps x 16 substeps, writing the per-step
checkpoints) followed by the window adjoint (reverse over the 32 steps, each
step's substeps recomputed from its checkpoint).  value = N * h / time.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference] [--workload W]

Timed form (``value``): BATCHED, the configured variant (per-control-step
checkpoints, substeps recomputed in the adjoint), launch shape chosen by the
library's autotuner on this batch, both launches captured in one CUDA graph,
inputs resident in HBM, L2 flushed (256 MB write) before every timed step,
CUDA events on the launching stream, median over the timed steps.  Also
reported: the same window with the window tape (every substep record kept in
HBM, no recompute), the episodic window, the PLAIN form (one env per thread,
one kernel per stage per substep) on the same inputs for the speed-up, and
``e2e``: the measurement through the public API with pinned host buffers
(host->device copies of q0, qd0 and the actions and device->host copies of the
rewards and of the action and initial-state gradients inside the timed region).

--impl reference times the FP64 CPU oracle (forward + exact adjoint) on the
host cores on a bounded sample of the same workload.
--profile-case runs a few windows of a workload with no timing, for profiler
captures.
Under torchrun each rank simulates its own environments (weak scaling, no
collective on the data path); rank 0 prints the line.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "env-steps/s fwd+adjoint over 32-step window, batched vs plain; grad rel err<=1e-3"
WORKLOAD = "ant-2048"
H = 32
FLUSH_BYTES = 256 << 20

# FP32 lanes per SM and flops per lane per cycle (one FMA) of the GB300's SMs;
# the FP32 peak is derived from these, the device's SM count and the maximum
# SM clock sampled during the run (fp32_peak_tflops).
FP32_LANES_PER_SM = 128
FLOPS_PER_LANE_CYCLE = 2
DEFAULT_SM_MAX_MHZ = 2070.0

# FP32 work per env-step, counted with ncu on the one-environment-per-thread
# (PLAIN) stage kernels over one window step: thread-level FADD + FMUL +
# 2 x FFMA, i.e. the work that form executes (it includes whatever redundant
# work that form does; the FP64 oracle is no op count of this algorithm: it
# builds M from per-link Jacobians and the bias by vector Newton-Euler, which
# is other and more work).  "forward": one forward step (K substeps);
# "reverse": the reverse-only part of one adjoint step; the recomputing
# adjoint kernel executes one forward recompute + the reverse.
FLOPS_PER_ENV_STEP = {
    "ant": {"forward": 134692, "recompute": 134556, "reverse": 172338},
}

# Algorithmic HBM bytes per env-step (FP32) of one step-level call, the
# accounting of the hot-path table: the forward reads the state and the action
# and writes the next state and the reward; the adjoint reads the checkpoint,
# the action, the next state's cotangent and the reward cotangent and writes the
# state and action cotangents (ant-like model: 268 + 416 = 684 B).  The window
# kernels move less (the state stays on chip between steps).  The substep
# records a kernel keeps in the workspace (one step's worth for the recomputing
# adjoint, the whole window with the window tape) are scratch traffic, reported
# beside.
def algo_bytes_per_env_step(model):
    s = model.nq + model.nv
    return {"forward": 4 * (2 * s + model.na + 1), "adjoint": 4 * (3 * s + 2 * model.na + 1)}


# DRAM traffic (read + write) per launch of the model-specialised batched
# kernels on the full ant-2048 h = 32 window, from a one-pass ncu capture
# (dram__bytes_read.sum + dram__bytes_write.sum of one launch of each kernel);
# None where no capture of the current kernels exists.  The recomputing
# adjoint's traffic is mostly its per-step substep records (about 91 MB per
# step for 2048 environments) written back from L2 as they are replaced step
# after step.
TRAFFIC_BYTES_PER_LAUNCH = {"ant-2048": {"forward": 2.407168e6 + 0.0, "adjoint_recompute": 201.74336e6 + 2316.516608e6,
                                         "adjoint_tape": None}}


def fp32_peak_tflops(n_sms: int, sm_mhz: float) -> float:
    return n_sms * FP32_LANES_PER_SM * FLOPS_PER_LANE_CYCLE * sm_mhz * 1e6 / 1e12


def measured_hbm_gbs():
    """Measured HBM copy bandwidth (MEASURED_PEAKS.json next to this file: a
    STREAM-style copy measured on GB300s of the same kind), else the fallback
    figure."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"]), "measured (MEASURED_PEAKS.json hbm_gbs)"
    except (OSError, ValueError, KeyError):
        return 6800.0, "fallback 6.8 TB/s"


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=40)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    p.add_argument("--plain-steps", type=int, default=20)
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--workload", default=None, help=f"workload name (default {WORKLOAD}; mtu-512 with --policy)")
    p.add_argument("--grad-check-envs", type=int, default=4,
                   help="sampled environments of every group checked against the oracle (0: skip)")
    p.add_argument("--autotune-ms", type=int, default=5000,
                   help="wall-clock budget of the library's launch-shape search on the timed batch (0: default shape)")
    p.add_argument("--no-specialize", action="store_true",
                   help="time the generic batched kernels instead of the ones compiled for the workload's model")
    p.add_argument("--profile-case", action="store_true",
                   help="run --pc-reps windows of the workload through the public API, no timing or checks "
                        "(for profiler captures)")
    p.add_argument("--pc-envs", type=int, default=0, help="profile case: environments of the first group "
                                                          "(the others scaled alike; 0: the workload's)")
    p.add_argument("--pc-form", default="batched", choices=["batched", "plain"])
    p.add_argument("--pc-h", type=int, default=32)
    p.add_argument("--pc-reps", type=int, default=1)
    p.add_argument("--pc-tape", type=int, default=0, help="profile case: 1 keeps the window tape (batched)")
    p.add_argument("--pc-lanes", type=int, default=0)
    p.add_argument("--pc-warps", type=int, default=0)
    p.add_argument("--h-sweep", default="",
                   help="window-length study instead of the contract line: comma-separated h values; "
                        "N = samples // h environments of the workload's first model (see --samples)")
    p.add_argument("--samples", type=int, default=65536,
                   help="env-steps per window of the --h-sweep study (N x h)")
    p.add_argument("--shac-episodes", type=int, default=0,
                   help="time learning episodes of the short-horizon actor-critic learner instead of the contract "
                        "line (the paper's per-episode forward / backward / critic split)")
    p.add_argument("--shac-envs", type=int, default=64)
    p.add_argument("--policy", action="store_true",
                   help="config 5 with the policy MLP in the loop (workload mtu-512): graph-captured window of "
                        "policy + library steps + autograd through the step adjoints, timed beside the step loop "
                        "without the network and the open-loop window")
    args = p.parse_args()
    if args.workload is None:
        args.workload = "mtu-512" if args.policy else WORKLOAD
    return args


# ------------------------------------------------------------------ clocks --
class ClockSampler:
    """nvidia-smi samples (100 ms) during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for n, v in zip(names, parts[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


# --------------------------------------------------------------- reference --
def host_cpu_model() -> str:
    """The host CPU's model name as lscpu reports it (Arm cores report no name
    in /proc/cpuinfo), else the machine type."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.strip().startswith("Model name:"):
                return ln.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    import platform
    return platform.machine()


def oracle_window_rate(model, n_envs: int, seed: int = 0, target_s: float = 12.0):
    """env-steps/s of the FP64 oracle (window forward + exact adjoint) on a
    bounded sample of the workload: hs steps of n environments, starting from
    one environment per oracle thread (the oracle runs environments in
    parallel) and grown (steps first, up to the 32-step window, then
    environments) until the sample takes about target_s / 4 .. target_s of
    wall time; a whole workload that runs faster is repeated until it does.
    Returns (rate, n, hs, threads, seconds, repeats)."""
    from paper_2204_07137_gb300 import inputs as I
    from oracle import oracle
    o = oracle.Oracle(model)

    def run(n, hs):
        q0, qd0 = I.initial_state(model, n, seed)
        act = I.window_actions(model, n, hs, seed)
        t0 = time.perf_counter()
        qt, qdt, rw = o.window_forward(q0.T, qd0.T, act.transpose(0, 2, 1))
        o.window_adjoint(qt, qdt, act.transpose(0, 2, 1), np.ones((hs, n)), np.zeros((n, model.nq)),
                         np.zeros((n, model.nv)))
        return time.perf_counter() - t0

    threads = oracle.num_threads()
    n, hs = max(1, min(threads, n_envs)), 1
    dt = run(n, hs)
    while dt < target_s / 4 and (hs < H or n < n_envs):
        grow = min(8.0, target_s / max(dt, 1e-3))
        if hs < H:
            hs = min(H, max(hs + 1, int(hs * grow)))
        else:
            n = min(n_envs, max(n + 1, int(n * grow)))
        dt = run(n, hs)
    reps = 1
    if dt < target_s / 4:   # the whole workload: repeat it
        reps = max(1, int(math.ceil(target_s / 4 / max(dt, 1e-6))))
        dt += sum(run(n, hs) for _ in range(reps - 1))
    return n * hs * reps / dt, n, hs, threads, dt, reps


def oracle_workload_rate(groups, seed: int = 0, target_s: float = 12.0):
    """env-steps/s of the oracle on a whole workload: each articulation group
    sampled on its own (target_s split by group), combined as the whole job's
    env-steps over the sum of the groups' times, sum N_g / sum (N_g / r_g).
    Returns (rate, threads, seconds sampled, sample description)."""
    per = target_s / len(groups)
    total_n, total_t, dts, parts, threads = 0, 0.0, 0.0, [], 1
    for model, n_g in groups:
        r, n, hs, threads, dt, reps = oracle_window_rate(model, n_g, seed=seed, target_s=per)
        total_n += n_g
        total_t += n_g / r
        dts += dt
        parts.append(f"{n} of {n_g} envs ({model.name}) x {hs} steps" + (f" x {reps} runs" if reps > 1 else ""))
    return total_n / total_t, threads, dts, "; ".join(parts)


def reference_main(args, rank, world):
    from paper_2204_07137_gb300 import inputs as I
    if rank != 0:
        return
    wl = I.workload(args.workload)
    n_total = sum(n for _, n in wl.groups)
    # warm-up: W untimed runs of a small sample (one environment, one step of
    # each group) load the oracle and touch its code paths
    for s in range(args.warmup):
        oracle_workload_rate([(m, 1) for m, _ in wl.groups], seed=1000 + s, target_s=0.0)
    rates, samples = [], []
    for s in range(args.steps):
        r, threads, dt, desc = oracle_workload_rate(wl.groups, seed=s, target_s=min(12.0, 60.0 / max(1, args.steps)))
        rates.append(r)
        samples.append(desc)
    value = statistics.median(rates)
    model = wl.groups[0][0]
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "env-steps/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * n_total * H / value,
        "ms_per_step_basis": f"extrapolated to the whole workload ({n_total} environments x {H} steps) from the "
                            f"median rate of the timed samples ({samples[0]} per timed step)",
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": wl.name, "n_envs": n_total, "h": H,
                   "substeps": model.substeps if len(wl.groups) == 1 else [m.substeps for m, _ in wl.groups],
                   "form": "FP64 CPU oracle, forward + dual-number exact adjoint"},
        "cpu_baseline": {"value": value, "unit": "env-steps/s", "cores": threads, "kind": "oracle",
                         "cpu_model": host_cpu_model(), "sample": f"{samples[0]} per timed step (extrapolated)"},
        "e2e": {"value": value, "unit": "env-steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# --------------------------------------------------------------- ranks ---
def shard_seed(rank: int) -> int:
    """Each rank simulates its own environments (weak scaling): the input
    seed of a rank's shard."""
    return rank


def max_over_ranks(values, dist, device=None):
    """Element-wise maximum of per-rank timings (the slowest rank sets the
    job time); identity without a process group."""
    if dist is None:
        return list(values)
    import torch
    t = torch.tensor([float(v) for v in values], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return t.tolist()


# -------------------------------------------------------- h-sweep study ---
def h_sweep_main(args):
    """Window-length study (the paper's horizon study: every variant draws
    the same number of samples per learning episode, N x h fixed): for each
    h, N = samples // h environments run the graph-captured forward + adjoint
    window (window tape kept, the kernels specialised for the model unless
    --no-specialize); one JSON line with env-steps/s, ms per window and the
    kernel split per h (medians of the timed windows).  L2 flushed before each
    timed window."""
    import torch
    from paper_2204_07137_gb300 import build, inputs as I
    from paper_2204_07137_gb300.sim import Simulator

    build.build()
    dev = torch.device("cuda", 0)
    model = I.workload(args.workload).groups[0][0]
    flush = torch.empty(FLUSH_BYTES, dtype=torch.uint8, device=dev)
    stream = torch.cuda.Stream(device=dev)
    rows = []
    for h in [int(x) for x in args.h_sweep.split(",")]:
        N = max(1, args.samples // h)
        sim = Simulator([(model, N)], form="batched", h_max=h)
        sim.set_window_tape(True)
        if not args.no_specialize:
            sim.specialize()
        q0, qd0 = (torch.from_numpy(np.ascontiguousarray(x.reshape(-1))).to(dev) for x in I.initial_state(model, N, 0))
        act = torch.from_numpy(I.window_actions(model, N, h, 0).reshape(h, -1)).to(dev).contiguous()
        rbar = torch.full((h, N), 1.0 / (N * h), device=dev)
        zq = torch.zeros(h + 1, sim.q_size, device=dev)
        zqd = torch.zeros(h + 1, sim.qd_size, device=dev)
        with torch.cuda.stream(stream):
            f = sim.window_forward(q0, qd0, act, stream=stream)
            a = sim.window_adjoint(f[0], f[1], act, rbar, zq, zqd, stream=stream)
        stream.synchronize()
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.stream(stream):
            with torch.cuda.graph(graph, stream=stream):
                sim.window_forward(q0, qd0, act, out=f, stream=stream)
                sim.window_adjoint(f[0], f[1], act, rbar, zq, zqd, out=a, stream=stream)
        stream.synchronize()
        times = {}
        with torch.cuda.stream(stream):
            for name, fn in (("window", graph.replay),
                             ("forward", lambda: sim.window_forward(q0, qd0, act, out=f, stream=stream)),
                             ("adjoint", lambda: sim.window_adjoint(f[0], f[1], act, rbar, zq, zqd, out=a,
                                                                    stream=stream))):
                for _ in range(args.warmup):
                    fn()
                ts = []
                for _ in range(args.steps):
                    flush.zero_()
                    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    e0.record(stream)
                    fn()
                    e1.record(stream)
                    e1.synchronize()
                    ts.append(e0.elapsed_time(e1))
                times[name] = float(np.median(ts))
        assert sim.status() == 0 and torch.isfinite(a[2]).all()
        rows.append({"h": h, "n_envs": N, "env_steps_per_s": N * h / (times["window"] * 1e-3),
                     "ms_per_window": times["window"], "ms_forward": times["forward"], "ms_adjoint": times["adjoint"],
                     "lanes_per_env": sim.get_launch(0)[0]})
        del sim
    print(json.dumps({"study": "window length h, N x h fixed", "model": model.name, "samples": args.samples,
                      "kernels": "generic" if args.no_specialize else "model-specialised",
                      "dtype": "f32", "data": "synthetic", "rows": rows}), flush=True)


# ------------------------------------------------------ learner episodes ---
# The paper's per-learning-episode times (N = 64, h = 32, TITAN X; forward,
# backward, critic in seconds): context for --shac-episodes, other hardware.
PAPER_EPISODE_S = {"cartpole": (0.15, 0.23, 0.34), "ant": (0.25, 0.37, 0.32), "humanoid": (0.91, 1.97, 0.32),
                   "mtu": (0.82, 1.66, 0.33)}


def shac_main(args):
    """Learning episodes of Algorithm 1 on the workload's first model with the
    paper's N and h: per-episode forward (rollout + policy loss), backward
    (analytic gradient + actor step) and critic (targets + fit) times, after
    two warm-up episodes; one JSON line."""
    import torch
    from paper_2204_07137_gb300 import build, inputs as I
    from paper_2204_07137_gb300.shac import SHAC

    build.build()
    model = I.workload(args.workload).groups[0][0]
    agent = SHAC(model, n_envs=args.shac_envs, h=H, episodes=args.shac_episodes + 2, seed=0)
    for _ in range(2):
        agent.episode()
    hist = [agent.episode() for _ in range(args.shac_episodes)]
    mean = {k: float(np.mean([s[k] for s in hist])) for k in ("t_forward", "t_backward", "t_critic")}
    tot = sum(mean.values())
    print(json.dumps({"study": "learning episode time (Algorithm 1)", "model": model.name, "n_envs": args.shac_envs,
                      "h": H, "episodes": args.shac_episodes, "seconds_per_episode": mean, "total_s": tot,
                      "env_steps_per_s": args.shac_envs * H / tot,
                      "mean_reward_first_last": [hist[0]["mean_reward"], hist[-1]["mean_reward"]],
                      "paper_titan_x_s": PAPER_EPISODE_S.get(model.name), "dtype": "f32", "data": "synthetic"}),
          flush=True)


# ------------------------------------------------------------------- GPU ---
def workload_inputs(sim, groups, seed, h, dev):
    """Seeded initial state and actions of every group, packed."""
    import torch
    from paper_2204_07137_gb300 import inputs as I
    q0 = sim.pack([I.initial_state(m, n, seed)[0] for m, n in groups], "q")
    qd0 = sim.pack([I.initial_state(m, n, seed)[1] for m, n in groups], "qd")
    act = torch.cat([torch.from_numpy(I.window_actions(m, n, h, seed).reshape(h, -1)) for m, n in groups],
                    dim=1).to(dev).contiguous()
    return q0, qd0, act


class Timer:
    """CUDA-event timing on one stream: W warm-up runs, then K timed runs, each
    after an L2 flush; the median of the K per-run times (ms), max over ranks
    by the caller.  Barrier + synchronize on both sides of the timed region."""

    def __init__(self, stream, flush, dist):
        self.stream, self.flush, self.dist = stream, flush, dist

    def __call__(self, fn, steps, warmup):
        import torch
        with torch.cuda.stream(self.stream):
            for _ in range(warmup):
                fn()
            self.stream.synchronize()
            if self.dist is not None:
                self.dist.barrier()
            torch.cuda.synchronize()
            ts = []
            for _ in range(steps):
                self.flush.zero_()
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(self.stream)
                fn()
                e1.record(self.stream)
                e1.synchronize()
                ts.append(e0.elapsed_time(e1))
            torch.cuda.synchronize()
            if self.dist is not None:
                self.dist.barrier()
        return statistics.median(ts)


def capture_window(sim, q0, qd0, act, rbar, zq, zqd, stream):
    """Eager forward + adjoint window (outputs allocated), then both captured
    into one CUDA graph writing the same outputs."""
    import torch
    with torch.cuda.stream(stream):
        outf = sim.window_forward(q0, qd0, act, stream=stream)
        outa = sim.window_adjoint(outf[0], outf[1], act, rbar, zq, zqd, stream=stream)
    stream.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.stream(stream):
        with torch.cuda.graph(graph, stream=stream):
            sim.window_forward(q0, qd0, act, out=outf, stream=stream)
            sim.window_adjoint(outf[0], outf[1], act, rbar, zq, zqd, out=outa, stream=stream)
    stream.synchronize()
    return graph, outf, outa


def gpu_main(args, rank, world, dist):
    import torch
    from paper_2204_07137_gb300 import build, inputs as I
    from paper_2204_07137_gb300.sim import Simulator

    build.build()
    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", 0)))
    torch.cuda.set_device(dev)
    wl = I.workload(args.workload)
    groups = wl.groups
    n_envs = wl.n_envs
    n_sms = torch.cuda.get_device_properties(dev).multi_processor_count

    def make(form):
        return Simulator(groups, form=form, h_max=H)

    seed = shard_seed(rank)
    sim = make("batched")   # the configured variant: per-step checkpoints, substeps recomputed in the adjoint
    q0, qd0, act = workload_inputs(sim, groups, seed, H, dev)
    # loss = mean reward over the window: reward cotangent 1 / (N h)
    rbar = torch.full((H, n_envs), 1.0 / (n_envs * H), device=dev)
    zq = torch.zeros(H + 1, sim.q_size, device=dev)
    zqd = torch.zeros(H + 1, sim.qd_size, device=dev)
    flush = torch.empty(FLUSH_BYTES, dtype=torch.uint8, device=dev)
    stream = torch.cuda.Stream(device=dev)
    timed = Timer(stream, flush, dist)

    # ---- launch shape: the library's measured search on this batch
    default_shape = [sim.get_launch(g) for g in range(len(groups))]
    tune = None
    if args.autotune_ms > 0:
        g0, _, _ = capture_window(sim, q0, qd0, act, rbar, zq, zqd, stream)
        ms_default = timed(g0.replay, 5, 2)
        del g0
        shape = sim.autotune_native(budget_ms=args.autotune_ms, stream=stream, q0=q0, qd0=qd0, act=act)
        tune = {"default": {"lanes_per_env": [l for l, _ in default_shape], "warps_per_cta": default_shape[0][1],
                            "ms_per_window": ms_default},
                "chosen": {"lanes_per_env": [l for l, _ in shape], "warps_per_cta": shape[0][1]},
                "search": "coordinate descent over lanes per environment (each group) then warps per CTA, "
                          f"h = 8 windows of the workload's inputs (median of 3; a change needs a 3 % gain), budget "
                          f"{args.autotune_ms} ms",
                "note": "ms_per_window of each shape: graph replay of the h = 32 window with the generic kernels "
                        "(before any specialisation), median of 5"}
        g1, _, _ = capture_window(sim, q0, qd0, act, rbar, zq, zqd, stream)
        tune["chosen"]["ms_per_window"] = timed(g1.replay, 5, 2)
        del g1
    # kernels compiled for this model and launch shape (single-group batches);
    # the search then re-times the warps per CTA with them (it keeps the team
    # size they were compiled for)
    spec_s = None
    if len(groups) == 1 and not args.no_specialize:
        t0 = time.perf_counter()
        sim.specialize()
        spec_s = time.perf_counter() - t0
        if tune is not None:
            w_gen = sim.get_launch(0)[1]
            sim.autotune_native(budget_ms=args.autotune_ms, stream=stream, q0=q0, qd0=qd0, act=act)
            tune["specialised"] = {"warps_per_cta": sim.get_launch(0)[1], "generic_choice": w_gen,
                                   "search": "warps per CTA with the specialised kernels, same rule"}
    shape = [sim.get_launch(g) for g in range(len(groups))]

    # ---- the configured variant: graph-captured forward + recomputing adjoint
    graph, outf, outa = capture_window(sim, q0, qd0, act, rbar, zq, zqd, stream)
    sampler = ClockSampler(dev.index) if rank == 0 else None
    if sampler:
        sampler.start()
    ms_window = timed(graph.replay, args.steps, args.warmup)
    clocks = sampler.stop() if sampler else None

    # per-kernel durations (eager launches, same stream) for the roofline
    def one_fwd():
        sim.window_forward(q0, qd0, act, out=outf, stream=stream)

    def one_adj():
        sim.window_adjoint(outf[0], outf[1], act, rbar, zq, zqd, out=outa, stream=stream)

    ms_fwd = timed(one_fwd, max(5, args.steps // 2), 1)
    ms_adj = timed(one_adj, max(5, args.steps // 2), 1)

    # ---- the same window with the window tape (every substep record of the
    # forward kept in HBM; the adjoint reads them instead of recomputing)
    tsim = make("batched")
    for g, (l, w) in enumerate(shape):
        tsim.set_launch(g, l, w)
    ws_step = tsim.workspace.numel()
    tsim.set_window_tape(True)
    if spec_s is not None:
        tsim.specialize()
    tape_bytes = (tsim.workspace.numel() - ws_step) / (H * (n_envs + 31 * len(groups)))
    tgraph, toutf, touta = capture_window(tsim, q0, qd0, act, rbar, zq, zqd, stream)
    ms_tape = timed(tgraph.replay, args.steps, args.warmup)
    ms_tape_adj = timed(lambda: tsim.window_adjoint(toutf[0], toutf[1], act, rbar, zq, zqd, out=touta, stream=stream),
                        max(5, args.steps // 2), 1)
    graph.replay()
    tgraph.replay()
    torch.cuda.synchronize()
    same = all(torch.equal(x, y) for x, y in zip(tuple(outf) + tuple(outa), tuple(toutf) + tuple(touta)))
    del tgraph, tsim

    # ---- episodic window (early termination with in-kernel reset, gradient
    # cut at resets), graph captured like the main window: the task heights and
    # horizons of the models, seeded reset states, episode counters spread over
    # the horizon
    rules = [I.episode_rule(m) for m, _ in groups]
    qr = sim.pack([I.initial_state(m, n, seed + 1)[0] for m, n in groups], "q")
    qdr = sim.pack([I.initial_state(m, n, seed + 1)[1] for m, n in groups], "qd")
    ep0 = np.concatenate([np.random.default_rng(seed).integers(0, hz, n) for (m, n), (_, hz) in zip(groups, rules)])
    ep_step = torch.from_numpy(ep0.astype(np.int32)).to(dev)
    th, hz = [r[0] for r in rules], [r[1] for r in rules]
    with torch.cuda.stream(stream):
        oef = sim.window_forward_episodic(q0, qd0, act, qr, qdr, th, hz, ep_step, stream=stream)
        oea = sim.window_adjoint_episodic(oef[0], oef[1], act, oef[3], rbar, zq, zqd, stream=stream)
    stream.synchronize()
    graph_ep = torch.cuda.CUDAGraph()
    with torch.cuda.stream(stream):
        with torch.cuda.graph(graph_ep, stream=stream):
            sim.window_forward_episodic(q0, qd0, act, qr, qdr, th, hz, ep_step, out=oef, stream=stream)
            sim.window_adjoint_episodic(oef[0], oef[1], act, oef[3], rbar, zq, zqd, out=oea, stream=stream)
    stream.synchronize()
    ms_episodic = timed(graph_ep.replay, args.steps, args.warmup)
    done_frac = float(oef[3].float().mean())
    del graph_ep

    # the outputs the CPU leg checks (sampled gradients of every group)
    graph.replay()
    torch.cuda.synchronize()
    check_data = None
    if rank == 0 and not args.no_cpu_baseline and args.grad_check_envs > 0:
        check_data = [x.detach().clone() for x in tuple(outf) + tuple(outa)]

    # ---- plain form on the same inputs
    plain = make("plain")
    pf = plain.window_forward(q0, qd0, act, stream=stream)
    pa = plain.window_adjoint(pf[0], pf[1], act, rbar, zq, zqd, stream=stream)
    stream.synchronize()

    def plain_step():
        plain.window_forward(q0, qd0, act, out=pf, stream=stream)
        plain.window_adjoint(pf[0], pf[1], act, rbar, zq, zqd, out=pa, stream=stream)

    ms_plain = timed(plain_step, args.plain_steps, args.warmup)
    del plain

    # ---- end to end through the public API with pinned host buffers
    hq0 = q0.cpu().pin_memory()
    hqd0 = qd0.cpu().pin_memory()
    hact = act.cpu().pin_memory()
    dq0, dqd0, dact = torch.empty_like(q0), torch.empty_like(qd0), torch.empty_like(act)
    hrew = torch.empty(H, n_envs).pin_memory()
    hab = torch.empty(H, sim.act_size).pin_memory()
    hq0b = torch.empty(sim.q_size).pin_memory()
    hqd0b = torch.empty(sim.qd_size).pin_memory()

    def e2e_step():
        dq0.copy_(hq0, non_blocking=True)
        dqd0.copy_(hqd0, non_blocking=True)
        dact.copy_(hact, non_blocking=True)
        f = sim.window_forward(dq0, dqd0, dact, out=outf, stream=stream)
        a = sim.window_adjoint(f[0], f[1], dact, rbar, zq, zqd, out=outa, stream=stream)
        hrew.copy_(f[2], non_blocking=True)
        hq0b.copy_(a[0], non_blocking=True)
        hqd0b.copy_(a[1], non_blocking=True)
        hab.copy_(a[2], non_blocking=True)

    ms_e2e = timed(e2e_step, args.steps, args.warmup)
    h2d = 4 * (q0.numel() + qd0.numel() + act.numel())
    d2h = 4 * (hrew.numel() + hab.numel() + hq0b.numel() + hqd0b.numel())

    # max over ranks
    ms_window, ms_plain, ms_e2e, ms_fwd, ms_adj, ms_episodic, ms_tape, ms_tape_adj = max_over_ranks(
        [ms_window, ms_plain, ms_e2e, ms_fwd, ms_adj, ms_episodic, ms_tape, ms_tape_adj], dist, dev)
    if rank != 0:
        return
    env_steps = n_envs * H * world
    value = env_steps / (ms_window * 1e-3)
    plain_value = env_steps / (ms_plain * 1e-3)
    sm_max = (clocks or {}).get("sm_max_mhz") or DEFAULT_SM_MAX_MHZ
    sm_med = (clocks or {}).get("sm_mhz") or sm_max
    peak = fp32_peak_tflops(n_sms, sm_max)
    peak_src = (f"derived FP32 peak: {n_sms} SMs (device query) x {FP32_LANES_PER_SM} lanes x "
                f"{FLOPS_PER_LANE_CYCLE} flop x {sm_max:.0f} MHz (maximum SM clock sampled)")
    model0 = groups[0][0]
    counts = FLOPS_PER_ENV_STEP.get(model0.name) if len(groups) == 1 else None
    bytes_alg = algo_bytes_per_env_step(model0) if len(groups) == 1 else None
    per_launch = n_envs * H
    dominant, ms_dom = ("adjoint", ms_adj) if ms_adj >= ms_fwd else ("forward", ms_fwd)
    dom_flops = None
    if counts:
        dom_flops = counts["recompute"] + counts["reverse"] if dominant == "adjoint" else counts["forward"]
    achieved = None if dom_flops is None else dom_flops * per_launch / (ms_dom * 1e-3) / 1e12
    traffic = TRAFFIC_BYTES_PER_LAUNCH.get(wl.name, {}).get("adjoint_recompute" if dominant == "adjoint"
                                                             else "forward")
    if spec_s is None:   # the capture is of the specialised kernels
        traffic = None
    hbm_peak, hbm_src = measured_hbm_gbs()
    dom_bytes = None if bytes_alg is None else bytes_alg[dominant] * per_launch
    # the window's work (forward + recompute + reverse) over each form's window time
    wf = None if counts is None else counts["forward"] + counts["recompute"] + counts["reverse"]

    def window_roofline(ms, flops_per_env_step):
        if flops_per_env_step is None:
            return None
        a = flops_per_env_step * env_steps / (ms * 1e-3) / 1e12
        return {"bound": "alu", "achieved": a, "peak": peak, "unit": "TFLOP/s", "frac": a / peak,
                "flops_per_env_step": flops_per_env_step, "peak_source": peak_src}

    line = {
        "metric": METRIC, "value": value, "unit": "env-steps/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_window, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": wl.name, "n_envs_per_gpu": n_envs, "h": H,
                   "substeps": model0.substeps if len(groups) == 1 else [m.substeps for m, _ in groups],
                   "form": "batched; per-control-step checkpoints, substeps recomputed in the adjoint; forward + "
                           "adjoint captured in one CUDA graph",
                   "kernels": "model-specialised (run-time compiled for this model and launch shape, "
                              f"{spec_s:.1f} s)" if spec_s is not None else "generic",
                   "lanes_per_env": [l for l, _ in shape], "warps_per_cta": shape[0][1],
                   "timing": "median of the timed steps", "l2": "flushed (256 MB write) before each timed step",
                   "parallelism": f"env-sharded replicas x{world}"},
        "autotune": tune,
        "plain_form": {"value": plain_value, "unit": "env-steps/s", "ms_per_step": ms_plain,
                       "steps": args.plain_steps, "window_roofline": window_roofline(ms_plain, wf)},
        "window_roofline": window_roofline(ms_window, wf),
        "speedup_vs_plain": value / plain_value,
        "window_tape": {"value": env_steps / (ms_tape * 1e-3), "unit": "env-steps/s", "ms_per_step": ms_tape,
                        "bitwise_equal_to_recompute": bool(same),
                        "tape_bytes_per_env_step": tape_bytes,
                        "workspace_bytes": int(ws_step + tape_bytes * H * (n_envs + 31 * len(groups))),
                        "ms_adjoint_kernel": ms_tape_adj,
                        "window_roofline": window_roofline(ms_tape, None if counts is None else
                                                           counts["forward"] + counts["reverse"]),
                        "scratch_vs_algorithmic_bytes": None if bytes_alg is None else
                        (tape_bytes + bytes_alg["adjoint"]) / bytes_alg["adjoint"],
                        "note": "the forward keeps every substep record in HBM and the adjoint reads them back "
                                "instead of recomputing each step's substeps; same results bit for bit"},
        "episodic": {"value": env_steps / (ms_episodic * 1e-3), "unit": "env-steps/s", "ms_per_step": ms_episodic,
                     "done_frac": done_frac,
                     "rule": "root below the task height or the task horizon; seeded reset states; "
                             "forward + adjoint with the gradient cut at resets, one CUDA graph"},
        "kernels_ms": {"k_batched_forward": ms_fwd, "k_batched_adjoint (recompute)": ms_adj},
        "gpu_launches": 2 * args.steps,
        "clocks": clocks,
        "e2e": {"value": env_steps / (ms_e2e * 1e-3), "unit": "env-steps/s", "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h},
        "roofline": {"bound": "alu", "kernel": f"k_batched<{1 if dominant == 'adjoint' else 0}> ({dominant}"
                                               f"{', recomputing' if dominant == 'adjoint' else ''})",
                     "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                     "frac": None if achieved is None else achieved / peak,
                     "frac_at_median_clock": None if achieved is None else
                     achieved / fp32_peak_tflops(n_sms, sm_med),
                     "peak_source": peak_src, "traffic": traffic,
                     "flops_per_env_step": dom_flops,
                     "flops_source": "FP32 work the one-environment-per-thread form executes for the same "
                                     "stages (ncu count of FADD + FMUL + 2 FFMA)",
                     "units_per_launch": per_launch,
                     "hbm": None if dom_bytes is None else
                     {"achieved": dom_bytes / (ms_dom * 1e-3) / 1e9, "peak": hbm_peak, "unit": "GB/s",
                      "frac": dom_bytes / (ms_dom * 1e-3) / 1e9 / hbm_peak,
                      "algo_bytes_per_env_step": bytes_alg[dominant],
                      "algo_bytes_total_per_env_step": bytes_alg["forward"] + bytes_alg["adjoint"],
                      "peak_source": hbm_src}},
    }
    if not args.no_cpu_baseline:
        # CPU leg: the FP64 oracle timed on the host cores, and the gradient
        # validity gate (sampled environments of every group against it)
        r, threads, dt, desc = oracle_workload_rate(groups, seed=0, target_s=12.0)
        line["cpu_baseline"] = {"value": r, "unit": "env-steps/s", "cores": threads, "kind": "oracle",
                                "cpu_model": host_cpu_model(),
                                "sample": f"{desc}, forward + exact adjoint, {dt:.1f} s; rate extrapolated to the "
                                          f"workload",
                                "single_core": oracle_single_core_rate(args.workload)}
        if check_data is not None:
            cf, ca = check_data[:3], check_data[3:]
            line["grad_rel_err"] = gradient_check(sim, groups, cf, ca, act, rbar, n_sample=args.grad_check_envs)
    print(json.dumps(line), flush=True)


def oracle_single_core_rate(workload: str):
    """The oracle's env-steps/s on one host core (a child process with one
    OpenMP thread, a bounded sample of about 4 s); None if it fails."""
    code = ("import json, sys; sys.path.insert(0, sys.argv[1]); import bench; "
            "from paper_2204_07137_gb300 import inputs as I; "
            "r, t, dt, desc = bench.oracle_workload_rate(I.workload(sys.argv[2]).groups, seed=0, target_s=4.0); "
            "print(json.dumps({'value': r, 'unit': 'env-steps/s', 'cores': t, "
            "'sample': f'{desc}, {dt:.1f} s'}))")
    try:
        out = subprocess.run([sys.executable, "-c", code, ROOT, workload], capture_output=True, text=True,
                             timeout=300, env={**os.environ, "OMP_NUM_THREADS": "1"})
        return json.loads(out.stdout.strip().splitlines()[-1])
    except (subprocess.SubprocessError, ValueError, IndexError):
        return None


# Gradient validity gate per sampled environment: relative error <= 1e-3, or
# <= GRAD_FLOOR_FACTOR x the environment's FP32 floor (environments whose own
# gradient moves by more than 1e-4 when the oracle's operations are rounded at
# FP32's unit roundoff: a contact, friction or limit switch within rounding of
# its threshold somewhere in the window).
GRAD_RTOL = 1e-3
GRAD_FLOOR_RUNS = 3
GRAD_FLOOR_FACTOR = 10.0


def gradient_check(sim, groups, outf, outa, act, rbar, n_sample: int = 4):
    """Per group: the maximum over sampled environments of the per-environment
    relative error (2-norm) of the window gradients (action and initial-state
    cotangents) against the FP64 oracle adjoint run on the GPU checkpoints."""
    from oracle import oracle
    qt_all, qdt_all = sim.unpack(outf[0], "q"), sim.unpack(outf[1], "qd")
    a_all = sim.unpack(act, "act")
    ga_all, gq_all, gqd_all = sim.unpack(outa[2], "act"), sim.unpack(outa[0], "q"), sim.unpack(outa[1], "qd")
    rb_all = rbar.cpu().numpy()
    out, off = {}, 0
    for gi, (model, N) in enumerate(groups):
        o = oracle.Oracle(model)
        envs = np.sort(np.random.default_rng(gi).choice(N, size=min(n_sample, N), replace=False))
        qt = qt_all[gi][:, :, envs]
        qdt = qdt_all[gi][:, :, envs]
        a = a_all[gi][:, :, envs]
        rb = rb_all[:, off + envs]
        qb, qdb, ab = o.window_adjoint(qt.transpose(0, 2, 1), qdt.transpose(0, 2, 1), a.transpose(0, 2, 1), rb,
                                       np.zeros((len(envs), model.nq)), np.zeros((len(envs), model.nv)))
        g_a = ga_all[gi][:, :, envs].transpose(2, 0, 1).reshape(len(envs), -1)
        got = np.concatenate([g_a, gq_all[gi][:, envs].T, gqd_all[gi][:, envs].T], axis=1)
        ref = np.concatenate([ab.transpose(1, 0, 2).reshape(len(envs), -1), qb, qdb], axis=1)
        rel = np.linalg.norm(got - ref, axis=1) / np.linalg.norm(ref, axis=1)
        # FP32 floor of each environment's gradient along the same checkpoints:
        # the oracle's own largest deviation over GRAD_FLOOR_RUNS runs with every
        # operation perturbed at FP32's unit roundoff (Monte Carlo Arithmetic)
        floor = np.zeros(len(envs))
        for k in range(GRAD_FLOOR_RUNS):
            mc = o.mca_window_adjoint(qt.transpose(0, 2, 1), qdt.transpose(0, 2, 1), a.transpose(0, 2, 1), rb,
                                      np.zeros((len(envs), model.nq)), np.zeros((len(envs), model.nv)),
                                      seed=11 + k, tangents=False)
            mref = np.concatenate([mc[2].transpose(1, 0, 2).reshape(len(envs), -1), mc[0], mc[1]], axis=1)
            floor = np.maximum(floor, np.linalg.norm(mref - ref, axis=1) / np.linalg.norm(ref, axis=1))
        ok = rel <= np.maximum(GRAD_RTOL, GRAD_FLOOR_FACTOR * floor)
        out[f"{gi}:{model.name}"] = {"max": float(rel.max()), "envs": envs.tolist(), "rel": rel.tolist(),
                                     "fp32_floor": floor.tolist(), "within_gate": bool(ok.all())}
        off += N
    return out


def policy_main(args, rank, world, dist):
    """Config 5 with the policy in the loop: the window of h = 32 steps in which
    every step's actions come from the MLP (obs -> 256 -> 128 -> muscles) and
    the loss's gradient flows through the library's step adjoints into the
    policy parameters (one CUDA graph: forward, loss, backward).  Timed beside
    the same step loop with given actions (no network; gradient with respect
    to the actions) and the open-loop window calls (two launches).  Each rank
    its own shard (weak scaling); env-steps/s = N h / time."""
    import torch
    from paper_2204_07137_gb300 import build, inputs as I
    from paper_2204_07137_gb300.policy import PolicyMLP, observation_size, policy_window_loss
    from paper_2204_07137_gb300.sim import Simulator

    build.build()
    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", 0)))
    torch.cuda.set_device(dev)
    wl = I.workload(args.workload)
    if len(wl.groups) != 1 or not wl.groups[0][0].n_muscles:
        raise SystemExit("--policy needs a single muscle-actuated group (mtu-512)")
    model, N = wl.groups[0]
    seed = shard_seed(rank)
    sim = Simulator(wl.groups, form="batched", h_max=1)
    g = torch.Generator().manual_seed(seed)
    pol = PolicyMLP(observation_size(model), model.na, generator=g).to(dev)
    params = list(pol.parameters())
    q0 = sim.pack([I.initial_state(model, N, seed)[0]], "q")
    qd0 = sim.pack([I.initial_state(model, N, seed)[1]], "qd")
    acts = torch.from_numpy(I.window_actions(model, N, H, seed).reshape(H, -1)).to(dev).contiguous()
    # the library's launch-shape search on this workload, as for the contract line
    if args.autotune_ms > 0:
        sim.autotune_native(budget_ms=args.autotune_ms, q0=q0, qd0=qd0, act=acts)
    if not args.no_specialize:
        sim.specialize()
        if args.autotune_ms > 0:
            sim.autotune_native(budget_ms=args.autotune_ms, q0=q0, qd0=qd0, act=acts)
    shape = sim.get_launch(0)
    acts.requires_grad_(True)
    flush = torch.empty(FLUSH_BYTES, dtype=torch.uint8, device=dev)
    stream = torch.cuda.Stream(device=dev)
    timed = Timer(stream, flush, dist)

    def capture(fn):
        with torch.cuda.stream(stream):
            for _ in range(2):
                fn()
        stream.synchronize()
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.stream(stream):
            with torch.cuda.graph(graph, stream=stream):
                out = fn()
        stream.synchronize()
        return graph, out

    def with_policy():
        loss = policy_window_loss(sim, pol, q0, qd0, H)
        return (loss,) + tuple(torch.autograd.grad(loss, params))

    def without_policy():
        loss = policy_window_loss(sim, pol, q0, qd0, H, actions=acts)
        return loss, torch.autograd.grad(loss, [acts])[0]

    g_pol, out_pol = capture(with_policy)
    g_act, out_act = capture(without_policy)
    wsim = Simulator(wl.groups, form="batched", h_max=H)
    wsim.set_launch(0, shape[0], shape[1])
    if not args.no_specialize:
        wsim.specialize()
    rbar = torch.full((H, N), 1.0 / (N * H), device=dev)
    zq = torch.zeros(H + 1, wsim.q_size, device=dev)
    zqd = torch.zeros(H + 1, wsim.qd_size, device=dev)
    a_det = acts.detach()
    g_win, _, outa = capture_window(wsim, q0, qd0, a_det, rbar, zq, zqd, stream)
    sampler = ClockSampler(dev.index) if rank == 0 else None
    if sampler:
        sampler.start()
    ms_pol = timed(g_pol.replay, args.steps, args.warmup)
    clocks = sampler.stop() if sampler else None
    ms_act = timed(g_act.replay, args.steps, args.warmup)
    ms_win = timed(g_win.replay, args.steps, args.warmup)
    torch.cuda.synchronize()
    finite = all(bool(torch.isfinite(x).all()) for x in tuple(out_pol) + tuple(out_act) + tuple(outa))
    ms_pol, ms_act, ms_win = max_over_ranks([ms_pol, ms_act, ms_win], dist, dev)
    if rank != 0:
        return
    env_steps = N * H * world
    n_params = sum(p.numel() for p in params)
    line = {
        "metric": METRIC + " (policy in the loop)", "value": env_steps / (ms_pol * 1e-3), "unit": "env-steps/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_pol,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": wl.name + " policy-in-the-loop", "n_envs_per_gpu": N, "h": H,
                   "substeps": model.substeps, "policy": f"MLP {observation_size(model)}-256-128-{model.na}, ELU, "
                                                       f"sigmoid; {n_params} parameters, weights ~ N(0, 0.05)",
                   "form": "per step: observation, MLP, library step (shac_step); backward: autograd through "
                           "the library's step adjoint (substeps recomputed) into the MLP; one CUDA graph",
                   "lanes_per_env": shape[0], "warps_per_cta": shape[1],
                   "kernels": "generic" if args.no_specialize else "model-specialised",
                   "timing": "median of the timed steps", "l2": "flushed (256 MB write) before each timed step"},
        "without_policy": {"value": env_steps / (ms_act * 1e-3), "unit": "env-steps/s", "ms_per_step": ms_act,
                           "form": "the same step loop with given actions, gradient w.r.t. the actions"},
        "open_loop_window": {"value": env_steps / (ms_win * 1e-3), "unit": "env-steps/s", "ms_per_step": ms_win,
                             "form": "shac_window_forward + shac_window_adjoint, one CUDA graph"},
        "finite": finite, "clocks": clocks,
        "gpu_launches": 2 * H * args.steps,
    }
    print(json.dumps(line), flush=True)


def profile_case_main(args):
    """A few windows of a workload through the public API, no timing and no
    checks, for profiler captures (the ncu commands recorded with the kernel
    summaries): --pc-envs environments of the first group (the others scaled
    alike), --pc-form, --pc-h steps, --pc-reps windows, --pc-tape, --pc-lanes /
    --pc-warps (0: the library's default shape)."""
    import torch
    from paper_2204_07137_gb300 import build, inputs as I
    from paper_2204_07137_gb300.sim import Simulator
    build.build()
    wl = I.workload(args.workload)
    scale = args.pc_envs / wl.groups[0][1] if args.pc_envs > 0 else 1.0
    groups = [(m, max(1, int(round(n * scale)))) for m, n in wl.groups]
    h = args.pc_h
    sim = Simulator(groups, form=args.pc_form, h_max=h)
    if args.pc_lanes or args.pc_warps:
        sim.set_launch(-1, args.pc_lanes, args.pc_warps)
    if args.pc_form == "batched" and args.pc_tape:
        sim.set_window_tape(True)
    if args.pc_form == "batched" and len(groups) == 1 and not args.no_specialize:
        sim.specialize()
    dev = sim.device
    q0, qd0, act = workload_inputs(sim, groups, 0, h, dev)
    rb = torch.ones(h, sim.n_envs, device=dev)
    zq = torch.zeros(h + 1, sim.q_size, device=dev)
    zqd = torch.zeros(h + 1, sim.qd_size, device=dev)
    for _ in range(args.pc_reps):
        f = sim.window_forward(q0, qd0, act)
        sim.window_adjoint(f[0], f[1], act, rb, zq, zqd)
    torch.cuda.synchronize()
    assert bool(torch.isfinite(f[0]).all())


def main():
    args = parse()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist_mod
        backend = "gloo" if args.impl == "reference" else "nccl"
        if backend == "nccl":
            import torch
            torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", 0)))
        dist_mod.init_process_group(backend)
        dist = dist_mod
    try:
        if args.impl == "reference":
            reference_main(args, rank, world)
        elif args.profile_case:
            if rank == 0:
                profile_case_main(args)
        elif args.policy:
            policy_main(args, rank, world, dist)
        elif args.h_sweep:
            if rank == 0:
                h_sweep_main(args)
        elif args.shac_episodes > 0:
            if rank == 0:
                shac_main(args)
        else:
            gpu_main(args, rank, world, dist)
    finally:
        if dist is not None:
            dist.destroy_process_group()


if __name__ == "__main__":
    main()
