"""Full-size workloads in the launch configuration the bench times (batched
form, launch shape chosen by the library's autotuner, kernels compiled for the
model and that shape when the batch has one group, per-step checkpoints,
substeps recomputed in the adjoint), h = 32: sampled environments of every
articulation group checked against the FP64 oracle -

  * every step of the window from the GPU's own checkpoints, elementwise
    (1e-4 relative / 1e-5 absolute), or within the FP32 floor of its state;
  * the window gradients (initial-state and action cotangents of the mean
    window reward), relative 2-norm error per environment <= 1e-3, or within
    10 x the environment's FP32 floor (the oracle's own largest gradient
    deviation over 3 Monte Carlo Arithmetic runs at FP32's unit roundoff) for
    an environment whose gradient is itself that sensitive; the
    distribution and the floors recorded for the session summary;
  * every environment of the batch finite.
"""
import numpy as np
import pytest

from helpers import (GRAD_FLOOR_FACTOR, GRAD_FLOOR_RUNS, GRAD_LOG, GRAD_RTOL, assert_state_close, grad_rel_per_env,
                     oracle_step_with_floor)
from paper_2204_07137_gb300 import inputs as I

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

H = 32
# (workload, sampled environments per group)
FULL = [("ant-2048", 16), ("humanoid-1024", 64), ("mtu-512", 16), ("hetero-4096-2048-1024", 8),
        ("halfcheetah-2048", 8), ("hopper-2048", 8), ("cartpole-64", 16)]


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2204_07137_gb300 import build
    build.build()


@pytest.mark.parametrize("workload,n_sample", FULL)
def test_full_size_window_matches_oracle(oracle_mod, workload, n_sample):
    from paper_2204_07137_gb300.sim import Simulator
    wl = I.workload(workload)
    sim = Simulator(wl.groups, form="batched", h_max=H)
    q0 = sim.pack([I.initial_state(m, n, 0)[0] for m, n in wl.groups], "q")
    qd0 = sim.pack([I.initial_state(m, n, 0)[1] for m, n in wl.groups], "qd")
    act = torch.cat([torch.from_numpy(I.window_actions(m, n, H, 0).reshape(H, -1)) for m, n in wl.groups],
                    dim=1).cuda().contiguous()
    # the bench's launch configuration: the search on these inputs, specialisation, the warps re-searched
    sim.autotune_native(budget_ms=3000, q0=q0, qd0=qd0, act=act)
    if len(wl.groups) == 1:
        sim.specialize()
        sim.autotune_native(budget_ms=3000, q0=q0, qd0=qd0, act=act)
    rb = torch.full((H, wl.n_envs), 1.0 / (wl.n_envs * H), device="cuda")
    zq = torch.zeros(H + 1, sim.q_size, device="cuda")
    zqd = torch.zeros(H + 1, sim.qd_size, device="cuda")
    qt, qdt, rw = sim.window_forward(q0, qd0, act)
    g0, gd0, ga = sim.window_adjoint(qt, qdt, act, rb, zq, zqd)
    torch.cuda.synchronize()
    for x in (qt, qdt, rw, g0, gd0, ga):
        assert torch.isfinite(x).all()
    assert sim.status() == 0
    qt_g, qdt_g, a_g = sim.unpack(qt, "q"), sim.unpack(qdt, "qd"), sim.unpack(act, "act")
    g0_g, gd0_g, ga_g = sim.unpack(g0, "q"), sim.unpack(gd0, "qd"), sim.unpack(ga, "act")
    rw_all, rb_all = rw.cpu().numpy(), rb.cpu().numpy()
    off = 0
    for gi, (m, N) in enumerate(wl.groups):
        o = oracle_mod.Oracle(m)
        envs = np.sort(np.random.default_rng(1000 + gi).choice(N, size=min(n_sample, N), replace=False))
        ne = len(envs)
        gq = qt_g[gi][:, :, envs].astype(np.float64).transpose(0, 2, 1)     # [h+1, ne, nq]
        gqd = qdt_g[gi][:, :, envs].astype(np.float64).transpose(0, 2, 1)
        a = a_g[gi][:, :, envs].astype(np.float64).transpose(0, 2, 1)       # [h, ne, na]
        tag = f"{workload} {m.name}"
        # every step from the GPU checkpoints
        (rq, rqd, rr), (fq, fqd, fr) = oracle_step_with_floor(o, gq[:-1].reshape(-1, m.nq),
                                                              gqd[:-1].reshape(-1, m.nv), a.reshape(-1, m.na))
        assert_state_close(gq[1:].reshape(-1, m.nq), rq, f"full {tag} q", fq)
        assert_state_close(gqd[1:].reshape(-1, m.nv), rqd, f"full {tag} qd", fqd)
        assert_state_close(rw_all[:, off + envs].reshape(-1), rr, f"full {tag} reward", fr)
        # window gradients of the sampled environments
        rbs = rb_all[:, off + envs]
        z = (np.zeros((ne, m.nq)), np.zeros((ne, m.nv)))
        ex = o.window_adjoint(gq, gqd, a, rbs, *z)

        def flat(qb, qdb, ab):
            return np.concatenate([ab.transpose(1, 0, 2).reshape(ne, -1), qb, qdb], axis=1)
        ref = flat(*ex)
        got = flat(g0_g[gi][:, envs].T, gd0_g[gi][:, envs].T, ga_g[gi][:, :, envs].transpose(0, 2, 1))
        rel = grad_rel_per_env(got, ref)
        floor = np.zeros(ne)
        for k in range(GRAD_FLOOR_RUNS):
            mc = o.mca_window_adjoint(gq, gqd, a, rbs, *z, seed=11 + k, tangents=False)
            floor = np.maximum(floor, grad_rel_per_env(flat(*mc), ref))
        bound = np.maximum(GRAD_RTOL, GRAD_FLOOR_FACTOR * floor)
        above = rel > GRAD_RTOL
        GRAD_LOG.append((f"{tag} (h {H})", ne, float(rel.max()), float(np.percentile(rel, 99)),
                         float(np.median(rel)), int(above.sum()), float(floor.max()), float(np.median(floor)),
                         int((above & (rel <= bound)).sum())))
        bad = np.argwhere(~(rel <= bound)).ravel()
        assert bad.size == 0, (f"{tag}: window gradients of {bad.size} / {ne} environments outside rel {GRAD_RTOL} and "
                               f"outside {GRAD_FLOOR_FACTOR} x their FP32 floor: envs {envs[bad].tolist()} "
                               f"rel {rel[bad]} floor {floor[bad]}")
        off += N
