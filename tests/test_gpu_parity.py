"""GPU (FP32, through the C ABI) against the FP64 oracle on the same seeded
inputs: per-step states and rewards, step adjoints, window adjoints, both
execution forms; sizes span several work items with a ragged tail."""
import numpy as np
import pytest

from helpers import (airborne, assert_grad_close, assert_state_close, model_by_name,
                     oracle_step_with_floor, seeded_case)
from paper_2204_07137_gb300 import inputs as I

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2204_07137_gb300 import build
    build.build()


def make_sim(groups, form, h_max=32):
    from paper_2204_07137_gb300.sim import Simulator
    return Simulator(groups, form=form, h_max=h_max)


def orc(oracle_mod, model):
    return oracle_mod.Oracle(model)


def T(x):
    return torch.from_numpy(np.ascontiguousarray(np.asarray(x, np.float32).reshape(-1))).cuda()


# (model name, N, airborne?) -- N chosen to leave a ragged last work item
CASES = [("cartpole", 37, False), ("ant", 23, False), ("ant", 9, True), ("humanoid", 5, False),
         ("humanoid", 3, True), ("mtu", 3, False), ("halfcheetah", 19, False), ("hopper", 21, False)]


@pytest.mark.parametrize("form", ["plain", "batched"])
@pytest.mark.parametrize("name,N,air", CASES)
def test_step_matches_oracle(oracle_mod, form, name, N, air):
    m = model_by_name(name)
    if air:
        m = airborne(m)
    sim = make_sim([(m, N)], form)
    o = orc(oracle_mod, m)
    for seed, kind in ((0, "initial"), (1, "random")):
        q, qd, a = seeded_case(m, N, seed, kind)
        qn, qdn, r = sim.step(T(q), T(qd), T(a))
        torch.cuda.synchronize()
        (rq, rqd, rr), (fq, fqd, fr) = oracle_step_with_floor(o, q.T, qd.T, a.T)
        assert_state_close(qn.cpu().numpy().reshape(m.nq, N).T, rq, f"step {name}/{form} q seed {seed}", fq)
        assert_state_close(qdn.cpu().numpy().reshape(m.nv, N).T, rqd, f"step {name}/{form} qd seed {seed}", fqd)
        assert_state_close(r.cpu().numpy(), rr, f"step {name}/{form} reward seed {seed}", fr)
    assert sim.status() == 0


@pytest.mark.parametrize("form", ["plain", "batched"])
@pytest.mark.parametrize("name,N,air", CASES)
def test_step_adjoint_matches_oracle(oracle_mod, form, name, N, air):
    m = model_by_name(name)
    if air:
        m = airborne(m)
    sim = make_sim([(m, N)], form)
    o = orc(oracle_mod, m)
    q, qd, a = seeded_case(m, N, 2, "initial")
    rng = np.random.default_rng(5)
    qb = rng.normal(size=(m.nq, N)).astype(np.float32)
    qdb = rng.normal(size=(m.nv, N)).astype(np.float32)
    rb = rng.normal(size=N).astype(np.float32)
    gq, gqd, ga = sim.step_adjoint(T(q), T(qd), T(a), T(qb), T(qdb), T(rb))
    torch.cuda.synchronize()
    rq, rqd, ra = o.step_vjp(q.T, qd.T, a.T, qb.T, qdb.T, rb)
    got = np.concatenate([gq.cpu().numpy().reshape(m.nq, N), gqd.cpu().numpy().reshape(m.nv, N),
                          ga.cpu().numpy().reshape(m.na, N)])
    ref = np.concatenate([rq.T, rqd.T, ra.T])
    assert_grad_close(got, ref, f"{name}/{form} step adjoint")


WINDOW_CASES = [("cartpole", 37, False, 32), ("ant", 11, False, 32), ("ant", 5, True, 32),
                ("humanoid", 3, False, 6), ("mtu", 2, False, 4), ("halfcheetah", 7, False, 16),
                ("hopper", 9, False, 16)]


@pytest.mark.parametrize("form", ["plain", "batched"])
@pytest.mark.parametrize("name,N,air,h", WINDOW_CASES)
def test_window_matches_oracle(oracle_mod, form, name, N, air, h):
    """Window forward: every step checked from the GPU's own checkpoint;
    contact-free cases also compare the whole trajectory.  Window adjoint:
    the oracle adjoint runs on the GPU checkpoints (per-env norm-wise)."""
    m = model_by_name(name)
    if air:
        m = airborne(m)
    sim = make_sim([(m, N)], form, h_max=h)
    o = orc(oracle_mod, m)
    q0, qd0 = I.initial_state(m, N, 3)
    act = I.window_actions(m, N, h, 3)
    qt, qdt, rw = sim.window_forward(T(q0), T(qd0), T(act).view(h, -1))
    torch.cuda.synchronize()
    gq = qt.cpu().numpy().reshape(h + 1, m.nq, N)
    gqd = qdt.cpu().numpy().reshape(h + 1, m.nv, N)
    grw = rw.cpu().numpy()
    assert np.array_equal(gq[0], q0) and np.array_equal(gqd[0], qd0)
    # per step from the GPU checkpoints
    sq = gq[:-1].transpose(0, 2, 1).reshape(-1, m.nq)
    sqd = gqd[:-1].transpose(0, 2, 1).reshape(-1, m.nv)
    sa = act.transpose(0, 2, 1).reshape(-1, m.na)
    (rq, rqd, rr), (fq, fqd, fr) = oracle_step_with_floor(o, sq, sqd, sa)
    assert_state_close(gq[1:].transpose(0, 2, 1).reshape(-1, m.nq), rq, f"window {name}/{form} q", fq)
    assert_state_close(gqd[1:].transpose(0, 2, 1).reshape(-1, m.nv), rqd, f"window {name}/{form} qd", fqd)
    assert_state_close(grw.reshape(-1), rr, f"window {name}/{form} reward", fr)
    if name == "cartpole" or air:
        oq, oqd, orw = o.window_forward(q0.T, qd0.T, act.transpose(0, 2, 1))
        assert_state_close(gq.transpose(0, 2, 1), oq, f"{name}/{form} trajectory q", rtol=1e-3, atol=1e-4)
    # window adjoint with random cotangents on rewards and on the final state
    rng = np.random.default_rng(7)
    rb = rng.normal(size=(h, N)).astype(np.float32)
    qtb = np.zeros((h + 1, m.nq, N), np.float32)
    qdtb = np.zeros((h + 1, m.nv, N), np.float32)
    qtb[-1] = rng.normal(size=(m.nq, N))
    qdtb[-1] = rng.normal(size=(m.nv, N))
    qtb[h // 2] = rng.normal(size=(m.nq, N))      # a mid-window checkpoint read directly
    g0, gd0, ga = sim.window_adjoint(qt, qdt, T(act).view(h, -1), T(rb).view(h, -1), T(qtb).view(h + 1, -1),
                                     T(qdtb).view(h + 1, -1))
    torch.cuda.synchronize()
    # oracle: chain step VJPs over the GPU checkpoints, adding the direct checkpoint cotangents
    qbar = qtb[-1].T.astype(np.float64)
    qdbar = qdtb[-1].T.astype(np.float64)
    abar = np.zeros((h, N, m.na))
    for t in range(h - 1, -1, -1):
        qbar, qdbar, abar[t] = o.step_vjp(gq[t].T, gqd[t].T, act[t].T, qbar, qdbar, rb[t])
        qbar = qbar + qtb[t].T
        qdbar = qdbar + qdtb[t].T
    got = np.concatenate([g0.cpu().numpy().reshape(m.nq, N), gd0.cpu().numpy().reshape(m.nv, N),
                          ga.cpu().numpy().reshape(h * m.na, N)])
    ref = np.concatenate([qbar.T, qdbar.T, abar.transpose(0, 2, 1).reshape(h * m.na, N)])
    assert_grad_close(got, ref, f"{name}/{form} window adjoint")


def test_plain_and_batched_agree_and_graph_replay_is_bitwise(oracle_mod):
    m = I.ant()
    N, h = 13, 8
    sp = make_sim([(m, N)], "plain", h)
    sb = make_sim([(m, N)], "batched", h)
    q0, qd0 = I.initial_state(m, N, 4)
    act = T(I.window_actions(m, N, h, 4)).view(h, -1)
    a = sp.window_forward(T(q0), T(qd0), act)
    b = sb.window_forward(T(q0), T(qd0), act)
    torch.cuda.synchronize()
    for x, y in zip(a, b):
        assert torch.isfinite(x).all() and torch.isfinite(y).all()
        np.testing.assert_allclose(x.cpu().numpy(), y.cpu().numpy(), rtol=1e-4, atol=1e-4)
    # CUDA-graph capture of the batched forward + adjoint window, replayed
    q0t, qd0t = T(q0), T(qd0)
    rb = torch.ones(h, N, device="cuda")
    qtb = torch.zeros(h + 1, sb.q_size, device="cuda")
    qdtb = torch.zeros(h + 1, sb.qd_size, device="cuda")
    outf = sb.window_forward(q0t, qd0t, act)
    outa = sb.window_adjoint(outf[0], outf[1], act, rb, qtb, qdtb)
    ref = [t.clone() for t in outf + outa]
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    g = torch.cuda.CUDAGraph()
    with torch.cuda.stream(s):
        with torch.cuda.graph(g, stream=s):
            sb.window_forward(q0t, qd0t, act, out=outf, stream=s)
            sb.window_adjoint(outf[0], outf[1], act, rb, qtb, qdtb, out=outa, stream=s)
    torch.cuda.current_stream().wait_stream(s)
    for _ in range(2):
        for t in outf + outa:
            t.zero_()
        g.replay()
        torch.cuda.synchronize()
        for x, y in zip(outf + outa, ref):
            assert torch.equal(x, y)


def test_heterogeneous_batch_equals_homogeneous_runs(oracle_mod):
    """One persistent launch over cartpole + ant + humanoid groups gives, per
    environment, exactly the results of each group run alone."""
    groups = [(I.cartpole(), 40), (I.ant(), 7), (I.humanoid(), 3)]
    h = 3
    het = make_sim(groups, "batched", h)
    q0 = [I.initial_state(m, n, 6)[0] for m, n in groups]
    qd0 = [I.initial_state(m, n, 6)[1] for m, n in groups]
    acts = [I.window_actions(m, n, h, 6) for m, n in groups]
    act_flat = np.concatenate([a.reshape(h, -1) for a in acts], axis=1)
    out = het.window_forward(het.pack(q0, "q"), het.pack(qd0, "qd"), T(act_flat).view(h, -1))
    qs = het.unpack(out[0], "q")
    rws = np.split(out[2].cpu().numpy(), np.cumsum([n for _, n in groups])[:-1], axis=1)
    for gi, (m, n) in enumerate(groups):
        s1 = make_sim([(m, n)], "batched", h)
        o1 = s1.window_forward(T(q0[gi]), T(qd0[gi]), T(acts[gi]).view(h, -1))
        np.testing.assert_array_equal(qs[gi], o1[0].cpu().numpy().reshape(h + 1, m.nq, n))
        np.testing.assert_array_equal(rws[gi], o1[2].cpu().numpy())


def test_autograd_window_gradient_matches_step_chain(oracle_mod):
    """SimWindow's backward equals chaining SimStep backward over the window."""
    from paper_2204_07137_gb300.sim import SimStep, SimWindow
    m = I.ant()
    N, h = 6, 5
    sim = make_sim([(m, N)], "batched", h)
    q0, qd0 = I.initial_state(m, N, 8)
    act = T(I.window_actions(m, N, h, 8)).view(h, -1).requires_grad_(True)
    qd0t = T(qd0).requires_grad_(True)
    qt, qdt, rw = SimWindow.apply(sim, T(q0), qd0t, act)
    loss = rw.sum() + (qt[-1] ** 2).sum() + qdt[h // 2].sum()
    loss.backward()
    g_act, g_qd0 = act.grad.clone(), qd0t.grad.clone()
    act2 = act.detach().clone().requires_grad_(True)
    qd_leaf = T(qd0).requires_grad_(True)
    q, qd = T(q0), qd_leaf
    qds = [qd]
    total = 0.0
    for t in range(h):
        q, qd, r = SimStep.apply(sim, q, qd, act2[t])
        qds.append(qd)
        total = total + r.sum()
    total = total + (q ** 2).sum() + qds[h // 2].sum()
    total.backward()
    np.testing.assert_allclose(g_act.cpu().numpy(), act2.grad.cpu().numpy(), rtol=1e-4, atol=1e-5)
    np.testing.assert_allclose(g_qd0.cpu().numpy(), qd_leaf.grad.cpu().numpy(), rtol=1e-4, atol=1e-5)


@pytest.mark.parametrize("lanes", [1, 4, 16, 32])
def test_team_sizes_match_oracle(oracle_mod, lanes):
    """Every team size (lanes per environment), including teams narrower than
    the DOF count (shared-memory dense stages), matches the oracle."""
    m = I.ant()
    N = 21
    sim = make_sim([(m, N)], "batched", 2)
    sim.set_launch(0, lanes, 0)
    assert sim.get_launch(0)[0] == lanes
    o = orc(oracle_mod, m)
    q, qd, a = seeded_case(m, N, 9, "initial")
    qn, qdn, r = sim.step(T(q), T(qd), T(a))
    torch.cuda.synchronize()
    (rq, rqd, rr), (fq, fqd, fr) = oracle_step_with_floor(o, q.T, qd.T, a.T)
    assert_state_close(qn.cpu().numpy().reshape(m.nq, N).T, rq, f"lanes {lanes} q", fq)
    assert_state_close(qdn.cpu().numpy().reshape(m.nv, N).T, rqd, f"lanes {lanes} qd", fqd)
    rng = np.random.default_rng(3)
    qb, qdb, rb = (rng.normal(size=s).astype(np.float32) for s in ((m.nq, N), (m.nv, N), N))
    gq, gqd, ga = sim.step_adjoint(T(q), T(qd), T(a), T(qb), T(qdb), T(rb))
    torch.cuda.synchronize()
    sq, sqd, sa = o.step_vjp(q.T, qd.T, a.T, qb.T, qdb.T, rb)
    got = np.concatenate([gq.cpu().numpy().reshape(m.nq, N), gqd.cpu().numpy().reshape(m.nv, N),
                          ga.cpu().numpy().reshape(m.na, N)])
    assert_grad_close(got, np.concatenate([sq.T, sqd.T, sa.T]), f"lanes {lanes} adjoint")
