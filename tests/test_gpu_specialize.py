"""Model-specialised batched kernels (shac_batch_specialize): the batched
kernels compiled at run time with one model's counts and scratch offsets and
the team size as constants.  They must compute what the generic kernels
compute: every step against the FP64 oracle (the same gate as the generic
kernels), the window gradients against the generic kernels', the window tape
bit for bit against their own recompute, a CUDA graph replayed bit for bit;
the generic kernels take over when the launch shape changes; batches they do
not cover are refused."""
import numpy as np
import pytest

from helpers import (airborne, assert_grad_close, assert_state_close, model_by_name, oracle_step_with_floor)
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


def _window(sim, m, N, h, seed):
    q0, qd0 = I.initial_state(m, N, seed)
    act = T(I.window_actions(m, N, h, seed)).view(h, -1)
    rng = np.random.default_rng(seed)
    rb = T(rng.normal(size=(h, N))).view(h, -1)
    zq = torch.zeros(h + 1, sim.q_size, device="cuda")
    zqd = torch.zeros(h + 1, sim.qd_size, device="cuda")
    f = sim.window_forward(T(q0), T(qd0), act)
    g = sim.window_adjoint(f[0], f[1], act, rb, zq, zqd)
    torch.cuda.synchronize()
    return act, f, g


CASES = [("cartpole", 37, False), ("ant", 23, False), ("ant", 9, True), ("humanoid", 5, False), ("mtu", 3, False),
         ("halfcheetah", 19, False), ("hopper", 21, False)]


@pytest.mark.parametrize("name,N,air", CASES)
def test_specialised_window_matches_oracle_and_generic(oracle_mod, name, N, air):
    from paper_2204_07137_gb300.sim import Simulator
    m = model_by_name(name)
    if air:
        m = airborne(m)
    h = 4
    gen = Simulator([(m, N)], form="batched", h_max=h)
    spc = Simulator([(m, N)], form="batched", h_max=h)
    spc.specialize()
    act, f, g = _window(spc, m, N, h, 3)
    _, fg, gg = _window(gen, m, N, h, 3)
    assert spc.status() == 0 and gen.status() == 0
    o = oracle_mod.Oracle(m)
    gq = f[0].cpu().numpy().reshape(h + 1, m.nq, N).transpose(0, 2, 1)
    gqd = f[1].cpu().numpy().reshape(h + 1, m.nv, N).transpose(0, 2, 1)
    a = act.cpu().numpy().reshape(h, m.na, N).transpose(0, 2, 1)
    (rq, rqd, rr), (fq, fqd, fr) = oracle_step_with_floor(o, gq[:-1].reshape(-1, m.nq), gqd[:-1].reshape(-1, m.nv),
                                                          a.reshape(-1, m.na))
    assert_state_close(gq[1:].reshape(-1, m.nq), rq, f"specialised {name} q", fq)
    assert_state_close(gqd[1:].reshape(-1, m.nv), rqd, f"specialised {name} qd", fqd)
    assert_state_close(f[2].cpu().numpy().reshape(-1), rr, f"specialised {name} reward", fr)
    # the generic kernels on the same inputs: the same window up to FP32 rounding
    got = np.concatenate([x.cpu().numpy().reshape(-1, N) for x in g])
    ref = np.concatenate([x.cpu().numpy().reshape(-1, N) for x in gg])
    assert_grad_close(got, ref, f"specialised {name} window gradient vs generic", rtol=1e-3)
    np.testing.assert_allclose(f[0].cpu().numpy(), fg[0].cpu().numpy(), rtol=1e-3, atol=1e-4)


def test_specialised_tape_graph_and_fallback():
    from paper_2204_07137_gb300.sim import Simulator
    m, N, h = I.ant(), 40, 6
    rec = Simulator([(m, N)], form="batched", h_max=h)
    rec.specialize()
    tap = Simulator([(m, N)], form="batched", h_max=h)
    tap.set_window_tape(True)
    tap.specialize()
    a1, f1, g1 = _window(rec, m, N, h, 5)
    a2, f2, g2 = _window(tap, m, N, h, 5)
    for x, y in zip(tuple(f1) + tuple(g1), tuple(f2) + tuple(g2)):
        assert torch.equal(x, y)
    # graph capture of the specialised forward + adjoint window, replayed bit for bit
    q0, qd0 = (T(x) for x in I.initial_state(m, N, 7))
    act = T(I.window_actions(m, N, h, 7)).view(h, -1)
    rb = torch.ones(h, N, device="cuda")
    zq = torch.zeros(h + 1, rec.q_size, device="cuda")
    zqd = torch.zeros(h + 1, rec.qd_size, device="cuda")
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        outf = rec.window_forward(q0, qd0, act, stream=s)
        outa = rec.window_adjoint(outf[0], outf[1], act, rb, zq, zqd, stream=s)
    s.synchronize()
    ref = [t.clone() for t in tuple(outf) + tuple(outa)]
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.stream(s):
        with torch.cuda.graph(graph, stream=s):
            rec.window_forward(q0, qd0, act, out=outf, stream=s)
            rec.window_adjoint(outf[0], outf[1], act, rb, zq, zqd, out=outa, stream=s)
    torch.cuda.current_stream().wait_stream(s)
    for _ in range(2):
        for t in tuple(outf) + tuple(outa):
            t.zero_()
        graph.replay()
        torch.cuda.synchronize()
        for x, y in zip(tuple(outf) + tuple(outa), ref):
            assert torch.equal(x, y)
    # another team size: the generic kernels run (no key mismatch is raised)
    rec.set_launch(0, 32, 0)
    _, f3, g3 = _window(rec, m, N, h, 5)
    assert rec.status() == 0
    for x, y in zip(tuple(f3) + tuple(g3), tuple(f1) + tuple(g1)):
        np.testing.assert_allclose(x.cpu().numpy(), y.cpu().numpy(), rtol=1e-3, atol=1e-4)


def test_specialisation_refuses_what_it_does_not_cover():
    from paper_2204_07137_gb300 import _lib
    from paper_2204_07137_gb300.sim import Simulator
    for sim in (Simulator([(I.cartpole(), 8), (I.ant(), 4)], form="batched", h_max=2),
                Simulator([(I.ant(), 4)], form="plain", h_max=2)):
        with pytest.raises(_lib.ShacError) as e:
            sim.specialize()
        assert e.value.status == 6   # SHAC_ERR_UNSUPPORTED
    sim = Simulator([(I.ant(), 4)], form="batched", h_max=2)
    sim.specialize(True)
    sim.specialize(False)
    assert _lib.load().shac_batch_specialize(sim.batch, 2) == 1   # SHAC_ERR_INVALID_ARG


def test_autotune_on_a_specialised_batch_keeps_its_team_size():
    """After specialisation the launch-shape search keeps the team size the
    kernels were compiled for and only moves the warps per CTA; the window it
    leaves behind computes what the generic kernels compute."""
    from paper_2204_07137_gb300.sim import Simulator
    m, N, h = I.ant(), 96, 4
    spc = Simulator([(m, N)], form="batched", h_max=h)
    spc.set_launch(0, 16, 4)
    spc.specialize()
    shape = spc.autotune_native(budget_ms=3000)
    assert shape[0][0] == 16 and shape[0][1] in (1, 2, 4, 8)
    gen = Simulator([(m, N)], form="batched", h_max=h)
    gen.set_launch(0, 16, 4)
    _, f, g = _window(spc, m, N, h, 11)
    _, fg, gg = _window(gen, m, N, h, 11)
    assert spc.status() == 0 and gen.status() == 0
    for x, y in zip(tuple(f) + tuple(g), tuple(fg) + tuple(gg)):
        np.testing.assert_allclose(x.cpu().numpy(), y.cpu().numpy(), rtol=1e-3, atol=1e-4)
