"""Degenerate and extreme sizes through the C ABI: a single environment (a
team or a plain warp with one live lane) and the largest model the library
accepts (32 DOF) against the FP64 oracle, and an empty articulation group
inside a batch, which must change nothing for the others."""
import numpy as np
import pytest

from helpers import (assert_grad_close, assert_state_close, long_chain, model_by_name, oracle_step_with_floor,
                     seeded_case)
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


def make_sim(groups, form, h_max=4):
    from paper_2204_07137_gb300.sim import Simulator
    return Simulator(groups, form=form, h_max=h_max)


@pytest.mark.parametrize("form", ["plain", "batched"])
@pytest.mark.parametrize("name", ["cartpole", "ant", "humanoid"])
def test_single_environment_step_and_adjoint(oracle_mod, form, name):
    m = model_by_name(name)
    sim = make_sim([(m, 1)], form)
    o = oracle_mod.Oracle(m)
    q, qd, a = seeded_case(m, 1, 4, "initial")
    qn, qdn, r = sim.step(T(q), T(qd), T(a))
    torch.cuda.synchronize()
    (rq, rqd, rr), (fq, fqd, fr) = oracle_step_with_floor(o, q.T, qd.T, a.T)
    assert_state_close(qn.cpu().numpy().reshape(m.nq, 1).T, rq, f"one env {name}/{form} q", fq)
    assert_state_close(qdn.cpu().numpy().reshape(m.nv, 1).T, rqd, f"one env {name}/{form} qd", fqd)
    assert_state_close(r.cpu().numpy(), rr, f"one env {name}/{form} reward", fr)
    rng = np.random.default_rng(8)
    qb = rng.normal(size=(m.nq, 1)).astype(np.float32)
    qdb = rng.normal(size=(m.nv, 1)).astype(np.float32)
    rb = rng.normal(size=1).astype(np.float32)
    gq, gqd, ga = sim.step_adjoint(T(q), T(qd), T(a), T(qb), T(qdb), T(rb))
    torch.cuda.synchronize()
    sq, sqd, sa = o.step_vjp(q.T, qd.T, a.T, qb.T, qdb.T, rb)
    got = np.concatenate([gq.cpu().numpy().reshape(m.nq, 1), gqd.cpu().numpy().reshape(m.nv, 1),
                          ga.cpu().numpy().reshape(m.na, 1)])
    assert_grad_close(got, np.concatenate([sq.T, sqd.T, sa.T]), f"{name}/{form} step adjoint")
    assert sim.status() == 0


@pytest.mark.parametrize("form", ["plain", "batched"])
def test_empty_group_changes_nothing(form):
    """cart-pole 5 + ant 0 + hopper 3 in one batch: the window of every live
    environment equals the batch without the empty group, bit for bit."""
    h = 3
    full = [(I.cartpole(), 5), (I.ant(), 0), (I.hopper(), 3)]
    live = [full[0], full[2]]
    outs = []
    for groups in (full, live):
        sim = make_sim(groups, form, h)
        q0 = sim.pack([I.initial_state(m, n, 9)[0] for m, n in groups], "q")
        qd0 = sim.pack([I.initial_state(m, n, 9)[1] for m, n in groups], "qd")
        act = np.concatenate([I.window_actions(m, n, h, 9).reshape(h, -1) for m, n in groups], axis=1)
        f = sim.window_forward(q0, qd0, T(act).view(h, -1))
        rb = torch.ones(h, sim.n_envs, device="cuda")
        zq = torch.zeros(h + 1, sim.q_size, device="cuda")
        zqd = torch.zeros(h + 1, sim.qd_size, device="cuda")
        g = sim.window_adjoint(f[0], f[1], T(act).view(h, -1), rb, zq, zqd)
        torch.cuda.synchronize()
        assert sim.status() == 0
        outs.append([x.cpu().numpy() for x in list(f) + list(g)])
    for a, b in zip(*outs):
        np.testing.assert_array_equal(a, b)


@pytest.mark.parametrize("form", ["plain", "batched"])
def test_largest_model_step_and_adjoint(oracle_mod, form):
    """32 DOF, the compiled maximum: the batched form runs its widest
    register dense path (32 rows, one environment per warp)."""
    m = long_chain(26)
    assert m.nv == 32
    N = 3
    sim = make_sim([(m, N)], form)
    o = oracle_mod.Oracle(m)
    q, qd = I.initial_state(m, N, 2)
    a = I.window_actions(m, N, 1, 2)[0]
    qn, qdn, r = sim.step(T(q), T(qd), T(a))
    torch.cuda.synchronize()
    (rq, rqd, rr), (fq, fqd, fr) = oracle_step_with_floor(o, q.T, qd.T, a.T)
    assert_state_close(qn.cpu().numpy().reshape(m.nq, N).T, rq, f"chain32/{form} q", fq)
    assert_state_close(qdn.cpu().numpy().reshape(m.nv, N).T, rqd, f"chain32/{form} qd", fqd)
    rng = np.random.default_rng(3)
    qb = rng.normal(size=(m.nq, N)).astype(np.float32)
    qdb = rng.normal(size=(m.nv, N)).astype(np.float32)
    rb = rng.normal(size=N).astype(np.float32)
    gq, gqd, ga = sim.step_adjoint(T(q), T(qd), T(a), T(qb), T(qdb), T(rb))
    torch.cuda.synchronize()
    sq, sqd, sa = o.step_vjp(q.T, qd.T, a.T, qb.T, qdb.T, rb)
    got = np.concatenate([gq.cpu().numpy().reshape(m.nq, N), gqd.cpu().numpy().reshape(m.nv, N),
                          ga.cpu().numpy().reshape(m.na, N)])
    assert_grad_close(got, np.concatenate([sq.T, sqd.T, sa.T]), f"chain32/{form} step adjoint")
    assert sim.status() == 0


@pytest.mark.parametrize("form", ["plain", "batched"])
def test_two_env_ranges_equal_one_run(form):
    """Environment sharding by offsets (the multi-GPU split is replicas over
    env ranges): a window over environments [0, 11) and another over [11, 23),
    fed the matching slices of the inputs, give bit for bit the full 23-env
    window's states, rewards and cotangents."""
    m, N, h, cut = I.ant(), 23, 4, 11
    q0, qd0 = I.initial_state(m, N, 12)
    act = I.window_actions(m, N, h, 12)                 # [h, na, N]
    rng = np.random.default_rng(4)
    rb = rng.normal(size=(h, N)).astype(np.float32)

    def window(sl):
        n = sl.stop - sl.start
        sim = make_sim([(m, n)], form, h)
        a = T(act[:, :, sl]).view(h, -1)
        f = sim.window_forward(T(q0[:, sl]), T(qd0[:, sl]), a)
        zq = torch.zeros(h + 1, sim.q_size, device="cuda")
        zqd = torch.zeros(h + 1, sim.qd_size, device="cuda")
        g = sim.window_adjoint(f[0], f[1], a, T(rb[:, sl]).view(h, n), zq, zqd)
        torch.cuda.synchronize()
        assert sim.status() == 0
        qt = f[0].cpu().numpy().reshape(h + 1, m.nq, n)
        qdt = f[1].cpu().numpy().reshape(h + 1, m.nv, n)
        ab = g[2].cpu().numpy().reshape(h, m.na, n)
        return [qt, qdt, f[2].cpu().numpy(), g[0].cpu().numpy().reshape(m.nq, n),
                g[1].cpu().numpy().reshape(m.nv, n), ab]

    full = window(slice(0, N))
    parts = [window(slice(0, cut)), window(slice(cut, N))]
    for k, x in enumerate(full):
        np.testing.assert_array_equal(x, np.concatenate([parts[0][k], parts[1][k]], axis=-1), err_msg=str(k))
