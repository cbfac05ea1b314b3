"""Episodic window on the GPU (Sec. 3.2 reset on early termination with the
gradient cut at the reset; appendix A.3 termination rules) against the FP64
oracle, step by step from the GPU's own checkpoints, and its adjoint against
the oracle's episodic window adjoint.  The termination decision is a float
comparison deciding an integer: where the oracle's root height lies within
1e-3 of the task height both decisions are accepted, and the GPU's is used
for the expected state."""
import numpy as np
import pytest

from helpers import airborne, assert_grad_close, assert_state_close, oracle_step_with_floor
from paper_2204_07137_gb300 import inputs as I

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

MARGIN = 1e-3


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2204_07137_gb300 import build
    build.build()


def T(x):
    return torch.from_numpy(np.ascontiguousarray(np.asarray(x, np.float32).reshape(-1))).cuda()


def _height_index(m):
    """q index of the root height: q[2] for a free root, else height_q."""
    return 2 if int(m.joint_type[0]) == 0 else int(m.height_q)


def _case(name, N, h, seed):
    """Seeded reset states, random episode counters and a short horizon so
    both rules fire.  Models with a height rule fly without their contacts,
    started from root heights spread just around the task height, so that the
    root falls through it during the window on smooth dynamics."""
    m = getattr(I, name)()
    thr, _ = I.episode_rule(m)
    if thr > -np.inf:
        m = airborne(m)
    q0, qd0 = I.initial_state(m, N, seed)
    q0 = q0.copy()
    if thr > -np.inf:
        q0[_height_index(m)] = np.linspace(thr - 0.02, thr + 0.1, N).astype(np.float32)
    qr, qdr = I.initial_state(m, N, seed + 1)
    act = I.window_actions(m, N, h, seed + 2)
    H = 5
    ep0 = np.random.default_rng(seed).integers(0, H, N).astype(np.int32)
    return m, thr, q0, qd0, qr, qdr, act, H, ep0


def _run(m, N, h, thr, q0, qd0, qr, qdr, act, H, ep0):
    from paper_2204_07137_gb300.sim import Simulator
    sim = Simulator([(m, N)], form="batched", h_max=h)
    ep = torch.from_numpy(ep0.copy()).cuda()
    out = sim.window_forward_episodic(T(q0), T(qd0), T(act).view(h, -1), T(qr), T(qdr), [thr], [H], ep)
    torch.cuda.synchronize()
    return sim, ep, out


@pytest.mark.parametrize("name,N", [("ant", 37), ("humanoid", 9), ("cartpole", 21), ("hopper", 13)])
def test_episodic_window_matches_oracle_step_by_step(oracle_mod, name, N):
    h = 8
    m, thr, q0, qd0, qr, qdr, act, H, ep0 = _case(name, N, h, seed=3)
    sim, ep, (qt, qdt, rw, done) = _run(m, N, h, thr, q0, qd0, qr, qdr, act, H, ep0)
    gq = qt.cpu().numpy().reshape(h + 1, m.nq, N).transpose(0, 2, 1)
    gqd = qdt.cpu().numpy().reshape(h + 1, m.nv, N).transpose(0, 2, 1)
    grw = rw.cpu().numpy()
    gd = done.cpu().numpy().astype(bool)
    assert np.array_equal(gq[0], q0.T) and np.array_equal(gqd[0], qd0.T)
    o = oracle_mod.Oracle(m)
    a = act.transpose(0, 2, 1)
    e = ep0.astype(np.int64)
    hq = _height_index(m) if thr > -np.inf else -1
    fired = 0
    for t in range(h):
        (pq, pqd, pr), (fq, fqd, fr) = oracle_step_with_floor(o, gq[t], gqd[t], a[t])
        assert_state_close(grw[t], pr, f"episodic {name} reward step {t}", fr)
        e = e + 1
        by_len = e >= H
        by_height = (pq[:, hq] < thr) if hq >= 0 else np.zeros(N, bool)
        clear = by_len | (np.abs(pq[:, hq] - thr) > MARGIN) if hq >= 0 else np.ones(N, bool)
        np.testing.assert_array_equal(gd[t][clear], (by_len | by_height)[clear], err_msg=f"{name} done step {t}")
        fired += int(gd[t].sum())
        d = gd[t]
        np.testing.assert_array_equal(gq[t + 1][d], qr.T[d])      # reset states copied bit for bit
        np.testing.assert_array_equal(gqd[t + 1][d], qdr.T[d])
        if (~d).any():
            assert_state_close(gq[t + 1][~d], pq[~d], f"episodic {name} q step {t}", fq[~d])
            assert_state_close(gqd[t + 1][~d], pqd[~d], f"episodic {name} qd step {t}", fqd[~d])
        e[d] = 0
    assert fired > 0
    np.testing.assert_array_equal(ep.cpu().numpy(), e)

    # adjoint: reward and checkpoint cotangents, against the oracle's episodic
    # adjoint on the GPU checkpoints and done mask
    rng = np.random.default_rng(5)
    rb = rng.normal(size=(h, N)).astype(np.float32)
    qtb = rng.normal(size=(h + 1, m.nq, N)).astype(np.float32) * 0.1
    qdtb = rng.normal(size=(h + 1, m.nv, N)).astype(np.float32) * 0.1
    g0, gd0, ga = sim.window_adjoint_episodic(qt, qdt, T(act).view(h, -1), done, T(rb).view(h, N),
                                              T(qtb).view(h + 1, -1), T(qdtb).view(h + 1, -1))
    torch.cuda.synchronize()
    qb, qdb, ab = o.window_adjoint_episodic(gq, gqd, a, gd.astype(np.uint8), rb, qtb.transpose(0, 2, 1),
                                            qdtb.transpose(0, 2, 1))
    got = np.concatenate([g0.cpu().numpy().reshape(m.nq, N), gd0.cpu().numpy().reshape(m.nv, N),
                          ga.cpu().numpy().reshape(h * m.na, N)])
    ref = np.concatenate([qb.T, qdb.T, ab.transpose(0, 2, 1).reshape(h * m.na, N)])
    assert_grad_close(got, ref, f"{name} episodic window gradient")


def test_without_resets_equals_the_plain_window():
    """No height rule, no horizon: the episodic window and its adjoint give
    the plain window's results bit for bit, no done flags, and e + h."""
    h, N = 6, 19
    m, thr, q0, qd0, qr, qdr, act, H, ep0 = _case("ant", N, h, seed=7)
    sim, ep, (qt, qdt, rw, done) = _run(m, N, h, -np.inf, q0, qd0, qr, qdr, act, 0, ep0)
    pt, pdt, prw = sim.window_forward(T(q0), T(qd0), T(act).view(h, -1))
    torch.cuda.synchronize()
    assert torch.equal(qt, pt) and torch.equal(qdt, pdt) and torch.equal(rw, prw)
    assert int(done.sum()) == 0
    np.testing.assert_array_equal(ep.cpu().numpy(), ep0 + h)
    rb = torch.randn(h, N, device="cuda")
    zq, zqd = torch.randn_like(qt), torch.randn_like(qdt)
    e1 = sim.window_adjoint_episodic(qt, qdt, T(act).view(h, -1), done, rb, zq, zqd)
    e2 = sim.window_adjoint(qt, qdt, T(act).view(h, -1), rb, zq, zqd)
    torch.cuda.synchronize()
    for x, y in zip(e1, e2):
        assert torch.equal(x, y)


def test_episodic_rejects_the_plain_form():
    from paper_2204_07137_gb300 import _lib
    from paper_2204_07137_gb300.sim import Simulator
    m = I.cartpole()
    N, h = 4, 2
    sim = Simulator([(m, N)], form="plain", h_max=h)
    q0, qd0 = I.initial_state(m, N, 0)
    ep = torch.zeros(N, dtype=torch.int32, device="cuda")
    with pytest.raises(_lib.ShacError, match="UNSUPPORTED"):
        sim.window_forward_episodic(T(q0), T(qd0), T(I.window_actions(m, N, h, 0)).view(h, -1), T(q0), T(qd0),
                                    [-np.inf], [3], ep)
