"""Pins of the oracle's episodic window (Sec. 3.2: reset on early termination,
gradient cut at the reset; appendix A.3: termination below a task height or
at the task horizon) against facts that do not come from the oracle itself:
the integer schedule of horizon resets, exact reset states, exact zeros of
the gradient across a reset, and central finite differences of the episodic
window loss."""
import numpy as np

from paper_2204_07137_gb300 import inputs as I


def _env_major(q, qd):
    return q.T.astype(np.float64), qd.T.astype(np.float64)


def test_horizon_reset_schedule_is_exact(oracle_mod):
    """No height rule (cart-pole): with horizon H and e0 steps already taken,
    environment i ends its episode exactly at the steps t with
    (e0_i + t + 1) % H == 0, restarts from its reset state bit for bit, and
    leaves the window with e = (e0 + h) % H."""
    m = I.cartpole()
    o = oracle_mod.Oracle(m)
    N, h, H = 4, 9, 3
    q0, qd0 = _env_major(*I.initial_state(m, N, seed=1))
    qr, qdr = _env_major(*I.random_state(m, N, seed=2))
    act = I.window_actions(m, N, h, seed=3).transpose(0, 2, 1)
    e0 = np.array([0, 1, 2, 0])
    qt, qdt, rw, done, e, q_pre, qd_pre = o.window_forward_episodic(q0, qd0, act, qr, qdr, -np.inf, H, e0)
    t = np.arange(h)[:, None]
    np.testing.assert_array_equal(done, ((e0[None, :] + t + 1) % H == 0).astype(np.uint8))
    np.testing.assert_array_equal(e, (e0 + h) % H)
    for tt in range(h):
        for i in range(N):
            if done[tt, i]:
                np.testing.assert_array_equal(qt[tt + 1, i], qr[i])
                np.testing.assert_array_equal(qdt[tt + 1, i], qdr[i])
            else:
                np.testing.assert_array_equal(qt[tt + 1, i], q_pre[tt, i])


def test_height_rule_on_a_free_root(oracle_mod):
    """Ant-like model: a torso started well below the task height ends its
    episode after the first step and restarts from the reset state; one
    started well above it, in the air, does not."""
    m = I.ant()
    o = oracle_mod.Oracle(m)
    thr, _ = I.episode_rule(m)
    q0, qd0 = _env_major(*I.initial_state(m, 2, seed=0))
    q0[0, 2] = 0.05
    q0[1, 2] = 1.5
    qr, qdr = _env_major(*I.initial_state(m, 2, seed=4))
    act = I.window_actions(m, 2, 1, seed=5).transpose(0, 2, 1)
    qt, qdt, rw, done, e, q_pre, _ = o.window_forward_episodic(q0, qd0, act, qr, qdr, thr, 0, np.zeros(2))
    assert q_pre[0, 0, 2] < thr - 0.1 and q_pre[0, 1, 2] > thr + 0.5
    np.testing.assert_array_equal(done[0], [1, 0])
    np.testing.assert_array_equal(qt[1, 0], qr[0])
    np.testing.assert_array_equal(e, [0, 1])


def test_no_gradient_crosses_a_reset(oracle_mod):
    """With a reset after step 2, rewards after the reset do not depend on
    the start state or on actions up to step 2: their cotangents there are
    exactly zero."""
    m = I.cartpole()
    o = oracle_mod.Oracle(m)
    N, h = 2, 6
    q0, qd0 = _env_major(*I.initial_state(m, N, seed=6))
    qr, qdr = _env_major(*I.random_state(m, N, seed=7))
    act = I.window_actions(m, N, h, seed=8).transpose(0, 2, 1)
    qt, qdt, rw, done, e, _, _ = o.window_forward_episodic(q0, qd0, act, qr, qdr, -np.inf, 3, np.zeros(N))
    assert done[2].all() and not done[:2].any()
    rb = np.zeros((h, N))
    rb[3:] = np.random.default_rng(0).normal(size=(h - 3, N))
    zq, zqd = np.zeros((h + 1, N, m.nq)), np.zeros((h + 1, N, m.nv))
    qb, qdb, ab = o.window_adjoint_episodic(qt, qdt, act, done, rb, zq, zqd)
    assert np.all(qb == 0.0) and np.all(qdb == 0.0) and np.all(ab[:3] == 0.0)
    assert np.abs(ab[3:]).max() > 0.0


def test_episodic_adjoint_matches_finite_differences(oracle_mod):
    """L = sum_t w_t r_t + <c, q_traj[h]> over an episodic cart-pole window
    with a horizon reset after step 1 (a decision that does not depend on the
    state, so finite differences do not cross it): the episodic adjoint equals
    central differences of L in the start state and every action."""
    m = I.cartpole()
    o = oracle_mod.Oracle(m)
    N, h = 1, 4
    q0, qd0 = _env_major(*I.initial_state(m, N, seed=9))
    qr, qdr = _env_major(*I.random_state(m, N, seed=10))
    act = I.window_actions(m, N, h, seed=11).transpose(0, 2, 1).astype(np.float64)
    rng = np.random.default_rng(2)
    w = rng.normal(size=(h, N))
    cq, cqd = rng.normal(size=(N, m.nq)), rng.normal(size=(N, m.nv))

    def run(q0_, qd0_, act_):
        return o.window_forward_episodic(q0_, qd0_, act_, qr, qdr, -np.inf, 2, np.zeros(N))

    def loss(q0_, qd0_, act_):
        qt, qdt, rw = run(q0_, qd0_, act_)[:3]
        return float((w * rw).sum() + (cq * qt[-1]).sum() + (cqd * qdt[-1]).sum())

    qt, qdt, rw, done, _, _, _ = run(q0, qd0, act)
    assert done[1].all() and done[3].all() and not done[0].any() and not done[2].any()
    qtb, qdtb = np.zeros((h + 1, N, m.nq)), np.zeros((h + 1, N, m.nv))
    qtb[h], qdtb[h] = cq, cqd
    qb, qdb, ab = o.window_adjoint_episodic(qt, qdt, act, done, w, qtb, qdtb)
    eps = 1e-6
    for arr, grad in ((q0, qb), (qd0, qdb), (act, ab)):
        flat = arr.reshape(-1)
        g = grad.reshape(-1)
        for i in range(flat.size):
            old = flat[i]
            flat[i] = old + eps
            lp = loss(q0, qd0, act)
            flat[i] = old - eps
            lm = loss(q0, qd0, act)
            flat[i] = old
            np.testing.assert_allclose(g[i], (lp - lm) / (2 * eps), rtol=1e-6, atol=1e-7)


def test_discount_restarts_after_a_reset():
    """Eq. policy_loss weights gamma^(t - t0), t0 = the first step of the
    current episode inside the window (Sec. 3.2: the discount restarts at a
    reset), written out by hand for one pattern of resets."""
    torch = __import__("pytest").importorskip("torch")
    from paper_2204_07137_gb300.sim import episode_discounts
    g = 0.9
    done = torch.tensor([[0, 1], [1, 0], [0, 0], [0, 1], [0, 0]], dtype=torch.uint8)
    w = episode_discounts(done, g).numpy()
    ref = np.array([[1, 1], [g, 1], [1, g], [g, g * g], [g * g, 1]], np.float32)
    np.testing.assert_allclose(w, ref, rtol=1e-7)
