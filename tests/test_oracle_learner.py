"""Pins of the oracle's TD-lambda targets (Sec. 3.2, Eq. td-lambda) against
facts that hold independently of the formula as written: its lambda = 0 and
lambda = 1 limits (one-step TD target and the discounted return to the window
end), the backward recursion target_t = r_t + gamma((1 - lambda) V_{t+1} +
lambda target_{t+1}) that the geometric weights imply, and the fact that
nothing after an episode's end reaches the targets before it."""
import numpy as np
import pytest


@pytest.fixture(scope="module")
def orc():
    from oracle import oracle
    return oracle


def _data(h=9, N=5, p_done=0.2, seed=0):
    rng = np.random.default_rng(seed)
    r = rng.normal(size=(h, N))
    v = rng.normal(scale=5.0, size=(h + 1, N))
    d = rng.random((h, N)) < p_done
    return r, v, d


def test_lambda_zero_is_the_one_step_target(orc):
    r, v, d = _data()
    g = 0.97
    out = orc.td_lambda(r, v, d, g, 0.0)
    ref = r + np.where(d, 0.0, g * v[1:])
    np.testing.assert_allclose(out, ref, rtol=1e-13, atol=1e-13)


def test_lambda_one_is_the_discounted_return_to_the_window_end(orc):
    r, v, _ = _data()
    h, N = r.shape
    g = 0.9
    out = orc.td_lambda(r, v, None, g, 1.0)
    for t in range(h):
        ref = sum(g ** l * r[t + l] for l in range(h - t)) + g ** (h - t) * v[h]
        np.testing.assert_allclose(out[t], ref, rtol=1e-12)


@pytest.mark.parametrize("p_done", [0.0, 0.3])
def test_backward_recursion_holds(orc, p_done):
    r, v, d = _data(h=12, N=6, p_done=p_done, seed=3)
    h = r.shape[0]
    g, lam = 0.99, 0.95
    out = orc.td_lambda(r, v, d, g, lam)
    nxt = v[h]                                   # target_h := V(s_h) closes the recursion
    for t in range(h - 1, -1, -1):
        ref = r[t] + np.where(d[t], 0.0, g * ((1 - lam) * v[t + 1] + lam * nxt))
        np.testing.assert_allclose(out[t], ref, rtol=1e-12, atol=1e-12)
        nxt = out[t]


def test_nothing_after_an_episode_end_reaches_earlier_targets(orc):
    r, v, d = _data(h=10, N=1, p_done=0.0, seed=4)
    d[4, 0] = True
    base = orc.td_lambda(r, v, d, 0.99, 0.95)
    r2, v2 = r.copy(), v.copy()
    r2[5:] += 3.0
    v2[5:] -= 7.0
    other = orc.td_lambda(r2, v2, d, 0.99, 0.95)
    np.testing.assert_array_equal(base[:5], other[:5])
    assert np.abs(base[5:] - other[5:]).min() > 0
