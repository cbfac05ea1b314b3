"""Pins of the oracle's FP32 floor (Monte Carlo Arithmetic: every operation
result perturbed by a random relative amount of at most u).  The floor is
trusted only if (1) with u = 0 it is the exact oracle bit for bit, (2) it is a
first-order effect, growing in proportion to u, (3) on a Cholesky solve, the
textbook case, it grows with the matrix's condition number and stays inside
the classical error bound of that solve."""
import numpy as np
import pytest

from helpers import model_by_name, seeded_case

U32 = 2.0 ** -24


@pytest.mark.parametrize("name", ["cartpole", "ant", "humanoid", "hopper"])
def test_zero_perturbation_is_the_exact_oracle(oracle_mod, name):
    m = model_by_name(name)
    o = oracle_mod.Oracle(m)
    q, qd, a = seeded_case(m, 3, 1, "initial")
    ex = o.step(q.T, qd.T, a.T)
    for x, y in zip(o.mca_step(q.T, qd.T, a.T, seed=4, u=0.0), ex):
        np.testing.assert_array_equal(x, y)
    h = 2
    from paper_2204_07137_gb300 import inputs as I
    q0, qd0 = I.initial_state(m, 2, 0)
    act = I.window_actions(m, 2, h, 0).transpose(0, 2, 1)
    qt, qdt, _ = o.window_forward(q0.T, qd0.T, act)
    rb = np.ones((h, 2))
    z = (np.zeros((2, m.nq)), np.zeros((2, m.nv)))
    ref = o.window_adjoint(qt, qdt, act, rb, *z)
    for tangents in (False, True):
        got = o.mca_window_adjoint(qt, qdt, act, rb, *z, seed=4, u=0.0, tangents=tangents)
        for x, y in zip(got, ref):
            np.testing.assert_array_equal(x, y)


def test_floor_is_first_order_in_u(oracle_mod):
    """Deviation at u and at u / 64: ratio 64 within a factor 2 (rounding
    errors propagate linearly), on the ant-like model in contact."""
    m = model_by_name("ant")
    o = oracle_mod.Oracle(m)
    q, qd, a = seeded_case(m, 8, 2, "initial")
    ex = o.step(q.T, qd.T, a.T)

    def dev(u):
        d = []
        for k in range(4):
            y = o.mca_step(q.T, qd.T, a.T, seed=k, u=u)
            d.append(np.linalg.norm(y[1] - ex[1]))
        return np.mean(d)

    r = dev(U32) / dev(U32 / 64)
    assert 32 < r < 128, r


def _spd(n, cond, rng):
    Q, _ = np.linalg.qr(rng.normal(size=(n, n)))
    ev = np.geomspace(1.0, cond, n)
    return (Q * ev) @ Q.T


@pytest.mark.parametrize("n", [6, 14, 28])
def test_cholesky_floor_tracks_the_condition_number(oracle_mod, n):
    """x = A^-1 b in Monte Carlo Arithmetic at u = 2^-24: the relative error
    stays below the classical forward bound (3n + 1) u kappa(A) of a
    Cholesky solve (backward error |dA| <= gamma_{3n+1} |L||L^T|), is not
    vanishingly small against kappa u, and grows with kappa."""
    rng = np.random.default_rng(n)
    errs = {}
    for cond in (1e1, 1e5):
        A = _spd(n, cond, rng)
        b = rng.normal(size=n)
        x = np.linalg.solve(A, b)
        e = max(np.linalg.norm(oracle_mod.mca_chol_solve(A, b, seed=s) - x) / np.linalg.norm(x) for s in range(6))
        kappa = np.linalg.cond(A)
        assert e <= (3 * n + 1) * U32 * kappa, (cond, e)
        assert e >= 1e-3 * U32 * kappa, (cond, e)
        errs[cond] = e
    assert errs[1e5] > 100 * errs[1e1]
