"""Pins of the FP64 oracle against facts fixed by mechanics and the paper,
not by the oracle itself (closed forms, exact discrete solutions, invariants,
library routines, brute-force finite differences).

Each test names the part of the simulator (paper Sec. 3.1) it pins.
"""
import math

import numpy as np
import pytest

from paper_2204_07137_gb300 import inputs as I


def _orc(oracle_mod, model):
    return oracle_mod.Oracle(model)


def single_body(shape="sphere", radius=0.1, mass=None, contact=False, ke=0.0, kd=0.0, kt=0.0, mu=0.0,
                gravity=(0, 0, -9.81), dt=1.0 / 60.0, substeps=1, inertia=None):
    b = I._Builder("body")
    m, c, Ib = I.sphere_mass_inertia(radius, 1000.0)
    if mass is not None:
        Ib = Ib * (mass / m)
        m = mass
    if inertia is not None:
        Ib = np.asarray(inertia)
    link = b.link(-1, I.FREE, mass=m, com=c, inertia=Ib)
    if contact:
        b.contact(link, (0, 0, 0), radius)
    return b.finish(act_dof=[], act_gear=[], dt=dt, substeps=substeps, ke=ke, kd=kd, kt=kt, mu=mu,
                    gravity=gravity)


def pendulum(d=0.7, mass=2.0, I_com=0.05, dt=1.0 / 60.0, substeps=16, axis=(0, 1, 0), com=None,
             limit=None, k_limit=0.0):
    b = I._Builder("pendulum")
    b.link(-1, I.REVOLUTE, axis=axis, mass=mass, com=com if com is not None else (0, 0, -d),
           inertia=np.diag([I_com, I_com, I_com]), limit=limit)
    return b.finish(act_dof=[0], act_gear=[1.0], dt=dt, substeps=substeps, k_limit=k_limit)


# --------------------------------------------------------------- closed forms

@pytest.mark.parametrize("th,thd,xd", [(0.3, -0.7, 0.5), (-1.2, 2.0, -1.0), (2.5, 0.1, 0.0)])
def test_cartpole_mass_matrix_and_bias_closed_form(oracle_mod, th, thd, xd):
    """Cart-pole with a uniform rod pole (theta from upright, l = L/2):
    M = [[mc+mp, mp l cos], [mp l cos, mp L^2/3]],
    c = [-mp l sin thd^2, -mp g l sin] (Lagrange's equations)."""
    m = I.cartpole()
    o = _orc(oracle_mod, m)
    mc, mp, L = float(m.mass[0]), float(m.mass[1]), 1.0
    l = L / 2
    q = np.array([0.3, th])
    qd = np.array([xd, thd])
    M = o.mass_matrix(q)
    Mref = np.array([[mc + mp, mp * l * math.cos(th)], [mp * l * math.cos(th), mp * L * L / 3]])
    # the rod inertia about its COM is stored in float32
    np.testing.assert_allclose(M, Mref, rtol=1e-7, atol=1e-9)
    c = o.inverse_dynamics(q, qd, np.zeros(2))
    cref = np.array([-mp * l * math.sin(th) * thd ** 2, -mp * 9.81 * l * math.sin(th)])
    np.testing.assert_allclose(c, cref, rtol=1e-6, atol=1e-9)


@pytest.mark.parametrize("name", ["ant", "humanoid", "mtu", "halfcheetah", "hopper"])
def test_kinetic_energy_equals_half_qd_M_qd(oracle_mod, name):
    """0.5 qd^T M qd equals sum_i (0.5 m_i |v_ci|^2 + 0.5 w_i^T I_i w_i),
    the latter from link velocities (independent of the mass matrix)."""
    m = getattr(I, name)()
    o = _orc(oracle_mod, m)
    q, qd = I.random_state(m, 3, seed=1)
    for e in range(3):
        M = o.mass_matrix(q[:, e])
        em = o.energy_momentum(q[:, e], qd[:, e])
        T = 0.5 * qd[:, e].astype(np.float64) @ M @ qd[:, e].astype(np.float64)
        np.testing.assert_allclose(T, em["T"], rtol=1e-11)
        assert np.allclose(M, M.T, atol=1e-12)
        assert np.linalg.eigvalsh(M).min() > 0


@pytest.mark.parametrize("name", ["cartpole", "ant", "humanoid", "mtu", "halfcheetah", "hopper"])
def test_newton_euler_difference_is_mass_matrix(oracle_mod, name):
    """ID(q, qd, qdd) - ID(q, qd, 0) = M(q) qdd: ties the Newton-Euler
    recursion to the Jacobian-based mass matrix."""
    m = getattr(I, name)()
    o = _orc(oracle_mod, m)
    q, qd = I.random_state(m, 2, seed=2)
    rng = np.random.default_rng(0)
    for e in range(2):
        qdd = rng.normal(size=m.nv)
        a = rng.uniform(0, 1, size=max(1, m.na))
        lhs = o.inverse_dynamics(q[:, e], qd[:, e], qdd, a) - o.inverse_dynamics(q[:, e], qd[:, e], np.zeros(m.nv), a)
        rhs = o.mass_matrix(q[:, e]) @ qdd
        np.testing.assert_allclose(lhs, rhs, rtol=1e-10, atol=1e-10 * np.abs(rhs).max())


def test_cholesky_matches_numpy(oracle_mod):
    rng = np.random.default_rng(3)
    for n in (1, 2, 7, 14, 27, 28):
        A = rng.normal(size=(n, n))
        A = A @ A.T + n * np.eye(n)
        np.testing.assert_allclose(oracle_mod.cholesky(A), np.linalg.cholesky(A), rtol=1e-12, atol=1e-12)


def test_capsule_inertia_matches_quadrature():
    """Closed-form capsule inertia (inputs module) vs a midpoint quadrature of the solid."""
    r, length = 0.08, 0.3
    m, c, Ifull = I.capsule_mass_inertia(r, (0, 0, -length / 2), (0, 0, length / 2), 1000.0)
    n = 120
    xs = (np.arange(n) + 0.5) / n * 2 * r - r
    zs = (np.arange(2 * n) + 0.5) / (2 * n) * (length + 2 * r) - (length / 2 + r)
    X, Y, Z = np.meshgrid(xs, xs, zs, indexing="ij")
    dz = np.clip(np.abs(Z) - length / 2, 0, None)
    inside = X ** 2 + Y ** 2 + dz ** 2 <= r * r
    dv = (2 * r / n) ** 2 * (length + 2 * r) / (2 * n)
    mq = inside.sum() * dv * 1000.0
    Ixx = ((Y ** 2 + Z ** 2) * inside).sum() * dv * 1000.0
    Izz = ((X ** 2 + Y ** 2) * inside).sum() * dv * 1000.0
    np.testing.assert_allclose(mq, m, rtol=3e-3)
    np.testing.assert_allclose(Ixx, Ifull[0, 0], rtol=5e-3)
    np.testing.assert_allclose(Izz, Ifull[2, 2], rtol=5e-3)


# ------------------------------------------------------- exact discrete motion

def test_free_fall_exact_discrete_solution(oracle_mod):
    """Semi-implicit Euler under gravity: v_n = v0 - n g h,
    z_n = z0 + n v0 h - g h^2 n (n + 1) / 2 (velocity first, then position)."""
    K = 8
    m = single_body(substeps=K)
    o = _orc(oracle_mod, m)
    g, h = -float(m.gravity[2]), m.dt / K   # the float32-stored values the oracle sees
    q = np.array([[0.1, -0.2, 3.0, 0, 0, 0, 1.0]])
    v0 = 0.7
    qd = np.array([[0, 0, 0, 0.3, -0.1, v0]])
    qt, qdt, _ = o.window_forward(q, qd, np.zeros((5, 1, 0)))
    for t in range(6):
        n = t * K
        np.testing.assert_allclose(qdt[t, 0, 5], v0 - n * g * h, rtol=0, atol=1e-12)
        np.testing.assert_allclose(qt[t, 0, 2], 3.0 + n * v0 * h - g * h * h * n * (n + 1) / 2, atol=1e-12)
        np.testing.assert_allclose(qt[t, 0, 0], 0.1 + 0.3 * n * h, atol=1e-12)


def test_torque_free_spin_angle_per_substep(oracle_mod):
    """Spin about a principal axis of a symmetric body: the normalised
    first-order quaternion update turns by exactly 2 atan(|w| h / 2) per substep."""
    K = 4
    m = single_body(substeps=K, gravity=(0, 0, 0))
    o = _orc(oracle_mod, m)
    h = m.dt / K
    w = 5.0
    axis = np.array([1.0, 2.0, 2.0]) / 3.0
    q = np.array([[0, 0, 0, 0, 0, 0, 1.0]])
    qd = np.concatenate([w * axis, [0, 0, 0]])[None]
    qt, qdt, _ = o.window_forward(q, qd, np.zeros((3, 1, 0)))
    for t in range(4):
        quat = qt[t, 0, 3:7]
        angle = 2 * math.atan2(np.linalg.norm(quat[:3]), quat[3])
        np.testing.assert_allclose(angle, t * K * 2 * math.atan(w * h / 2), atol=1e-12)
        if t:
            np.testing.assert_allclose(quat[:3] / np.linalg.norm(quat[:3]), axis, atol=1e-12)
        np.testing.assert_allclose(qdt[t, 0, :3], w * axis, atol=1e-12)


def test_small_angle_pendulum_discrete_frequency(oracle_mod):
    """Physical pendulum, theta0 = 1e-3: semi-implicit Euler on the linearised
    equation theta'' = -w^2 theta, w^2 = m g d / I_pivot, is the linear map
    (theta, v) -> ((1 - h^2 w^2) theta + h v, v - h w^2 theta); the oracle must
    follow its powers to O(theta0^3)."""
    K = 16
    d, mass, Ic = 0.7, 2.0, 0.05
    m = pendulum(d=d, mass=mass, I_com=Ic, substeps=K)
    o = _orc(oracle_mod, m)
    h = m.dt / K
    Ipiv = Ic + mass * d * d
    w2 = mass * 9.81 * d / Ipiv
    A = np.array([[1 - h * h * w2, h], [-h * w2, 1.0]])
    th0 = 1e-3
    steps = 40
    qt, qdt, _ = o.window_forward(np.array([[th0]]), np.array([[0.0]]), np.zeros((steps, 1, 1)))
    x = np.array([th0, 0.0])
    for t in range(steps + 1):
        np.testing.assert_allclose(qt[t, 0, 0], x[0], atol=th0 * 2e-6)
        x = np.linalg.matrix_power(A, K) @ x
    # discrete frequency cos(phi) = 1 - (w h)^2 / 2 -> continuous period as h -> 0
    phi = math.acos(1 - w2 * h * h / 2)
    period = 2 * math.pi * h / phi
    assert abs(period - 2 * math.pi * math.sqrt(Ipiv / (mass * 9.81 * d))) < 1e-3


# ----------------------------------------------------- conservation / convergence

def _airborne_ant(substeps):
    m = I.ant(substeps=substeps)
    return m.replace(contact_link=m.contact_link[:0], contact_pos=m.contact_pos[:0],
                     contact_radius=m.contact_radius[:0])


def _energy_drift(oracle_mod, substeps, steps=30):
    m = _airborne_ant(substeps)
    o = _orc(oracle_mod, m)
    q, qd = I.random_state(m, 1, seed=5, vel_scale=2.0)
    q = q.astype(np.float64).T
    qd = qd.astype(np.float64).T
    qt, qdt, _ = o.window_forward(q, qd, np.zeros((steps, 1, m.na)))
    E = []
    for t in range(steps + 1):
        em = o.energy_momentum(qt[t, 0], qdt[t, 0])
        E.append(em["T"] + em["V"])
    E = np.array(E)
    return np.abs(E - E[0]).max() / abs(E[0])


def test_energy_drift_bounded_and_first_order(oracle_mod):
    """Gravity on, contact/limits/damping off, no actuation: the relative energy
    error stays small and halves when the step halves (first-order scheme)."""
    e1 = _energy_drift(oracle_mod, 16)
    e2 = _energy_drift(oracle_mod, 32)
    assert e1 < 2e-2
    assert 1.6 < e1 / e2 < 2.5


def _momentum_drift(oracle_mod, substeps, steps=20):
    m = _airborne_ant(substeps).replace(gravity=np.zeros(3, np.float32))
    o = _orc(oracle_mod, m)
    q, qd = I.random_state(m, 1, seed=6, vel_scale=1.0)
    q = q.astype(np.float64).T
    qd = qd.astype(np.float64).T
    act = I.window_actions(m, 1, steps, seed=6).astype(np.float64).transpose(0, 2, 1) * 0.2
    qt, qdt, _ = o.window_forward(q, qd, act)
    em0 = o.energy_momentum(qt[0, 0], qdt[0, 0])
    dP = dH = 0.0
    for t in range(steps + 1):
        em = o.energy_momentum(qt[t, 0], qdt[t, 0])
        dP = max(dP, np.abs(em["P"] - em0["P"]).max())
        dH = max(dH, np.abs(em["H"] - em0["H"]).max())
    return dP, dH


def test_momentum_conserved_to_first_order(oracle_mod):
    """Gravity and contact off, random internal joint torques: total linear and
    angular momentum are invariants of the continuous system; the discrete drift
    shrinks at first order in the step."""
    p1, h1 = _momentum_drift(oracle_mod, 16)
    p2, h2 = _momentum_drift(oracle_mod, 32)
    assert p1 < 5.0 and h1 < 5.0
    assert 1.6 < p1 / p2 < 2.5
    assert 1.6 < h1 / h2 < 2.5


# ----------------------------------------------------------- contact and limits

def test_resting_sphere_equilibrium_penetration(oracle_mod):
    """Sphere resting on the plane: the normal penalty balances gravity at
    d* = -m g / k_n; a sphere placed there at rest stays there."""
    mass, r, ke = 3.0, 0.1, 4e4
    m = single_body(mass=mass, radius=r, contact=True, ke=ke, kd=1e3, kt=1e3, mu=0.75)
    o = _orc(oracle_mod, m)
    mass, r, ke, g = float(m.mass[0]), float(m.contact_radius[0]), m.ke, -float(m.gravity[2])
    dstar = -mass * g / ke
    q = np.array([0, 0, r + dstar, 0, 0, 0, 1.0])
    qdd = o.forward_accel(q, np.zeros(6), np.zeros(0))
    np.testing.assert_allclose(qdd, 0, atol=1e-12)
    # above / below the equilibrium the net force points back to it
    assert o.forward_accel(q + np.array([0, 0, 1e-4, 0, 0, 0, 0]), np.zeros(6), np.zeros(0))[5] < 0
    assert o.forward_accel(q - np.array([0, 0, 1e-4, 0, 0, 0, 0]), np.zeros(6), np.zeros(0))[5] > 0
    # damping opposes penetration velocity
    down = o.forward_accel(q, np.array([0, 0, 0, 0, 0, -0.5]), np.zeros(0))[5]
    up = o.forward_accel(q, np.array([0, 0, 0, 0, 0, 0.5]), np.zeros(0))[5]
    assert down > 0 > up


def test_sliding_friction_deceleration_mu_g(oracle_mod):
    """Sphere sliding without spin at the equilibrium depth, saturated friction:
    the COM decelerates at exactly mu g opposite to the slip."""
    mass, r, ke, mu = 3.0, 0.1, 4e4, 0.75
    m = single_body(mass=mass, radius=r, contact=True, ke=ke, kd=1e3, kt=1e3, mu=mu)
    o = _orc(oracle_mod, m)
    mass, r, ke, g, mu = float(m.mass[0]), float(m.contact_radius[0]), m.ke, -float(m.gravity[2]), m.mu
    dstar = -mass * g / ke
    q = np.array([0, 0, r + dstar, 0, 0, 0, 1.0])
    v = np.array([3.0, -4.0]) / 5.0 * 2.0
    qdd = o.forward_accel(q, np.array([0, 0, 0, v[0], v[1], 0]), np.zeros(0))
    np.testing.assert_allclose(qdd[3:5], -mu * g * v / np.linalg.norm(v), rtol=1e-10)
    np.testing.assert_allclose(qdd[5], 0.0, atol=1e-10)
    # slow slip: viscous branch -k_t v_t / m
    vs = np.array([1e-3, 0.0])
    qdd = o.forward_accel(q, np.array([0, 0, 0, vs[0], vs[1], 0]), np.zeros(0))
    np.testing.assert_allclose(qdd[3], -m.kt * vs[0] / mass, rtol=1e-10)


def test_joint_limit_static_hang(oracle_mod):
    """Horizontal arm against an upper limit at 0: equilibrium where the limit
    penalty cancels the gravity torque, k (0 - q*) + m g d cos q* = 0."""
    d, mass, k = 0.5, 2.0, 1e4
    m = pendulum(d=d, mass=mass, com=(d, 0, 0), limit=(-1.0, 0.0), k_limit=k)
    o = _orc(oracle_mod, m)
    d, mass, k = float(m.com[0, 0]), float(m.mass[0]), m.k_limit
    qs = 0.0
    for _ in range(50):
        qs = mass * -float(m.gravity[2]) * d * math.cos(qs) / k
    qdd = o.forward_accel(np.array([qs]), np.zeros(1), np.zeros(1))
    np.testing.assert_allclose(qdd, 0, atol=1e-10)
    # inside the limits there is no penalty; below the lower limit it pushes up
    assert o.joint_forces(np.array([-0.5]), np.zeros(1), np.zeros(1))[0] == 0.0
    np.testing.assert_allclose(o.joint_forces(np.array([-1.1]), np.zeros(1), np.zeros(1))[0], k * 0.1, rtol=1e-6)


def test_muscle_generalised_force_is_minus_F_dlength_dq(oracle_mod):
    """A contractile force F along the via-point path does virtual work
    -F dl, so its generalised force is tau = -F dl/dq (FD of the path length)."""
    b = I._Builder("arm")
    l0 = b.link(-1, I.REVOLUTE, axis=(0, 1, 0), mass=1.0, com=(0, 0, -0.2), inertia=np.eye(3) * 0.01)
    l1 = b.link(l0, I.REVOLUTE, axis=(1, 0, 0), pos=(0, 0, -0.4), mass=1.0, com=(0, 0, -0.2),
                inertia=np.eye(3) * 0.01)
    l2 = b.link(l1, I.REVOLUTE, axis=(0, 0.6, 0.8), pos=(0, 0, -0.4), mass=0.5, com=(0, 0, -0.1),
                inertia=np.eye(3) * 0.01)
    b.muscle(700.0, [(l0, (0.05, 0.02, -0.1)), (l1, (0.04, -0.03, -0.2)), (l2, (0.02, 0.05, -0.1))])
    b.muscle(300.0, [(l0, (-0.05, 0.0, -0.3)), (l2, (-0.03, 0.01, -0.15))])
    m = b.finish(act_dof=[], act_gear=[], dt=1 / 60, substeps=1, gravity=(0, 0, 0))
    o = _orc(oracle_mod, m)
    q = np.array([0.3, -0.4, 0.7])
    qd = np.zeros(3)
    act = np.array([0.6, 0.9])
    # generalised muscle force = -(ID with the muscle forces) at qd = qdd = 0
    tau = -o.inverse_dynamics(q, qd, np.zeros(3), act)
    eps = 1e-6
    ref = np.zeros(3)
    for j in range(3):
        dq = np.zeros(3)
        dq[j] = eps
        dl = (o.muscle_lengths(q + dq) - o.muscle_lengths(q - dq)) / (2 * eps)
        ref[j] = -(act * m.muscle_fmax.astype(np.float64)) @ dl
    np.testing.assert_allclose(tau, ref, rtol=1e-6, atol=1e-6)   # central-difference truncation


# --------------------------------------------------------- derivatives (brute force)

def _fd_jacobian(o, q, qd, a, eps):
    m = o.model
    x0 = np.concatenate([q, qd, a])
    nin = x0.size

    def f(x):
        qn, qdn, r = o.step(x[None, :m.nq], x[None, m.nq:m.nq + m.nv], x[None, m.nq + m.nv:])
        return np.concatenate([qn[0], qdn[0], r])

    J = np.zeros((m.nq + m.nv + 1, nin))
    for i in range(nin):
        dx = np.zeros(nin)
        dx[i] = eps
        J[:, i] = (f(x0 + dx) - f(x0 - dx)) / (2 * eps)
    return J


@pytest.mark.parametrize("case", ["cartpole", "ant_air", "ant_contact", "humanoid_air", "mtu_air",
                                  "halfcheetah_contact", "hopper_air"])
def test_step_jacobian_matches_central_differences(oracle_mod, case):
    """The exact (dual-number) step Jacobian of Eq. backward against central
    finite differences of the FP64 step, on inputs whose branch decisions
    (contact, friction regime, limits) are far from their thresholds."""
    if case == "cartpole":
        m = I.cartpole()
        q, qd = I.initial_state(m, 1, seed=3)
    elif case == "ant_contact":
        m = I.ant(substeps=4)
        q, qd = I.initial_state(m, 1, seed=3)
        q[2] -= 0.01      # every foot well inside the contact branch
        qd[3:5] = 1.0     # saturated friction at the feet
    elif case == "halfcheetah_contact":
        m = I.halfcheetah(substeps=4)
        q, qd = I.initial_state(m, 1, seed=3, joint_range=0.0)
        q[1] -= 0.01      # the four foot spheres well inside the contact branch, torso ends above
        qd[:] = 0.0
        qd[0] = 1.0       # saturated friction at the feet
    else:
        base = {"ant_air": I.ant, "humanoid_air": I.humanoid, "mtu_air": I.mtu, "hopper_air": I.hopper}[case]()
        m = base.replace(contact_link=base.contact_link[:0], contact_pos=base.contact_pos[:0],
                         contact_radius=base.contact_radius[:0], substeps=4,
                         q_lower=np.full_like(base.q_lower, -I.BIG), q_upper=np.full_like(base.q_upper, I.BIG))
        q, qd = I.random_state(m, 1, seed=4, vel_scale=0.5)
    o = _orc(oracle_mod, m)
    a = I.window_actions(m, 1, 1, seed=3)[0]
    if m.n_muscles:
        a = np.clip(a, 0.05, 0.95)
    q, qd, a = (x[:, 0].astype(np.float64) for x in (q, qd, a))
    J = o.step_jacobian(q[None], qd[None], a[None])[0]
    Jfd = _fd_jacobian(o, q, qd, a, 1e-6)
    scale = np.abs(J).max()
    np.testing.assert_allclose(J, Jfd, rtol=2e-5, atol=2e-6 * max(scale, 1.0))


def test_window_adjoint_matches_finite_differences(oracle_mod):
    """Window loss L = sum_t w_t r_t + <c_q, q_h> + <c_qd, qd_h> over 6 cartpole
    steps: the chained step adjoints (appendix A.1 recursion) give the same
    gradient as central differences of the whole window."""
    m = I.cartpole()
    o = _orc(oracle_mod, m)
    h = 6
    q0, qd0 = I.initial_state(m, 1, seed=8)
    act = I.window_actions(m, 1, h, seed=8)
    q0, qd0 = q0.T.astype(np.float64), qd0.T.astype(np.float64)
    act = act.transpose(0, 2, 1).astype(np.float64)
    rng = np.random.default_rng(1)
    w = rng.normal(size=(h, 1))
    cq, cqd = rng.normal(size=(1, m.nq)), rng.normal(size=(1, m.nv))

    def loss(q0_, qd0_, act_):
        qt, qdt, rw = o.window_forward(q0_, qd0_, act_)
        return float((w * rw).sum() + (cq * qt[-1]).sum() + (cqd * qdt[-1]).sum())

    qt, qdt, rw = o.window_forward(q0, qd0, act)
    qb, qdb, ab = o.window_adjoint(qt, qdt, act, w, cq, cqd)
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


def test_reward_shapes(oracle_mod):
    """Appendix A.3 reward shapes at a state where every term is known:
    ant at rest, upright, height h: r = 0.1 * 1 + 1 * 1 + (h - 0.27);
    cart-pole config loss -(theta^2 + 0.1 x^2)."""
    m = I.ant(substeps=1).replace(dt=1e-9, gravity=np.zeros(3, np.float32))
    m = m.replace(contact_link=m.contact_link[:0], contact_pos=m.contact_pos[:0], contact_radius=m.contact_radius[:0])
    o = _orc(oracle_mod, m)
    q = np.zeros((1, 15)); q[0, 2] = 0.6; q[0, 6] = 1.0
    qd = np.zeros((1, 14)); qd[0, 3] = 1.5
    _, _, r = o.step(q, qd, np.zeros((1, 8)))
    np.testing.assert_allclose(r[0], 1.5 + 0.1 + 1.0 + (0.6 - 0.27), atol=1e-6)
    c = I.cartpole()
    oc = _orc(oracle_mod, c.replace(dt=1e-12, gravity=np.zeros(3, np.float32)))
    _, _, r = oc.step(np.array([[0.2, -0.3]]), np.zeros((1, 2)), np.zeros((1, 1)))
    np.testing.assert_allclose(r[0], -(0.09 + 0.1 * 0.04), atol=1e-9)


def test_planar_reward_shapes(oracle_mod):
    """Appendix A.3 HalfCheetah v_x - 0.1 |a|^2 and Hopper v_x + R_height +
    R_angle - 0.1 |a|^2 at states where every term is known (no gravity,
    vanishing step): hopper height change -0.4 gives D = clip(-0.1) and
    R_height = -200 D^2 = -2; pitch 0.2 gives R_angle = -(0.2 / (pi / 6))^2;
    at height change +0.5, D clips to 0.3."""
    def still(m):
        m = m.replace(dt=1e-12, gravity=np.zeros(3, np.float32))
        return _orc(oracle_mod, m.replace(contact_link=m.contact_link[:0], contact_pos=m.contact_pos[:0],
                                          contact_radius=m.contact_radius[:0]))
    oc = still(I.halfcheetah(substeps=1))
    qd = np.zeros((1, 9)); qd[0, 0] = 1.5
    _, _, r = oc.step(np.zeros((1, 9)), qd, np.full((1, 6), 0.5))
    np.testing.assert_allclose(r[0], 1.5 - 0.1 * 6 * 0.25, atol=1e-6)
    oh = still(I.hopper(substeps=1))
    q = np.zeros((2, 6)); q[0, 1] = -0.4; q[0, 2] = 0.2; q[1, 1] = 0.5
    qd = np.zeros((2, 6)); qd[:, 0] = 1.5
    _, _, r = oh.step(q, qd, np.full((2, 3), 0.5))
    np.testing.assert_allclose(r, [1.5 - 2.0 - (0.2 / (math.pi / 6)) ** 2 - 0.075, 1.5 + 0.3 - 0.075], atol=1e-6)


def test_oracle_forest_steps_as_its_separate_trees(oracle_mod):
    """A model of two trees hanging from the world (parent -1 past link 0):
    its step equals the step of each tree as a model of its own, the reward
    their sum (the trees share nothing but the ground)."""
    from helpers import forest, forest_trees, seeded_case
    m = forest()
    ma, mb = forest_trees()
    for seed, kind in ((0, "initial"), (1, "random")):
        q, qd, a = seeded_case(m, 5, seed, kind)
        rq, rqd, rr = oracle_mod.Oracle(m).step(q.T, qd.T, a.T)
        qa, qda, ra = oracle_mod.Oracle(ma).step(q[:2].T, qd[:2].T, a[:1].T)
        qb, qdb, rb = oracle_mod.Oracle(mb).step(q[2:].T, qd[2:].T, a[1:].T)
        np.testing.assert_allclose(rq, np.concatenate([qa, qb], 1), rtol=1e-12, atol=1e-12)
        np.testing.assert_allclose(rqd, np.concatenate([qda, qdb], 1), rtol=1e-12, atol=1e-12)
        np.testing.assert_allclose(rr, ra + rb, rtol=1e-12, atol=1e-12)
