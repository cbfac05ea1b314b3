"""Shared test helpers: seeded cases, layout conversion, tolerance checks."""
import numpy as np

from paper_2204_07137_gb300 import inputs as I

# Per-step state tolerance (elementwise) and window-gradient tolerance
# (norm-wise per environment) for the FP32 GPU path against the FP64 oracle.
STATE_RTOL, STATE_ATOL = 1e-4, 1e-5
GRAD_RTOL = 1e-3


def assert_state_close(got, ref, what, rtol=STATE_RTOL, atol=STATE_ATOL):
    """State parity.  2-D arrays hold one environment state per row and are
    compared normwise per row: ||got - ref||_inf <= atol + rtol ||ref||_inf
    (the bound FP32 conditioning of the step allows: kappa(M) eps_32 is up to
    6e-5, so a near-zero component of a state cannot hold a 1e-4 bound of its
    own).  1-D arrays (rewards, one scalar per environment) are compared
    elementwise.  Non-finite values always fail."""
    got = np.asarray(got, np.float64)
    ref = np.asarray(ref, np.float64)
    assert np.isfinite(ref).all(), f"{what}: reference not finite"
    if ref.ndim == 1:
        err = np.abs(got - ref)
        bound = atol + rtol * np.abs(ref)
    else:
        got = got.reshape(-1, got.shape[-1])
        ref = ref.reshape(-1, ref.shape[-1])
        err = np.max(np.abs(got - ref), axis=1)
        bound = atol + rtol * np.max(np.abs(ref), axis=1)
    bad = ~(err <= bound)          # NaN counts as a mismatch
    if bad.any():
        idx = np.argwhere(bad)[:5].ravel()
        raise AssertionError(f"{what}: {bad.sum()} / {bad.size} states outside |d| <= {atol} + {rtol}|ref| "
                             f"(normwise per state); worst ratio {np.max(err / bound):.3g}; first rows "
                             f"{idx.tolist()}")


def elementwise_violation_fraction(got, ref, rtol=STATE_RTOL, atol=STATE_ATOL):
    """Fraction of components outside the elementwise form of the bound (diagnostic)."""
    got = np.asarray(got, np.float64)
    ref = np.asarray(ref, np.float64)
    return float(np.mean(~(np.abs(got - ref) <= atol + rtol * np.abs(ref))))


def assert_grad_close(got, ref, what, rtol=GRAD_RTOL, axis_env=-1):
    """Norm-wise per environment: |g - g*|_2 <= rtol |g*|_2 (env on the last axis)."""
    got = np.moveaxis(np.asarray(got, np.float64), axis_env, 0).reshape(np.shape(got)[axis_env], -1)
    ref = np.moveaxis(np.asarray(ref, np.float64), axis_env, 0).reshape(np.shape(ref)[axis_env], -1)
    assert np.isfinite(ref).all(), f"{what}: reference not finite"
    num = np.linalg.norm(got - ref, axis=1)
    den = np.linalg.norm(ref, axis=1)
    bad = ~(num <= rtol * np.maximum(den, 1e-30))   # NaN counts as a mismatch
    if bad.any():
        e = np.argwhere(bad)[:5].ravel()
        raise AssertionError(f"{what}: {bad.sum()} / {bad.size} envs outside rel {rtol}; envs {e.tolist()} "
                             f"rel err {(num / np.maximum(den, 1e-30))[e]}")


def airborne(m):
    """The model without contacts (contact-free configuration)."""
    return m.replace(contact_link=m.contact_link[:0], contact_pos=m.contact_pos[:0],
                     contact_radius=m.contact_radius[:0])


def model_by_name(name):
    return {"cartpole": I.cartpole, "ant": I.ant, "humanoid": I.humanoid, "mtu": I.mtu,
            "halfcheetah": I.halfcheetah, "hopper": I.hopper}[name]()


def seeded_case(model, n, seed, kind="initial"):
    """(q [nq,N], qd [nv,N], act [na,N]) float32."""
    if kind == "initial":
        q, qd = I.initial_state(model, n, seed)
    else:
        q, qd = I.random_state(model, n, seed, pos_scale=0.3, vel_scale=0.5)
        if model.root_z != 1.0 or model.name in ("ant", "humanoid", "mtu"):
            q[2] = model.root_z + np.float32(0.3)   # above the ground
    act = I.window_actions(model, n, 1, seed)[0]
    return q, qd, act


def long_chain(n_hinges):
    """A free root (sphere, r 0.1 m) carrying one chain of n_hinges hinges
    (alternating y / x axes, 0.05 m capsules): nv = 6 + n_hinges.  Armature
    0.1 keeps cond(M + diag(arm)) near 200, under the ant-like model's, so
    FP32 parity holds at the usual tolerances."""
    b = I._Builder("chain")
    m, c, J = I.sphere_mass_inertia(0.1, 1000.0)
    parent = b.link(-1, I.FREE, mass=m, com=c, inertia=J)
    for k in range(n_hinges):
        mk, ck, Jk = I.capsule_mass_inertia(0.02, (0, 0, 0), (0, 0, -0.05), 1000.0)
        parent = b.link(parent, I.REVOLUTE, axis=(0, 1, 0) if k % 2 == 0 else (1, 0, 0),
                        pos=(0, 0, -0.1 if k == 0 else -0.05), mass=mk, com=ck, inertia=Jk)
    nv = 6 + n_hinges
    return b.finish(act_dof=list(range(6, nv)), act_gear=[5.0] * n_hinges, dt=I.CONTROL_DT, substeps=4,
                    armature=0.1, damping=0.1, root_z=5.0)
