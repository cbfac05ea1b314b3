"""Shared test helpers: seeded cases, layout conversion, tolerance checks."""
import numpy as np

from paper_2204_07137_gb300 import inputs as I

# Per-step state tolerance (elementwise) and window-gradient tolerance
# (norm-wise per environment) for the FP32 GPU path against the FP64 oracle.
STATE_RTOL, STATE_ATOL = 1e-4, 1e-5
GRAD_RTOL = 1e-3


def assert_state_close(got, ref, what, rtol=STATE_RTOL, atol=STATE_ATOL):
    got = np.asarray(got, np.float64)
    ref = np.asarray(ref, np.float64)
    assert np.isfinite(ref).all(), f"{what}: reference not finite"
    err = np.abs(got - ref)
    bound = atol + rtol * np.abs(ref)
    bad = ~(err <= bound)          # NaN counts as a mismatch
    if bad.any():
        idx = np.argwhere(bad)[:5]
        raise AssertionError(f"{what}: {bad.sum()} / {bad.size} elements outside |d| <= {atol} + {rtol}|ref|; "
                             f"worst ratio {np.max(err / bound):.3g}; first {idx.tolist()} "
                             f"got {got[bad][:5]} ref {ref[bad][:5]}")


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
    return {"cartpole": I.cartpole, "ant": I.ant, "humanoid": I.humanoid, "mtu": I.mtu}[name]()


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
