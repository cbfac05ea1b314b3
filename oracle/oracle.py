"""ctypes wrapper of the FP64 CPU oracle (test infrastructure only).

Only the tests, ``__graft_entry__.smoke()`` and the bench's CPU-baseline /
reference leg use this module.  The oracle follows Sec. 3.1 of the paper (the
simulator F, Eq. fwd_dynamics, the contact and joint-limit equations,
Cholesky, semi-implicit Euler) and Eq. backward / appendix A.1 for the
adjoint; see ``shac_oracle.cpp`` for the per-function citations.

Arrays at this interface are environment-major ([N][dim]); the helpers
``soa``/``aos`` convert from/to the structure-of-arrays layout ([dim][N]) the
CUDA library uses.  Inputs are promoted to float64 as given, so passing the
float32 values the GPU sees gives both sides identical inputs.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import sys

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "shac_oracle.cpp")
_LIB = os.path.join(_HERE, "liboracle.so")

_i32p = ctypes.POINTER(ctypes.c_int32)
_f64p = ctypes.POINTER(ctypes.c_double)


class OrcDesc(ctypes.Structure):
    _fields_ = [
        ("n_links", ctypes.c_int32), ("parent", _i32p), ("joint_type", _i32p),
        ("joint_axis", _f64p), ("joint_pos", _f64p), ("joint_quat", _f64p),
        ("mass", _f64p), ("com", _f64p), ("inertia", _f64p),
        ("n_contacts", ctypes.c_int32), ("contact_link", _i32p), ("contact_pos", _f64p),
        ("contact_radius", _f64p),
        ("q_lower", _f64p), ("q_upper", _f64p), ("armature", _f64p), ("damping", _f64p),
        ("k_limit", ctypes.c_double),
        ("n_tact", ctypes.c_int32), ("act_dof", _i32p), ("act_gear", _f64p),
        ("n_muscles", ctypes.c_int32), ("muscle_ptr", _i32p), ("via_link", _i32p),
        ("via_pos", _f64p), ("muscle_fmax", _f64p),
        ("dt", ctypes.c_double), ("substeps", ctypes.c_int32), ("gravity", ctypes.c_double * 3),
        ("ke", ctypes.c_double), ("kd", ctypes.c_double), ("kt", ctypes.c_double), ("mu", ctypes.c_double),
        ("rw_q", _f64p), ("rw_qd", _f64p), ("reward_coef", ctypes.c_double * 10),
        ("height_q", ctypes.c_int32), ("vx_dof", ctypes.c_int32),
    ]


def build(force: bool = False) -> str:
    """Compile liboracle.so with g++ (-O2, OpenMP).  Portable flags only."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        cmd = ["g++", "-O2", "-std=c++17", "-fopenmp", "-fPIC", "-shared", _SRC, "-o", _LIB + ".tmp"]
        subprocess.check_call(cmd)
        os.replace(_LIB + ".tmp", _LIB)
    return _LIB


_lib = None


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB)
        D = ctypes.POINTER(OrcDesc)
        i32 = ctypes.c_int32
        L.orc_step.argtypes = [D, i32, _f64p, _f64p, _f64p, _f64p, _f64p, _f64p]
        L.orc_step_jacobian.argtypes = [D, i32, _f64p, _f64p, _f64p, _f64p]
        L.orc_step_vjp.argtypes = [D, i32, _f64p, _f64p, _f64p, _f64p, _f64p, _f64p, _f64p, _f64p, _f64p]
        L.orc_window_forward.argtypes = [D, i32, i32, _f64p, _f64p, _f64p, _f64p, _f64p, _f64p]
        L.orc_window_adjoint.argtypes = [D, i32, i32, _f64p, _f64p, _f64p, _f64p, _f64p, _f64p,
                                         _f64p, _f64p, _f64p]
        L.orc_forward_accel.argtypes = [D, _f64p, _f64p, _f64p, _f64p]
        L.orc_mass_matrix.argtypes = [D, _f64p, _f64p]
        L.orc_inverse_dynamics.argtypes = [D, _f64p, _f64p, _f64p, _f64p, i32, _f64p]
        L.orc_joint_forces.argtypes = [D, _f64p, _f64p, _f64p, _f64p]
        L.orc_energy_momentum.argtypes = [D, _f64p, _f64p, _f64p]
        L.orc_link_poses.argtypes = [D, _f64p, _f64p, _f64p, _f64p]
        L.orc_muscle_lengths.argtypes = [D, _f64p, _f64p]
        L.orc_cholesky.argtypes = [i32, _f64p, _f64p]
        L.orc_num_threads.restype = ctypes.c_int
        u64, f64 = ctypes.c_uint64, ctypes.c_double
        L.orc_mca_step.argtypes = [D, i32, _f64p, _f64p, _f64p, _f64p, _f64p, _f64p, u64, f64]
        L.orc_mca_window_adjoint.argtypes = [D, i32, i32, _f64p, _f64p, _f64p, _f64p, _f64p, _f64p,
                                             _f64p, _f64p, _f64p, u64, f64, i32]
        L.orc_mca_chol_solve.argtypes = [i32, _f64p, _f64p, _f64p, u64, f64]
        _lib = L
    return _lib


def num_threads() -> int:
    return int(lib().orc_num_threads())


# Unit roundoff of FP32 (round to nearest): the relative size of the Monte
# Carlo Arithmetic perturbations that stand for FP32 rounding.
U_FP32 = 2.0 ** -24


def mca_chol_solve(A, b, seed: int, u: float = U_FP32):
    """x = A^{-1} b by Cholesky in Monte Carlo Arithmetic (see shac_oracle.cpp)."""
    A, pA = _d(A)
    b, pb = _d(b)
    x = np.zeros(b.shape[0])
    lib().orc_mca_chol_solve(int(b.shape[0]), pA, pb, x.ctypes.data_as(_f64p), int(seed), float(u))
    return x


def _d(a):
    a = np.ascontiguousarray(np.asarray(a, np.float64))
    return a, a.ctypes.data_as(_f64p)


def _i(a):
    a = np.ascontiguousarray(np.asarray(a, np.int32))
    return a, a.ctypes.data_as(_i32p)


class Oracle:
    """The oracle bound to one articulation model (an ``inputs.ArticulationModel``)."""

    def __init__(self, model):
        self.model = model
        keep = []

        def d(x):
            arr, p = _d(x)
            keep.append(arr)
            return p

        def i(x):
            arr, p = _i(x)
            keep.append(arr)
            return p

        m = model
        desc = OrcDesc()
        desc.n_links = m.n_links
        desc.parent = i(m.parent)
        desc.joint_type = i(m.joint_type)
        desc.joint_axis = d(m.joint_axis)
        desc.joint_pos = d(m.joint_pos)
        desc.joint_quat = d(m.joint_quat)
        desc.mass = d(m.mass)
        desc.com = d(m.com)
        desc.inertia = d(m.inertia)
        desc.n_contacts = m.n_contacts
        desc.contact_link = i(m.contact_link if m.n_contacts else np.zeros(1, np.int32))
        desc.contact_pos = d(m.contact_pos if m.n_contacts else np.zeros(3))
        desc.contact_radius = d(m.contact_radius if m.n_contacts else np.zeros(1))
        desc.q_lower = d(m.q_lower)
        desc.q_upper = d(m.q_upper)
        desc.armature = d(m.armature)
        desc.damping = d(m.damping)
        desc.k_limit = float(m.k_limit)
        desc.n_tact = m.n_tact
        desc.act_dof = i(m.act_dof if m.n_tact else np.zeros(1, np.int32))
        desc.act_gear = d(m.act_gear if m.n_tact else np.zeros(1))
        desc.n_muscles = m.n_muscles
        desc.muscle_ptr = i(m.muscle_ptr)
        desc.via_link = i(m.via_link if m.via_link.size else np.zeros(1, np.int32))
        desc.via_pos = d(m.via_pos if m.via_pos.size else np.zeros(3))
        desc.muscle_fmax = d(m.muscle_fmax if m.n_muscles else np.zeros(1))
        desc.dt = float(m.dt)
        desc.substeps = int(m.substeps)
        for k in range(3):
            desc.gravity[k] = float(m.gravity[k])
        desc.ke, desc.kd, desc.kt, desc.mu = float(m.ke), float(m.kd), float(m.kt), float(m.mu)
        desc.rw_q = d(m.rw_q)
        desc.rw_qd = d(m.rw_qd)
        for k in range(10):
            desc.reward_coef[k] = float(m.reward_coef[k])
        desc.height_q = int(m.height_q)
        desc.vx_dof = int(m.vx_dof)
        self._keep = keep
        self.desc = desc
        self.nq, self.nv, self.na = m.nq, m.nv, m.na

    # ---- batched (env-major) -------------------------------------------
    def step(self, q, qd, a):
        q, pq = _d(q); qd, pqd = _d(qd); a, pa = _d(a)
        N = q.shape[0]
        qn = np.zeros((N, self.nq)); qdn = np.zeros((N, self.nv)); r = np.zeros(N)
        lib().orc_step(ctypes.byref(self.desc), N, pq, pqd, pa, _d(qn)[1], _d(qdn)[1], _d(r)[1])
        return qn, qdn, r

    def step_jacobian(self, q, qd, a):
        q, pq = _d(q); qd, pqd = _d(qd); a, pa = _d(a)
        N = q.shape[0]
        J = np.zeros((N, self.nq + self.nv + 1, self.nq + self.nv + self.na))
        lib().orc_step_jacobian(ctypes.byref(self.desc), N, pq, pqd, pa, J.ctypes.data_as(_f64p))
        return J

    def step_vjp(self, q, qd, a, qn_bar, qdn_bar, r_bar):
        arrs = [_d(x) for x in (q, qd, a, qn_bar, qdn_bar, r_bar)]
        N = arrs[0][0].shape[0]
        qb = np.zeros((N, self.nq)); qdb = np.zeros((N, self.nv)); ab = np.zeros((N, self.na))
        lib().orc_step_vjp(ctypes.byref(self.desc), N, *[p for _, p in arrs],
                           qb.ctypes.data_as(_f64p), qdb.ctypes.data_as(_f64p), ab.ctypes.data_as(_f64p))
        return qb, qdb, ab

    def window_forward(self, q0, qd0, act):
        """q0 [N,nq], qd0 [N,nv], act [h,N,na] -> q_traj [h+1,N,nq], qd_traj, rew [h,N]."""
        q0, p0 = _d(q0); qd0, pd0 = _d(qd0); act, pa = _d(act)
        h, N = act.shape[0], act.shape[1]
        qt = np.zeros((h + 1, N, self.nq)); qdt = np.zeros((h + 1, N, self.nv)); rw = np.zeros((h, N))
        lib().orc_window_forward(ctypes.byref(self.desc), N, h, p0, pd0, pa,
                                 qt.ctypes.data_as(_f64p), qdt.ctypes.data_as(_f64p), rw.ctypes.data_as(_f64p))
        return qt, qdt, rw

    def window_adjoint(self, q_traj, qd_traj, act, r_bar, qT_bar, qdT_bar):
        arrs = [_d(x) for x in (q_traj, qd_traj, act, r_bar, qT_bar, qdT_bar)]
        h, N = arrs[2][0].shape[0], arrs[2][0].shape[1]
        qb = np.zeros((N, self.nq)); qdb = np.zeros((N, self.nv)); ab = np.zeros((h, N, self.na))
        lib().orc_window_adjoint(ctypes.byref(self.desc), N, h, *[p for _, p in arrs],
                                 qb.ctypes.data_as(_f64p), qdb.ctypes.data_as(_f64p), ab.ctypes.data_as(_f64p))
        return qb, qdb, ab

    # ---- episodic window ---------------------------------------------------
    # Sec. 3.2: the environment is reset when its task terminates early, and the
    # gradient is cut at the reset.  Appendix A.3: a task terminates when the
    # root falls below a task height, or at the task horizon.  Written plainly
    # on top of step / step_vjp: one step at a time, the decision and the reset
    # taken in float64 on the oracle's own state.
    def window_forward_episodic(self, q0, qd0, act, q_reset, qd_reset, term_height, max_episode_steps, ep0):
        """q0 [N,nq], qd0 [N,nv], act [h,N,na], q_reset/qd_reset like q0/qd0,
        ep0 [N] steps since each environment's last reset.  After step t:
        e += 1; done = (root height < term_height: q[2] for a free root, else
        q[height_q] when height_q >= 0) or
        (max_episode_steps > 0 and e >= max_episode_steps); a done environment
        restarts from its reset state with e = 0.
        -> q_traj [h+1,N,nq] (states after any reset), qd_traj, rew [h,N] (rewards
        before the reset), done [h,N] (uint8), e [N], and the states before the
        reset q_pre [h,N,nq], qd_pre."""
        act = np.asarray(act, np.float64)
        h, N = act.shape[0], act.shape[1]
        hq = 2 if int(self.model.joint_type[0]) == 0 else int(self.model.height_q)   # root height coordinate
        q = np.array(q0, np.float64); qd = np.array(qd0, np.float64)
        qr = np.asarray(q_reset, np.float64); qdr = np.asarray(qd_reset, np.float64)
        e = np.array(ep0, np.int64)
        qt = [q.copy()]; qdt = [qd.copy()]; rw = np.zeros((h, N)); done = np.zeros((h, N), np.uint8)
        q_pre = np.zeros((h, N, self.nq)); qd_pre = np.zeros((h, N, self.nv))
        for t in range(h):
            q, qd, rw[t] = self.step(q, qd, act[t])
            q_pre[t], qd_pre[t] = q, qd
            e = e + 1
            d = np.zeros(N, bool)
            if hq >= 0:
                d |= q[:, hq] < term_height
            if max_episode_steps > 0:
                d |= e >= max_episode_steps
            done[t] = d
            e[d] = 0
            q = np.where(d[:, None], qr, q)
            qd = np.where(d[:, None], qdr, qd)
            qt.append(q.copy()); qdt.append(qd.copy())
        return np.stack(qt), np.stack(qdt), rw, done, e, q_pre, qd_pre

    def window_adjoint_episodic(self, q_traj, qd_traj, act, done, r_bar, q_traj_bar, qd_traj_bar):
        """Reverse of the episodic window over its checkpoints (q_traj [h+1,N,nq]
        after resets) and done mask: where done[t] the cotangent of the state
        after step t is dropped (a reset state is a constant), then step t is
        reversed with its reward cotangent r_bar[t].  q_traj_bar [h+1,N,nq] are
        the direct cotangents of the checkpoints.  -> q0_bar, qd0_bar, act_bar [h,N,na]."""
        act = np.asarray(act, np.float64)
        h, N = act.shape[0], act.shape[1]
        qb = np.array(q_traj_bar[h], np.float64); qdb = np.array(qd_traj_bar[h], np.float64)
        ab = np.zeros((h, N, self.na))
        for t in range(h - 1, -1, -1):
            cut = np.asarray(done[t]).astype(bool)
            qb[cut] = 0.0
            qdb[cut] = 0.0
            sq, sqd, ab[t] = self.step_vjp(q_traj[t], qd_traj[t], act[t], qb, qdb, r_bar[t])
            qb = sq + q_traj_bar[t]
            qdb = sqd + qd_traj_bar[t]
        return qb, qdb, ab

    # ---- single state ------------------------------------------------------
    def forward_accel(self, q, qd, a):
        out = np.zeros(self.nv)
        lib().orc_forward_accel(ctypes.byref(self.desc), _d(q)[1], _d(qd)[1], _d(a)[1], out.ctypes.data_as(_f64p))
        return out

    def mass_matrix(self, q):
        out = np.zeros((self.nv, self.nv))
        q, pq = _d(q)
        lib().orc_mass_matrix(ctypes.byref(self.desc), pq, out.ctypes.data_as(_f64p))
        return out

    def inverse_dynamics(self, q, qd, qdd, a=None, with_ext=True):
        if a is None:
            a = np.zeros(max(1, self.na))
        out = np.zeros(self.nv)
        q, pq = _d(q); qd, pqd = _d(qd); qdd, pqdd = _d(qdd); a, pa = _d(a)
        lib().orc_inverse_dynamics(ctypes.byref(self.desc), pq, pqd, pqdd, pa, int(with_ext),
                                   out.ctypes.data_as(_f64p))
        return out

    def joint_forces(self, q, qd, a):
        out = np.zeros(self.nv)
        q, pq = _d(q); qd, pqd = _d(qd); a, pa = _d(a)
        lib().orc_joint_forces(ctypes.byref(self.desc), pq, pqd, pa, out.ctypes.data_as(_f64p))
        return out

    def energy_momentum(self, q, qd):
        out = np.zeros(11)
        q, pq = _d(q); qd, pqd = _d(qd)
        lib().orc_energy_momentum(ctypes.byref(self.desc), pq, pqd, out.ctypes.data_as(_f64p))
        return dict(T=out[0], V=out[1], P=out[2:5].copy(), H=out[5:8].copy(), com=out[8:11].copy())

    def link_poses(self, q):
        L = self.model.n_links
        R = np.zeros((L, 3, 3)); o = np.zeros((L, 3)); c = np.zeros((L, 3))
        q, pq = _d(q)
        lib().orc_link_poses(ctypes.byref(self.desc), pq, R.ctypes.data_as(_f64p),
                             o.ctypes.data_as(_f64p), c.ctypes.data_as(_f64p))
        return R, o, c

    def muscle_lengths(self, q):
        out = np.zeros(max(1, self.model.n_muscles))
        q, pq = _d(q)
        lib().orc_muscle_lengths(ctypes.byref(self.desc), pq, out.ctypes.data_as(_f64p))
        return out[: self.model.n_muscles]

    # ---- FP32 error floor (Monte Carlo Arithmetic; see shac_oracle.cpp) ----
    def mca_step(self, q, qd, a, seed: int, u: float = U_FP32):
        """step() with every operation perturbed at relative size u (seeded
        per environment); u = 0 gives step() exactly."""
        q, pq = _d(q); qd, pqd = _d(qd); a, pa = _d(a)
        N = q.shape[0]
        qn = np.zeros((N, self.nq)); qdn = np.zeros((N, self.nv)); r = np.zeros(N)
        lib().orc_mca_step(ctypes.byref(self.desc), N, pq, pqd, pa, qn.ctypes.data_as(_f64p),
                           qdn.ctypes.data_as(_f64p), r.ctypes.data_as(_f64p), int(seed), float(u))
        return qn, qdn, r

    def mca_window_adjoint(self, q_traj, qd_traj, act, r_bar, qT_bar, qdT_bar, seed: int, u: float = U_FP32,
                           tangents: bool = True):
        """window_adjoint() with each step's Jacobian taken along a perturbed
        evaluation of the step (values perturbed at relative size u; with
        tangents, every operation of the derivative computation as well)."""
        arrs = [_d(x) for x in (q_traj, qd_traj, act, r_bar, qT_bar, qdT_bar)]
        h, N = arrs[2][0].shape[0], arrs[2][0].shape[1]
        qb = np.zeros((N, self.nq)); qdb = np.zeros((N, self.nv)); ab = np.zeros((h, N, self.na))
        lib().orc_mca_window_adjoint(ctypes.byref(self.desc), N, h, *[p for _, p in arrs],
                                     qb.ctypes.data_as(_f64p), qdb.ctypes.data_as(_f64p), ab.ctypes.data_as(_f64p),
                                     int(seed), float(u), int(bool(tangents)))
        return qb, qdb, ab

    def step_floor(self, q, qd, a, runs: int = 3, seed: int = 0):
        """Per-component FP32 floor of one step: the largest deviation from the
        exact result over `runs` Monte Carlo Arithmetic runs.
        -> (exact (qn, qdn, r), floor (fq, fqd, fr))."""
        ex = self.step(q, qd, a)
        fl = [np.zeros_like(x) for x in ex]
        for k in range(runs):
            for f, y, x in zip(fl, self.mca_step(q, qd, a, seed=seed * 1000 + k), ex):
                np.maximum(f, np.abs(y - x), out=f)
        return ex, tuple(fl)


def cholesky(A):
    A, pa = _d(A)
    n = A.shape[0]
    Lc = np.zeros((n, n))
    lib().orc_cholesky(n, pa, Lc.ctypes.data_as(_f64p))
    return Lc


def aos(x):
    """[dim][N] (or [t][dim][N]) -> [N][dim] (or [t][N][dim]) float64."""
    x = np.asarray(x, np.float64)
    return np.ascontiguousarray(np.swapaxes(x, -1, -2))


soa = aos

if __name__ == "__main__":
    build(force="--force" in sys.argv)
    print(_LIB)


# ---- learner (Sec. 3.2) -------------------------------------------------------

def td_lambda(reward, value, done, gamma, lam):
    """Critic targets of Eq. td-lambda, term by term: for each state s_t of the
    window, the (1 - lambda)-weighted average of its k-step returns
    G_t^k = sum_{l<k} gamma^l r_{t+l} + gamma^k V(s_{t+k}) plus the weight
    lambda^(H-1) on the longest one, H the number of steps left in the state's
    episode inside the window.  An episode that ends at step `end` (done) takes
    no bootstrap after its last reward; otherwise the window end bootstraps
    with V(s_h).  reward [h, N], value [h+1, N], done [h, N] or None -> [h, N]."""
    reward = np.asarray(reward, np.float64)
    value = np.asarray(value, np.float64)
    h, N = reward.shape
    done = np.zeros((h, N), bool) if done is None else np.asarray(done).astype(bool)
    out = np.zeros((h, N))
    for e in range(N):
        for t in range(h):
            end = t
            while end < h - 1 and not done[end, e]:
                end += 1
            terminal = bool(done[end, e])
            H = end - t + 1

            def G(k):
                g = sum(gamma ** l * reward[t + l, e] for l in range(k))
                if k < H or not terminal:
                    g += gamma ** k * value[t + k, e]
                return g

            out[t, e] = (1 - lam) * sum(lam ** (k - 1) * G(k) for k in range(1, H)) + lam ** (H - 1) * G(H)
    return out
