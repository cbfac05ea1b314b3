"""Seeded synthetic workloads: articulation descriptions and window inputs.

This module is shared by the CUDA path, the tests, the bench and the CPU
oracle.  It holds model *construction* only (joint trees, masses, inertias,
contact spheres, limits, gears, muscles, seeds) and none of the simulator's
arithmetic: no kinematics, dynamics, contact, integration or reward code lives
here.

The paper's own task models (Sec. 4 and appendix A.3: CartPole, Ant,
Humanoid, Humanoid MTU) are not available, so each builder below is a
synthetic stand-in with the sizes the paper's tasks have (DOF counts,
contact counts, action sizes; appendix A.3 observation tables give 1/8/21/152
actions).  Conventions (shared reading of the paper, Sec. 3.1):

* z is up, gravity (0, 0, -9.81), ground plane z = 0.
* Joint types: FREE (6 DOF, root only), REVOLUTE, PRISMATIC, FIXED.
* Free joint coordinates: q = (p_world[3], quat xyzw[4]),
  qd = (omega_body[3], v_body[3]) -- body-frame angular velocity and the
  body-frame velocity of the link origin.
* Every link frame sits at its joint; ``joint_pos``/``joint_quat`` place the
  joint frame in the parent link frame; ``joint_axis`` is a unit vector in the
  joint frame.  ``com`` and ``inertia`` (xx, yy, zz, xy, xz, yz about the
  COM) are in the link frame.
* All float parameters are stored as float32: the GPU consumes them as is and
  the FP64 oracle promotes the same rounded values.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Sequence, Tuple

import numpy as np

FREE, REVOLUTE, PRISMATIC, FIXED = 0, 1, 2, 3
JOINT_NDOF = {FREE: 6, REVOLUTE: 1, PRISMATIC: 1, FIXED: 0}
JOINT_NQ = {FREE: 7, REVOLUTE: 1, PRISMATIC: 1, FIXED: 0}

# reward_coef slots (see ArticulationModel.reward_coef)
RC_W_ACT, RC_W_V, RC_W_UP, RC_W_HEAD, RC_H0, RC_LO, RC_HI, RC_NEG2, RC_NEG1, RC_POS = range(10)
N_REWARD_COEF = 10
BIG = 1.0e30


@dataclasses.dataclass
class ArticulationModel:
    """One articulation type (a joint tree plus its contact and actuation data).

    Reward (evaluated on the post-step state with the step's action):
      r = - sum_j rw_q[j] q_j^2 - sum_j rw_qd[j] qd_j^2 - w_act * |a|^2
          + w_v * vx + R_h + [free root only] w_up * up_z + w_head * head_x
      R_h = c_neg2*D^2 + c_neg1*D  if D < 0  else  c_pos*D,
      D = clip(root_z - h0, lo, hi)
    where, with a free root, vx is the world x-velocity of the root origin,
    root_z = q[2], up_z the world z component of the root's z axis and head_x
    the world x component of the root's x axis; without one (planar models on
    x / z slide joints) vx = qd[vx_dof] and root_z = q[height_q], each term
    dropped when its index is -1 (appendix A.3 reward shapes).
    """

    name: str
    parent: np.ndarray          # int32 [L]; -1 = world; parent[i] < i
    joint_type: np.ndarray      # int32 [L]
    joint_axis: np.ndarray      # f32 [L,3]
    joint_pos: np.ndarray       # f32 [L,3]
    joint_quat: np.ndarray      # f32 [L,4] xyzw
    mass: np.ndarray            # f32 [L]
    com: np.ndarray             # f32 [L,3]
    inertia: np.ndarray         # f32 [L,6]
    contact_link: np.ndarray    # int32 [C]
    contact_pos: np.ndarray     # f32 [C,3]
    contact_radius: np.ndarray  # f32 [C]
    q_lower: np.ndarray         # f32 [nv]  (-BIG = none)
    q_upper: np.ndarray         # f32 [nv]  (+BIG = none)
    armature: np.ndarray        # f32 [nv]
    damping: np.ndarray         # f32 [nv]
    k_limit: float
    act_dof: np.ndarray         # int32 [n_tact]
    act_gear: np.ndarray        # f32 [n_tact]
    muscle_ptr: np.ndarray      # int32 [M+1]
    via_link: np.ndarray        # int32 [V]
    via_pos: np.ndarray         # f32 [V,3]
    muscle_fmax: np.ndarray     # f32 [M]
    dt: float                   # control step
    substeps: int
    gravity: np.ndarray         # f32 [3]
    ke: float
    kd: float
    kt: float
    mu: float
    rw_q: np.ndarray            # f32 [nq]
    rw_qd: np.ndarray           # f32 [nv]
    reward_coef: np.ndarray     # f32 [10]
    root_z: float = 1.0         # initial root height of the standing pose
    height_q: int = -1          # q index of the root height (models without a free root)
    vx_dof: int = -1            # qd index of the forward velocity (models without a free root)

    @property
    def n_links(self) -> int:
        return int(self.parent.shape[0])

    @property
    def nq(self) -> int:
        return int(sum(JOINT_NQ[int(t)] for t in self.joint_type))

    @property
    def nv(self) -> int:
        return int(sum(JOINT_NDOF[int(t)] for t in self.joint_type))

    @property
    def n_tact(self) -> int:
        return int(self.act_dof.shape[0])

    @property
    def n_muscles(self) -> int:
        return int(self.muscle_ptr.shape[0] - 1)

    @property
    def na(self) -> int:
        return self.n_tact + self.n_muscles

    @property
    def n_contacts(self) -> int:
        return int(self.contact_link.shape[0])

    def q_start(self) -> np.ndarray:
        out, acc = [], 0
        for t in self.joint_type:
            out.append(acc)
            acc += JOINT_NQ[int(t)]
        return np.asarray(out, np.int32)

    def dof_start(self) -> np.ndarray:
        out, acc = [], 0
        for t in self.joint_type:
            out.append(acc)
            acc += JOINT_NDOF[int(t)]
        return np.asarray(out, np.int32)

    def replace(self, **kw) -> "ArticulationModel":
        return dataclasses.replace(self, **kw)


# ---------------------------------------------------------------------------
# Builder helpers (model construction only)
# ---------------------------------------------------------------------------

def quat_axis_angle(axis: Sequence[float], angle: float) -> np.ndarray:
    a = np.asarray(axis, np.float64)
    a = a / np.linalg.norm(a)
    s = math.sin(angle / 2.0)
    return np.array([a[0] * s, a[1] * s, a[2] * s, math.cos(angle / 2.0)])


def _rot_of_quat(qx, qy, qz, qw) -> np.ndarray:
    # used only to place fixed frames while building models
    return np.array([
        [1 - 2 * (qy * qy + qz * qz), 2 * (qx * qy - qz * qw), 2 * (qx * qz + qy * qw)],
        [2 * (qx * qy + qz * qw), 1 - 2 * (qx * qx + qz * qz), 2 * (qy * qz - qx * qw)],
        [2 * (qx * qz - qy * qw), 2 * (qy * qz + qx * qw), 1 - 2 * (qx * qx + qy * qy)],
    ])


def capsule_mass_inertia(radius: float, p0: Sequence[float], p1: Sequence[float], density: float):
    """Mass, COM and inertia (about COM, 6-vector) of a solid capsule whose
    segment runs from p0 to p1 (a cylinder of that length capped by two
    hemispheres), in the frame p0/p1 are given in.  Closed form: cylinder plus
    two hemispheres shifted by the parallel-axis theorem."""
    p0 = np.asarray(p0, np.float64)
    p1 = np.asarray(p1, np.float64)
    seg = p1 - p0
    length = float(np.linalg.norm(seg))
    r = float(radius)
    m_cyl = density * math.pi * r * r * length
    m_hemi = density * (2.0 / 3.0) * math.pi * r ** 3
    mass = m_cyl + 2.0 * m_hemi
    i_axis = m_cyl * r * r / 2.0 + 2.0 * (2.0 / 5.0) * m_hemi * r * r
    shift = length / 2.0 + 3.0 * r / 8.0
    i_trans = (m_cyl * (r * r / 4.0 + length * length / 12.0)
               + 2.0 * ((83.0 / 320.0) * m_hemi * r * r + m_hemi * shift * shift))
    if length > 0:
        u = seg / length
    else:
        u = np.array([0.0, 0.0, 1.0])
    full = i_trans * np.eye(3) + (i_axis - i_trans) * np.outer(u, u)
    com = 0.5 * (p0 + p1)
    return mass, com, full


def sphere_mass_inertia(radius: float, density: float):
    m = density * 4.0 / 3.0 * math.pi * radius ** 3
    i = 2.0 / 5.0 * m * radius * radius
    return m, np.zeros(3), i * np.eye(3)


def _sym6(full: np.ndarray) -> np.ndarray:
    return np.array([full[0, 0], full[1, 1], full[2, 2], full[0, 1], full[0, 2], full[1, 2]])


def combine_bodies(parts):
    """Combine (mass, com, full_inertia_about_com) parts rigidly attached to one link."""
    m = sum(p[0] for p in parts)
    if m == 0:
        return 0.0, np.zeros(3), np.zeros((3, 3))
    c = sum(p[0] * np.asarray(p[1]) for p in parts) / m
    I = np.zeros((3, 3))
    for pm, pc, pI in parts:
        d = np.asarray(pc) - c
        I += pI + pm * (np.dot(d, d) * np.eye(3) - np.outer(d, d))
    return m, c, I


class _Builder:
    def __init__(self, name: str):
        self.name = name
        self.links = []
        self.contacts = []
        self.muscles = []       # list of (fmax, [(link, pos), ...])
        self.limits = {}        # link -> (lo, hi)

    def link(self, parent, jtype, axis=(0, 0, 1), pos=(0, 0, 0), quat=(0, 0, 0, 1),
             mass=0.0, com=(0, 0, 0), inertia=None, limit=None):
        if inertia is None:
            inertia = np.zeros((3, 3))
        ax = np.asarray(axis, np.float64)
        ax = ax / np.linalg.norm(ax)
        self.links.append(dict(parent=parent, jtype=jtype, axis=ax, pos=np.asarray(pos, np.float64),
                               quat=np.asarray(quat, np.float64), mass=float(mass),
                               com=np.asarray(com, np.float64), inertia=_sym6(np.asarray(inertia))))
        idx = len(self.links) - 1
        if limit is not None:
            self.limits[idx] = limit
        return idx

    def contact(self, link, pos, radius):
        self.contacts.append((link, np.asarray(pos, np.float64), float(radius)))

    def muscle(self, fmax, vias):
        self.muscles.append((float(fmax), list(vias)))

    def fixed_pose(self, link):
        """World pose of a link with every joint coordinate at zero and an
        identity root at the origin (placement helper for builders)."""
        chain = []
        i = link
        while i >= 0:
            chain.append(i)
            i = self.links[i]["parent"]
        R = np.eye(3)
        p = np.zeros(3)
        for i in reversed(chain):
            L = self.links[i]
            if L["jtype"] == FREE:
                continue
            p = p + R @ L["pos"]
            R = R @ _rot_of_quat(*L["quat"])
        return R, p

    def finish(self, *, act_dof, act_gear, dt, substeps, ke=0.0, kd=0.0, kt=0.0, mu=0.0,
               k_limit=0.0, armature=0.0, damping=0.0, rw_q=None, rw_qd=None,
               reward_coef=None, gravity=(0.0, 0.0, -9.81), root_z=1.0, height_q=-1,
               vx_dof=-1) -> ArticulationModel:
        f32 = np.float32
        L = len(self.links)
        jt = np.array([l["jtype"] for l in self.links], np.int32)
        nv = int(sum(JOINT_NDOF[int(t)] for t in jt))
        nq = int(sum(JOINT_NQ[int(t)] for t in jt))
        q_lower = np.full(nv, -BIG, f32)
        q_upper = np.full(nv, BIG, f32)
        ds = 0
        for i, l in enumerate(self.links):
            if i in self.limits:
                assert JOINT_NDOF[l["jtype"]] == 1
                q_lower[ds], q_upper[ds] = self.limits[i]
            ds += JOINT_NDOF[l["jtype"]]
        ptr = [0]
        vlink, vpos, fmax = [], [], []
        for fm, vias in self.muscles:
            for lk, p in vias:
                vlink.append(lk)
                vpos.append(p)
            ptr.append(len(vlink))
            fmax.append(fm)
        rc = np.zeros(N_REWARD_COEF, f32) if reward_coef is None else np.asarray(reward_coef, f32)
        return ArticulationModel(
            name=self.name,
            parent=np.array([l["parent"] for l in self.links], np.int32),
            joint_type=jt,
            joint_axis=np.array([l["axis"] for l in self.links], f32).reshape(L, 3),
            joint_pos=np.array([l["pos"] for l in self.links], f32).reshape(L, 3),
            joint_quat=np.array([l["quat"] for l in self.links], f32).reshape(L, 4),
            mass=np.array([l["mass"] for l in self.links], f32),
            com=np.array([l["com"] for l in self.links], f32).reshape(L, 3),
            inertia=np.array([l["inertia"] for l in self.links], f32).reshape(L, 6),
            contact_link=np.array([c[0] for c in self.contacts], np.int32),
            contact_pos=np.array([c[1] for c in self.contacts], f32).reshape(-1, 3),
            contact_radius=np.array([c[2] for c in self.contacts], f32),
            q_lower=q_lower, q_upper=q_upper,
            armature=np.broadcast_to(np.asarray(armature, f32), (nv,)).copy(),
            damping=np.broadcast_to(np.asarray(damping, f32), (nv,)).copy(),
            k_limit=float(np.float32(k_limit)),
            act_dof=np.asarray(act_dof, np.int32),
            act_gear=np.asarray(act_gear, f32),
            muscle_ptr=np.asarray(ptr, np.int32),
            via_link=np.asarray(vlink, np.int32),
            via_pos=np.asarray(vpos, f32).reshape(-1, 3),
            muscle_fmax=np.asarray(fmax, f32),
            dt=float(np.float32(dt)), substeps=int(substeps),
            gravity=np.asarray(gravity, f32),
            ke=float(np.float32(ke)), kd=float(np.float32(kd)), kt=float(np.float32(kt)),
            mu=float(np.float32(mu)),
            rw_q=np.zeros(nq, f32) if rw_q is None else np.asarray(rw_q, f32),
            rw_qd=np.zeros(nv, f32) if rw_qd is None else np.asarray(rw_qd, f32),
            reward_coef=rc,
            root_z=float(root_z),
            height_q=int(height_q),
            vx_dof=int(vx_dof),
        )


def _loco_coef(w_act, w_v, w_up, w_head, h0, lo, hi, neg2, neg1, pos):
    return [w_act, w_v, w_up, w_head, h0, lo, hi, neg2, neg1, pos]


# ---------------------------------------------------------------------------
# The five workload articulations
# ---------------------------------------------------------------------------

CONTROL_DT = 1.0 / 60.0


def cartpole(substeps: int = 4) -> ArticulationModel:
    """Cart (prismatic along x, 1 kg) + pole (revolute about y, 0.1 kg uniform
    rod of 1 m, theta = 0 upright).  One action: cart force, gear 100 N.
    Reward -(theta^2 + 0.1 x^2) (config loss); no contact."""
    b = _Builder("cartpole")
    cart = b.link(-1, PRISMATIC, axis=(1, 0, 0), mass=1.0,
                  inertia=np.diag([0.01, 0.01, 0.01]))
    mp, L = 0.1, 1.0
    b.link(cart, REVOLUTE, axis=(0, 1, 0), mass=mp, com=(0, 0, L / 2),
           inertia=np.diag([mp * L * L / 12, mp * L * L / 12, 1e-5]))
    return b.finish(act_dof=[0], act_gear=[100.0], dt=CONTROL_DT, substeps=substeps,
                    rw_q=[0.1, 1.0], reward_coef=_loco_coef(0, 0, 0, 0, 0, -BIG, BIG, 0, 0, 0))


ANT_DENSITY = 5.0 * 200.0   # "density 5 kg/m^3 scaled": scale 200, so that explicit contact damping stays stable
ANT_FOOT_PENETRATION = 0.002


def ant(substeps: int = 16, density: float = ANT_DENSITY) -> ArticulationModel:
    """Ant-like quadruped: free torso (sphere r 0.25) + 4 x (hip yaw, knee
    pitch) hinges; thigh capsules 0.3 m, shin capsules 0.5 m, radius 0.08;
    contact spheres at the 4 shin ends and the torso centre (5 contacts);
    ke 4e4, kd 1e3, mu 0.75, kt 1e3 (kt not given by the paper); gear 200.
    Reward: appendix A.3 Ant, v_x + 0.1 up + heading + (h - 0.27)."""
    b = _Builder("ant")
    m, c, I = sphere_mass_inertia(0.25, density)
    torso = b.link(-1, FREE, mass=m, com=c, inertia=I)
    b.contact(torso, (0, 0, 0), 0.25)
    r = 0.08
    shin_end = np.array([0.5 * math.cos(math.pi / 4), 0.0, -0.5 * math.sin(math.pi / 4)])
    for k in range(4):
        phi = math.pi / 4 + k * math.pi / 2
        m1, c1, I1 = capsule_mass_inertia(r, (0, 0, 0), (0.3, 0, 0), density)
        hip = b.link(torso, REVOLUTE, axis=(0, 0, 1),
                     pos=(0.25 * math.cos(phi), 0.25 * math.sin(phi), 0.0),
                     quat=quat_axis_angle((0, 0, 1), phi), mass=m1, com=c1, inertia=I1)
        m2, c2, I2 = capsule_mass_inertia(r, (0, 0, 0), shin_end, density)
        knee = b.link(hip, REVOLUTE, axis=(0, 1, 0), pos=(0.3, 0, 0), mass=m2, com=c2, inertia=I2)
        b.contact(knee, shin_end, r)
    foot_z = -0.5 * math.sin(math.pi / 4) - r
    nq = 15
    return b.finish(act_dof=list(range(6, 14)), act_gear=[200.0] * 8, dt=CONTROL_DT,
                    substeps=substeps, ke=4e4, kd=1e3, kt=1e3, mu=0.75,
                    rw_q=np.zeros(nq), root_z=-foot_z - ANT_FOOT_PENETRATION,
                    reward_coef=_loco_coef(0.0, 1.0, 0.1, 1.0, 0.27, -BIG, BIG, 0.0, 1.0, 1.0))


PLANAR_DENSITY = 1000.0
PLANAR_ARMATURE = 0.05     # joint armature (kg m^2), not stated by the paper
PLANAR_DAMPING = 1.0       # joint damping (N m s/rad), not stated by the paper


def _planar_root(b, z0, torso_p0, torso_p1, radius):
    """Planar root: slide along world x, slide along world z (frame at height
    z0, so q[1] is the height change from the initial pose), hinge about y
    carrying the torso capsule.  Returns the torso link."""
    sx = b.link(-1, PRISMATIC, axis=(1, 0, 0))
    sz = b.link(sx, PRISMATIC, axis=(0, 0, 1), pos=(0, 0, z0))
    m, c, I = capsule_mass_inertia(radius, torso_p0, torso_p1, PLANAR_DENSITY)
    return b.link(sz, REVOLUTE, axis=(0, 1, 0), mass=m, com=c, inertia=I)


def _planar_limb(b, parent, pos, p1, radius, limit):
    """Hinge about y at pos (parent frame) with a capsule from its origin to p1."""
    m, c, I = capsule_mass_inertia(radius, (0, 0, 0), p1, PLANAR_DENSITY)
    return b.link(parent, REVOLUTE, axis=(0, 1, 0), pos=pos, mass=m, com=c, inertia=I, limit=limit)


def halfcheetah(substeps: int = 16) -> ArticulationModel:
    """Planar two-legged runner (stand-in for appendix A.3 HalfCheetah): x / z
    slides and a pitch hinge carrying a 1 m torso capsule (radius 0.05), and
    per leg a thigh (0.25 m), shin (0.25 m) and forward foot (0.15 m) on y
    hinges (6 actuated DOFs, gear 100, limits +-1 rad at k_limit 1e3);
    contact spheres at both ends of each foot and of the torso; ke 4e4,
    kd 1e3, kt 1e3, mu 0.75.  Reward v_x - 0.1 |a|^2 (A.3); no early termination."""
    b = _Builder("halfcheetah")
    r = 0.05
    z0 = 0.5 + r - 0.002
    torso = _planar_root(b, z0, (-0.5, 0, 0), (0.5, 0, 0), r)
    for x in (-0.5, 0.5):
        thigh = _planar_limb(b, torso, (x, 0, 0), (0, 0, -0.25), r, (-1.0, 1.0))
        shin = _planar_limb(b, thigh, (0, 0, -0.25), (0, 0, -0.25), r, (-1.0, 1.0))
        foot = _planar_limb(b, shin, (0, 0, -0.25), (0.15, 0, 0), r, (-1.0, 1.0))
        b.contact(foot, (0, 0, 0), r)
        b.contact(foot, (0.15, 0, 0), r)
    b.contact(torso, (-0.5, 0, 0), r)
    b.contact(torso, (0.5, 0, 0), r)
    return b.finish(act_dof=list(range(3, 9)), act_gear=[100.0] * 6, dt=CONTROL_DT, substeps=substeps,
                    ke=4e4, kd=1e3, kt=1e3, mu=0.75, k_limit=1e3, armature=PLANAR_ARMATURE,
                    damping=PLANAR_DAMPING, root_z=z0, height_q=1, vx_dof=0,
                    reward_coef=_loco_coef(0.1, 1.0, 0.0, 0.0, 0.0, -BIG, BIG, 0.0, 0.0, 0.0))


def hopper(substeps: int = 16) -> ArticulationModel:
    """Planar one-legged hopper (stand-in for appendix A.3 Hopper): x / z
    slides and a pitch hinge carrying a 0.4 m upright torso capsule (radius
    0.05), then thigh (0.45 m), leg (0.5 m) and a horizontal foot (0.39 m) on y
    hinges (3 actuated DOFs, gear 200, limits +-1 rad at k_limit 1e3); contact
    spheres at both foot ends, the knee and the top of the torso.  Reward (A.3): v_x + R_height + R_angle -
    0.1 |a|^2 with R_height = -200 D^2 (D < 0), D (D >= 0),
    D = clip(h + 0.3, -1, 0.3), h the height change of the root, and
    R_angle = -(theta / 30 deg)^2 (the paper's constant 1 is dropped: it does
    not change any gradient)."""
    b = _Builder("hopper")
    r = 0.05
    z0 = 0.95 + r - 0.002
    torso = _planar_root(b, z0, (0, 0, 0), (0, 0, 0.4), r)
    thigh = _planar_limb(b, torso, (0, 0, 0), (0, 0, -0.45), r, (-1.0, 1.0))
    leg = _planar_limb(b, thigh, (0, 0, -0.45), (0, 0, -0.5), r, (-1.0, 1.0))
    m, c, I = capsule_mass_inertia(r, (-0.13, 0, 0), (0.26, 0, 0), PLANAR_DENSITY)
    foot = b.link(leg, REVOLUTE, axis=(0, 1, 0), pos=(0, 0, -0.5), mass=m, com=c, inertia=I, limit=(-1.0, 1.0))
    b.contact(foot, (-0.13, 0, 0), r)
    b.contact(foot, (0.26, 0, 0), r)
    b.contact(leg, (0, 0, 0), r)
    b.contact(torso, (0, 0, 0.4), r)
    rw_q = np.zeros(6)
    rw_q[2] = 1.0 / (math.pi / 6) ** 2
    return b.finish(act_dof=[3, 4, 5], act_gear=[200.0] * 3, dt=CONTROL_DT, substeps=substeps,
                    ke=4e4, kd=1e3, kt=1e3, mu=0.75, k_limit=1e3, armature=PLANAR_ARMATURE,
                    damping=PLANAR_DAMPING, root_z=z0, height_q=1, vx_dof=0, rw_q=rw_q,
                    reward_coef=_loco_coef(0.1, 1.0, 0.0, 0.0, -0.3, -1.0, 0.3, -200.0, 0.0, 1.0))


HUMANOID_TOTAL_MASS = 40.0
HUMANOID_ARMATURE = 0.05     # joint armature (kg m^2), not stated by the paper
HUMANOID_DAMPING = 5.0       # joint damping (N m s/rad), not stated by the paper
MTU_ARMATURE = 0.05
MTU_DAMPING = 5.0


def humanoid(substeps: int = 48, seed: int = 0) -> ArticulationModel:
    """Humanoid-like: free torso + 21 revolute DOFs over 13 capsule bodies
    (multi-DOF joints as chains of revolute joints through massless links),
    total mass 40 kg, 10 capsule-end contact spheres, joint limits as a stiff
    penalty (k_limit 1e4, ranges seeded), per-joint gears 50-200 (seeded).
    Reward: forward velocity of the torso (config 3)."""
    rng = np.random.default_rng(np.random.SeedSequence([2204, 7137, 3, seed]))
    b = _Builder("humanoid")
    parts = []   # (link, p0, p1, radius) capsules, filled below; masses scaled at the end

    def chain(parent, pos, axes, limits):
        """Revolute chain at one joint site; returns the last link."""
        cur = parent
        for j, ax in enumerate(axes):
            cur = b.link(cur, REVOLUTE, axis=ax, pos=pos if j == 0 else (0, 0, 0),
                         limit=limits[j])
        return cur

    def lim(scale_lo, scale_hi):
        lo = -float(rng.uniform(scale_lo, scale_hi))
        hi = float(rng.uniform(scale_lo, scale_hi))
        return (lo, hi)

    torso = b.link(-1, FREE)
    parts.append((torso, (0, 0, -0.1), (0, 0, 0.2), 0.09))
    lwaist = chain(torso, (0, 0, -0.15), [(0, 0, 1), (0, 1, 0)], [lim(0.5, 1.0), lim(0.5, 1.0)])
    parts.append((lwaist, (0, 0, 0.0), (0, 0, -0.1), 0.07))
    pelvis = chain(lwaist, (0, 0, -0.1), [(1, 0, 0)], [lim(0.5, 1.0)])
    parts.append((pelvis, (0, -0.1, -0.05), (0, 0.1, -0.05), 0.09))
    b.contact(pelvis, (0, -0.1, -0.05), 0.09)
    b.contact(pelvis, (0, 0.1, -0.05), 0.09)
    for side in (-1.0, 1.0):
        thigh = chain(pelvis, (0, 0.1 * side, -0.1), [(1, 0, 0), (0, 0, 1), (0, 1, 0)],
                      [lim(0.5, 1.5), lim(0.5, 1.5), lim(0.5, 1.5)])
        parts.append((thigh, (0, 0, 0), (0, 0, -0.4), 0.06))
        shin = chain(thigh, (0, 0, -0.42), [(0, 1, 0)], [lim(1.0, 1.5)])
        parts.append((shin, (0, 0, 0), (0, 0, -0.4), 0.05))
        b.contact(shin, (0, 0, -0.4), 0.05)
        foot = chain(shin, (0, 0, -0.45), [(0, 1, 0), (1, 0, 0)], [lim(0.5, 1.0), lim(0.5, 1.0)])
        parts.append((foot, (-0.05, 0, 0), (0.15, 0, 0), 0.04))
        b.contact(foot, (-0.05, 0, 0), 0.04)
        b.contact(foot, (0.15, 0, 0), 0.04)
        uarm = chain(torso, (0, 0.17 * side, 0.15), [(1, 0, 0), (0, 1, 0)], [lim(0.8, 1.5), lim(0.8, 1.5)])
        parts.append((uarm, (0, 0, 0), (0, 0.05 * side, -0.28), 0.045))
        larm = chain(uarm, (0, 0.05 * side, -0.3), [(0, 1, 0)], [lim(1.0, 1.5)])
        parts.append((larm, (0, 0, 0), (0, 0, -0.25), 0.04))
        b.contact(larm, (0, 0, -0.25), 0.04)
    # masses: unit density, then scaled to the total
    raw = [capsule_mass_inertia(r, p0, p1, 1.0) for (_, p0, p1, r) in parts]
    scale = HUMANOID_TOTAL_MASS / sum(x[0] for x in raw)
    for (lk, _, _, _), (m, c, I) in zip(parts, raw):
        b.links[lk]["mass"] = m * scale
        b.links[lk]["com"] = c
        b.links[lk]["inertia"] = _sym6(I * scale)
    nv = 27
    n_act = 21
    # per-joint gears in 50..200 by joint kind (DOF order: waist 2, pelvis 1,
    # then per side thigh 3, shin 1, foot 2, upper arm 2, lower arm 1)
    side = [200.0] * 3 + [150.0] + [50.0] * 2 + [100.0] * 2 + [50.0]
    gears = np.array([200.0, 200.0, 200.0] + side + side)
    assert gears.size == n_act
    lowest = min(b.fixed_pose(lk)[1][2] + b.fixed_pose(lk)[0][2] @ p - r for (lk, p, r) in b.contacts)
    arm = np.full(nv, HUMANOID_ARMATURE)
    arm[:6] = 0.0
    damp = np.full(nv, HUMANOID_DAMPING)
    damp[:6] = 0.0
    return b.finish(root_z=-lowest - 0.002,
                    act_dof=list(range(6, 6 + n_act)), act_gear=gears, dt=CONTROL_DT,
                    substeps=substeps, ke=4e4, kd=1e3, kt=1e3, mu=0.75, k_limit=1e4,
                    armature=arm, damping=damp, rw_q=np.zeros(28), rw_qd=np.zeros(nv),
                    reward_coef=_loco_coef(0.0, 1.0, 0.0, 0.0, 0.0, -BIG, BIG, 0.0, 0.0, 0.0))


def mtu(substeps: int = 32, seed: int = 0, n_muscles: int = 152) -> ArticulationModel:
    """Muscle-actuated lower body: free pelvis + 8 bodies (per leg femur,
    tibia, talus, toes), 22 revolute DOFs (3+3+3+2 per leg), n_muscles
    line-of-action muscles with 2-4 via points fixed in adjacent or
    next-adjacent bodies, force = activation * Fmax, Fmax ~ U(200, 1500) N.
    4 contact spheres (heel and toe of each foot).  Reward: appendix A.3
    Humanoid MTU shape with h0 = 0.51 scaled to this model's pelvis height."""
    rng = np.random.default_rng(np.random.SeedSequence([2204, 7137, 5, seed]))
    b = _Builder("mtu")
    dens = 1000.0
    parts = []
    pelvis = b.link(-1, FREE)
    parts.append((pelvis, (0, -0.09, 0), (0, 0.09, 0), 0.08))
    bodies = [pelvis]     # massive bodies (muscle attachment candidates), in tree order
    body_parent = {pelvis: None}
    body_len = {pelvis: (np.array([0, -0.09, 0.0]), np.array([0, 0.09, 0.0]))}

    def chain(parent, pos, axes):
        cur = parent
        for j, ax in enumerate(axes):
            cur = b.link(cur, REVOLUTE, axis=ax, pos=pos if j == 0 else (0, 0, 0))
        return cur

    for side in (-1.0, 1.0):
        femur = chain(pelvis, (0, 0.09 * side, -0.02), [(1, 0, 0), (0, 0, 1), (0, 1, 0)])
        parts.append((femur, (0, 0, -0.02), (0, 0, -0.40), 0.06))
        tibia = chain(femur, (0, 0, -0.42), [(0, 1, 0), (1, 0, 0), (0, 0, 1)])
        parts.append((tibia, (0, 0, -0.02), (0, 0, -0.38), 0.05))
        talus = chain(tibia, (0, 0, -0.42), [(0, 1, 0), (1, 0, 0), (0, 0, 1)])
        parts.append((talus, (-0.05, 0, -0.03), (0.10, 0, -0.03), 0.04))
        toes = chain(talus, (0.12, 0, -0.03), [(0, 1, 0), (1, 0, 0)])
        parts.append((toes, (0.0, 0, 0.0), (0.06, 0, 0.0), 0.03))
        b.contact(talus, (-0.05, 0, -0.03), 0.04)
        b.contact(toes, (0.06, 0, 0.0), 0.03)
        for lk, par, seg in ((femur, pelvis, ((0, 0, -0.02), (0, 0, -0.40))),
                             (tibia, femur, ((0, 0, -0.02), (0, 0, -0.38))),
                             (talus, tibia, ((-0.05, 0, -0.03), (0.10, 0, -0.03))),
                             (toes, talus, ((0, 0, 0), (0.06, 0, 0)))):
            bodies.append(lk)
            body_parent[lk] = par
            body_len[lk] = (np.asarray(seg[0], np.float64), np.asarray(seg[1], np.float64))
    for (lk, p0, p1, r) in parts:
        m, c, I = capsule_mass_inertia(r, p0, p1, dens)
        b.links[lk]["mass"] = m
        b.links[lk]["com"] = c
        b.links[lk]["inertia"] = _sym6(I)

    def ancestors(body):
        out = []
        p = body_parent[body]
        while p is not None:
            out.append(p)
            p = body_parent[p]
        return out

    def via_on(body):
        p0, p1 = body_len[body]
        t = rng.uniform(0.1, 0.9)
        off = rng.uniform(-0.04, 0.04, size=3)
        return (body, p0 + t * (p1 - p0) + off)

    for _ in range(n_muscles):
        # pick a distal body and a proximal body one or two levels up
        while True:
            dist = bodies[int(rng.integers(1, len(bodies)))]
            anc = ancestors(dist)
            depth = int(rng.integers(1, 3))
            if len(anc) >= depth:
                prox = anc[depth - 1]
                break
        n_via = int(rng.integers(2, 5))
        path = [prox] + ([anc[0]] if depth == 2 else []) + [dist]
        vias = [via_on(path[0])]
        middle = n_via - 2
        for k in range(middle):
            vias.append(via_on(path[min(1 + k, len(path) - 1)] if len(path) > 2 else path[-1]))
        vias.append(via_on(path[-1]))
        b.muscle(float(rng.uniform(200.0, 1500.0)), vias)
    lowest = min(b.fixed_pose(lk)[1][2] + b.fixed_pose(lk)[0][2] @ p - r for (lk, p, r) in b.contacts)
    h0 = -lowest - 0.002 - 0.05
    arm = np.full(28, MTU_ARMATURE)
    arm[:6] = 0.0
    damp = np.full(28, MTU_DAMPING)
    damp[:6] = 0.0
    return b.finish(root_z=-lowest - 0.002,
                    act_dof=[], act_gear=[], dt=CONTROL_DT, substeps=substeps,
                    ke=4e4, kd=1e3, kt=1e3, mu=0.75, armature=arm, damping=damp,
                    rw_q=np.zeros(29), rw_qd=np.zeros(28),
                    reward_coef=_loco_coef(0.001, 1.0, 0.1, 1.0, h0, -1.0, 0.05, -200.0, 0.0, 4.0))


# ---------------------------------------------------------------------------
# Seeded window inputs
# ---------------------------------------------------------------------------

def _rng(*key):
    return np.random.default_rng(np.random.SeedSequence([2204, 7137] + [int(k) for k in key]))


def initial_state(model: ArticulationModel, n_envs: int, seed: int = 0,
                  joint_range: float | None = None) -> Tuple[np.ndarray, np.ndarray]:
    """q0 [nq, N], qd0 [nv, N] float32 (structure of arrays)."""
    rng = _rng(11, seed, model.nq, model.nv)
    nq, nv = model.nq, model.nv
    q = np.zeros((nq, n_envs), np.float64)
    qd = np.zeros((nv, n_envs), np.float64)
    if model.name == "cartpole":
        q[:] = rng.uniform(-0.1, 0.1, size=(nq, n_envs))
        qd[:] = rng.uniform(-0.1, 0.1, size=(nv, n_envs))
    elif int(model.joint_type[0]) != FREE:   # planar: x, z (height change), pitch, joints
        rng_j = 0.1 if joint_range is None else joint_range
        q[2:] = rng.uniform(-rng_j, rng_j, size=(nq - 2, n_envs))
        qd[:] = rng.uniform(-0.1, 0.1, size=(nv, n_envs))
    else:
        rng_j = 0.2 if model.name == "ant" else 0.1
        if joint_range is not None:
            rng_j = joint_range
        q[2] = model.root_z
        q[6] = 1.0
        q[7:] = rng.uniform(-rng_j, rng_j, size=(nq - 7, n_envs))
    return q.astype(np.float32), qd.astype(np.float32)


def window_actions(model: ArticulationModel, n_envs: int, h: int, seed: int = 0) -> np.ndarray:
    """Actions [h, na, N] float32: U(-1, 1) torques (times the model gear) or
    U(0, 1) muscle activations."""
    rng = _rng(13, seed, model.na, h)
    if model.n_muscles > 0 and model.n_tact == 0:
        a = rng.uniform(0.0, 1.0, size=(h, model.na, n_envs))
    else:
        a = rng.uniform(-1.0, 1.0, size=(h, model.na, n_envs))
    return a.astype(np.float32)


def random_state(model: ArticulationModel, n_envs: int, seed: int, pos_scale=0.5, vel_scale=1.0):
    """Generic random state (for pins and parity of free-flying cases):
    root anywhere, random unit quaternion, random joint angles and velocities."""
    rng = _rng(17, seed, model.nq)
    nq, nv = model.nq, model.nv
    q = np.zeros((nq, n_envs))
    qd = rng.uniform(-vel_scale, vel_scale, size=(nv, n_envs))
    qs = model.q_start()
    for i, t in enumerate(model.joint_type):
        s = qs[i]
        if t == FREE:
            q[s:s + 3] = rng.uniform(-pos_scale, pos_scale, size=(3, n_envs))
            qq = rng.normal(size=(4, n_envs))
            q[s + 3:s + 7] = qq / np.linalg.norm(qq, axis=0)
        elif t in (REVOLUTE, PRISMATIC):
            q[s] = rng.uniform(-pos_scale, pos_scale, size=n_envs)
    return q.astype(np.float32), qd.astype(np.float32)


# ---------------------------------------------------------------------------
# Workload configurations (the five evaluation workloads)
# ---------------------------------------------------------------------------

@dataclasses.dataclass
class Workload:
    name: str
    groups: List[Tuple[ArticulationModel, int]]
    h: int = 32

    @property
    def n_envs(self) -> int:
        return sum(n for _, n in self.groups)


def workload(name: str, scale: float = 1.0) -> Workload:
    """Named workloads; ``scale`` shrinks the env counts (for parity cases)."""
    def n(x):
        return max(1, int(round(x * scale)))
    if name == "cartpole-64":
        return Workload(name, [(cartpole(), n(64))])
    if name == "ant-2048":
        return Workload(name, [(ant(), n(2048))])
    if name == "humanoid-1024":
        return Workload(name, [(humanoid(), n(1024))])
    if name == "hetero-4096-2048-1024":
        return Workload(name, [(cartpole(), n(4096)), (ant(), n(2048)), (humanoid(), n(1024))])
    if name == "mtu-512":
        return Workload(name, [(mtu(), n(512))])
    if name == "halfcheetah-2048":
        return Workload(name, [(halfcheetah(), n(2048))])
    if name == "hopper-2048":
        return Workload(name, [(hopper(), n(2048))])
    raise KeyError(name)


WORKLOADS = ["cartpole-64", "ant-2048", "humanoid-1024", "hetero-4096-2048-1024", "mtu-512", "halfcheetah-2048",
             "hopper-2048"]

# Episode rules of the tasks (appendix A.3): root height below which the task
# terminates early (-inf: no early termination) and the task horizon in control
# steps.  The root of the ant-like model is the torso, of the humanoid-like model
# the torso, of the muscle model the pelvis; the planar models' root height is
# the height change of their z slide.
EPISODE_RULES = {"cartpole": (-np.inf, 240), "ant": (0.27, 1000), "humanoid": (0.74, 1000), "mtu": (0.46, 1000),
                 "halfcheetah": (-np.inf, 1000), "hopper": (-0.45, 1000)}


def episode_rule(model: ArticulationModel) -> Tuple[float, int]:
    """(termination height, task horizon) of a model built by this module."""
    return EPISODE_RULES[model.name]

