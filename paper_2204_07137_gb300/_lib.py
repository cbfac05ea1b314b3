"""ctypes binding of libshacsim.so (include/shacsim.h): argument marshalling only.

Every call here forwards to the C ABI with the same name; no step of the
simulator runs in Python.  Loading fails loudly if the library is missing:
there is no fallback path.
"""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libshacsim.so")

_i32p = ctypes.POINTER(ctypes.c_int32)
_f32p = ctypes.POINTER(ctypes.c_float)
_vp = ctypes.c_void_p

SHAC_OK = 0
STATUS_NAMES = {0: "SHAC_OK", 1: "SHAC_ERR_INVALID_ARG", 2: "SHAC_ERR_MODEL", 3: "SHAC_ERR_CUDA",
                4: "SHAC_ERR_NONFINITE", 5: "SHAC_ERR_CAPACITY", 6: "SHAC_ERR_UNSUPPORTED"}
FORM_PLAIN, FORM_BATCHED = 0, 1

# every symbol include/shacsim.h declares
EXPORTED = [
    "shac_model_create", "shac_model_destroy", "shac_model_dims", "shac_batch_create", "shac_batch_destroy",
    "shac_batch_dims", "shac_batch_workspace_bytes", "shac_step", "shac_step_adjoint", "shac_window_forward",
    "shac_window_adjoint", "shac_window_forward_episodic", "shac_window_adjoint_episodic", "shac_batch_set_launch",
    "shac_batch_get_launch", "shac_batch_set_window_tape", "shac_get_status", "shac_status_string",
    "shac_step_adjoint_static", "shac_td_lambda", "shac_autotune", "shac_autotune_workspace_bytes",
    "shac_batch_specialize",
]


class ShacModelDesc(ctypes.Structure):
    _fields_ = [
        ("n_links", ctypes.c_int32), ("parent", _i32p), ("joint_type", _i32p),
        ("joint_axis", _f32p), ("joint_pos", _f32p), ("joint_quat", _f32p),
        ("mass", _f32p), ("com", _f32p), ("inertia", _f32p),
        ("n_contacts", ctypes.c_int32), ("contact_link", _i32p), ("contact_pos", _f32p),
        ("contact_radius", _f32p),
        ("q_lower", _f32p), ("q_upper", _f32p), ("k_limit", ctypes.c_float),
        ("armature", _f32p), ("joint_damping", _f32p),
        ("n_tact", ctypes.c_int32), ("act_dof", _i32p), ("act_gear", _f32p),
        ("n_muscles", ctypes.c_int32), ("muscle_ptr", _i32p), ("via_link", _i32p), ("via_pos", _f32p),
        ("muscle_fmax", _f32p),
        ("dt", ctypes.c_float), ("substeps", ctypes.c_int32), ("gravity", ctypes.c_float * 3),
        ("ke", ctypes.c_float), ("kd", ctypes.c_float), ("kt", ctypes.c_float), ("mu", ctypes.c_float),
        ("rw_q", _f32p), ("rw_qd", _f32p), ("reward_coef", ctypes.c_float * 10),
        ("height_q", ctypes.c_int32), ("vx_dof", ctypes.c_int32),
    ]


class ShacError(RuntimeError):
    def __init__(self, status: int, where: str):
        super().__init__(f"{where}: {STATUS_NAMES.get(status, status)} ({status_string(status)})")
        self.status = status


_lib = None


def load(path: str = LIB_PATH):
    """Load the CUDA library (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"libshacsim.so not found at {path}; run paper_2204_07137_gb300.build.build()")
    L = ctypes.CDLL(path)
    L.shac_model_create.argtypes = [ctypes.POINTER(ShacModelDesc), ctypes.POINTER(_vp)]
    L.shac_model_create.restype = ctypes.c_int
    L.shac_model_destroy.argtypes = [_vp]
    L.shac_model_destroy.restype = None
    L.shac_model_dims.argtypes = [_vp, _i32p, _i32p, _i32p]
    L.shac_model_dims.restype = None
    L.shac_batch_create.argtypes = [ctypes.POINTER(_vp), _i32p, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                    ctypes.POINTER(_vp)]
    L.shac_batch_create.restype = ctypes.c_int
    L.shac_batch_destroy.argtypes = [_vp]
    L.shac_batch_destroy.restype = None
    i64p = ctypes.POINTER(ctypes.c_int64)
    L.shac_batch_dims.argtypes = [_vp, i64p, i64p, i64p, i64p]
    L.shac_batch_dims.restype = None
    L.shac_batch_workspace_bytes.argtypes = [_vp]
    L.shac_batch_workspace_bytes.restype = ctypes.c_size_t
    L.shac_step.argtypes = [_vp, _vp, _vp] + [_vp] * 6
    L.shac_step.restype = ctypes.c_int
    L.shac_step_adjoint.argtypes = [_vp, _vp, _vp] + [_vp] * 9
    L.shac_step_adjoint.restype = ctypes.c_int
    L.shac_step_adjoint_static.argtypes = [_vp, _vp] + [_vp] * 9
    L.shac_step_adjoint_static.restype = ctypes.c_int
    L.shac_window_forward.argtypes = [_vp, _vp, _vp, ctypes.c_int32] + [_vp] * 6
    L.shac_window_forward.restype = ctypes.c_int
    L.shac_window_adjoint.argtypes = [_vp, _vp, _vp, ctypes.c_int32] + [_vp] * 9
    L.shac_window_adjoint.restype = ctypes.c_int
    L.shac_window_forward_episodic.argtypes = [_vp, _vp, _vp, ctypes.c_int32] + [_vp] * 12
    L.shac_window_forward_episodic.restype = ctypes.c_int
    L.shac_window_adjoint_episodic.argtypes = [_vp, _vp, _vp, ctypes.c_int32] + [_vp] * 10
    L.shac_window_adjoint_episodic.restype = ctypes.c_int
    L.shac_batch_set_launch.argtypes = [_vp, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32]
    L.shac_batch_set_launch.restype = ctypes.c_int
    L.shac_td_lambda.argtypes = [_vp, ctypes.c_int32, ctypes.c_int64, _vp, _vp, _vp, ctypes.c_float, ctypes.c_float,
                                 _vp]
    L.shac_td_lambda.restype = ctypes.c_int
    L.shac_batch_set_window_tape.argtypes = [_vp, ctypes.c_int32]
    L.shac_batch_set_window_tape.restype = ctypes.c_int
    L.shac_autotune.argtypes = [_vp, _vp, _vp, ctypes.c_int32, _vp, _vp, _vp]
    L.shac_autotune.restype = ctypes.c_int
    L.shac_batch_specialize.argtypes = [_vp, ctypes.c_int32]
    L.shac_batch_specialize.restype = ctypes.c_int
    L.shac_autotune_workspace_bytes.argtypes = [_vp]
    L.shac_autotune_workspace_bytes.restype = ctypes.c_size_t
    L.shac_batch_get_launch.argtypes = [_vp, ctypes.c_int32, _i32p, _i32p]
    L.shac_batch_get_launch.restype = ctypes.c_int
    L.shac_get_status.argtypes = [_vp, _vp, ctypes.POINTER(ctypes.c_uint32), ctypes.c_int32]
    L.shac_get_status.restype = ctypes.c_int
    L.shac_status_string.argtypes = [ctypes.c_int]
    L.shac_status_string.restype = ctypes.c_char_p
    _lib = L
    return L


def status_string(status: int) -> str:
    try:
        return load().shac_status_string(int(status)).decode()
    except Exception:  # library not loadable: still give a readable message
        return STATUS_NAMES.get(status, str(status))


def check(status: int, where: str) -> None:
    if status != SHAC_OK:
        raise ShacError(status, where)


class ModelHandle:
    """A shac_model created from an ``inputs.ArticulationModel``."""

    def __init__(self, model):
        import numpy as np
        L = load()
        keep = []

        def f(x, n_min=1):
            a = np.ascontiguousarray(np.asarray(x, np.float32).reshape(-1))
            if a.size < n_min:
                a = np.zeros(n_min, np.float32)
            keep.append(a)
            return a.ctypes.data_as(_f32p)

        def i(x, n_min=1):
            a = np.ascontiguousarray(np.asarray(x, np.int32).reshape(-1))
            if a.size < n_min:
                a = np.zeros(n_min, np.int32)
            keep.append(a)
            return a.ctypes.data_as(_i32p)

        m = model
        d = ShacModelDesc()
        d.n_links = m.n_links
        d.parent, d.joint_type = i(m.parent), i(m.joint_type)
        d.joint_axis, d.joint_pos, d.joint_quat = f(m.joint_axis), f(m.joint_pos), f(m.joint_quat)
        d.mass, d.com, d.inertia = f(m.mass), f(m.com), f(m.inertia)
        d.n_contacts = m.n_contacts
        d.contact_link, d.contact_pos, d.contact_radius = i(m.contact_link), f(m.contact_pos), f(m.contact_radius)
        d.q_lower, d.q_upper, d.k_limit = f(m.q_lower), f(m.q_upper), float(m.k_limit)
        d.armature, d.joint_damping = f(m.armature), f(m.damping)
        d.n_tact = m.n_tact
        d.act_dof, d.act_gear = i(m.act_dof), f(m.act_gear)
        d.n_muscles = m.n_muscles
        d.muscle_ptr, d.via_link, d.via_pos, d.muscle_fmax = i(m.muscle_ptr), i(m.via_link), f(m.via_pos), f(m.muscle_fmax)
        d.dt, d.substeps = float(m.dt), int(m.substeps)
        for k in range(3):
            d.gravity[k] = float(m.gravity[k])
        d.ke, d.kd, d.kt, d.mu = float(m.ke), float(m.kd), float(m.kt), float(m.mu)
        d.rw_q, d.rw_qd = f(m.rw_q), f(m.rw_qd)
        for k in range(10):
            d.reward_coef[k] = float(m.reward_coef[k])
        d.height_q = int(m.height_q)
        d.vx_dof = int(m.vx_dof)
        h = _vp()
        check(L.shac_model_create(ctypes.byref(d), ctypes.byref(h)), "shac_model_create")
        self.handle = h
        self.model = model
        nq, nv, na = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
        L.shac_model_dims(h, ctypes.byref(nq), ctypes.byref(nv), ctypes.byref(na))
        self.nq, self.nv, self.na = nq.value, nv.value, na.value

    def __del__(self):
        try:
            if self.handle:
                load().shac_model_destroy(self.handle)
                self.handle = None
        except Exception:
            pass


def ptr(t) -> int:
    """Device pointer of a torch tensor (or 0 for None)."""
    return 0 if t is None else int(t.data_ptr())
