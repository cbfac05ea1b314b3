"""PyTorch-facing API of the GB300 simulator (thin wrapper over libshacsim.so).

PyTorch supplies device memory and streams; every stage of the step and of its
adjoint runs in the library's CUDA kernels.  Arrays are flat structure-of-arrays
buffers (see include/shacsim.h): a state block is the concatenation over groups
of [dim][N_g]; trajectories add a leading time axis.
"""
from __future__ import annotations

import ctypes
from typing import List, Sequence, Tuple

import numpy as np
import torch

from . import _lib

FORMS = {"plain": _lib.FORM_PLAIN, "batched": _lib.FORM_BATCHED}


class Simulator:
    """A batch of articulation groups on the current CUDA device.

    groups: sequence of (inputs.ArticulationModel, n_envs).
    form:   "batched" (fused persistent kernel) or "plain" (thread per env,
            kernel per stage per substep).
    """

    def __init__(self, groups: Sequence[Tuple[object, int]], form: str = "batched", h_max: int = 32,
                 device=None):
        if not torch.cuda.is_available():
            raise RuntimeError("the simulator needs a CUDA device")
        self.device = torch.device("cuda", torch.cuda.current_device()) if device is None else torch.device(device)
        L = _lib.load()
        self.groups = [(m, int(n)) for m, n in groups]
        self.form = form
        self.h_max = int(h_max)
        self._models = [_lib.ModelHandle(m) for m, _ in self.groups]
        handles = (ctypes.c_void_p * len(self._models))(*[mh.handle.value for mh in self._models])
        counts = (ctypes.c_int32 * len(self._models))(*[n for _, n in self.groups])
        b = ctypes.c_void_p()
        with torch.cuda.device(self.device):
            _lib.check(L.shac_batch_create(handles, counts, len(self._models), FORMS[form], self.h_max,
                                           ctypes.byref(b)), "shac_batch_create")
        self.batch = b
        qs, qds, acs, ne = (ctypes.c_int64() for _ in range(4))
        L.shac_batch_dims(b, ctypes.byref(qs), ctypes.byref(qds), ctypes.byref(acs), ctypes.byref(ne))
        self.q_size, self.qd_size, self.act_size, self.n_envs = qs.value, qds.value, acs.value, ne.value
        self._alloc_workspace()

    def _alloc_workspace(self):
        nbytes = int(_lib.load().shac_batch_workspace_bytes(self.batch))
        self.workspace = torch.empty(max(nbytes, 256), dtype=torch.uint8, device=self.device)
        assert self.workspace.data_ptr() % 256 == 0

    def __del__(self):
        try:
            if getattr(self, "batch", None):
                _lib.load().shac_batch_destroy(self.batch)
                self.batch = None
        except Exception:
            pass

    # ------------------------------------------------------------ launches --
    def set_launch(self, group: int = -1, lanes_per_env: int = 0, warps_per_cta: int = 0):
        _lib.check(_lib.load().shac_batch_set_launch(self.batch, group, lanes_per_env, warps_per_cta),
                   "shac_batch_set_launch")
        self._alloc_workspace()

    def set_window_tape(self, keep: bool = True):
        """Keep every substep record of the forward window for the window
        adjoint (no recompute; much larger workspace; see shacsim.h for the
        contract: the adjoint must follow its forward on the same buffers)."""
        _lib.check(_lib.load().shac_batch_set_window_tape(self.batch, int(bool(keep))), "shac_batch_set_window_tape")
        self._alloc_workspace()

    def autotune_native(self, budget_ms: int = 2000, stream=None, q0=None, qd0=None, act=None):
        """The library's own measured launch-shape search (shac_autotune):
        lanes per environment for each group, then warps per CTA, timed as short
        windows (min(h_max, 8) steps) from q0, qd0 with actions act (CUDA float32
        tensors in the window calls' layouts; act's first min(h_max, 8) steps are
        used), or from the rest configuration where one is None; the fastest
        shape stays applied (after specialize(): the team size stays, the warps
        per CTA are searched with the specialised kernels).  The search's buffers
        are a temporary torch allocation of shac_autotune_workspace_bytes.
        Synchronises; not for a stream capture."""
        L = _lib.load()
        h = min(self.h_max, 8)

        def ptr(t, n):
            if t is None:
                return None
            t = t.reshape(-1)
            if t.dtype != torch.float32 or not t.is_cuda or not t.is_contiguous() or t.numel() < n:
                raise ValueError("autotune inputs must be contiguous CUDA float32 tensors of the window layout")
            return ctypes.c_void_p(t.data_ptr())
        args = (ptr(q0, self.q_size), ptr(qd0, self.qd_size), ptr(act, h * self.act_size))
        nbytes = int(L.shac_autotune_workspace_bytes(self.batch))
        tmp = torch.empty(max(nbytes, 256), dtype=torch.uint8, device=self.device)
        assert tmp.data_ptr() % 256 == 0
        _lib.check(L.shac_autotune(self.batch, self._stream(stream), ctypes.c_void_p(tmp.data_ptr()), int(budget_ms),
                                   *args), "shac_autotune")
        del tmp
        self._alloc_workspace()
        return [self.get_launch(g) for g in range(len(self.groups))]

    def specialize(self, enable: bool = True):
        """Use (or stop using) batched kernels compiled at run time for this
        batch's model and current team size (shac_batch_specialize): a few
        seconds the first time per model layout and team size in a process.
        Single-group batched simulators only."""
        _lib.check(_lib.load().shac_batch_specialize(self.batch, int(bool(enable))), "shac_batch_specialize")

    def get_launch(self, group: int) -> Tuple[int, int]:
        l, w = ctypes.c_int32(), ctypes.c_int32()
        _lib.check(_lib.load().shac_batch_get_launch(self.batch, group, ctypes.byref(l), ctypes.byref(w)),
                   "shac_batch_get_launch")
        return l.value, w.value

    def _stream(self, stream=None):
        s = torch.cuda.current_stream(self.device) if stream is None else stream
        return ctypes.c_void_p(s.cuda_stream)

    def _ws(self):
        return ctypes.c_void_p(self.workspace.data_ptr())

    def _check(self, t, n, name):
        if t is None:
            raise ValueError(f"{name} is required")
        if not (t.is_cuda and t.dtype == torch.float32 and t.is_contiguous() and t.numel() == n):
            raise ValueError(f"{name}: expected contiguous float32 CUDA tensor with {n} elements, "
                             f"got {tuple(t.shape)} {t.dtype} {t.device}")
        return ctypes.c_void_p(t.data_ptr())

    # ----------------------------------------------------------- C-ABI calls --
    def step(self, q, qd, act, out=None, stream=None):
        """One control step -> (q_next, qd_next, reward)."""
        if out is None:
            out = (torch.empty(self.q_size, device=self.device), torch.empty(self.qd_size, device=self.device),
                   torch.empty(self.n_envs, device=self.device))
        args = [self._check(q, self.q_size, "q"), self._check(qd, self.qd_size, "qd"),
                self._check(act, self.act_size, "act"), self._check(out[0], self.q_size, "q_next"),
                self._check(out[1], self.qd_size, "qd_next"), self._check(out[2], self.n_envs, "reward")]
        _lib.check(_lib.load().shac_step(self.batch, self._stream(stream), self._ws(), *args), "shac_step")
        return out

    def step_adjoint(self, q, qd, act, q_next_bar, qd_next_bar, reward_bar, out=None, stream=None):
        """Eq. backward for one step -> (q_bar, qd_bar, act_bar)."""
        if out is None:
            out = (torch.empty(self.q_size, device=self.device), torch.empty(self.qd_size, device=self.device),
                   torch.empty(self.act_size, device=self.device))
        args = [self._check(q, self.q_size, "q"), self._check(qd, self.qd_size, "qd"),
                self._check(act, self.act_size, "act"), self._check(q_next_bar, self.q_size, "q_next_bar"),
                self._check(qd_next_bar, self.qd_size, "qd_next_bar"),
                self._check(reward_bar, self.n_envs, "reward_bar"),
                self._check(out[0], self.q_size, "q_bar"), self._check(out[1], self.qd_size, "qd_bar"),
                self._check(out[2], self.act_size, "act_bar")]
        _lib.check(_lib.load().shac_step_adjoint(self.batch, self._stream(stream), self._ws(), *args),
                   "shac_step_adjoint")
        return out

    def window_forward(self, q0, qd0, act, out=None, stream=None):
        """act [h, act_size] -> (q_traj [h+1, q_size], qd_traj, reward [h, n_envs])."""
        h = int(act.shape[0])
        if out is None:
            out = (torch.empty(h + 1, self.q_size, device=self.device),
                   torch.empty(h + 1, self.qd_size, device=self.device),
                   torch.empty(h, self.n_envs, device=self.device))
        args = [self._check(q0, self.q_size, "q0"), self._check(qd0, self.qd_size, "qd0"),
                self._check(act, h * self.act_size, "act"), self._check(out[0], (h + 1) * self.q_size, "q_traj"),
                self._check(out[1], (h + 1) * self.qd_size, "qd_traj"),
                self._check(out[2], h * self.n_envs, "reward")]
        _lib.check(_lib.load().shac_window_forward(self.batch, self._stream(stream), self._ws(), h, *args),
                   "shac_window_forward")
        return out

    def window_adjoint(self, q_traj, qd_traj, act, reward_bar, q_traj_bar, qd_traj_bar, out=None, stream=None):
        """Reverse over the window -> (q0_bar, qd0_bar, act_bar [h, act_size])."""
        h = int(act.shape[0])
        if out is None:
            out = (torch.empty(self.q_size, device=self.device), torch.empty(self.qd_size, device=self.device),
                   torch.empty(h, self.act_size, device=self.device))
        args = [self._check(q_traj, (h + 1) * self.q_size, "q_traj"),
                self._check(qd_traj, (h + 1) * self.qd_size, "qd_traj"),
                self._check(act, h * self.act_size, "act"), self._check(reward_bar, h * self.n_envs, "reward_bar"),
                self._check(q_traj_bar, (h + 1) * self.q_size, "q_traj_bar"),
                self._check(qd_traj_bar, (h + 1) * self.qd_size, "qd_traj_bar"),
                self._check(out[0], self.q_size, "q0_bar"), self._check(out[1], self.qd_size, "qd0_bar"),
                self._check(out[2], h * self.act_size, "act_bar")]
        _lib.check(_lib.load().shac_window_adjoint(self.batch, self._stream(stream), self._ws(), h, *args),
                   "shac_window_adjoint")
        return out

    def window_forward_episodic(self, q0, qd0, act, q_reset, qd_reset, term_height, max_episode_steps,
                                episode_step, out=None, stream=None):
        """Window with early termination and reset (see shacsim.h).
        term_height, max_episode_steps: one value per group (-inf / 0: no such
        rule); episode_step: int32 CUDA tensor [n_envs], updated in place.
        -> (q_traj [h+1, q_size], qd_traj, reward [h, n_envs], done uint8 [h, n_envs])."""
        h = int(act.shape[0])
        if out is None:
            out = (torch.empty(h + 1, self.q_size, device=self.device),
                   torch.empty(h + 1, self.qd_size, device=self.device),
                   torch.empty(h, self.n_envs, device=self.device),
                   torch.empty(h, self.n_envs, dtype=torch.uint8, device=self.device))
        if not (episode_step.is_cuda and episode_step.dtype == torch.int32 and episode_step.is_contiguous()
                and episode_step.numel() == self.n_envs):
            raise ValueError(f"episode_step: expected contiguous int32 CUDA tensor with {self.n_envs} elements")
        d = out[3]
        if not (d.is_cuda and d.dtype == torch.uint8 and d.is_contiguous() and d.numel() == h * self.n_envs):
            raise ValueError(f"done: expected contiguous uint8 CUDA tensor with {h * self.n_envs} elements")
        th, hz = list(term_height), list(max_episode_steps)
        if len(th) != len(self.groups) or len(hz) != len(self.groups):
            raise ValueError(f"term_height, max_episode_steps: expected {len(self.groups)} values (one per group)")
        th_c = (ctypes.c_float * len(th))(*[float(x) for x in th])
        hz_c = (ctypes.c_int32 * len(hz))(*[int(x) for x in hz])
        args = [self._check(q0, self.q_size, "q0"), self._check(qd0, self.qd_size, "qd0"),
                self._check(act, h * self.act_size, "act"), self._check(q_reset, self.q_size, "q_reset"),
                self._check(qd_reset, self.qd_size, "qd_reset"), ctypes.cast(th_c, ctypes.c_void_p),
                ctypes.cast(hz_c, ctypes.c_void_p), ctypes.c_void_p(episode_step.data_ptr()),
                self._check(out[0], (h + 1) * self.q_size, "q_traj"),
                self._check(out[1], (h + 1) * self.qd_size, "qd_traj"),
                self._check(out[2], h * self.n_envs, "reward"), ctypes.c_void_p(d.data_ptr())]
        _lib.check(_lib.load().shac_window_forward_episodic(self.batch, self._stream(stream), self._ws(), h, *args),
                   "shac_window_forward_episodic")
        return out

    def window_adjoint_episodic(self, q_traj, qd_traj, act, done, reward_bar, q_traj_bar, qd_traj_bar, out=None,
                                stream=None):
        """Reverse of an episodic window: no gradient crosses a reset (done mask
        of the forward) -> (q0_bar, qd0_bar, act_bar [h, act_size])."""
        h = int(act.shape[0])
        if out is None:
            out = (torch.empty(self.q_size, device=self.device), torch.empty(self.qd_size, device=self.device),
                   torch.empty(h, self.act_size, device=self.device))
        if not (done.is_cuda and done.dtype == torch.uint8 and done.is_contiguous() and done.numel() == h * self.n_envs):
            raise ValueError(f"done: expected contiguous uint8 CUDA tensor with {h * self.n_envs} elements")
        args = [self._check(q_traj, (h + 1) * self.q_size, "q_traj"),
                self._check(qd_traj, (h + 1) * self.qd_size, "qd_traj"),
                self._check(act, h * self.act_size, "act"), ctypes.c_void_p(done.data_ptr()),
                self._check(reward_bar, h * self.n_envs, "reward_bar"),
                self._check(q_traj_bar, (h + 1) * self.q_size, "q_traj_bar"),
                self._check(qd_traj_bar, (h + 1) * self.qd_size, "qd_traj_bar"),
                self._check(out[0], self.q_size, "q0_bar"), self._check(out[1], self.qd_size, "qd0_bar"),
                self._check(out[2], h * self.act_size, "act_bar")]
        _lib.check(_lib.load().shac_window_adjoint_episodic(self.batch, self._stream(stream), self._ws(), h, *args),
                   "shac_window_adjoint_episodic")
        return out

    def status(self, clear: bool = False, stream=None) -> int:
        """Sticky device flags (bit 0: a non-finite state was produced). Synchronises."""
        v = ctypes.c_uint32()
        st = _lib.load().shac_get_status(self.batch, self._stream(stream), ctypes.byref(v), int(clear))
        if st not in (_lib.SHAC_OK, 4):
            _lib.check(st, "shac_get_status")
        return v.value

    # ------------------------------------------------------------- layout --
    def pack(self, per_group: List[np.ndarray], kind: str) -> torch.Tensor:
        """Concatenate per-group [dim_g, N_g] arrays into one flat device block."""
        parts = [np.asarray(a, np.float32).reshape(-1) for a in per_group]
        return torch.from_numpy(np.concatenate(parts)).to(self.device)

    def dims(self, kind: str) -> List[int]:
        attr = {"q": "nq", "qd": "nv", "act": "na"}[kind]
        return [getattr(m, attr) for m, _ in self.groups]

    def unpack(self, flat, kind: str) -> List[np.ndarray]:
        """Split a flat block (numpy or tensor; leading axes kept) into per-group [.., dim_g, N_g]."""
        x = flat.detach().cpu().numpy() if isinstance(flat, torch.Tensor) else np.asarray(flat)
        out, off = [], 0
        for (m, n), d in zip(self.groups, self.dims(kind)):
            out.append(x[..., off:off + d * n].reshape(x.shape[:-1] + (d, n)))
            off += d * n
        return out


def episode_discounts(done: torch.Tensor, gamma: float) -> torch.Tensor:
    """Reward weights gamma^(t - t0) of the policy loss (Eq. policy_loss) with the
    discount restarted after every reset (Sec. 3.2): done [h, N] (uint8, from
    window_forward_episodic) -> [h, N] float32 whose row 0 is all ones and
    whose row t + 1 is 1 where step t ended an episode, else gamma x row t."""
    h = int(done.shape[0])
    w = torch.ones(tuple(done.shape), dtype=torch.float32, device=done.device)
    for t in range(1, h):
        w[t] = torch.where(done[t - 1].bool(), torch.ones_like(w[t]), w[t - 1] * gamma)
    return w


# ------------------------------------------------------------ autograd --

class SimStep(torch.autograd.Function):
    """s_{t+1}, r_t = F(s_t, a_t) as a differentiable layer (appendix A.1):
    backward is the library's step adjoint (Eq. backward)."""

    @staticmethod
    def forward(ctx, sim: Simulator, q, qd, act):
        q, qd, act = q.contiguous(), qd.contiguous(), act.contiguous()
        stream = torch.cuda.current_stream(sim.device)
        qn, qdn, r = sim.step(q, qd, act, stream=stream)
        ctx.sim = sim
        ctx.stream = stream
        ctx.save_for_backward(q, qd, act)
        return qn, qdn, r

    @staticmethod
    def backward(ctx, gq, gqd, gr):
        sim = ctx.sim
        q, qd, act = ctx.saved_tensors
        # the adjoint runs on the forward's stream (also inside a graph capture)
        with torch.cuda.stream(ctx.stream):
            z = lambda n, g: torch.zeros(n, device=sim.device) if g is None else g.contiguous()
            qb, qdb, ab = sim.step_adjoint(q, qd, act, z(sim.q_size, gq), z(sim.qd_size, gqd), z(sim.n_envs, gr),
                                           stream=ctx.stream)
        return None, qb, qdb, ab


class SimWindow(torch.autograd.Function):
    """A whole open-loop window: forward writes the per-step checkpoints (the
    tape), backward recomputes substeps from them (window adjoint)."""

    @staticmethod
    def forward(ctx, sim: Simulator, q0, qd0, act):
        q0, qd0, act = q0.contiguous(), qd0.contiguous(), act.contiguous()
        stream = torch.cuda.current_stream(sim.device)
        q_traj, qd_traj, rew = sim.window_forward(q0, qd0, act, stream=stream)
        ctx.sim = sim
        ctx.stream = stream
        ctx.save_for_backward(q_traj, qd_traj, act)
        return q_traj, qd_traj, rew

    @staticmethod
    def backward(ctx, gq, gqd, gr):
        sim = ctx.sim
        q_traj, qd_traj, act = ctx.saved_tensors
        h = act.shape[0]
        with torch.cuda.stream(ctx.stream):
            gq = torch.zeros_like(q_traj) if gq is None else gq.contiguous()
            gqd = torch.zeros_like(qd_traj) if gqd is None else gqd.contiguous()
            gr = torch.zeros(h, sim.n_envs, device=sim.device) if gr is None else gr.contiguous()
            q0b, qd0b, ab = sim.window_adjoint(q_traj, qd_traj, act, gr, gq, gqd, stream=ctx.stream)
        return None, q0b, qd0b, ab
