"""The step adjoint for callers that cannot allocate device memory
(shac_step_adjoint_static): its scratch is a fixed array compiled into the
library instead of a caller workspace.  Checked through the C ABI against
shac_step_adjoint on two calls in a row (the array keeps the previous call's
contents, which must not leak into the next result).  This file is collected
last on purpose."""
import ctypes

import numpy as np
import pytest

from helpers import assert_grad_close
from paper_2204_07137_gb300 import inputs as I

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def test_static_scratch_step_adjoint_matches_workspace_version():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2204_07137_gb300 import _lib, build
    from paper_2204_07137_gb300.sim import Simulator
    build.build()
    L = _lib.load()
    m = I.ant()
    N = 96
    sim = Simulator([(m, N)], form="batched", h_max=1)
    assert _lib.load().shac_batch_workspace_bytes(sim.batch) <= 64 << 20
    T = lambda x: torch.from_numpy(np.ascontiguousarray(np.asarray(x, np.float32).reshape(-1))).cuda()
    stream = torch.cuda.current_stream()
    for call, seed in enumerate((11, 12)):
        q, qd = I.initial_state(m, N, seed)
        a = I.window_actions(m, N, 1, seed)[0]
        rng = np.random.default_rng(seed)
        qb, qdb, rb = (T(rng.normal(size=s)) for s in ((m.nq, N), (m.nv, N), N))
        ref = sim.step_adjoint(T(q), T(qd), T(a), qb, qdb, rb)
        out = [torch.full_like(r, float("nan")) for r in ref]
        st = L.shac_step_adjoint_static(sim.batch, ctypes.c_void_p(stream.cuda_stream),
                                        *[ctypes.c_void_p(t.data_ptr()) for t in (T(q), T(qd), T(a), qb, qdb, rb)],
                                        *[ctypes.c_void_p(t.data_ptr()) for t in out])
        assert st == 0, _lib.status_string(st)
        torch.cuda.synchronize()
        got = np.concatenate([out[0].cpu().numpy().reshape(m.nq, N), out[1].cpu().numpy().reshape(m.nv, N),
                              out[2].cpu().numpy().reshape(m.na, N)])
        exp = np.concatenate([ref[0].cpu().numpy().reshape(m.nq, N), ref[1].cpu().numpy().reshape(m.nv, N),
                              ref[2].cpu().numpy().reshape(m.na, N)])
        assert_grad_close(got, exp, f"static-scratch step adjoint, call {call}")


def test_static_scratch_rejects_batches_beyond_its_size():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2204_07137_gb300 import _lib
    from paper_2204_07137_gb300.sim import Simulator
    m = I.ant()
    sim = Simulator([(m, 4096)], form="batched", h_max=1)
    assert _lib.load().shac_batch_workspace_bytes(sim.batch) > 64 << 20
    z = torch.zeros(max(sim.q_size, sim.qd_size, sim.act_size, sim.n_envs), device="cuda")
    p = ctypes.c_void_p(z.data_ptr())
    st = _lib.load().shac_step_adjoint_static(sim.batch, ctypes.c_void_p(torch.cuda.current_stream().cuda_stream),
                                              *([p] * 9))
    assert st == 5   # SHAC_ERR_CAPACITY, nothing launched
