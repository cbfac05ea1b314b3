"""The step adjoint for callers that cannot allocate device memory
(shac_step_adjoint_static): its scratch is a fixed array compiled into the
library instead of a caller workspace.  Checked through the C ABI against
shac_step_adjoint: both run the same kernels in the same launch shape on the
same inputs, so the results must agree bit for bit.  The array keeps the
previous call's contents; a first call on a larger batch with other inputs
fills it with different records, so stale contents would show in the next
results.  This file is collected last on purpose."""
import ctypes

import numpy as np
import pytest

from paper_2204_07137_gb300 import inputs as I

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def T(x):
    return torch.from_numpy(np.ascontiguousarray(np.asarray(x, np.float32).reshape(-1))).cuda()


def _inputs(m, N, seed):
    q, qd = I.initial_state(m, N, seed)
    a = I.window_actions(m, N, 1, seed)[0]
    rng = np.random.default_rng(seed)
    qb, qdb, rb = (rng.normal(size=s) for s in ((m.nq, N), (m.nv, N), N))
    # every buffer bound to a name that lives across the call
    return [T(x) for x in (q, qd, a, qb, qdb, rb)]


def _static_call(sim, inputs):
    from paper_2204_07137_gb300 import _lib
    stream = torch.cuda.current_stream()
    out = [torch.full((n,), float("nan"), device="cuda") for n in (sim.q_size, sim.qd_size, sim.act_size)]
    st = _lib.load().shac_step_adjoint_static(sim.batch, ctypes.c_void_p(stream.cuda_stream),
                                              *[ctypes.c_void_p(t.data_ptr()) for t in inputs],
                                              *[ctypes.c_void_p(t.data_ptr()) for t in out])
    assert st == 0, _lib.status_string(st)
    torch.cuda.synchronize()
    return out


def _workspace_call(sim, inputs):
    ref = sim.step_adjoint(*inputs)
    torch.cuda.synchronize()
    return ref


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2204_07137_gb300 import build
    build.build()


def test_static_scratch_step_adjoint_matches_workspace_version():
    from paper_2204_07137_gb300 import _lib
    from paper_2204_07137_gb300.sim import Simulator
    m = I.ant()
    # fill the array with another batch's records first
    big = Simulator([(m, 320)], form="batched", h_max=1)
    _static_call(big, _inputs(m, 320, 99))
    N = 96
    sim = Simulator([(m, N)], form="batched", h_max=1)
    assert _lib.load().shac_batch_workspace_bytes(sim.batch) <= 64 << 20
    for call, seed in enumerate((11, 12)):
        x = _inputs(m, N, seed)
        ref = _workspace_call(sim, x)
        got = _static_call(sim, x)
        for g, r, name in zip(got, ref, ("q_bar", "qd_bar", "act_bar")):
            assert torch.isfinite(r).all()
            np.testing.assert_array_equal(g.cpu().numpy(), r.cpu().numpy(), err_msg=f"call {call} {name}")


def test_static_scratch_ignores_the_window_tape():
    """With the window tape on, the workspace grows beyond the array, but step
    calls never use the tape: the call is accepted and matches bit for bit."""
    from paper_2204_07137_gb300 import _lib
    from paper_2204_07137_gb300.sim import Simulator
    m = I.ant()
    N = 512
    sim = Simulator([(m, N)], form="batched", h_max=32)
    sim.set_window_tape(True)
    assert _lib.load().shac_batch_workspace_bytes(sim.batch) > 64 << 20
    x = _inputs(m, N, 21)
    ref = _workspace_call(sim, x)
    got = _static_call(sim, x)
    for g, r in zip(got, ref):
        np.testing.assert_array_equal(g.cpu().numpy(), r.cpu().numpy())


def test_static_scratch_rejects_batches_beyond_its_size():
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
