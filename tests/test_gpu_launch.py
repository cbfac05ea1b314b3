"""Launch shapes of the batched kernels from a fresh CUDA context.

Shared memory per CTA grows with the warps per CTA; between 44 and 48 KB of
dynamic shared memory the kernels' static part pushes a CTA over the default
48 KB and the opt-in attribute is required.  Attributes persist in a process,
so the sweep runs in a fresh child process, smallest CTA first."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r"""
import sys, numpy as np, torch
sys.path.insert(0, sys.argv[1])
from paper_2204_07137_gb300 import inputs as I
from paper_2204_07137_gb300.sim import Simulator
T = lambda x: torch.from_numpy(np.ascontiguousarray(np.asarray(x, np.float32).reshape(-1))).cuda()
for name in ("ant", "humanoid", "mtu"):
    m = getattr(I, name)()
    for warps in range(1, 9):
        N = 8 * warps + 3
        sim = Simulator([(m, N)], form="batched", h_max=1)
        sim.set_launch(0, 0, warps)
        lanes, w_used = sim.get_launch(0)
        q0, qd0 = I.initial_state(m, N, 0)
        act = T(I.window_actions(m, N, 1, 0)).view(1, -1)
        qt, qdt, r = sim.window_forward(T(q0), T(qd0), act)
        g = sim.window_adjoint(qt, qdt, act, torch.ones(1, N, device="cuda"),
                               torch.zeros_like(qt), torch.zeros_like(qdt))
        torch.cuda.synchronize()
        assert all(torch.isfinite(x).all() for x in (qt, qdt, r) + tuple(g)), (name, warps)
        print(name, warps, lanes, w_used)
print("ok")
"""


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2204_07137_gb300 import build
    build.build()


def test_every_cta_size_launches_in_a_fresh_context():
    out = subprocess.run([sys.executable, "-c", CHILD, ROOT], capture_output=True, text=True, timeout=600)
    assert out.returncode == 0, out.stdout[-2000:] + out.stderr[-4000:]
    assert out.stdout.strip().endswith("ok")


LANES = (1, 2, 4, 8, 16, 32)
WARPS = (1, 2, 4, 8)


def _window_inputs(sim, h):
    from paper_2204_07137_gb300 import inputs as I
    q0 = sim.pack([I.initial_state(m, n, 0)[0] for m, n in sim.groups], "q")
    qd0 = sim.pack([I.initial_state(m, n, 0)[1] for m, n in sim.groups], "qd")
    act = torch.cat([torch.from_numpy(I.window_actions(m, n, h, 0).reshape(h, -1)) for m, n in sim.groups],
                    dim=1).cuda().contiguous()
    return q0, qd0, act


@pytest.mark.parametrize("tape", [False, True])
def test_native_autotune_keeps_a_valid_shape(tape):
    """shac_autotune (the library's measured search) on a heterogeneous batch,
    with and without the window tape (timed from the caller's window inputs
    with the tape, from the rest configuration without): a valid shape is left
    applied, the windows it times (in the caller's buffer of
    shac_autotune_workspace_bytes) do not disturb the caller's inputs, and the
    retuned batch gives the same
    window up to FP32 reassociation inside a team; a non-positive budget is
    rejected."""
    import numpy as np
    from paper_2204_07137_gb300 import _lib
    from paper_2204_07137_gb300.sim import Simulator
    groups = [(_inputs().cartpole(), 40), (_inputs().ant(), 13)]
    tuned = Simulator(groups, form="batched", h_max=2)
    ref = Simulator(groups, form="batched", h_max=2)
    if tape:
        tuned.set_window_tape(True)
        ref.set_window_tape(True)
    L = _lib.load()
    assert L.shac_autotune_workspace_bytes(tuned.batch) > L.shac_batch_workspace_bytes(tuned.batch)
    q0, qd0, act = _window_inputs(ref, 2)
    keep = [t.clone() for t in (q0, qd0, act)]
    shapes = tuned.autotune_native(budget_ms=5000, **({"q0": q0, "qd0": qd0, "act": act} if tape else {}))
    assert len(shapes) == 2
    assert all(l in LANES and w in WARPS for l, w in shapes)
    assert all(torch.equal(a, b) for a, b in zip(keep, (q0, qd0, act)))
    a = tuned.window_forward(q0, qd0, act)
    b = ref.window_forward(q0, qd0, act)
    torch.cuda.synchronize()
    for u, v in zip(a, b):
        np.testing.assert_allclose(u.cpu().numpy(), v.cpu().numpy(), rtol=1e-4, atol=1e-3)
    assert tuned.status() == 0
    with pytest.raises(_lib.ShacError) as e:
        tuned.autotune_native(budget_ms=0)
    assert e.value.status == 1


def _inputs():
    from paper_2204_07137_gb300 import inputs
    return inputs
