"""Window tape (the forward window keeps every substep record; the adjoint
reads them instead of recomputing): results bit for bit equal to the
recomputing adjoint, for single models, a heterogeneous batch and the
episodic window; step-level calls unaffected.  Parity of the recomputing
path with the FP64 oracle is covered in test_gpu_parity / test_gpu_episodic."""
import numpy as np
import pytest

from paper_2204_07137_gb300 import inputs as I

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2204_07137_gb300 import build
    build.build()


def _inputs(sim, groups, h, seed):
    q0 = sim.pack([I.initial_state(m, n, seed)[0] for m, n in groups], "q")
    qd0 = sim.pack([I.initial_state(m, n, seed)[1] for m, n in groups], "qd")
    act = torch.cat([torch.from_numpy(I.window_actions(m, n, h, seed).reshape(h, -1)) for m, n in groups],
                    dim=1).cuda().contiguous()
    g = torch.Generator(device="cuda").manual_seed(seed)
    rb = torch.randn(h, sim.n_envs, device="cuda", generator=g)
    qtb = 0.1 * torch.randn(h + 1, sim.q_size, device="cuda", generator=g)
    qdtb = 0.1 * torch.randn(h + 1, sim.qd_size, device="cuda", generator=g)
    return q0, qd0, act, rb, qtb, qdtb


@pytest.mark.parametrize("spec,h", [
    ([("ant", 37)], 5),
    ([("humanoid", 9)], 3),
    ([("mtu", 3)], 2),
    ([("hopper", 21)], 4),
    ([("cartpole", 40), ("ant", 13), ("humanoid", 5)], 3),
])
def test_taped_window_equals_recomputing_window(spec, h):
    from paper_2204_07137_gb300.sim import Simulator
    groups = [(getattr(I, name)(), n) for name, n in spec]
    ref = Simulator(groups, form="batched", h_max=h + 2)
    tap = Simulator(groups, form="batched", h_max=h + 2)
    small = tap.workspace.numel()
    tap.set_window_tape(True)
    assert tap.workspace.numel() > small
    q0, qd0, act, rb, qtb, qdtb = _inputs(ref, groups, h, seed=4)
    f1 = ref.window_forward(q0, qd0, act)
    a1 = ref.window_adjoint(f1[0], f1[1], act, rb, qtb, qdtb)
    f2 = tap.window_forward(q0, qd0, act)
    a2 = tap.window_adjoint(f2[0], f2[1], act, rb, qtb, qdtb)
    a3 = tap.window_adjoint(f2[0], f2[1], act, rb, qtb, qdtb)    # the tape is read, not consumed
    torch.cuda.synchronize()
    for x, y in zip(f1, f2):
        assert torch.equal(x, y)
    for x, y, z in zip(a1, a2, a3):
        assert torch.equal(x, y) and torch.equal(y, z)
    # step-level calls never touch the tape
    s1 = ref.step_adjoint(q0, qd0, act[0], qtb[1], qdtb[1], rb[0])
    s2 = tap.step_adjoint(q0, qd0, act[0], qtb[1], qdtb[1], rb[0])
    torch.cuda.synchronize()
    for x, y in zip(s1, s2):
        assert torch.equal(x, y)


def test_taped_episodic_window_equals_recomputing_one():
    from paper_2204_07137_gb300.sim import Simulator
    m, N, h = I.ant(), 29, 6
    groups = [(m, N)]
    ref = Simulator(groups, form="batched", h_max=h)
    tap = Simulator(groups, form="batched", h_max=h)
    tap.set_window_tape(True)
    q0, qd0, act, rb, qtb, qdtb = _inputs(ref, groups, h, seed=5)
    qr = ref.pack([I.initial_state(m, N, 6)[0]], "q")
    qdr = ref.pack([I.initial_state(m, N, 6)[1]], "qd")
    ep0 = torch.from_numpy(np.random.default_rng(0).integers(0, 4, N).astype(np.int32)).cuda()
    outs = []
    for sim in (ref, tap):
        ep = ep0.clone()
        f = sim.window_forward_episodic(q0, qd0, act, qr, qdr, [0.27], [4], ep)
        a = sim.window_adjoint_episodic(f[0], f[1], act, f[3], rb, qtb, qdtb)
        outs.append((f, a, ep))
    torch.cuda.synchronize()
    (f1, a1, e1), (f2, a2, e2) = outs
    assert int(f1[3].sum()) > 0 and torch.equal(e1, e2)
    for x, y in zip(tuple(f1) + tuple(a1), tuple(f2) + tuple(a2)):
        assert torch.equal(x, y)


def test_window_tape_is_batched_only():
    from paper_2204_07137_gb300 import _lib
    from paper_2204_07137_gb300.sim import Simulator
    sim = Simulator([(I.cartpole(), 4)], form="plain", h_max=2)
    with pytest.raises(_lib.ShacError, match="UNSUPPORTED"):
        sim.set_window_tape(True)
