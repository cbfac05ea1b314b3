"""The learner's observation vector against the sizes of the appendix A.3
observation tables (tests/golden/observation_sizes.txt).  The muscle model's
table describes the paper's own skeleton (22 angles, 18 velocities), not the
synthetic one here, and is not compared."""
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "observation_sizes.txt")


def _sizes():
    out = {}
    for ln in open(GOLDEN):
        ln = ln.strip()
        if not ln or ln.startswith("#"):
            continue
        task, rows, _, total = ln.split()
        assert sum(int(x) for x in rows.split("+")) == int(total)
        out[task] = int(total)
    return out


@pytest.mark.parametrize("task", ["cartpole", "halfcheetah", "hopper", "ant", "humanoid"])
def test_observation_size_matches_the_table(task):
    from paper_2204_07137_gb300 import inputs as I, shac
    m = getattr(I, task)()
    q, qd = I.initial_state(m, 3, 0)
    a = torch.zeros(3, m.na)
    o = shac.observation(m, torch.from_numpy(q), torch.from_numpy(qd), a)
    assert tuple(o.shape) == (3, _sizes()[task])


def test_planar_observation_leaves_out_the_forward_position():
    from paper_2204_07137_gb300 import inputs as I, shac
    m = I.hopper()
    q, qd = I.initial_state(m, 2, 1)
    o1 = shac.observation(m, torch.from_numpy(q), torch.from_numpy(qd))
    q[0] += np.float32(3.0)   # move forward along x
    o2 = shac.observation(m, torch.from_numpy(q), torch.from_numpy(qd))
    assert torch.equal(o1, o2)


def test_last_actions_are_observed_by_torque_models():
    from paper_2204_07137_gb300 import inputs as I, shac
    m = I.ant()
    q, qd = I.initial_state(m, 2, 1)
    a = torch.arange(2 * m.na, dtype=torch.float32).view(2, m.na)
    o = shac.observation(m, torch.from_numpy(q), torch.from_numpy(qd), a)
    assert torch.equal(o[:, -m.na:], a)
