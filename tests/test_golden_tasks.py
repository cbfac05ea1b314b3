"""Task horizons, early-termination heights and reward constants of the
synthetic models against appendix A.3 (tests/golden/task_rules.txt).  The
reward vector is r = -c0 |a|^2 + c1 vx + c2 up + c3 heading +
Rh(clip(z - c4, c5, c6)), Rh(D) = c7 D^2 + c8 D (D < 0), c9 D (D >= 0)."""
import math
import os

import pytest

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "task_rules.txt")


def _rules():
    out = {}
    for ln in open(GOLDEN):
        ln = ln.strip()
        if not ln or ln.startswith("#"):
            continue
        task, key, val = ln.split()
        out.setdefault(task, {})[key] = None if val == "none" else float(val)
    return out


@pytest.mark.parametrize("task", ["cartpole", "halfcheetah", "hopper", "ant", "humanoid", "mtu"])
def test_horizon_and_termination(task):
    from paper_2204_07137_gb300 import inputs as I
    rule = _rules()[task]
    height, horizon = I.episode_rule(getattr(I, task)())
    assert horizon == rule["horizon"]
    if rule["termination"] is None:
        assert height == -math.inf
    else:
        assert height == pytest.approx(rule["termination"], abs=1e-7)


@pytest.mark.parametrize("task", ["halfcheetah", "hopper", "ant", "mtu"])
def test_reward_constants(task):
    from paper_2204_07137_gb300 import inputs as I
    c = [float(x) for x in getattr(I, task)().reward_coef]
    rule = _rules()[task]
    assert c[1] == 1.0                                   # forward velocity, weight 1 everywhere
    keys = {"reward_action_weight": (0, 1.0), "reward_up_weight": (2, 1.0), "height_offset": (4, -1.0),
            "height_clip_low": (5, 1.0), "height_clip_high": (6, 1.0), "height_penalty_below": (7, 1.0),
            "height_slope_above": (9, 1.0)}
    for key, val in rule.items():
        if key in keys:
            k, sign = keys[key]
            assert c[k] == pytest.approx(sign * val, rel=1e-6), (task, key)
    if task in ("ant", "mtu"):
        assert c[3] == 1.0                               # heading projection, weight 1
