"""Host logic of bench.py that needs no GPU: the oracle baseline of a mixed
batch is the whole job's env-steps over the sum of the groups' times."""
import os
import sys
from types import SimpleNamespace

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def test_mixed_batch_rate_is_total_envs_over_summed_group_times(monkeypatch):
    import bench
    rates = {"a": 1000.0, "b": 10.0, "c": 0.5}
    seen = []

    def fake(model, n_envs, seed=0, target_s=12.0):
        seen.append((model.name, n_envs, target_s))
        return rates[model.name], 3, 2, 16, 1.0, 1

    monkeypatch.setattr(bench, "oracle_window_rate", fake)
    groups = [(SimpleNamespace(name="a"), 4096), (SimpleNamespace(name="b"), 2048), (SimpleNamespace(name="c"), 1024)]
    r, threads, dt, desc = bench.oracle_workload_rate(groups, seed=0, target_s=9.0)
    want = (4096 + 2048 + 1024) / (4096 / 1000.0 + 2048 / 10.0 + 1024 / 0.5)
    assert abs(r - want) <= 1e-12 * want
    assert threads == 16 and dt == 3.0
    assert [s[:2] for s in seen] == [("a", 4096), ("b", 2048), ("c", 1024)]
    assert all(abs(s[2] - 3.0) < 1e-12 for s in seen)   # the time budget is split over the groups
    assert "(a)" in desc and "(b)" in desc and "(c)" in desc


def test_single_group_rate_is_the_group_rate(monkeypatch):
    import bench
    monkeypatch.setattr(bench, "oracle_window_rate", lambda m, n, seed=0, target_s=12.0: (123.0, 8, 4, 16, 2.0, 1))
    r, threads, dt, desc = bench.oracle_workload_rate([(SimpleNamespace(name="ant"), 2048)])
    assert abs(r - 123.0) <= 1e-12 * 123.0 and dt == 2.0 and desc.startswith("8 of 2048 envs (ant) x 4 steps")
