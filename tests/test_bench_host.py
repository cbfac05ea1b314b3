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


def test_reference_arm_line_keeps_the_contract(monkeypatch, capsys):
    """--impl reference: one JSON line on rank 0 with the contract's keys, the
    oracle's median rate as value, its cpu_baseline and a zero-byte e2e; the
    other ranks print nothing."""
    import json
    import bench
    calls = []

    def fake(groups, seed=0, target_s=12.0):
        calls.append((len(groups), seed, target_s))
        return 100.0 + seed, 16, 2.0, "4 of 2048 envs (ant) x 32 steps, forward + exact adjoint, 2.0 s"

    monkeypatch.setattr(bench, "oracle_workload_rate", fake)
    args = SimpleNamespace(workload="ant-2048", gpus=1, steps=3, warmup=2)
    bench.reference_main(args, 1, 2)
    assert capsys.readouterr().out == "" and not calls
    bench.reference_main(args, 0, 1)
    line = json.loads(capsys.readouterr().out.strip())
    for k in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in line, k
    assert line["impl"] == "reference" and line["metric"] == bench.METRIC and line["unit"] == "env-steps/s"
    assert line["value"] == 101.0   # median of the three timed samples 100, 101, 102
    assert line["config"]["workload"] == "ant-2048" and line["higher_is_better"] is True
    assert line["cpu_baseline"]["value"] == line["value"] and line["cpu_baseline"]["kind"] == "oracle"
    assert line["cpu_baseline"]["cores"] == 16
    assert line["e2e"] == {"value": 101.0, "unit": "env-steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    assert abs(line["ms_per_step"] - 1e3 * 2048 * bench.H / 101.0) < 1e-9
    assert len(calls) == 2 + 3 and all(c[0] == 1 for c in calls[:2])   # warm-up on a one-environment sample


def test_default_workload_and_fp32_peak(monkeypatch):
    import bench
    monkeypatch.setattr(sys, "argv", ["bench.py"])
    assert bench.parse().workload == bench.WORKLOAD == "ant-2048"
    monkeypatch.setattr(sys, "argv", ["bench.py", "--policy"])
    assert bench.parse().workload == "mtu-512"
    monkeypatch.setattr(sys, "argv", ["bench.py", "--policy", "--workload", "mtu-512"])
    assert bench.parse().workload == "mtu-512"
    # 152 SMs x 128 FP32 lanes x 2 flop (FMA) x 2070 MHz
    assert abs(bench.fp32_peak_tflops(152, 2070.0) - 152 * 128 * 2 * 2.07e9 / 1e12) < 1e-9
    ab = bench.algo_bytes_per_env_step(SimpleNamespace(nq=15, nv=14, na=8))
    assert ab == {"forward": 4 * (2 * 29 + 8 + 1), "adjoint": 4 * (3 * 29 + 2 * 8 + 1)}   # 268 B and 416 B
