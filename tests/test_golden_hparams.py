"""The learner's hyperparameters against the values the paper prints in its
appendix tables (tab:optimal_params, tab:general_params), transcribed in
tests/golden/shac_hyperparameters.txt."""
import inspect
import os

import pytest

pytest.importorskip("torch")

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "shac_hyperparameters.txt")


def _table():
    rows = {}
    for ln in open(GOLDEN):
        ln = ln.strip()
        if not ln or ln.startswith("#"):
            continue
        table, task, key, val = ln.split()
        rows[(table, task, key)] = tuple(int(x) for x in val.split(",")) if table == "network" else float(val)
    return rows


def test_per_task_and_general_settings_match_the_paper():
    from paper_2204_07137_gb300 import shac
    rows = _table()
    for (table, task, key), val in rows.items():
        if table == "network" or key not in ("actor_lr", "critic_lr", "alpha", "episodes"):
            continue
        hp = shac.GENERAL_HPARAMS if table == "general" else shac.PAPER_HPARAMS[task]
        assert hp[key] == pytest.approx(val, rel=0, abs=0), (table, task, key)
    # a task the tables do not list takes the general setting
    for key in ("actor_lr", "critic_lr", "alpha"):
        assert shac.GENERAL_HPARAMS[key] == rows[("general", "any", key)]


def test_learner_defaults_match_the_paper():
    from paper_2204_07137_gb300 import shac
    rows = _table()
    d = {k: p.default for k, p in inspect.signature(shac.SHAC.__init__).parameters.items()}
    assert d["h"] == rows[("general", "any", "h")]
    assert d["n_envs"] == rows[("general", "any", "N")]
    assert d["gamma"] == rows[("general", "any", "gamma")]
    assert d["lam"] == rows[("general", "any", "lambda")]
    assert d["critic_iters"] == rows[("general", "any", "critic_iters")]
    assert d["critic_minibatches"] == rows[("general", "any", "critic_minibatches")]
    assert tuple(d["betas"]) == (rows[("optimal", "cartpole", "adam_beta1")],
                                 rows[("optimal", "cartpole", "adam_beta2")])


def test_network_sizes_match_the_paper():
    from paper_2204_07137_gb300 import shac
    for (table, task, key), val in _table().items():
        if table != "network":
            continue
        pol, vf = shac.PAPER_NETWORKS[task]
        assert (pol if key == "policy" else vf) == val, (task, key)


def test_hidden_layers_are_elu_then_layer_norm():
    import torch
    from paper_2204_07137_gb300 import shac
    net = shac.mlp([5, 64, 32, 1])
    kinds = [type(m) for m in net]
    assert kinds == [torch.nn.Linear, torch.nn.ELU, torch.nn.LayerNorm, torch.nn.Linear, torch.nn.ELU,
                     torch.nn.LayerNorm, torch.nn.Linear]
