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
        rows[(table, task, key)] = float(val)
    return rows


def test_per_task_and_general_settings_match_the_paper():
    from paper_2204_07137_gb300 import shac
    rows = _table()
    for (table, task, key), val in rows.items():
        if key not in ("actor_lr", "critic_lr", "alpha", "episodes"):
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
