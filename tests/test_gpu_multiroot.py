"""A model with several roots (links other than 0 hanging from the world) and a
branching subtree with fixed and prismatic joints, a contact and a joint
limit: the team form's tree sums, ancestor sums and poses by rows skip a root's
missing parent, so its step and step adjoint must match the FP64 oracle at
every team size (narrower than three lanes included), in the PLAIN form and in
a model-specialised build."""
import numpy as np
import pytest

from helpers import assert_grad_close, assert_state_close, forest, oracle_step_with_floor, seeded_case

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

N = 37   # ragged work items at every team size


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2204_07137_gb300 import build
    build.build()


def T(x):
    return torch.from_numpy(np.ascontiguousarray(np.asarray(x, np.float32).reshape(-1))).cuda()


FORMS = [("plain", 0, False), ("batched", 2, False), ("batched", 4, False), ("batched", 8, False),
         ("batched", 16, False), ("batched", 8, True)]


def _sim(m, form, lanes, spec):
    from paper_2204_07137_gb300.sim import Simulator
    sim = Simulator([(m, N)], form=form, h_max=4)
    if form == "batched":
        sim.set_launch(0, lanes, 0)
        if spec:
            sim.specialize()
    return sim


@pytest.mark.parametrize("form,lanes,spec", FORMS)
def test_multi_root_step_matches_oracle(oracle_mod, form, lanes, spec):
    m = forest()
    sim = _sim(m, form, lanes, spec)
    o = oracle_mod.Oracle(m)
    tag = f"forest/{form}/T{lanes}{'/spec' if spec else ''}"
    for seed, kind in ((0, "initial"), (1, "random")):
        q, qd, a = seeded_case(m, N, seed, kind)
        qn, qdn, r = sim.step(T(q), T(qd), T(a))
        torch.cuda.synchronize()
        (rq, rqd, rr), (fq, fqd, fr) = oracle_step_with_floor(o, q.T, qd.T, a.T)
        assert_state_close(qn.cpu().numpy().reshape(m.nq, N).T, rq, f"{tag} q seed {seed}", fq)
        assert_state_close(qdn.cpu().numpy().reshape(m.nv, N).T, rqd, f"{tag} qd seed {seed}", fqd)
        assert_state_close(r.cpu().numpy(), rr, f"{tag} reward seed {seed}", fr)
    assert sim.status() == 0


@pytest.mark.parametrize("form,lanes,spec", FORMS)
def test_multi_root_step_adjoint_matches_oracle(oracle_mod, form, lanes, spec):
    m = forest()
    sim = _sim(m, form, lanes, spec)
    o = oracle_mod.Oracle(m)
    q, qd, a = seeded_case(m, N, 2, "random")
    rng = np.random.default_rng(9)
    qb = rng.normal(size=(m.nq, N)).astype(np.float32)
    qdb = rng.normal(size=(m.nv, N)).astype(np.float32)
    rb = rng.normal(size=N).astype(np.float32)
    gq, gqd, ga = sim.step_adjoint(T(q), T(qd), T(a), T(qb), T(qdb), T(rb))
    torch.cuda.synchronize()
    rq, rqd, ra = o.step_vjp(q.T, qd.T, a.T, qb.T, qdb.T, rb)
    got = np.concatenate([gq.cpu().numpy().reshape(m.nq, N), gqd.cpu().numpy().reshape(m.nv, N),
                          ga.cpu().numpy().reshape(m.na, N)])
    ref = np.concatenate([rq.T, rqd.T, ra.T])
    assert_grad_close(got, ref, f"forest/{form}/T{lanes}{'/spec' if spec else ''} step adjoint")
    assert sim.status() == 0
