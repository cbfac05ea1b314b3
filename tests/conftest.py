import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a) and the built library")
    config.addinivalue_line("markers", "slow: longer CPU test")


@pytest.fixture(scope="session")
def oracle_mod():
    from oracle import oracle
    oracle.build()
    return oracle


def pytest_terminal_summary(terminalreporter, exitstatus, config):
    """Per comparison: components outside the elementwise state bound, the
    worst error over that bound and, where the FP32 floor was used, the worst
    error over the floor bound (must stay <= 1)."""
    try:
        from helpers import GRAD_LOG, PARITY_LOG
    except ImportError:
        return
    tr = terminalreporter
    if GRAD_LOG:
        tr.write_sep("-", "window gradients at full size: relative error per sampled environment")
        tr.write_line(f"{'window':44s} {'envs':>5s} {'max':>9s} {'p99':>9s} {'median':>9s} {'>1e-3':>6s} "
                      f"{'floor max':>9s} {'floor med':>9s} {'by floor':>8s}")
        for what, n, mx, p99, med, above, fmx, fmed, expl in GRAD_LOG:
            tr.write_line(f"{what[:44]:44s} {n:5d} {mx:9.3g} {p99:9.3g} {med:9.3g} {above:6d} {fmx:9.3g} {fmed:9.3g} "
                          f"{expl:8d}")
    if not PARITY_LOG:
        return
    tr.write_sep("-", "state parity: elementwise bound and FP32 floor")
    tr.write_line(f"{'comparison':60s} {'comps':>8s} {'outside':>8s} {'frac':>9s} {'err/bound':>9s} {'err/floor':>9s}")
    for what, n, nb, wb, wf in PARITY_LOG:
        tr.write_line(f"{what[:60]:60s} {n:8d} {nb:8d} {nb / max(n, 1):9.2e} {wb:9.3g} "
                      f"{'-' if wf is None else format(wf, '9.3g'):>9s}")
