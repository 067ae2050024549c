import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: takes more than a few seconds")


@pytest.fixture(scope="session")
def orc():
    import oracle

    oracle.lib()
    return oracle


def pytest_terminal_summary(terminalreporter):
    """The measured sensor errors of the GPU-vs-oracle comparisons: per sensor and
    precision, the largest floor coefficient c the cells needed beyond the relative
    tolerance (the floor is c(n) u scale, c(n) = C_EVAL + C_DRIFT sqrt(n + 1)), its ratio
    to the c(n) in force, and the largest err / tol."""
    try:
        from tests import parity
    except ImportError:
        return
    if not parity.REPORT:
        return
    import json

    path = os.environ.get("KSS_PARITY_REPORT")
    if path:
        with open(path, "w") as fh:
            json.dump(parity.REPORT, fh)
    agg = {}
    for r in parity.REPORT:
        k = (r["sensor"], r["prec"])
        a = agg.setdefault(k, {"n": 0, "c_needed": 0.0, "of_floor": 0.0, "tol": 0.0,
                               "err": 0.0})
        a["n"] += 1
        a["c_needed"] = max(a["c_needed"], r["c_needed"])
        a["of_floor"] = max(a["of_floor"], r["c_needed"] / r["c_floor"])
        a["tol"] = max(a["tol"], r["max_tol_ratio"])
        a["err"] = max(a["err"], r["max_err"])
    tr = terminalreporter
    tr.write_sep("-", "measured sensor errors (GPU vs FP64 oracle)")
    tr.write_line(f"{'sensor':10s}{'prec':6s}{'checks':>7s}{'max err':>12s}{'c needed':>11s}"
                  f"{'of floor':>10s}{'err/tol':>9s}")
    for (name, prec), a in sorted(agg.items()):
        tr.write_line(f"{name:10s}{prec:6s}{a['n']:7d}{a['err']:12.3e}{a['c_needed']:11.2f}"
                      f"{a['of_floor']:10.3f}{a['tol']:9.3f}")
