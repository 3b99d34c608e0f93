import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a) and the built CUDA library")
    config.addinivalue_line("markers", "slow: longer CPU test")


def pytest_sessionfinish(session, exitstatus):
    """With MPML_PRECISION_REPORT=<file>: write every element-wise parity check of the
    session (test, field, norm-relative error, max-relative error, tolerance) as JSON."""
    path = os.environ.get("MPML_PRECISION_REPORT")
    mod = sys.modules.get("tests._gpu")
    if not path or mod is None:
        return
    import json
    with open(path, "w") as fh:
        json.dump([{"test": t, "field": f, "norm_rel": a, "max_rel": b, "tol": tol} for t, f, a, b, tol in mod.REPORT],
                  fh, indent=0)
