import json
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")


@pytest.fixture(scope="session")
def oracle_lib():
    from oracle import Oracle
    return Oracle()


_REPORT = []


@pytest.fixture(scope="session")
def parity_report():
    """Collects the errors of the CUDA path against the oracle (one dict per
    case: what was compared and the largest errors).  With CK_PARITY_REPORT
    set to a path, the list is written there as JSON when the session ends."""
    return _REPORT


def pytest_sessionfinish(session, exitstatus):
    path = os.environ.get("CK_PARITY_REPORT")
    if path and _REPORT:
        os.makedirs(os.path.dirname(os.path.abspath(path)), exist_ok=True)
        with open(path, "w") as f:
            json.dump(_REPORT, f, indent=1)


def state_errors(y, yo):
    """Largest |dT|/T and |dY_k| between two batches of final states."""
    import numpy as np
    dT = np.abs(y[:, 0] - yo[:, 0]) / yo[:, 0]
    dY = np.abs(y[:, 1:] - yo[:, 1:])
    return float(dT.max()), float(dY.max())


def plain_relative(err, ref, floor=1e-20):
    """Plain relative error |gpu - oracle| / max(|oracle|, floor) per entry:
    the largest, how many entries exceed 1e-12 and the largest of those."""
    import numpy as np
    rel = err / np.maximum(np.abs(ref), floor)
    over = rel > 1e-12
    return {"max_plain_rel": float(rel.max()), "n_over_1e-12": int(over.sum()), "n_entries": int(rel.size),
            "worst_over": float(rel[over].max()) if over.any() else None}
