import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

GOLDEN = os.path.join(ROOT, "tests", "golden")


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: long CPU oracle runs (set PNM_SLOW=1 to run)")


def pytest_collection_modifyitems(config, items):
    if os.environ.get("PNM_SLOW") == "1":
        return
    skip = pytest.mark.skip(reason="slow oracle pin; set PNM_SLOW=1")
    for it in items:
        if "slow" in it.keywords:
            it.add_marker(skip)


def read_golden(name):
    """Rows of whitespace-separated fields from tests/golden/<name>, comments removed."""
    rows = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.split("#", 1)[0].strip()
            if line:
                rows.append(line.split())
    return rows


def minnesota_params():
    """(V_R, kappa_R, V_T, kappa_T, V_S, kappa_S, hbar^2/2m) from the golden fixture."""
    d = {k: float(v) for k, v in read_golden("minnesota.txt")}
    return (d["VR"], d["kR"], d["VT"], d["kT"], d["VS"], d["kS"], d["hbar2_2m"])
