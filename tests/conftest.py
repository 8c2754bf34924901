import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA device (runs on the GB300 box)")
    config.addinivalue_line("markers", "slow: longer CPU test")


def record(test: str, **values) -> None:
    """Append measured errors of a test as one JSON line to the file named by
    BM_TEST_REPORT (nothing when unset), so a run can show its margins."""
    path = os.environ.get("BM_TEST_REPORT")
    if not path:
        return
    import json
    with open(path, "a") as f:
        f.write(json.dumps({"test": test, **{k: (float(v) if hasattr(v, "__float__") else v)
                                             for k, v in values.items()}}) + "\n")
