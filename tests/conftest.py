import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: long-running CPU check")


def read_golden(name):
    """Rows of a whitespace-separated fixture under tests/golden ('#' comments)."""
    rows = []
    with open(os.path.join(ROOT, "tests", "golden", name)) as f:
        for line in f:
            line = line.split("#", 1)[0].strip()
            if line:
                rows.append(line.split())
    return rows


def exact_value(expr):
    """Evaluate a closed-form fixture entry such as (9+8*sqrt(10))/215."""
    import math
    return float(eval(expr, {"__builtins__": {}}, {"sqrt": math.sqrt}))
