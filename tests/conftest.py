import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (runs the CUDA path)")
    config.addinivalue_line("markers", "slow: full-size CPU work (tens of seconds)")


def golden_path(name: str) -> str:
    return os.path.join(ROOT, "tests", "golden", name)


def read_golden(name: str):
    """Non-comment, non-empty lines of a golden file, split on ';'."""
    out = []
    with open(golden_path(name)) as f:
        for line in f:
            s = line.strip()
            if not s or s.startswith("#"):
                continue
            out.append([p.strip() for p in s.split(";")])
    return out
