import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA device (GB300) and the built library")
    config.addinivalue_line("markers", "slow: longer CPU-only test")


def read_golden(name):
    """Numeric lines of a golden fixture, split into blocks at '#@ <label>' lines."""
    blocks, cur = {}, None
    with open(os.path.join(GOLDEN, name)) as fh:
        for line in fh:
            s = line.strip()
            if not s:
                continue
            if s.startswith("#@"):
                cur = s[2:].split()[0]
                blocks[cur] = []
                continue
            if s.startswith("#"):
                continue
            blocks.setdefault(cur, []).append([float(t) for t in s.split()])
    return {k: np.array(v) for k, v in blocks.items()}
