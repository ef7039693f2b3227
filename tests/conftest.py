import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

GOLDEN = os.path.join(ROOT, "tests", "golden")


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: takes more than a few seconds on CPU")


def load_golden_network(name):
    """Parse tests/golden/net_<name>.txt -> (n, stated facts, levels as lists of 0-based pairs)."""
    path = os.path.join(GOLDEN, f"net_{name}.txt")
    facts = {}
    levels = [[]]
    body = False
    with open(path) as f:
        for line in f:
            line = line.rstrip("\n")
            if line.startswith("#"):
                continue
            if not body:
                if line == "---":
                    body = True
                    continue
                key, val = line.split()
                facts[key] = int(val)
                continue
            if not line.strip():
                if levels[-1]:
                    levels.append([])
                continue
            i, j = line.split()
            levels[-1].append((int(i) - 1, int(j) - 1))
    if not levels[-1]:
        levels.pop()
    return facts["n"], facts, levels


@pytest.fixture(scope="session")
def golden_networks():
    names = ["best16", "opt10", "bn6", "bnl16", "bnp16"]
    return {name: load_golden_network(name) for name in names}
