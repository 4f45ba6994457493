import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (runs the sm_103a library)")


def parse_golden(path):
    """Parse tests/golden/*.txt: blank-line separated 'key: value' blocks."""
    blocks, cur = [], {}
    with open(path) as f:
        for line in f:
            line = line.strip()
            if line.startswith("#"):
                continue
            if not line:
                if cur:
                    blocks.append(cur)
                    cur = {}
                continue
            k, v = line.split(":", 1)
            cur[k.strip()] = v.strip()
    if cur:
        blocks.append(cur)
    return {b["example"]: b for b in blocks}


@pytest.fixture(scope="session")
def golden():
    return parse_golden(os.path.join(ROOT, "tests", "golden", "worked_examples.txt"))
