import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA device (B300, sm_103a)")


def load_golden(name):
    """Parse a tests/golden fixture: 'key: v v v / v v v' lines, '#' comments."""
    out = {}
    with open(os.path.join(ROOT, "tests", "golden", name)) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            key, val = line.split(":", 1)
            rows = [r.split() for r in val.split("/")]
            vals = [[float(x) for x in r] for r in rows]
            out.setdefault(key.strip(), []).append(vals)
    return out


@pytest.fixture(scope="session")
def golden():
    return load_golden
