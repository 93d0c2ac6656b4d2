import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA device (B300, sm_103a)")


def read_golden(name):
    """Parse a tests/golden/*.txt fixture: '# ...' comments, 'key = values' lines, or numeric rows."""
    path = os.path.join(ROOT, "tests", "golden", name)
    kv, rows = {}, []
    with open(path) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            if "=" in line:
                k, v = line.split("=", 1)
                kv[k.strip()] = [float(x) for x in v.split()]
            else:
                rows.append([float(x) for x in line.split()])
    return kv, rows


@pytest.fixture
def golden():
    return read_golden
