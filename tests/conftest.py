import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a) and the built library")
    config.addinivalue_line("markers", "slow: oracle runs that take more than a few seconds")


GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def read_golden(name):
    """Parse a golden poset fixture: 'key: value' lines, '#' comments, 'rel: i j' edges."""
    out = {"rel": []}
    with open(os.path.join(GOLDEN, name)) as fh:
        for line in fh:
            line = line.split("#", 1)[0].strip()
            if not line:
                continue
            key, val = (s.strip() for s in line.split(":", 1))
            if key == "rel":
                i, j = (int(x) for x in val.split())
                out["rel"].append((i, j))
            elif key in ("Nk", "L123"):
                out[key] = [int(x) for x in val.split()]
            elif key in ("phi", "Bphi"):
                out[key] = [float(x) for x in val.split()]
            elif key in ("S2", "S4") or key.startswith("Seps"):
                out[key] = float(val)
            else:
                out[key] = int(val)
    return out


@pytest.fixture
def golden():
    return read_golden
