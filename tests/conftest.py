import sys
from pathlib import Path

import pytest

ROOT = Path(__file__).resolve().parent.parent
if str(ROOT) not in sys.path:
    sys.path.insert(0, str(ROOT))

GOLDEN = Path(__file__).resolve().parent / "golden"


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: full-size workloads")


def read_golden(name: str) -> dict:
    """Parse a tests/golden/*.txt fixture: '# comment' lines, 'key values...' lines.
    Repeated keys collect into a list."""
    out: dict = {}
    for line in (GOLDEN / name).read_text().splitlines():
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        key, _, rest = line.partition(" ")
        if key in out:
            if not isinstance(out[key], list) or not out.get("_multi_" + key):
                out[key] = [out[key]]
                out["_multi_" + key] = True
            out[key].append(rest)
        else:
            out[key] = rest
    return out


@pytest.fixture(scope="session")
def golden():
    return read_golden
