import os
import sys
from pathlib import Path

import pytest

ROOT = Path(__file__).resolve().parent.parent
if str(ROOT) not in sys.path:
    sys.path.insert(0, str(ROOT))


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA device (B300, sm_103a)")
    config.addinivalue_line("markers", "slow: long statistical run")


@pytest.fixture(scope="session")
def orc():
    import oracle
    oracle.build()
    return oracle


def pytest_sessionfinish(session, exitstatus):
    """With XY_OBS_ERRLOG set, write the largest observable errors the GPU
    parity tests measured (gpu_helpers.measured_errors) to that file."""
    path = os.environ.get("XY_OBS_ERRLOG")
    if not path:
        return
    try:
        import gpu_helpers
    except ImportError:
        return
    errs = gpu_helpers.measured_errors()
    if errs:
        import json
        Path(path).parent.mkdir(parents=True, exist_ok=True)
        Path(path).write_text(json.dumps(errs, indent=1, sort_keys=True))
