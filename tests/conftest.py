import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: long-running CPU test")


def pytest_sessionfinish(session, exitstatus):
    """Write the parity errors the GPU tests measured (tests/gpu_helpers.py
    RECORDS) to LBM_RESULTS_DIR/parity_errors.json when that is set."""
    out = os.environ.get("LBM_RESULTS_DIR")
    mod = sys.modules.get("tests.gpu_helpers")
    if not out or mod is None or not getattr(mod, "RECORDS", None):
        return
    import json

    os.makedirs(out, exist_ok=True)
    with open(os.path.join(out, "parity_errors.json"), "w") as f:
        json.dump(mod.RECORDS, f, indent=0)
