import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA device (B300, sm_103a)")
    config.addinivalue_line("markers", "slow: long-running CPU test")


def _has_cuda():
    try:
        import torch
        return torch.cuda.is_available()
    except Exception:
        return False


def pytest_collection_modifyitems(config, items):
    if _has_cuda():
        return
    skip = pytest.mark.skip(reason="no CUDA device")
    for item in items:
        if "gpu" in item.keywords:
            item.add_marker(skip)


def pytest_sessionfinish(session, exitstatus):
    """With DVR_PARITY_REPORT=<path>, write every comparison the GPU parity
    tests made (per-element error with and without the kink slack, and the
    max-norm error) as JSON lines."""
    path = os.environ.get("DVR_PARITY_REPORT")
    helpers = sys.modules.get("tests.gpu_helpers")
    if not path or helpers is None:
        return
    import json
    with open(path, "w") as f:
        for what, e, raw, mx in helpers.RECORD:
            f.write(json.dumps({"what": what, "per_element": e, "per_element_no_slack": raw,
                                "max_norm": mx}) + "\n")
