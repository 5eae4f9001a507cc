import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA device (B300, sm_103a)")
    config.addinivalue_line("markers", "slow: long-running CPU test")


def _has_gpu() -> bool:
    try:
        import torch
        return torch.cuda.is_available()
    except Exception:
        return False


def pytest_collection_modifyitems(config, items):
    if _has_gpu():
        return
    skip = pytest.mark.skip(reason="no CUDA device")
    for item in items:
        if "gpu" in item.keywords:
            item.add_marker(skip)


def pytest_terminal_summary(terminalreporter):
    """Near-boundary counts of the parity checks that ran (oracle-flagged items
    excluded from the exact comparisons), also written as JSON to
    the file that $DIVAS_PARITY_JSON names, when it is set."""
    try:
        from tests import gpu_helpers
    except Exception:
        return
    rows = gpu_helpers.PARITY
    if not rows:
        return
    import json
    tr = terminalreporter
    tr.write_sep("-", "near-boundary items (flagged within 1e-6, excluded from exact checks)")
    for r in rows:
        tr.write_line(f"{r['check']}: {r['flagged']} of {r['items']} "
                      f"({100.0 * r['flagged_frac']:.3f}%), mismatches outside them "
                      f"{r['mismatches']}")
    path = os.environ.get("DIVAS_PARITY_JSON")
    if not path:
        return
    try:
        os.makedirs(os.path.dirname(os.path.abspath(path)), exist_ok=True)
        with open(path, "w") as f:
            json.dump(rows, f, indent=1)
    except OSError:
        pass
