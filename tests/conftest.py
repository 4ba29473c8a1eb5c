import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a) and the built CUDA library")


def pytest_collection_modifyitems(config, items):
    # GPU tests cannot run without a device; skip rather than fail on CPU-only hosts
    # when they are selected explicitly together with CPU tests.
    try:
        import torch
        has_gpu = torch.cuda.is_available()
    except Exception:  # pragma: no cover
        has_gpu = False
    if has_gpu:
        return
    skip = pytest.mark.skip(reason="no CUDA device")
    for it in items:
        if "gpu" in it.keywords:
            it.add_marker(skip)


def pytest_terminal_summary(terminalreporter):
    # the exception counts of the parity comparisons (keys on marginal rays,
    # near-edge hit ties), per test and in total
    try:
        import parity
    except ImportError:  # pragma: no cover
        return
    lines = parity.summary_lines()
    if lines:
        terminalreporter.write_sep("-", "parity exceptions")
        for line in lines:
            terminalreporter.write_line(line)
