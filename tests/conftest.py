import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a) and the built CUDA library")


def pytest_terminal_summary(terminalreporter):
    """Breakpoint flips of the GPU chains against Eq. 1 read literally (the
    plain sequential sum), per checked workload."""
    try:
        from _gpu import FLIP_LOG
    except ImportError:
        return
    if not FLIP_LOG:
        return
    terminalreporter.write_line("breakpoint flips vs plain-form Eq. 1 (label: flips / pieces checked):")
    for label, pieces, flips in FLIP_LOG:
        terminalreporter.write_line(f"  {label}: {flips} / {pieces}")
