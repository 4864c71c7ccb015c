"""Shared test setup.

Markers: ``gpu`` — needs a CUDA device and the built ``libmorph.so``.  Every
other test runs on the CPU (oracle pins, host logic, ABI symbol table).
"""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU and the built CUDA library")
    # a fresh checkout: compile the library first (nvcc cross-compiles
    # without a GPU; up-to-date builds return at once), so that the CPU tests
    # of the ABI and the GPU tests find it
    from paper_0712_0121_gb300 import build
    build.build_all()


GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def read_golden(name):
    """Parse a ``key: value`` fixture (``#`` comments)."""
    out = {}
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.split("#", 1)[0].strip()
            if not line:
                continue
            k, v = line.split(":", 1)
            out[k.strip()] = v.strip()
    return out
