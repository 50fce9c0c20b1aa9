"""Shared pytest configuration.

Markers:
  gpu   needs a CUDA device (GB300); everything else runs on the CPU.
  slow  a CPU test that takes more than a few seconds.
"""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA device; run with -m gpu")
    config.addinivalue_line("markers", "slow: CPU test taking more than a few seconds")
