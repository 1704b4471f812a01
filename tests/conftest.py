"""Test configuration: the ``gpu`` marker and shared fixtures.

``-m "not gpu"`` runs on any host: the oracle against its pins, the input
generators, host-side logic, and a load-and-export check of the C-ABI library.
``-m gpu`` runs the CUDA path against the oracle through the C ABI.
"""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a) and the built CUDA library")
    config.addinivalue_line("markers", "slow: large inputs (full benchmark sizes)")
