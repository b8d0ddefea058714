"""Test configuration: markers and import paths.

``-m "not gpu"`` runs the oracle pins, host logic and the C-ABI export check
on a machine without a GPU; ``-m gpu`` runs the CUDA parity tests."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
for p in (ROOT, os.path.join(ROOT, "oracle"), os.path.join(ROOT, "tests")):
    if p not in sys.path:
        sys.path.insert(0, p)


def pytest_sessionstart(session):
    """Builds the library (and the oracle) first when a checkout has none:
    the C-ABI and host-logic tests load it (without a GPU, no kernel runs)."""
    if not os.path.exists(os.path.join(ROOT, "paper_2207_03945_gb300", "libflock.so")):
        import __graft_entry__
        __graft_entry__.build()


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300) and the built library")
    config.addinivalue_line("markers", "slow: longer CPU test")
