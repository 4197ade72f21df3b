import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")


def pytest_sessionstart(session):
    """Builds the CUDA library (and the CPU oracle) when they are missing or
    stale, so the suite also runs on a fresh checkout; a no-op otherwise."""
    from oracle import build as obuild
    from paper_2604_19890_gb300 import build as sbuild
    obuild.build()
    sbuild.build()
