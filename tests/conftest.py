import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a) and the built library")


def pytest_sessionstart(session):
    # Host-only entry points of the library (coefficients, scheme digests,
    # the serving loop's footprints) are used by CPU tests too: make sure the
    # in-tree library exists (a no-op when it is up to date).
    from paper_1903_04946_gb300.build import build
    build()
