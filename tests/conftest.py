import os
import sys
import time

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

# GPU tests whose FP64 oracle references take tens of seconds (full-size
# 1M/3M-Gaussian frames checked on crops, finite differences, the storage
# precision report) run after every cheap GPU test.
_HEAVY = ("full_size", "finite_differences", "moment_storage_precision")


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")


def pytest_collection_modifyitems(config, items):
    """Host tests first, then cheap GPU tests, then the oracle-heavy GPU
    tests; tests/test_zz_no_alloc.py stays the last file, so that a run that
    stops at its first failure has run everything else before it."""
    def key(it):
        gpu = 1 if it.get_closest_marker("gpu") else 0
        last = 1 if os.path.basename(str(it.fspath)) == "test_zz_no_alloc.py" else 0
        heavy = 1 if gpu and any(h in it.name for h in _HEAVY) else 0
        return (last, gpu, heavy)
    items.sort(key=key)


_LOG = os.environ.get("MB3DGS_TEST_TIMES")


def pytest_runtest_logreport(report):
    # optional per-test wall times, appended as each test finishes (a run cut
    # off by a time limit still leaves the times of the finished tests)
    if _LOG and report.when == "call":
        with open(_LOG, "a") as f:
            f.write("%8.2f %s %s\n" % (report.duration, report.outcome, report.nodeid))
