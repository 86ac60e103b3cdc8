import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA device (B300, sm_103a)")
    config.addinivalue_line("markers", "slow: takes more than a few seconds on CPU")


def pytest_sessionfinish(session, exitstatus):
    """With ENUF_BOUNDS_REPORT set (a run of the tests on the checked build of
    the library), write the count of failed bounds checks and the first
    failure to that file as JSON."""
    path = os.environ.get("ENUF_BOUNDS_REPORT")
    if not path or "paper_2004_12484_b300" not in sys.modules:
        return
    import ctypes
    import json

    P = sys.modules["paper_2004_12484_b300"]
    lib = P.lib()
    fails = ctypes.c_ulonglong()
    where = ctypes.create_string_buffer(256)
    rc = lib.enuf_bounds_status(ctypes.byref(fails), where, 256, 0)
    with open(path, "w") as f:
        json.dump({"checked": lib.enuf_bounds_checked(), "rc": rc, "fails": fails.value,
                   "where": where.value.decode(), "library": P.LIB_PATH}, f)
