"""The checked build of the library (libenuf_check.so: every index the
kernels derive from particle data, bin counts, work lists or their thread
decomposition tested against its extent; a failed test is counted and the
access skipped, never trapped) takes the place of a memory checker.

Its self-test shows that a failing check refuses the access and is
recorded; then the GPU parity suites run again on the checked build (in a
child process, which selects the library by ENUF_BOUNDS_CHECK=1): every
comparison with the oracle must pass there too, and no check may fail.
"""
import ctypes
import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CHECK_LIB = os.path.join(ROOT, "paper_2004_12484_b300", "libenuf_check.so")

# the suites that drive every kernel variant: grid sizes 8-512, windows p = 2
# to 12, tile edges, staged / direct / TMA interpolation, fused and separate
# FFT passes, heavy tiles, chunked scans, all-pairs and cell real space,
# analytic-differentiation forces, smeared charges, time stepping, the
# structure-factor and FFT entry points, the failure paths, and the
# benchmark workloads at full size (the 512 grid's passes and the
# TMA-staged interpolation among them)
SUITES = ["test_gpu_parity.py", "test_gpu_fft.py", "test_gpu_ad.py", "test_gpu_dpd.py", "test_gpu_md.py",
          "test_gpu_autograd.py", "test_gpu_failures.py", "test_gpu_workloads.py"]


def test_selftest_refuses_and_records():
    lib = ctypes.CDLL(CHECK_LIB)
    lib.enuf_last_error.restype = ctypes.c_char_p
    assert lib.enuf_bounds_checked() == 1
    assert lib.enuf_bounds_selftest() == 0, lib.enuf_last_error()
    fails = ctypes.c_ulonglong(7)
    assert lib.enuf_bounds_status(ctypes.byref(fails), None, 0, 0) == 0
    assert fails.value == 0  # the self-test clears what it recorded


def test_parity_suites_on_the_checked_build(tmp_path):
    report = tmp_path / "bounds.json"
    env = dict(os.environ, ENUF_BOUNDS_CHECK="1", ENUF_BOUNDS_REPORT=str(report))
    cmd = [sys.executable, "-m", "pytest", "-q", "-x", "-m", "gpu", "-p", "no:cacheprovider",
           *[os.path.join(ROOT, "tests", s) for s in SUITES]]
    r = subprocess.run(cmd, cwd=ROOT, env=env, capture_output=True, text=True, timeout=1800)
    tail = (r.stdout + r.stderr)[-3000:]
    assert r.returncode == 0, tail
    rep = json.loads(report.read_text())
    assert rep["checked"] == 1 and rep["library"].endswith("libenuf_check.so"), rep
    assert rep["rc"] == 0 and rep["fails"] == 0, rep
