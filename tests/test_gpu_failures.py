"""Failure paths of the C ABI that need a CUDA context but fault nothing:
a device allocation that cannot succeed (ENUF_ENOMEM), a caller workspace
that is too small or misaligned (ENUF_EINVAL), and a plan created after
those failures working normally."""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2004_12484_b300 as P  # noqa: E402

DEV = torch.device("cuda", 0)
ENUF_EINVAL, ENUF_ENOMEM = -1, -3


def params(**kw):
    d = dict(L=(400.0, 400.0, 400.0), N=1000, alpha=0.3, r_c=9.0, M=32, p=4, precision="mixed")
    d.update(kw)
    return P.make_params(**d)


def test_allocation_failure_is_reported_as_enomem():
    lib = P.lib()
    # the largest N the parameters allow, in double precision: a workspace
    # well beyond the device's memory, so cudaMalloc must refuse it
    prm = params(N=2 ** 31 - 1, precision="fp64")
    nbytes = ctypes.c_size_t()
    assert lib.enuf_plan_workspace_bytes(ctypes.byref(prm), ctypes.byref(nbytes)) == 0
    total = torch.cuda.get_device_properties(DEV).total_memory
    assert nbytes.value > 1.5 * total
    h = ctypes.c_void_p()
    rc = lib.enuf_plan_create(ctypes.byref(prm), None, 1, ctypes.byref(h))
    assert rc == ENUF_ENOMEM
    assert b"cudaMalloc" in lib.enuf_last_error()
    assert not h.value


def test_too_small_or_misaligned_workspace_is_rejected():
    lib = P.lib()
    prm = params()
    nbytes = ctypes.c_size_t()
    assert lib.enuf_plan_workspace_bytes(ctypes.byref(prm), ctypes.byref(nbytes)) == 0
    h = ctypes.c_void_p()
    assert lib.enuf_plan_create(ctypes.byref(prm), None, 0, ctypes.byref(h)) == 0
    try:
        buf = torch.empty(nbytes.value + 512, dtype=torch.uint8, device=DEV)
        base = (buf.data_ptr() + 255) // 256 * 256
        assert lib.enuf_plan_set_workspace(h, ctypes.c_void_p(base), nbytes.value - 1) == ENUF_EINVAL
        assert b"too small" in lib.enuf_last_error()
        assert lib.enuf_plan_set_workspace(h, ctypes.c_void_p(base + 16), nbytes.value) == ENUF_EINVAL
        assert b"aligned" in lib.enuf_last_error()
        # a compute call without a workspace is refused, not run
        x = torch.zeros((1000, 3), device=DEV)
        q = torch.zeros((1000,), device=DEV)
        assert lib.enuf_compute(h, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(q.data_ptr()), None, None,
                                None, 0) == ENUF_EINVAL
    finally:
        lib.enuf_plan_destroy(h)


def test_plan_works_after_failures():
    g = np.random.default_rng(3)
    N = 1000
    pos = torch.tensor(g.uniform(0, 40.0, size=(N, 3)), dtype=torch.float32, device=DEV)
    q = torch.tensor(np.where(np.arange(N) % 2 == 0, 1.0, -1.0), dtype=torch.float32, device=DEV)
    plan = P.Plan(L=(40.0, 40.0, 40.0), N=N, alpha=0.3, r_c=9.0, M=32, p=4, device=DEV)
    parts, F, W, _ = plan.energy_forces(pos, q)
    assert np.isfinite(parts["E"]) and torch.isfinite(F).all()
