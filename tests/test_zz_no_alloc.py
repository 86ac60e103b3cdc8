"""The entry point that allocates no device memory (enuf_real_space_noalloc).

It exists for callers that cannot call cudaMalloc -- for example code inside
a framework whose device memory is held by its own pool allocator, or code
that must not allocate after set-up.  Its only scratch is a fixed array in
device memory, shared by every call.  This test calls it through the C ABI
twice in a row and checks each result against the library's main entry
point (the real-space part of enuf_energy_forces: E_real directly, the forces
and potentials as the full ones minus the reciprocal-space-only ones, minus
the self and background terms of the potential) and against the oracle's
real-space pair sum, at the same tolerances as the other parity tests.  The
file is named so that pytest collects it last.
"""
import ctypes

import numpy as np
import pytest

import oracle as O
import workloads as W

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2004_12484_b300 as P  # noqa: E402

DEV = torch.device("cuda", 0)
TOL = {"fp64": 1e-12, "mixed": 1e-5}


def rel_rms(a, b):
    return float(np.sqrt(((a - b) ** 2).sum() / (b ** 2).sum()))


def reference(d, precision, dt):
    kw = dict(L=d["L"], N=len(d["q"]), alpha=d["alpha"], r_c=d["r_c"], M=32, p=6, precision=precision, device=DEV)
    plan = P.Plan(**kw)
    tp = torch.tensor(d["pos"], dtype=dt, device=DEV)
    tq = torch.tensor(d["q"], dtype=dt, device=DEV)
    parts, F, Wf, phi = plan.energy_forces(tp, tq, phi=True)
    pk, Fk, Wk, phik = plan.energy_forces(tp, tq, phi=True, kspace_only=True)
    Fr = (F.double() - Fk.double()).cpu().numpy()
    Wr = Wf - Wk - parts["E_bg"] * np.eye(3)
    # the main entry point's potential also holds the self term -2 alpha q_i
    # / sqrt(pi) and the background term -pi Q / (V alpha^2)
    V = float(np.prod(d["L"]))
    q = np.asarray(d["q"], dtype=np.float64)
    phir = ((phi.double() - phik.double()).cpu().numpy() + 2.0 * d["alpha"] / np.sqrt(np.pi) * q
            + np.pi * q.sum() / (V * d["alpha"] ** 2))
    return parts["E_real"], Fr, Wr, phir, tp, tq


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_noalloc_matches_main_entry_point_twice(precision):
    d = W.rpm(N=6000, seed=41, M=32, p=6, r_c=10.0, alpha=0.3)
    dt = torch.float64 if precision == "fp64" else torch.float32
    if precision == "mixed":
        d["pos"], d["q"] = W.as_fp32(d["pos"], d["q"])
    E_ref, F_ref, W_ref, phi_ref, tp, tq = reference(d, precision, dt)
    Eo, Fo, phio, Wo = O.real_space(d["pos"], d["q"], d["L"], d["alpha"], d["r_c"])
    lib = P.lib()
    N = len(d["q"])
    L = (ctypes.c_double * 3)(*[float(x) for x in d["L"]])
    prec = P.FP64 if precision == "fp64" else P.MIXED
    tol = TOL[precision]
    for _ in range(2):
        F = torch.full((N, 3), float("nan"), dtype=dt, device=DEV)
        phi = torch.full((N,), float("nan"), dtype=dt, device=DEV)
        out = torch.full((10,), float("nan"), dtype=torch.float64, device=DEV)
        rc = lib.enuf_real_space_noalloc(ctypes.c_void_p(tp.data_ptr()), ctypes.c_void_p(tq.data_ptr()), N, L,
                                         d["alpha"], d["r_c"], 1.0, prec, ctypes.c_void_p(F.data_ptr()),
                                         ctypes.c_void_p(phi.data_ptr()), ctypes.c_void_p(out.data_ptr()),
                                         ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
        assert rc == 0, lib.enuf_last_error()
        torch.cuda.synchronize()
        o = out.cpu().numpy()
        etol = 1e-12 if precision == "fp64" else 1e-6
        Fn = F.double().cpu().numpy()
        phin = phi.double().cpu().numpy()
        Wn = o[1:].reshape(3, 3)
        # against the library's main entry point
        assert abs(o[0] / E_ref - 1) < etol
        assert rel_rms(Fn, F_ref) < tol
        assert rel_rms(phin, phi_ref) < tol
        assert np.abs(Wn - W_ref).max() < tol * np.abs(W_ref).max()
        # against the oracle's real-space pair sum (Eq. 17, Eq. 29)
        assert abs(o[0] / Eo - 1) < etol
        assert rel_rms(Fn, Fo) < tol
        assert rel_rms(phin, phio) < tol
        assert np.abs(Wn - Wo).max() < tol * np.abs(Wo).max()


def test_noalloc_rejects_sizes_beyond_its_scratch():
    lib = P.lib()
    N = 262144 + 1
    x = torch.zeros((N, 3), device=DEV)
    q = torch.zeros((N,), device=DEV)
    out = torch.zeros((10,), dtype=torch.float64, device=DEV)
    L = (ctypes.c_double * 3)(100.0, 100.0, 100.0)
    rc = lib.enuf_real_space_noalloc(ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(q.data_ptr()), N, L, 0.3,
                                     10.0, 1.0, P.MIXED, None, None, ctypes.c_void_p(out.data_ptr()), None)
    assert rc == -2  # ENUF_EUNSUPPORTED
    assert b"at most 262144" in lib.enuf_last_error()
