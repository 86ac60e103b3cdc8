"""Plain FP64 CPU oracle for the ENUF method -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It shares no code with the CUDA
library and never imports it.

The arithmetic lives in ``enuf_oracle.c`` (plain loops in IEEE double); this
module compiles it with gcc on first use and wraps each entry point with numpy
arrays.  Functions follow the paper (Yang et al., arXiv:2004.12484):

* :func:`direct_ewald` -- O1, the Ewald sum written out (Eq. 17, 22, 24-26,
  29, 41 in textbook form), optionally on a sampled subset of particles.
* :func:`nfft_ewald` -- O2, the reciprocal part by transposed / conjugated
  NFFT (Eq. 36-38, 41-42) plus the same real-space and self terms.
* :func:`nfft_ewald_ad`, :func:`kspace_nfft_ad` -- O2 with the forces as the
  analytic gradient of Eq. 38 (window derivative in the interpolation, one
  inverse FFT), the variant beside the ik forces of Eq. 41-42.
* ``slater=lambda_e`` in :func:`real_space`, :func:`direct_ewald` and
  :func:`nfft_ewald` -- the ENUF-DPD real-space correction for smeared
  Slater-type charges (Eq. 51-58), with :func:`slater_factors`.
* :func:`structure_factor_direct`, :func:`structure_factor_nfft`,
  :func:`fft1d`, :func:`fft3d`, :func:`window`, :func:`window_hat`,
  :func:`window_b`, :func:`image_sum` -- the individual steps, exposed so the
  tests can pin each of them.

Every function has a pin in ``tests/test_oracle_pins.py``; none is "parity
unpinned".
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "enuf_oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lib = None

_D = ctypes.POINTER(ctypes.c_double)
_I64 = ctypes.POINTER(ctypes.c_int64)


def build(force: bool = False) -> str:
    """Compile ``enuf_oracle.c`` into ``liboracle.so`` (gcc, OpenMP)."""
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-shared", "-fPIC", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB_PATH)
        L.orc_window_b.restype = ctypes.c_double
        L.orc_window_b.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int]
        L.orc_window.restype = ctypes.c_double
        L.orc_window.argtypes = [ctypes.c_double, ctypes.c_double]
        L.orc_window_hat.restype = ctypes.c_double
        L.orc_window_hat.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_double]
        L.orc_fft1d.argtypes = [ctypes.c_int, _D, ctypes.c_int]
        L.orc_fft3d.argtypes = [ctypes.c_int, _D, ctypes.c_int]
        L.orc_real_space.argtypes = [ctypes.c_int64, _D, _D, _D, ctypes.c_double, ctypes.c_double,
                                     ctypes.c_double, ctypes.c_int64, _I64, _D, _D, _D, _D]
        L.orc_real_space_slater.argtypes = [ctypes.c_int64, _D, _D, _D, ctypes.c_double, ctypes.c_double,
                                            ctypes.c_double, ctypes.c_double, ctypes.c_int64, _I64, _D, _D, _D, _D]
        L.orc_slater_factors.argtypes = [ctypes.c_double, ctypes.c_double, _D, _D]
        L.orc_self_and_background.argtypes = [ctypes.c_int64, _D, _D, ctypes.c_double, ctypes.c_double,
                                              _D, _D, _D]
        L.orc_kspace_direct.argtypes = [ctypes.c_int64, _D, _D, _D, ctypes.c_double, ctypes.c_double,
                                        ctypes.c_int, ctypes.c_int, _D, _D, _D, _D, ctypes.c_int64, _I64]
        L.orc_structure_factor_direct.argtypes = [ctypes.c_int64, _D, _D, _D, ctypes.c_int, _D]
        L.orc_structure_factor_nfft.argtypes = [ctypes.c_int64, _D, _D, _D, ctypes.c_int, ctypes.c_int,
                                                ctypes.c_int, _D]
        L.orc_spread.argtypes = [ctypes.c_int64, _D, _D, _D, ctypes.c_int, ctypes.c_int, ctypes.c_double, _D]
        L.orc_kspace_nfft.argtypes = [ctypes.c_int64, _D, _D, _D, ctypes.c_double, ctypes.c_double,
                                      ctypes.c_int, ctypes.c_int, ctypes.c_int, _D, _D, _D, _D]
        L.orc_kspace_nfft_ad.argtypes = [ctypes.c_int64, _D, _D, _D, ctypes.c_double, ctypes.c_double,
                                         ctypes.c_int, ctypes.c_int, ctypes.c_int, _D, _D, _D, _D]
        L.orc_window_deriv.restype = ctypes.c_double
        L.orc_window_deriv.argtypes = [ctypes.c_double, ctypes.c_double]
        L.orc_image_sum.restype = ctypes.c_double
        L.orc_image_sum.argtypes = [ctypes.c_int64, _D, _D, _D, ctypes.c_double, ctypes.c_int]
        L.orc_num_threads.restype = ctypes.c_int
        _lib = L
    return _lib


def _dp(a):
    return a.ctypes.data_as(_D) if a is not None else None


def _ip(a):
    return a.ctypes.data_as(_I64) if a is not None else None


def _arr(x, shape=None):
    a = np.ascontiguousarray(np.asarray(x, dtype=np.float64))
    if shape is not None:
        a = a.reshape(shape)
    return a


def _box(L):
    L = np.asarray(L, dtype=np.float64).reshape(-1)
    if L.size == 1:
        L = np.repeat(L, 3)
    return np.ascontiguousarray(L)


def num_threads() -> int:
    return int(lib().orc_num_threads())


# ---------------------------------------------------------------- window
def window_b(M: int, n_c: int, p: int) -> float:
    """Gaussian shape parameter b for sigma = M/(2 n_c), m = p/2."""
    return float(lib().orc_window_b(M, n_c, p))


def window(u, b: float):
    """phi(u) = (pi b)^(-1/2) exp(-u^2/b) in grid units."""
    u = np.atleast_1d(np.asarray(u, dtype=np.float64))
    return np.array([lib().orc_window(float(x), b) for x in u])


def window_hat(n, M: int, b: float):
    """M times the window's Fourier transform at integer frequency n."""
    n = np.atleast_1d(np.asarray(n, dtype=np.int64))
    return np.array([lib().orc_window_hat(int(x), M, b) for x in n])


# ---------------------------------------------------------------- FFT
def fft1d(x, sign: int = -1):
    a = np.ascontiguousarray(np.asarray(x, dtype=np.complex128)).copy()
    buf = a.view(np.float64)
    rc = lib().orc_fft1d(a.size, _dp(buf), sign)
    if rc != 0:
        raise ValueError("length must be a power of two")
    return a


def fft3d(x, sign: int = -1):
    """3D unnormalised FFT of a complex array indexed [z, y, x]."""
    a = np.ascontiguousarray(np.asarray(x, dtype=np.complex128)).copy()
    M = a.shape[0]
    assert a.shape == (M, M, M)
    rc = lib().orc_fft3d(M, _dp(a.view(np.float64)), sign)
    if rc != 0:
        raise ValueError("edge must be a power of two")
    return a


def spread(pos, q, L, M: int, p: int, n_c: int):
    """Spreading step only: the real grid g[z, y, x]."""
    pos = _arr(pos, (-1, 3)); q = _arr(q); L = _box(L)
    g = np.zeros((M, M, M), dtype=np.complex128)
    rc = lib().orc_spread(len(q), _dp(pos), _dp(q), _dp(L), M, p, window_b(M, n_c, p), _dp(g.view(np.float64)))
    if rc != 0:
        raise ValueError("bad arguments")
    return g.real.copy()


# ---------------------------------------------------------------- structure factors
def structure_factor_direct(pos, q, L, nc: int):
    """S(n) = sum_j q_j exp(-2 pi i n.x_j) on the cube |n_t| <= nc, indexed
    [nz+nc, ny+nc, nx+nc] (Eq. 37)."""
    pos = _arr(pos, (-1, 3)); q = _arr(q); L = _box(L)
    nn = 2 * nc + 1
    S = np.zeros((nn, nn, nn), dtype=np.complex128)
    lib().orc_structure_factor_direct(len(q), _dp(pos), _dp(q), _dp(L), nc, _dp(S.view(np.float64)))
    return S


def structure_factor_nfft(pos, q, L, M: int, p: int, nc: int):
    """S~(n) from the transposed NFFT (spread, FFT, scale), same indexing."""
    pos = _arr(pos, (-1, 3)); q = _arr(q); L = _box(L)
    nn = 2 * nc + 1
    S = np.zeros((nn, nn, nn), dtype=np.complex128)
    rc = lib().orc_structure_factor_nfft(len(q), _dp(pos), _dp(q), _dp(L), M, p, nc, _dp(S.view(np.float64)))
    if rc != 0:
        raise ValueError("bad NFFT parameters")
    return S


# ---------------------------------------------------------------- Ewald parts
@dataclass
class EwaldResult:
    E: float              # total energy
    E_real: float
    E_recip: float
    E_self: float
    E_background: float
    F: np.ndarray          # (n, 3) total force (real + reciprocal)
    phi: np.ndarray        # (n,) total potential dE/dq_i
    virial: np.ndarray     # (3, 3), W_ab = -dE/d eps_ab
    F_real: np.ndarray
    F_recip: np.ndarray
    phi_real: np.ndarray
    phi_recip: np.ndarray
    Q: float


def slater_factors(r, lambda_e):
    """ENUF-DPD correction factors (B_U, B_F) of Eq. 57-58 at distance r."""
    r = np.atleast_1d(np.asarray(r, dtype=np.float64))
    bu = np.zeros_like(r); bf = np.zeros_like(r)
    a, b = ctypes.c_double(), ctypes.c_double()
    for k, x in enumerate(r):
        lib().orc_slater_factors(float(x), float(lambda_e), ctypes.byref(a), ctypes.byref(b))
        bu[k], bf[k] = a.value, b.value
    return bu, bf


def real_space(pos, q, L, alpha, rc, ke=1.0, idx=None, slater=None):
    """Eq. 17 / Eq. 29: returns (E_R, F_R, phi_R, W_R); E_R and W_R are None
    when a subset ``idx`` is requested.  ``slater`` = lambda_e applies the
    ENUF-DPD factors of smeared Slater-type charges (Eq. 51-58) to every pair."""
    pos = _arr(pos, (-1, 3)); q = _arr(q); L = _box(L)
    N = len(q)
    if idx is not None:
        idx = np.ascontiguousarray(np.asarray(idx, dtype=np.int64))
        n = len(idx)
    else:
        n = N
    E = np.zeros(1); F = np.zeros((n, 3)); phi = np.zeros(n); W = np.zeros(9)
    if slater:
        lib().orc_real_space_slater(N, _dp(pos), _dp(q), _dp(L), alpha, rc, ke, float(slater),
                                    n if idx is not None else 0, _ip(idx), _dp(E), _dp(F), _dp(phi), _dp(W))
    else:
        lib().orc_real_space(N, _dp(pos), _dp(q), _dp(L), alpha, rc, ke, n if idx is not None else 0,
                             _ip(idx), _dp(E), _dp(F), _dp(phi), _dp(W))
    if idx is not None:
        return None, F, phi, None
    return float(E[0]), F, phi, W.reshape(3, 3)


def self_and_background(q, L, alpha, ke=1.0):
    q = _arr(q); L = _box(L)
    es = np.zeros(1); eb = np.zeros(1); Q = np.zeros(1)
    lib().orc_self_and_background(len(q), _dp(q), _dp(L), alpha, ke, _dp(es), _dp(eb), _dp(Q))
    return float(es[0]), float(eb[0]), float(Q[0])


def kspace_direct(pos, q, L, alpha, nmax, sphere=False, ke=1.0, idx=None):
    """O1 reciprocal part: (E_K, F_K, phi_K, W_K) over |n_t|<=nmax (cube) or
    |n|<=nmax (sphere).  With ``idx`` F/phi are only for those particles."""
    pos = _arr(pos, (-1, 3)); q = _arr(q); L = _box(L)
    N = len(q)
    if idx is not None:
        idx = np.ascontiguousarray(np.asarray(idx, dtype=np.int64))
    n = N if idx is None else len(idx)
    E = np.zeros(1); F = np.zeros((n, 3)); phi = np.zeros(n); W = np.zeros(9)
    rc = lib().orc_kspace_direct(N, _dp(pos), _dp(q), _dp(L), alpha, ke, int(nmax), int(bool(sphere)),
                                 _dp(E), _dp(F), _dp(phi), _dp(W), 0 if idx is None else n, _ip(idx))
    if rc != 0:
        raise MemoryError("oracle allocation failed")
    return float(E[0]), F, phi, W.reshape(3, 3)


def kspace_nfft(pos, q, L, alpha, M, p, nc=None, ke=1.0):
    """O2 reciprocal part: (E_K, F_K, phi_K, W_K) by NFFT."""
    pos = _arr(pos, (-1, 3)); q = _arr(q); L = _box(L)
    if nc is None:
        nc = M // 4
    N = len(q)
    E = np.zeros(1); F = np.zeros((N, 3)); phi = np.zeros(N); W = np.zeros(9)
    rc = lib().orc_kspace_nfft(N, _dp(pos), _dp(q), _dp(L), alpha, ke, M, p, nc, _dp(E), _dp(F), _dp(phi), _dp(W))
    if rc != 0:
        raise ValueError(f"bad NFFT parameters or allocation failure ({rc})")
    return float(E[0]), F, phi, W.reshape(3, 3)


def kspace_nfft_ad(pos, q, L, alpha, M, p, nc=None, ke=1.0):
    """O2-ad: the NFFT reciprocal energy of Eq. 38 with forces by analytic
    differentiation (one inverse FFT of the potential, window gradient in the
    interpolation); returns (E_K, F_K, phi_K, W_K) like :func:`kspace_nfft`."""
    pos = _arr(pos, (-1, 3)); q = _arr(q); L = _box(L)
    if nc is None:
        nc = M // 4
    N = len(q)
    E = np.zeros(1); F = np.zeros((N, 3)); phi = np.zeros(N); W = np.zeros(9)
    rc = lib().orc_kspace_nfft_ad(N, _dp(pos), _dp(q), _dp(L), alpha, ke, M, p, nc, _dp(E), _dp(F), _dp(phi),
                                  _dp(W))
    if rc != 0:
        raise ValueError(f"bad NFFT parameters or allocation failure ({rc})")
    return float(E[0]), F, phi, W.reshape(3, 3)


def window_deriv(u, b: float):
    """d phi/du of the Gaussian window in grid units."""
    u = np.atleast_1d(np.asarray(u, dtype=np.float64))
    return np.array([lib().orc_window_deriv(float(x), b) for x in u])


def nfft_ewald_ad(pos, q, L, alpha, rc, M, p, nc=None, ke=1.0) -> EwaldResult:
    """O2 with the reciprocal forces by analytic differentiation."""
    return _assemble(pos, q, L, alpha, rc, ke, kspace_nfft_ad(pos, q, L, alpha, M, p, nc, ke))


def _assemble(pos, q, L, alpha, rc, ke, kpart, idx=None, slater=None):
    Ek, Fk, phik, Wk = kpart
    Er, Fr, phir, Wr = real_space(pos, q, L, alpha, rc, ke, idx=idx, slater=slater)
    Es, Eb, Q = self_and_background(q, L, alpha, ke)
    qs = _arr(q) if idx is None else _arr(q)[np.asarray(idx)]
    V = float(np.prod(_box(L)))
    # d(E_self)/dq_i = -2 ke alpha/sqrt(pi) q_i ; d(E_bg)/dq_i = -ke pi Q/(V alpha^2)
    phi = phir + phik - 2.0 * ke * alpha / np.sqrt(np.pi) * qs - ke * np.pi * Q / (V * alpha * alpha)
    if idx is None:
        E = Er + Ek + Es + Eb
        W = Wr + Wk + Eb * np.eye(3)
    else:
        E = float("nan"); W = None; Er = float("nan")
    return EwaldResult(E=E, E_real=Er, E_recip=Ek, E_self=Es, E_background=Eb, F=Fr + Fk, phi=phi,
                       virial=W, F_real=Fr, F_recip=Fk, phi_real=phir, phi_recip=phik, Q=Q)


def direct_ewald(pos, q, L, alpha, rc, nmax, sphere=True, ke=1.0, idx=None, slater=None) -> EwaldResult:
    """O1: full Ewald sum with an explicit wave-vector set (``slater`` =
    lambda_e: the ENUF-DPD real-space factors, Eq. 57-58)."""
    return _assemble(pos, q, L, alpha, rc, ke, kspace_direct(pos, q, L, alpha, nmax, sphere, ke, idx=idx), idx,
                     slater=slater)


def nfft_ewald(pos, q, L, alpha, rc, M, p, nc=None, ke=1.0, slater=None) -> EwaldResult:
    """O2: Ewald sum with the reciprocal part by NFFT (``slater`` as in
    :func:`direct_ewald`)."""
    return _assemble(pos, q, L, alpha, rc, ke, kspace_nfft(pos, q, L, alpha, M, p, nc, ke), slater=slater)


def image_sum(pos, q, L, shell: int, ke=1.0) -> float:
    """Eq. 1 summed over image vectors |n| <= shell in spherical order."""
    pos = _arr(pos, (-1, 3)); q = _arr(q); L = _box(L)
    return float(lib().orc_image_sum(len(q), _dp(pos), _dp(q), _dp(L), ke, int(shell)))
