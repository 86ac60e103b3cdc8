"""ENUF on one B300: Ewald summation with the reciprocal-space sum evaluated by
non-uniform FFTs (Yang et al., arXiv:2004.12484), as hand-written sm_103a CUDA
kernels behind the C ABI of ``include/enuf.h``.

This module is the thin Python binding: it marshals torch tensors (device
memory and the current CUDA stream) into the C calls of ``libenuf.so`` and
turns error codes into exceptions.  Every step of the method runs in the
library's kernels; there is no Python or CPU fallback, and importing fails
loudly when the library has not been built.

    plan = Plan(L=(187.1,)*3, N=65536, alpha=0.2116, r_c=12.0, M=128, p=6)
    res = plan.compute(pos, q)            # asynchronous, device results
    E, F, W, phi = plan.energy_forces(pos, q)
    E = EnufEnergy.apply(pos, q, plan)    # differentiable in pos and q
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
# ENUF_BOUNDS_CHECK=1 in the environment selects the checked build of the
# library (bounds checks in every kernel; same entry points and results)
LIB_PATH = os.path.join(_HERE, "libenuf_check.so" if os.environ.get("ENUF_BOUNDS_CHECK") == "1" else "libenuf.so")

FP64 = 0
MIXED = 1
WANT_VIRIAL = 1
WANT_PHI = 2
REMOVE_NET_FORCE = 4
KSPACE_ONLY = 8
AD_FORCES = 16
NOUT = 16
OUT = dict(E=0, E_real=1, E_recip=2, E_self=3, E_bg=4, Q=5, virial=6, status=15)


class EnufError(RuntimeError):
    pass


class EnufParams(ctypes.Structure):
    _fields_ = [
        ("L", ctypes.c_double * 3),
        ("N", ctypes.c_int64),
        ("alpha", ctypes.c_double),
        ("r_c", ctypes.c_double),
        ("M", ctypes.c_int),
        ("p", ctypes.c_int),
        ("n_c", ctypes.c_int),
        ("precision", ctypes.c_int),
        ("coulomb_k", ctypes.c_double),
        ("flags", ctypes.c_int),
        ("slater_lambda", ctypes.c_double),
    ]


_lib = None
_vp = ctypes.c_void_p


def lib():
    """The loaded ``libenuf.so``; raises if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} is missing: build it with "
                              "`python -m paper_2004_12484_b300.build` (or __graft_entry__.build())")
        L = ctypes.CDLL(LIB_PATH)
        L.enuf_last_error.restype = ctypes.c_char_p
        L.enuf_bounds_status.argtypes = [ctypes.POINTER(ctypes.c_ulonglong), ctypes.c_char_p, ctypes.c_int,
                                         ctypes.c_int]
        L.enuf_version.restype = ctypes.c_char_p
        L.enuf_plan_workspace_bytes.argtypes = [ctypes.POINTER(EnufParams), ctypes.POINTER(ctypes.c_size_t)]
        L.enuf_md_run.argtypes = [_vp, _vp, _vp, _vp, _vp, _vp, ctypes.c_int, ctypes.c_double, ctypes.c_int,
                                  ctypes.c_int, _vp]
        L.enuf_backward_flags.argtypes = [_vp, _vp, _vp, _vp, _vp, _vp, ctypes.c_int]
        L.enuf_plan_create.argtypes = [ctypes.POINTER(EnufParams), _vp, ctypes.c_int, ctypes.POINTER(_vp)]
        L.enuf_plan_set_workspace.argtypes = [_vp, _vp, ctypes.c_size_t]
        L.enuf_plan_set_stream.argtypes = [_vp, _vp]
        L.enuf_plan_get_params.argtypes = [_vp, ctypes.POINTER(EnufParams)]
        L.enuf_plan_destroy.argtypes = [_vp]
        L.enuf_compute.argtypes = [_vp, _vp, _vp, _vp, _vp, _vp, ctypes.c_int]
        L.enuf_energy_forces.argtypes = [_vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, ctypes.c_int]
        L.enuf_energy_forces_host.argtypes = [_vp, _vp, _vp, _vp, _vp, _vp, _vp, ctypes.c_int]
        L.enuf_backward.argtypes = [_vp, _vp, _vp, _vp, _vp, _vp]
        L.enuf_last_timings.argtypes = [_vp, ctypes.POINTER(ctypes.c_char_p), ctypes.POINTER(ctypes.c_float), ctypes.c_int]
        L.enuf_launch_count.argtypes = [_vp, ctypes.c_int, ctypes.c_int]
        L.enuf_real_space_noalloc.argtypes = [_vp, _vp, ctypes.c_int64, ctypes.POINTER(ctypes.c_double),
                                              ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_int,
                                              _vp, _vp, _vp, _vp]
        L.enuf_structure_factor.argtypes = [_vp, _vp, _vp, _vp]
        L.enuf_fft_forward.argtypes = [_vp, _vp, _vp]
        _lib = L
    return _lib


def _check(rc):
    if rc != 0:
        raise EnufError(f"enuf error {rc}: {lib().enuf_last_error().decode()}")


def version() -> str:
    return lib().enuf_version().decode()


def make_params(L, N, alpha, r_c, M, p, n_c=0, precision="mixed", coulomb_k=1.0, slater_lambda=0.0) -> EnufParams:
    Lv = np.broadcast_to(np.asarray(L, dtype=np.float64).reshape(-1), (3,))
    prm = EnufParams()
    for t in range(3):
        prm.L[t] = float(Lv[t])
    prm.N = int(N)
    prm.alpha = float(alpha)
    prm.r_c = float(r_c)
    prm.M = int(M)
    prm.p = int(p)
    prm.n_c = int(n_c)
    prm.precision = {"fp64": FP64, "mixed": MIXED}.get(precision, precision) if isinstance(precision, str) \
        else int(precision)
    prm.coulomb_k = float(coulomb_k)
    prm.flags = 0
    prm.slater_lambda = float(slater_lambda)
    return prm


def workspace_bytes(**kw) -> int:
    prm = make_params(**kw)
    n = ctypes.c_size_t()
    _check(lib().enuf_plan_workspace_bytes(ctypes.byref(prm), ctypes.byref(n)))
    return n.value


class Plan:
    """An ENUF plan: fixed box, particle count and method parameters.  The
    device workspace is a torch tensor owned by the plan."""

    def __init__(self, L, N, alpha, r_c, M, p, n_c=0, precision="mixed", coulomb_k=1.0, device=None,
                 slater_lambda=0.0):
        import torch
        self.torch = torch
        self.device = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
        self.params = make_params(L, N, alpha, r_c, M, p, n_c, precision, coulomb_k, slater_lambda)
        self.dtype = torch.float64 if self.params.precision == FP64 else torch.float32
        self.N = int(N)
        nbytes = ctypes.c_size_t()
        _check(lib().enuf_plan_workspace_bytes(ctypes.byref(self.params), ctypes.byref(nbytes)))
        self.workspace_bytes = nbytes.value
        with torch.cuda.device(self.device):
            self._ws = torch.empty(nbytes.value + 256, dtype=torch.uint8, device=self.device)
            base = self._ws.data_ptr()
            aligned = (base + 255) // 256 * 256
            h = _vp()
            _check(lib().enuf_plan_create(ctypes.byref(self.params), _vp(torch.cuda.current_stream().cuda_stream), 0,
                                          ctypes.byref(h)))
            self._h = h
            _check(lib().enuf_plan_set_workspace(self._h, _vp(aligned), nbytes.value))
        got = EnufParams()
        _check(lib().enuf_plan_get_params(self._h, ctypes.byref(got)))
        self.n_c = got.n_c
        self.M, self.p = got.M, got.p
        self.alpha, self.r_c = got.alpha, got.r_c
        self.L = tuple(got.L)
        self.coulomb_k = got.coulomb_k
        self.precision = "fp64" if got.precision == FP64 else "mixed"

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and _lib is not None:
            _lib.enuf_plan_destroy(h)
            self._h = None

    # ----------------------------------------------------------- helpers
    def _sync_stream(self):
        _check(lib().enuf_plan_set_stream(self._h, _vp(self.torch.cuda.current_stream(self.device).cuda_stream)))

    def _dev(self, t, shape, name):
        torch = self.torch
        if not isinstance(t, torch.Tensor) or t.device != self.device or t.dtype != self.dtype:
            raise TypeError(f"{name} must be a {self.dtype} tensor on {self.device}")
        if tuple(t.shape) != shape or not t.is_contiguous():
            raise ValueError(f"{name} must be contiguous with shape {shape}")
        return t

    @staticmethod
    def flags(virial=True, phi=False, kspace_only=False, remove_net_force=False, ad=False) -> int:
        return ((WANT_VIRIAL if virial else 0) | (WANT_PHI if phi else 0) | (KSPACE_ONLY if kspace_only else 0)
                | (REMOVE_NET_FORCE if remove_net_force else 0) | (AD_FORCES if ad else 0))

    # ----------------------------------------------------------- calls
    def compute(self, pos, q, forces=True, phi=False, virial=True, kspace_only=False, remove_net_force=False,
                F=None, phi_out=None, out=None, ad=False):
        """Asynchronous evaluation on the current stream.  Returns
        (out[16] float64, F (N,3) or None, phi (N,) or None), all on the
        device.  ``ad=True`` takes the reciprocal forces by analytic
        differentiation (one inverse transform, window gradient)."""
        torch = self.torch
        self._dev(pos, (self.N, 3), "pos")
        self._dev(q, (self.N,), "q")
        if forces and F is None:
            F = torch.empty((self.N, 3), dtype=self.dtype, device=self.device)
        if phi and phi_out is None:
            phi_out = torch.empty((self.N,), dtype=self.dtype, device=self.device)
        if out is None:
            out = torch.empty((NOUT,), dtype=torch.float64, device=self.device)
        self._sync_stream()
        fl = self.flags(virial, phi, kspace_only, remove_net_force, ad)
        _check(lib().enuf_compute(self._h, _vp(pos.data_ptr()), _vp(q.data_ptr()),
                                  _vp(F.data_ptr() if forces else 0), _vp(phi_out.data_ptr() if phi else 0),
                                  _vp(out.data_ptr()), fl))
        return out, (F if forces else None), (phi_out if phi else None)

    def energy_forces(self, pos, q, phi=False, kspace_only=False, remove_net_force=False, ad=False):
        """Synchronous: returns (parts dict of floats, F tensor, virial 3x3
        numpy array, phi tensor or None)."""
        out, F, ph = self.compute(pos, q, True, phi, True, kspace_only, remove_net_force, ad=ad)
        h = out.cpu().numpy()
        st = int(h[OUT["status"]])
        if st & 1:
            raise EnufError("a position or charge is NaN or infinite")
        if st:
            raise EnufError(f"device status {st}")
        parts = {k: float(h[i]) for k, i in OUT.items() if k not in ("virial", "status")}
        return parts, F, h[6:15].reshape(3, 3).copy(), ph

    def __call__(self, pos, q, ad=False):
        """plan(pos, q) -> (E, F, virial): the total energy (float), the forces
        (device tensor, N x 3) and the 3 x 3 virial (numpy), synchronously."""
        parts, F, W, _ = self.energy_forces(pos, q, ad=ad)
        return parts["E"], F, W

    def energy_forces_host(self, pos_host, q_host, phi_host=None, F_host=None, kspace_only=False, ad=False):
        """End-to-end call with host (numpy or pinned torch CPU) buffers; the
        copies in and out are part of the call."""
        torch = self.torch
        fl = self.flags(True, phi_host is not None, kspace_only, ad=ad)
        E = ctypes.c_double()
        W = (ctypes.c_double * 9)()

        def ptr(a):
            if a is None:
                return 0
            if isinstance(a, torch.Tensor):
                assert a.device.type == "cpu" and a.dtype == self.dtype and a.is_contiguous()
                return a.data_ptr()
            assert a.dtype == (np.float64 if self.dtype == torch.float64 else np.float32) and a.flags.c_contiguous
            return a.ctypes.data

        self._sync_stream()
        _check(lib().enuf_energy_forces_host(self._h, _vp(ptr(pos_host)), _vp(ptr(q_host)), ctypes.byref(E),
                                             _vp(ptr(F_host)), W, _vp(ptr(phi_host)), fl))
        return E.value, np.array(W[:]).reshape(3, 3)

    def md_run(self, pos, vel, q, inv_mass, dt, nsteps, F=None, have_forces=False, ad=False,
               remove_net_force=False, kspace_only=False, energies=None):
        """nsteps velocity-Verlet steps on the device (pos and vel updated in
        place).  Returns (energies (nsteps, 4) float64 tensor: E_pot, E_kin,
        E_tot, status per step; F at the final positions)."""
        torch = self.torch
        self._dev(pos, (self.N, 3), "pos")
        self._dev(vel, (self.N, 3), "vel")
        self._dev(q, (self.N,), "q")
        self._dev(inv_mass, (self.N,), "inv_mass")
        if F is None:
            F = torch.empty((self.N, 3), dtype=self.dtype, device=self.device)
            have_forces = False
        if energies is None:
            energies = torch.empty((max(int(nsteps), 1), 4), dtype=torch.float64, device=self.device)
        fl = self.flags(False, False, kspace_only, remove_net_force, ad)
        self._sync_stream()
        _check(lib().enuf_md_run(self._h, _vp(pos.data_ptr()), _vp(vel.data_ptr()), _vp(q.data_ptr()),
                                 _vp(inv_mass.data_ptr()), _vp(F.data_ptr()), 1 if have_forces else 0, float(dt),
                                 int(nsteps), fl, _vp(energies.data_ptr())))
        return energies[:nsteps], F

    def backward(self, pos, q, gE=None, dpos=None, dq=None, ad=False):
        """dpos = -gE F, dq = gE phi (recomputed; gE a 1-element float64
        device tensor or None for 1).  ad=True: F by analytic differentiation,
        the exact gradient of the returned energy."""
        torch = self.torch
        self._dev(pos, (self.N, 3), "pos")
        self._dev(q, (self.N,), "q")
        if dpos is None:
            dpos = torch.empty((self.N, 3), dtype=self.dtype, device=self.device)
        if dq is None:
            dq = torch.empty((self.N,), dtype=self.dtype, device=self.device)
        g = 0
        if gE is not None:
            gE = gE.detach().to(device=self.device, dtype=torch.float64).reshape(1).contiguous()
            g = gE.data_ptr()
        self._sync_stream()
        _check(lib().enuf_backward_flags(self._h, _vp(pos.data_ptr()), _vp(q.data_ptr()), _vp(g),
                                         _vp(dpos.data_ptr()), _vp(dq.data_ptr()), AD_FORCES if ad else 0))
        self._keep = gE  # keep the scalar alive until the stream consumes it
        return dpos, dq

    def _spectrum(self):
        nn, kx = 2 * self.n_c + 1, self.n_c + 1
        ct = self.torch.complex128 if self.dtype == self.torch.float64 else self.torch.complex64
        return self.torch.empty((nn, nn, kx), dtype=ct, device=self.device)

    def structure_factor(self, pos, q):
        """S~(n) on the retained half cube, a (2 n_c + 1, 2 n_c + 1, n_c + 1)
        complex device tensor indexed [n_z + n_c, n_y + n_c, n_x] (synchronous)."""
        self._dev(pos, (self.N, 3), "pos")
        self._dev(q, (self.N,), "q")
        S = self._spectrum()
        self._sync_stream()
        _check(lib().enuf_structure_factor(self._h, _vp(pos.data_ptr()), _vp(q.data_ptr()), _vp(S.data_ptr())))
        return S

    def fft_forward(self, grid):
        """The library's forward FFT of a real (M, M, M) [z, y, x] device grid
        on the retained half cube (same indexing as structure_factor)."""
        M = self.M
        self._dev(grid, (M, M, M), "grid")
        G = self._spectrum()
        self._sync_stream()
        _check(lib().enuf_fft_forward(self._h, _vp(grid.data_ptr()), _vp(G.data_ptr())))
        return G

    def launch_count(self, flags: int, forces: bool = True) -> int:
        n = lib().enuf_launch_count(self._h, int(flags), 1 if forces else 0)
        if n < 0:
            _check(n)
        return n

    def timings(self):
        cap = 64
        names = (ctypes.c_char_p * cap)()
        times = (ctypes.c_float * cap)()
        n = lib().enuf_last_timings(self._h, names, times, cap)
        if n < 0:
            _check(n)
        return [(names[i].decode(), float(times[i])) for i in range(n)]


def real_space_noalloc(pos, q, L, alpha, r_c, coulomb_k=1.0, F=None, phi=None, out=None):
    """Real-space pair sum through the entry point that allocates no device
    memory inside the library (for callers that cannot allocate; see
    include/enuf.h).  pos, q: float32 or float64 CUDA tensors.  Returns
    (out[10] = E_real and its virial, F, phi) on the device; asynchronous on
    the current stream.  Buffers not given are allocated here by torch, in
    the caller's process, before the call."""
    import torch
    dt = pos.dtype
    prec = FP64 if dt == torch.float64 else MIXED
    N = q.shape[0]
    if F is None:
        F = torch.empty((N, 3), dtype=dt, device=pos.device)
    if phi is None:
        phi = torch.empty((N,), dtype=dt, device=pos.device)
    if out is None:
        out = torch.empty((10,), dtype=torch.float64, device=pos.device)
    Lv = (ctypes.c_double * 3)(*[float(x) for x in np.broadcast_to(np.asarray(L, dtype=np.float64).reshape(-1), (3,))])
    _check(lib().enuf_real_space_noalloc(_vp(pos.data_ptr()), _vp(q.data_ptr()), int(N), Lv, float(alpha),
                                         float(r_c), float(coulomb_k), prec, _vp(F.data_ptr()),
                                         _vp(phi.data_ptr()), _vp(out.data_ptr()),
                                         _vp(torch.cuda.current_stream(pos.device).cuda_stream)))
    return out, F, phi


def _autograd():
    import torch

    class EnufEnergy(torch.autograd.Function):
        """E(pos, q) as a differentiable torch function.  forward returns the
        total energy (0-dim float64); backward returns dE/dpos = -F and
        dE/dq = phi, recomputing the grids through the library (no grid is
        stored between the two passes).  apply(pos, q, plan, True) takes F by
        analytic differentiation: the exact gradient of the returned energy."""

        @staticmethod
        def forward(ctx, pos, q, plan, ad=False):
            if getattr(plan, "_eout", None) is None:
                plan._eout = torch.empty((NOUT,), dtype=torch.float64, device=plan.device)
            out, _, _ = plan.compute(pos.detach(), q.detach(), forces=False, phi=False, virial=False,
                                     out=plan._eout)
            ctx.plan = plan
            ctx.ad = bool(ad)
            ctx.save_for_backward(pos, q)
            return out[0].clone()

        @staticmethod
        def backward(ctx, gE):
            pos, q = ctx.saved_tensors
            dpos, dq = ctx.plan.backward(pos.detach().contiguous(), q.detach().contiguous(), gE, ad=ctx.ad)
            return dpos, dq, None, None

    return EnufEnergy


class _Lazy:
    _cls = None

    def __getattr__(self, k):
        if _Lazy._cls is None:
            _Lazy._cls = _autograd()
        return getattr(_Lazy._cls, k)


EnufEnergy = _Lazy()
