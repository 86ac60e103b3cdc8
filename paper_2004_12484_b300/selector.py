"""Parameter selection for ENUF plans (host logic).

The paper's procedure (Sec. 2.3.2 and Eq. 31-32): fix the accuracy delta and
the reciprocal cutoff n_c, obtain alpha and r_c from
    exp(-pi^2 n_c^2 / (alpha L)^2) <= delta,   erfc(alpha r_c) ~ exp(-alpha^2 r_c^2) <= delta,
and walk n_c upward until r_c suits the short-range cutoff.  This module
implements that search as a grid search over (alpha, r_c, M, p) -- n_c = M/4,
oversampling 2 -- that minimises a measured time model subject to an RMS
force-error estimate, and the legalisation of any proposed parameter set.

Error estimate (RMS force error per particle, absolute, for charges with
sum q^2 = Q in volume V):
  real-space truncation   dF_R^2 = q^2 (Q/V) int_{r_c}^inf 4 pi r^2 f(r)^2 dr,
                          f(r) = erfc(alpha r)/r^2 + 2 alpha/sqrt(pi) e^{-alpha^2 r^2}/r
  reciprocal truncation   dF_K^2 = q^2 (Q/V) 4 sqrt(pi/2) alpha erfc(k_c / (sqrt(2) alpha)),
                          k_c = 2 pi n_c / max(L)   (the sphere inside the kept cube)
  window (NFFT)           dF_W = eps_W(p) F_K,  eps_W = exp(-2 pi m (1 - 1/(2 sigma - 1))),
                          m = p/2, the Gaussian-window bound of the NFFT literature
                          (sigma = 2), F_K^2 = q^2 (Q/V) 4 sqrt(pi/2) alpha erf(...)
(both truncation terms follow from summing the neglected terms' variances for
uncorrelated positions; the window term is the relative accuracy of the
structure factor applied to the reciprocal force).  Errors are reported
relative to the force scale F0 = q_rms^2 rho^(2/3) (two typical charges at the
mean spacing), which stays finite for uniformly random positions where the
RMS of the total force does not.

Time model: t = sum of per-stage terms fitted to the library's own times on
this GPU (``timing_model.json``, written by ``calibrate.py``, which also
measures the window error).
"""
from __future__ import annotations

import json
import math
import os
from dataclasses import dataclass

import numpy as np
from scipy.special import erfc, erf

HERE = os.path.dirname(os.path.abspath(__file__))
TIMING_PATH = os.path.join(HERE, "timing_model.json")

GRID_SIZES = (16, 32, 64, 128, 256, 512)
WINDOWS = (2, 4, 6, 8, 10, 12)


@dataclass
class System:
    """What the selector needs to know about a system."""
    N: int
    L: tuple          # box edges
    Q: float          # sum of q^2
    charged_fraction: float = 1.0

    @property
    def V(self):
        return float(np.prod(self.L))

    @property
    def rho(self):
        return self.N / self.V

    @property
    def q2_mean(self):
        return self.Q / self.N

    @property
    def force_scale(self):
        """F0 = q_rms^2 rho^(2/3)."""
        return self.q2_mean * self.rho ** (2.0 / 3.0)


@dataclass
class Params:
    alpha: float
    r_c: float
    M: int
    p: int

    def as_dict(self):
        return dict(alpha=self.alpha, r_c=self.r_c, M=self.M, p=self.p, n_c=self.M // 4)


# ---------------------------------------------------------------- errors
# With x = alpha r the real-space integral becomes 4 pi alpha I(alpha r_c),
# I(u) = int_u^inf x^2 h(x)^2 dx, h(x) = erfc(x)/x^2 + 2/sqrt(pi) e^{-x^2}/x.
# I is tabulated once (Simpson's rule on a fine grid, integrated from the
# top down) and interpolated in log space.
def _build_real_table():
    x = np.linspace(1e-3, 14.0, 28001)
    h = erfc(x) / x ** 2 + 2.0 / math.sqrt(math.pi) * np.exp(-x * x) / x
    gx = x * x * h * h
    dx = x[1] - x[0]
    # cumulative trapezoid from the top, plus the tail beyond 14 (below 1e-80)
    seg = 0.5 * (gx[1:] + gx[:-1]) * dx
    tail = np.concatenate([np.cumsum(seg[::-1])[::-1], [0.0]])
    return x, np.log(np.maximum(tail, 1e-300))


_RX, _RLOGI = _build_real_table()


def real_integral(u):
    u = np.clip(np.asarray(u, dtype=np.float64), _RX[0], _RX[-1])
    return np.exp(np.interp(u, _RX, _RLOGI))


def real_error2(alpha, rc, sys_: System):
    """dF_R^2 per unit q_i^2 (vectorised over alpha, rc)."""
    alpha = np.asarray(alpha, dtype=np.float64)
    return sys_.Q / sys_.V * 4.0 * math.pi * alpha * real_integral(alpha * np.asarray(rc, dtype=np.float64))


def kspace_scale2(alpha, kc, sys_: System):
    return sys_.Q / sys_.V * 4.0 * math.sqrt(math.pi / 2.0) * np.asarray(alpha)


def kspace_error2(alpha, M, sys_: System):
    kc = 2.0 * math.pi * (np.asarray(M) // 4) / max(sys_.L)
    a = np.asarray(alpha, dtype=np.float64)
    return kspace_scale2(a, kc, sys_) * erfc(kc / (math.sqrt(2.0) * a))


def window_eps(p, sigma=2.0):
    """Relative RMS error of the reciprocal forces caused by the window: the
    values measured on this GPU by calibrate.py when present (window p
    against p = 12), else the Gaussian-window bound exp(-2 pi m (1 - 1/(2
    sigma - 1)))."""
    p = np.asarray(p)
    tab = _model().get("window_eps")
    if tab:
        return np.vectorize(lambda v: tab[str(int(v))])(p).astype(np.float64)
    m = p.astype(np.float64) / 2.0
    return np.exp(-2.0 * math.pi * m * (1.0 - 1.0 / (2.0 * sigma - 1.0)))


def window_error2(alpha, M, p, sys_: System):
    kc = 2.0 * math.pi * (np.asarray(M) // 4) / max(sys_.L)
    a = np.asarray(alpha, dtype=np.float64)
    fk2 = kspace_scale2(a, kc, sys_) * erf(kc / (math.sqrt(2.0) * a))
    return window_eps(p) ** 2 * fk2


def rms_force_error(prm: Params, sys_: System) -> float:
    """Estimated RMS force error relative to F0 = q_rms^2 rho^(2/3)."""
    e2 = (real_error2(prm.alpha, prm.r_c, sys_) + kspace_error2(prm.alpha, prm.M, sys_)
          + window_error2(prm.alpha, prm.M, prm.p, sys_))
    return float(np.sqrt(e2 * sys_.q2_mean)) / sys_.force_scale


# ---------------------------------------------------------------- time
DEFAULT_TIMING = {
    # seconds; fitted by calibrate.py on the GPU (these defaults are only a
    # placeholder shape used before calibration)
    "t0": 3.0e-5, "sort_per_particle": 2.0e-10, "spread_per_point": 2.5e-12,
    "gather_per_point": 3.5e-12, "fft_per_cell": 6.0e-11, "real_per_pair": 4.0e-12,
}


_MODEL = None


def _model():
    global _MODEL
    if _MODEL is None:
        _MODEL = {}
        if os.path.exists(TIMING_PATH):
            with open(TIMING_PATH) as f:
                _MODEL = json.load(f)
    return _MODEL


def load_timing():
    return dict(_model().get("coef", DEFAULT_TIMING))


def predicted_time(prm_alpha, rc, M, p, sys_: System, coef=None, kspace_only=False):
    """Seconds for one full evaluation (k-space + real space) on this GPU."""
    c = coef or load_timing()
    M = np.asarray(M, dtype=np.float64)
    p = np.asarray(p, dtype=np.float64)
    rc = np.asarray(rc, dtype=np.float64)
    N = sys_.N
    t = (c["t0"] + c["sort_per_particle"] * N + (c["spread_per_point"] + c["gather_per_point"]) * N * p ** 3
         + c["fft_per_cell"] * M ** 3)
    if not kspace_only:
        # linked cells of edge >= r_c: each particle visits 27 cells
        cell = np.maximum(rc, 1e-9)
        t = t + c["real_per_pair"] * N * sys_.rho * 27.0 * cell ** 3
    return t


# ---------------------------------------------------------------- search
def legal(prm: Params, sys_: System) -> Params:
    """Nearest parameter set the library accepts."""
    M = int(min(GRID_SIZES, key=lambda g: abs(math.log2(g) - math.log2(max(prm.M, 1e-9)))))
    p = int(min(WINDOWS, key=lambda w: abs(w - prm.p)))
    p = min(p, M)
    rc = float(min(max(prm.r_c, 1e-6), 0.5 * min(sys_.L)))
    a = float(max(prm.alpha, 1e-6))
    return Params(a, rc, M, p)


def grid_search(sys_: System, target: float, coef=None, n_alpha=48):
    """Time-optimal (alpha, r_c, M, p) whose estimated RMS force error
    (relative to F0) is at most `target`.  For each grid size and window, alpha
    runs over a log grid; r_c is the smallest cutoff that keeps the real-space
    error within its share.  Returns (Params, predicted seconds, estimate) or
    None if nothing in range meets the target."""
    coef = coef or load_timing()
    a_spacing = sys_.rho ** (-1.0 / 3.0)
    alphas = np.geomspace(0.05 / a_spacing, 6.0 / a_spacing, n_alpha)
    rc_max = 0.5 * min(sys_.L)
    rcs = np.geomspace(0.5 * a_spacing, rc_max, 96)
    rcs = rcs[rcs <= rc_max]
    tgt2 = (target * sys_.force_scale) ** 2 / sys_.q2_mean
    er_real = real_error2(alphas[:, None], rcs[None, :], sys_)  # (alpha, rc)
    best = None
    for M in GRID_SIZES:
        ek = kspace_error2(alphas, M, sys_)
        for p in WINDOWS:
            if p > M:
                continue
            ew = window_error2(alphas, M, p, sys_)
            budget = tgt2 - ek - ew  # left for the real-space error
            ok = er_real <= budget[:, None]
            has = ok.any(1) & (budget > 0)
            if not has.any():
                continue
            # smallest admissible r_c for each alpha (er_real decreases in rc)
            first = np.argmax(ok, axis=1)
            rc_sel = rcs[first]
            t = predicted_time(alphas, rc_sel, M, p, sys_, coef)
            t = np.where(has, t, np.inf)
            i = int(np.argmin(t))
            if np.isfinite(t[i]) and (best is None or t[i] < best[1]):
                prm = Params(float(alphas[i]), float(rc_sel[i]), M, p)
                best = (prm, float(t[i]), rms_force_error(prm, sys_))
    return best


def paper_procedure(sys_: System, delta: float, r_c: float, sigma_grid=2):
    """The paper's own recipe (Sec. 2.3.2, Eq. 31-32): with accuracy delta and
    a fixed short-range cutoff r_c, alpha = sqrt(-ln delta) / r_c (Eq. 32),
    then the smallest n_c with exp(-pi^2 n_c^2/(alpha L)^2) <= delta (Eq. 31),
    M = the smallest supported grid with M/4 >= n_c."""
    alpha = math.sqrt(-math.log(delta)) / r_c
    n_c = math.ceil(alpha * max(sys_.L) / math.pi * math.sqrt(-math.log(delta)))
    M = next((g for g in GRID_SIZES if g // 4 >= n_c), GRID_SIZES[-1])
    return Params(alpha, r_c, M, 6)


# ---------------------------------------------------------------- descriptors
def descriptor(sys_: System, target: float) -> np.ndarray:
    """The 6 inputs of the learned selector: log N, density, charged
    fraction, charge variance (mean q^2), box anisotropy (max/min edge),
    log10 target error."""
    L = np.asarray(sys_.L, dtype=np.float64)
    return np.array([math.log(sys_.N), sys_.rho, sys_.charged_fraction, sys_.q2_mean,
                     float(L.max() / L.min()), math.log10(target)], dtype=np.float64)
