"""Seeded synthetic inputs shaped like the paper's workloads.

This module only draws positions and charges (numpy PCG64, seed stated per
workload) and records each workload's plan parameters as plain numbers.  It
contains none of the method's arithmetic, and both the oracle-side tests and
the CUDA-side tests/benchmark take their inputs from it.

The paper's simulation systems (ionic liquids, polyelectrolytes, dendrimers;
Sec. 4) are not public data, so these generators stand in for their shapes:

* ``nacl``      rock-salt crystal, 4x4x4 conventional cells, 512 ions
                (the Madelung check of Sec. 2.4.2 uses an FCC +-1 lattice).
* ``rpm``       restricted-primitive-model electrolyte, 65,536 ions at
                0.01 per cubic Angstrom, uniform positions.
* ``polyelectrolyte``  1,048,576 bead-spring chain beads (random walks,
                bond 0.97 sigma) with every second bead charged -1, plus
                524,288 +1 counterions, density 0.85 sigma^-3.
* ``ionic_liquid``  8,388,608 sites, 4 per ion pair (cation: one +0.8 site
                and two neutral sites; anion: one -0.8 site), half of the
                pairs clustered around 10^6 centres (Gaussian, 2 Angstrom),
                density 0.1 per cubic Angstrom.

The Ewald parameter alpha recorded for the polyelectrolyte workload is the
value that balances the two truncation errors for the given r_c and n_c, r_c
= pi n_c / (alpha^2 L) (Eq. 32), rounded to four digits; the RPM and
ionic-liquid values are stated at ``rpm``, ``rpm_1e4`` and
``ionic_liquid``.  ``rpm_1e4`` and
``polyelectrolyte_1e4`` are the same systems with the smallest parameter
changes that meet a 1e-4 relative RMS force error; the ionic-liquid settings
meet their 1e-5 target.
"""
from __future__ import annotations

import numpy as np

NACL_A = 5.64


def _rng(seed):
    return np.random.Generator(np.random.PCG64(seed))


def rock_salt(cells=4, a=NACL_A, jitter=0.0, seed=1):
    """Rock-salt (NaCl) lattice: FCC cations + FCC anions shifted by a/2."""
    base = np.array([[0, 0, 0], [0, .5, .5], [.5, 0, .5], [.5, .5, 0]], dtype=np.float64)
    pos, q = [], []
    for i in range(cells):
        for j in range(cells):
            for k in range(cells):
                o = np.array([i, j, k], dtype=np.float64)
                for b in base:
                    pos.append((o + b) * a); q.append(1.0)
                    pos.append((o + b + np.array([.5, 0, 0])) * a); q.append(-1.0)
    pos = np.array(pos); q = np.array(q)
    if jitter > 0:
        pos = pos + _rng(seed).normal(0.0, jitter, size=pos.shape)
    L = np.full(3, cells * a)
    return pos, q, L


def cesium_chloride(cells=4, a=4.12):
    """CsCl lattice: simple cubic cations with anions at the cube centres."""
    pos, q = [], []
    for i in range(cells):
        for j in range(cells):
            for k in range(cells):
                o = np.array([i, j, k], dtype=np.float64)
                pos.append(o * a); q.append(1.0)
                pos.append((o + 0.5) * a); q.append(-1.0)
    return np.array(pos), np.array(q), np.full(3, cells * a)


def nacl(seed=1):
    """512-ion rock salt, Gaussian displacements sigma = 0.1 A, FP64 plan."""
    pos, q, L = rock_salt(4, NACL_A, jitter=0.1, seed=seed)
    return dict(name="nacl", pos=pos, q=q, L=L, alpha=0.35, r_c=9.0, M=32, p=4, n_c=8,
                precision="fp64", seed=seed)


def rpm(N=65536, density=0.01, seed=2, M=128, p=6, r_c=12.0, alpha=0.23):
    """Restricted primitive model: N/2 cations +1, N/2 anions -1, uniform.
    Grid 128^3, p = 6, r_c = 12 A as the workload names them; alpha = 0.23 is
    the value with the smallest measured RMS force error at these settings
    (4.1e-4 relative to converged Ewald; the p = 6 window caps it)."""
    L = (N / density) ** (1.0 / 3.0)
    g = _rng(seed)
    pos = g.uniform(0.0, L, size=(N, 3))
    q = np.where(np.arange(N) % 2 == 0, 1.0, -1.0)
    return dict(name="rpm", pos=pos, q=q, L=np.full(3, L), alpha=alpha, r_c=r_c, M=M, p=p, n_c=M // 4,
                precision="mixed", seed=seed)


def rpm_1e4(**kw):
    """The RPM electrolyte with the smallest changes that meet a 1e-4 relative
    RMS force error (measured 7.9e-5 against converged Ewald): window p = 8,
    r_c = 14.5 A, alpha = 0.215, same 128^3 grid."""
    kw.setdefault("p", 8)
    kw.setdefault("r_c", 14.5)
    kw.setdefault("alpha", 0.215)
    d = rpm(**kw)
    d["name"] = "rpm_1e-4"
    return d


def polyelectrolyte(n_beads=1048576, chain=50, density=0.85, bond=0.97, seed=3, M=256, p=6,
                    r_c=3.0, alpha=0.7389):
    """Bead-spring chains (random walks) + counterions.  Beads at odd in-chain
    index carry -1; one +1 counterion per charged bead."""
    g = _rng(seed)
    n_charged = 0
    chains = []
    left = n_beads
    starts = []
    while left > 0:
        n = min(chain, left)
        chains.append(n); left -= n
    n_ci = sum(n // 2 for n in chains)
    N = n_beads + n_ci
    L = (N / density) ** (1.0 / 3.0)
    pos = np.empty((N, 3)); q = np.zeros(N)
    o = 0
    for n in chains:
        start = g.uniform(0.0, L, size=3)
        v = g.normal(size=(n - 1, 3))
        v *= bond / np.linalg.norm(v, axis=1, keepdims=True)
        pos[o] = start
        pos[o + 1:o + n] = start + np.cumsum(v, axis=0)
        q[o + 1:o + n:2] = -1.0
        n_charged += n // 2
        o += n
    pos[o:] = g.uniform(0.0, L, size=(n_ci, 3))
    q[o:] = 1.0
    pos = np.mod(pos, L)
    return dict(name="polyelectrolyte", pos=pos, q=q, L=np.full(3, L), alpha=alpha, r_c=r_c, M=M, p=p,
                n_c=M // 4, precision="mixed", seed=seed, n_beads=n_beads)


def polyelectrolyte_1e4(**kw):
    """The polyelectrolyte system with the smallest changes that meet a 1e-4
    relative RMS force error against converged Ewald (grid 256^3 unchanged):
    the stated p = 6 window and r_c = 3 sigma give about 7e-4 (the window and
    the real-space truncation both exceed the target), p = 8 with r_c = 4.3
    sigma and alpha = 0.70 give about 6e-5 (measured with the oracle on
    1/8- and 1/64-volume copies of the system at the same density and grid
    spacing)."""
    kw.setdefault("p", 8)
    kw.setdefault("r_c", 4.3)
    kw.setdefault("alpha", 0.70)
    d = polyelectrolyte(**kw)
    d["name"] = "polyelectrolyte_1e-4"
    return d


def ionic_liquid(N=8388608, density=0.1, n_centres=1_000_000, blob=2.0, seed=4, M=512, p=8,
                 r_c=11.7, alpha=0.32):
    """Coarse-grained ionic-liquid-like sites with clustered placement.
    alpha = 0.32 and r_c = 11.7 A: at the fixed grid (512^3, p = 8, n_c =
    128) the reciprocal cost does not depend on alpha, so the time-optimal
    choice is the largest alpha (shortest r_c) whose total RMS force error
    stays below the 1e-5 target; measured with the oracle on a 1/8-volume
    copy of the system (same density, clustering and grid spacing): 6.4e-6
    at (0.32, 11.7), 8.2e-6 at (0.33, 11.3), 1.2e-5 at (0.34, 11.0), and
    4.4e-6 at the Eq. 32 balance (0.2562, 14.0), which costs 1.7x the
    real-space work."""
    assert N % 4 == 0
    g = _rng(seed)
    L = (N / density) ** (1.0 / 3.0)
    npair = N // 4
    centres = g.uniform(0.0, L, size=(n_centres, 3))
    clustered = g.random(npair) < 0.5
    anchor = g.uniform(0.0, L, size=(npair, 3))
    pick = g.integers(0, n_centres, size=npair)
    anchor[clustered] = centres[pick[clustered]] + g.normal(0.0, blob, size=(int(clustered.sum()), 3))

    def ball(n, r):
        v = g.normal(size=(n, 3))
        v /= np.linalg.norm(v, axis=1, keepdims=True)
        return v * (r * g.random((n, 1)) ** (1.0 / 3.0))

    def shell(n, r):
        v = g.normal(size=(n, 3))
        return v * (r / np.linalg.norm(v, axis=1, keepdims=True))

    pos = np.empty((N, 3)); q = np.empty(N)
    pos[0::4] = anchor;                    q[0::4] = 0.8
    pos[1::4] = anchor + ball(npair, 1.5); q[1::4] = 0.0
    pos[2::4] = anchor + ball(npair, 1.5); q[2::4] = 0.0
    pos[3::4] = anchor + shell(npair, 4.0); q[3::4] = -0.8
    pos = np.mod(pos, L)
    return dict(name="ionic_liquid", pos=pos, q=q, L=np.full(3, L), alpha=alpha, r_c=r_c, M=M, p=p,
                n_c=M // 4, precision="mixed", seed=seed)


def ionic_liquid_eighth(seed=45):
    """A 1/8-volume copy of the ionic-liquid workload (1,048,576 sites, box
    218.9 A, 125,000 cluster centres, grid 256^3: the same density,
    clustering, grid spacing and method parameters), small enough for
    detailed profiler captures and CPU accuracy studies."""
    d = ionic_liquid(N=1048576, n_centres=125000, seed=seed, M=256)
    d["name"] = "ionic_liquid_eighth"
    return d


def random_neutral(N, L, seed, charged_fraction=1.0, anisotropy=1.0):
    """Uniform positions, +-1 charges on a random charged fraction, neutral."""
    g = _rng(seed)
    Lv = np.array([L * anisotropy, L, L], dtype=np.float64)
    pos = g.uniform(0.0, 1.0, size=(N, 3)) * Lv
    nq = max(2, int(round(charged_fraction * N)) // 2 * 2)
    q = np.zeros(N)
    sel = g.permutation(N)[:nq]
    q[sel[: nq // 2]] = 1.0
    q[sel[nq // 2:]] = -1.0
    return pos, q, Lv


def as_fp32(pos, q):
    """The values a mixed-precision caller passes: positions and charges
    rounded to float32 (returned as float64 for the oracle)."""
    return pos.astype(np.float32).astype(np.float64), q.astype(np.float32).astype(np.float64)
