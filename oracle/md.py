"""Velocity-Verlet time stepping in FP64 -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this module; it shares no code with the CUDA library.

One step, with forces F = F(r) from a callable (any of the oracle's Ewald
sums):

    v <- v + (dt/2) F / m;   r <- r + dt v, wrapped into [0, L);
    F <- F(r);               v <- v + (dt/2) F / m.

The kinetic energy is 1/2 sum_i m_i |v_i|^2 (particles with 1/m = 0 are
fixed and carry none).
"""
from __future__ import annotations

import numpy as np


def verlet(pos, vel, inv_mass, L, dt, nsteps, forces, F=None):
    """Runs ``nsteps`` steps from (pos, vel).  ``forces(pos) -> (E_pot, F)``.
    Returns (pos, vel, F, energies) with energies[s] = (E_pot, E_kin, E_tot)
    after step s."""
    pos = np.array(pos, dtype=np.float64, copy=True).reshape(-1, 3)
    vel = np.array(vel, dtype=np.float64, copy=True).reshape(-1, 3)
    im = np.asarray(inv_mass, dtype=np.float64).reshape(-1)
    L = np.broadcast_to(np.asarray(L, dtype=np.float64).reshape(-1), (3,))
    if F is None:
        F = forces(pos)[1]
    F = np.array(F, dtype=np.float64, copy=True)
    energies = np.zeros((nsteps, 3))
    for s in range(nsteps):
        vel += 0.5 * dt * im[:, None] * F
        pos += dt * vel
        pos -= L * np.floor(pos / L)
        E, F = forces(pos)
        F = np.asarray(F, dtype=np.float64)
        vel += 0.5 * dt * im[:, None] * F
        moving = im > 0
        ke = 0.5 * np.sum((vel[moving] ** 2).sum(axis=1) / im[moving])
        energies[s] = (E, ke, E + ke)
    return pos, vel, F, energies
