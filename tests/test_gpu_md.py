"""The time-stepping harness (enuf_md_run: velocity Verlet, each step one
graph launch) against the FP64 oracle integrator driven by the oracle's
NFFT-Ewald forces, and the conservation laws along a trajectory.

System: a one-component plasma (all charges +1 with the neutralising
background), 3 A simple-cubic lattice with 0.2 A Gaussian displacements,
unit masses, Gaussian velocities (sigma 0.1), Gaussian units.  Repulsive
only, so the dynamics is smooth without a short-range potential.
"""
import numpy as np
import pytest

import oracle as O
from oracle import md as OMD

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2004_12484_b300 as P  # noqa: E402

DEV = torch.device("cuda", 0)


def ocp(n, a=3.0, jitter=0.2, vs=0.1, seed=1):
    g = np.random.default_rng(seed)
    x = (np.stack(np.meshgrid(*[np.arange(n)] * 3, indexing="ij"), -1).reshape(-1, 3) + 0.5) * a
    x += g.normal(scale=jitter, size=x.shape)
    v = g.normal(scale=vs, size=x.shape)
    v -= v.mean(0)
    return x, v, np.ones(len(x))


def device(a, dt):
    return torch.tensor(a, dtype=dt, device=DEV)


@pytest.mark.parametrize("ad", [False, True])
def test_md_fp64_matches_oracle_trajectory(ad):
    """64 ions, 20 steps of dt = 0.1: positions, velocities and the per-step
    energies of the FP64 plan against the oracle integrator with the
    oracle's NFFT-Ewald forces (ik, or analytic differentiation).  Each force
    agrees to about 1e-13; over 20 steps the trajectories stay within 1e-10."""
    x, v, q = ocp(4)
    L = np.full(3, 12.0)
    kw = dict(alpha=0.5, rc=5.9, M=16, p=6, nc=4)
    plan = P.Plan(L=L, N=len(q), alpha=kw["alpha"], r_c=kw["rc"], M=kw["M"], p=kw["p"], n_c=kw["nc"],
                  precision="fp64", device=DEV)
    tx, tv, tq = device(x, torch.float64), device(v, torch.float64), device(q, torch.float64)
    im = torch.ones(len(q), dtype=torch.float64, device=DEV)
    en, F = plan.md_run(tx, tv, tq, im, 0.1, 20, ad=ad)
    fn = O.nfft_ewald_ad if ad else O.nfft_ewald

    def forces(p):
        r = fn(p, q, L, **kw)
        return r.E, r.F

    px, pv, pF, pen = OMD.verlet(x, v, np.ones(len(q)), L, 0.1, 20, forces)
    gx = tx.cpu().numpy()
    d = np.abs(gx - px)
    assert np.minimum(d, L - d).max() < 1e-10
    assert np.abs(tv.cpu().numpy() - pv).max() < 1e-10
    assert np.abs(F.cpu().numpy() - pF).max() < 1e-10 * np.abs(pF).max()
    e = en.cpu().numpy()
    assert np.abs(e[:, :3] - pen).max() < 1e-10 * np.abs(pen[:, 0]).max()
    assert e[:, 3].max() == 0.0


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_md_momentum_and_energy_along_a_trajectory(precision):
    """512 ions for 20 time units (200 steps of 0.1).  Momentum: the ik
    forces sum to zero, so the total momentum stays at rounding level; the
    analytic-differentiation forces do not (the approximated energy is
    invariant only under shifts by whole grid cells), and with
    ENUF_REMOVE_NET_FORCE they do again.  Energy: the total stays within
    1e-3 (p = 6) and 2e-4 (p = 8) of the kinetic energy.  At p = 6 the drift
    does not shrink with dt (5.6e-4 at dt = 0.05 against 6.2e-4) and it
    falls with the window width, so it comes from the truncated window, whose
    energy jumps when a particle's support moves by a cell; from p = 8 on the
    integrator's error dominates (p = 8: 1.6e-4 at dt = 0.1, 7e-5 at 0.05;
    p = 10 and 12: 1.2e-4 at dt = 0.1).  The ik and the analytic-
    differentiation forces drift alike."""
    dtp = torch.float64 if precision == "fp64" else torch.float32
    mom_tol = 1e-12 if precision == "fp64" else 1e-3
    x, v, q = ocp(8)
    drift = {}
    for p in (6, 8):
        for ad, rnf in ((False, False), (True, False), (True, True)):
            plan = P.Plan(L=24.0, N=len(q), alpha=0.45, r_c=9.0, M=32, p=p, n_c=8, precision=precision,
                          device=DEV)
            tx, tv, tq = device(x, dtp), device(v, dtp), device(q, dtp)
            im = torch.ones(len(q), dtype=dtp, device=DEV)
            en, _ = plan.md_run(tx, tv, tq, im, 0.1, 200, ad=ad, remove_net_force=rnf)
            e = en.cpu().numpy()
            assert np.isfinite(e).all() and e[:, 3].max() == 0.0
            mom = np.abs(tv.double().sum(0).cpu().numpy()).max()
            if ad and not rnf:
                assert mom > 1e-4
            else:
                assert mom < mom_tol
            rel = np.abs(e[:, 2] - e[0, 2]).max() / e[:, 1].mean()
            drift[(p, ad, rnf)] = rel
    assert max(drift[(6, a, r)] for a, r in ((False, False), (True, False), (True, True))) < 1e-3
    assert max(drift[(8, a, r)] for a, r in ((False, False), (True, False), (True, True))) < 2e-4
    assert drift[(8, False, False)] < drift[(6, False, False)] / 3


def test_md_mixed_follows_fp64_and_replays_its_graph():
    """The mixed-precision trajectory stays close to the FP64 one over 50
    steps, and a second call with the same buffers replays the captured step
    (the step counter restarts, so the energies are written from row 0)."""
    x, v, q = ocp(6, seed=3)
    res = {}
    for prec, dtp in (("fp64", torch.float64), ("mixed", torch.float32)):
        plan = P.Plan(L=18.0, N=len(q), alpha=0.5, r_c=8.0, M=32, p=8, n_c=8, precision=prec, device=DEV)
        tx, tv, tq = device(x, dtp), device(v, dtp), device(q, dtp)
        im = torch.ones(len(q), dtype=dtp, device=DEV)
        F = torch.empty((len(q), 3), dtype=dtp, device=DEV)
        en = torch.empty((25, 4), dtype=torch.float64, device=DEV)
        e1, _ = plan.md_run(tx, tv, tq, im, 0.1, 25, F=F, energies=en)
        e1 = e1.cpu().numpy().copy()
        e2, _ = plan.md_run(tx, tv, tq, im, 0.1, 25, F=F, have_forces=True, energies=en)
        res[prec] = (tx.cpu().double().numpy(), np.concatenate([e1, e2.cpu().numpy()]))
    d = np.abs(res["mixed"][0] - res["fp64"][0])
    assert np.minimum(d, 18.0 - d).max() < 1e-3
    assert np.abs(res["mixed"][1][:, 2] - res["fp64"][1][:, 2]).max() < 1e-5 * np.abs(res["fp64"][1][:, 0]).max()
