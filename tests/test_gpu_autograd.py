"""The differentiable energy: backward returns dE/dr = -F and dE/dq = phi,
checked against the forward outputs, the oracle, and central differences."""
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


def test_backward_matches_forces_and_oracle_fp64():
    g = np.random.default_rng(31)
    N, L = 400, np.array([14.0, 15.0, 16.0])
    pos = g.uniform(0, 15, size=(N, 3))
    q = g.normal(size=N)
    q -= q.mean()
    kw = dict(alpha=0.45, r_c=6.0, M=32, p=8, n_c=8)
    plan = P.Plan(L=L, N=N, precision="fp64", device=DEV, **kw)
    tp = torch.tensor(pos, dtype=torch.float64, device=DEV, requires_grad=True)
    tq = torch.tensor(q, dtype=torch.float64, device=DEV, requires_grad=True)
    E = P.EnufEnergy.apply(tp, tq, plan)
    (2.5 * E).backward()
    ref = O.nfft_ewald(pos, q, L, kw["alpha"], kw["r_c"], kw["M"], kw["p"], kw["n_c"])
    assert abs(float(E.detach()) / ref.E - 1) < 1e-12
    assert np.abs(tp.grad.cpu().numpy() - (-2.5 * ref.F)).max() < 1e-11 * np.abs(ref.F).max()
    assert np.abs(tq.grad.cpu().numpy() - 2.5 * ref.phi).max() < 1e-11 * np.abs(ref.phi).max()


def test_dE_dq_central_difference_fp64():
    """E is quadratic in q: the central difference equals phi up to rounding."""
    d = W.rpm(N=2048, seed=32, M=32, p=6, r_c=9.0, alpha=0.35)
    plan = P.Plan(L=d["L"], N=2048, alpha=0.35, r_c=9.0, M=32, p=6, precision="fp64", device=DEV)
    tp = torch.tensor(d["pos"], dtype=torch.float64, device=DEV)
    tq = torch.tensor(d["q"], dtype=torch.float64, device=DEV)
    _, dq = plan.backward(tp, tq)
    dq = dq.cpu().numpy()
    h = 1e-3
    for i in [0, 17, 2047]:
        qp = tq.clone(); qp[i] += h
        qm = tq.clone(); qm[i] -= h
        ep = float(P.EnufEnergy.apply(tp, qp, plan))
        em = float(P.EnufEnergy.apply(tp, qm, plan))
        assert abs((ep - em) / (2 * h) - dq[i]) < 1e-9 * (1 + abs(dq[i]))


def test_dE_dr_central_difference_polyelectrolyte_like():
    """Central differences in positions (h = 1e-4 sigma) on 64 random beads of
    a polyelectrolyte-like system, through the autograd function.

    The ik forces (Eq. 41-42) are not the exact gradient of the NFFT energy:
    both approximate the exact Ewald force of the same frequency cube, each
    within the NFFT accuracy.  So the test checks (a) the difference quotient
    of the device energy against the difference quotient of the oracle's
    energy (same function, so they agree to rounding), and (b) that both the
    ik force and the difference quotient are within the NFFT accuracy of the
    direct Ewald force.  The truncated window makes the NFFT energy jump when
    a particle crosses a grid-cell boundary, and the real-space sum jumps when
    a pair crosses r_c; components whose difference interval contains such a
    crossing have no derivative and are skipped."""
    d = W.polyelectrolyte(n_beads=4000, seed=33, M=32, p=6, alpha=0.739)
    N = len(d["q"])
    L, pos, q = d["L"], d["pos"], d["q"]
    plan = P.Plan(L=L, N=N, alpha=d["alpha"], r_c=3.0, M=32, p=6, precision="fp64", device=DEV)
    tp = torch.tensor(pos, dtype=torch.float64, device=DEV)
    tq = torch.tensor(q, dtype=torch.float64, device=DEV)
    dpos, _ = plan.backward(tp, tq)
    dpos = dpos.cpu().numpy()
    beads = np.random.default_rng(34).choice(np.nonzero(q[: d["n_beads"]] != 0)[0], 64, replace=False)
    h = 1e-4
    fd = np.full((64, 3), np.nan)
    for k, i in enumerate(beads):
        for t in range(3):
            if np.floor(32 * (pos[i, t] + h) / L[t]) != np.floor(32 * (pos[i, t] - h) / L[t]):
                continue
            dr = pos - pos[i]
            dr -= L * np.round(dr / L)
            r = np.sqrt((dr ** 2).sum(1))
            r[i] = 0
            if np.any(np.abs(r - 3.0) < 2 * h):
                continue
            pp = tp.clone(); pp[i, t] += h
            pm = tp.clone(); pm[i, t] -= h
            fd[k, t] = (float(P.EnufEnergy.apply(pp, tq, plan)) - float(P.EnufEnergy.apply(pm, tq, plan))) / (2 * h)
    ok = ~np.isnan(fd)
    assert ok.sum() > 150
    # (a) the same difference quotients from the oracle's NFFT-Ewald energy
    checked = 0
    for k, i in enumerate(beads):
        for t in range(3):
            if not ok[k, t] or checked >= 6:
                continue
            pp = pos.copy(); pp[i, t] += h
            pm = pos.copy(); pm[i, t] -= h
            ep = O.nfft_ewald(pp, q, L, d["alpha"], 3.0, 32, 6, 8).E
            em = O.nfft_ewald(pm, q, L, d["alpha"], 3.0, 32, 6, 8).E
            assert abs((ep - em) / (2 * h) - fd[k, t]) < 1e-6 * (1 + abs(fd[k, t]))
            checked += 1
    # (b) both derivatives against the direct Ewald force of the same cube
    ref = O.direct_ewald(pos, q, L, d["alpha"], 3.0, 8, sphere=False, idx=beads)
    Fex = ref.F
    e_ik = np.sqrt(((-dpos[beads] - Fex) ** 2).sum() / (Fex ** 2).sum())
    e_fd = np.sqrt(((-fd - Fex)[ok] ** 2).sum() / (Fex[ok] ** 2).sum())
    err = np.sqrt(((fd - dpos[beads])[ok] ** 2).sum() / (dpos[beads][ok] ** 2).sum())
    assert e_ik < 2e-3 and e_fd < 1e-2, (e_ik, e_fd)
    assert err <= 1.05 * (e_ik + e_fd), (err, e_ik, e_fd)


def test_ad_gradient_is_exact_central_difference_fp64():
    """With forces by analytic differentiation the autograd gradient is the
    exact derivative of the returned energy: central differences (h = 1e-5)
    of the FP64 energy, real space included, agree to 1e-7 relative on 20
    components (those whose interval crosses a grid-cell face or r_c are
    skipped, where the energy has no derivative); the ik gradient of the same
    plan does not, at the window's accuracy."""
    g = np.random.default_rng(35)
    N, L = 300, np.array([14.0, 15.0, 16.0])
    pos = g.uniform(0, 1, size=(N, 3)) * L
    q = g.normal(size=N)
    q -= q.mean()
    M, rc = 32, 6.0
    plan = P.Plan(L=L, N=N, alpha=0.45, r_c=rc, M=M, p=4, n_c=8, precision="fp64", device=DEV)
    tp = torch.tensor(pos, dtype=torch.float64, device=DEV, requires_grad=True)
    tq = torch.tensor(q, dtype=torch.float64, device=DEV)
    E = P.EnufEnergy.apply(tp, tq, plan, True)
    E.backward()
    grad = tp.grad.cpu().numpy()
    dpos_ik, _ = plan.backward(tp.detach(), tq)
    dpos_ik = dpos_ik.cpu().numpy()
    h = 1e-5
    fd, an, ik = [], [], []
    for i in np.random.default_rng(36).choice(N, 40, replace=False):
        for t in range(3):
            if np.floor(M * (pos[i, t] + h) / L[t]) != np.floor(M * (pos[i, t] - h) / L[t]):
                continue
            dr = pos - pos[i]
            dr -= L * np.round(dr / L)
            r = np.sqrt((dr ** 2).sum(1))
            if np.any(np.abs(r - rc) < 2 * h):
                continue
            pp = tp.detach().clone(); pp[i, t] += h
            pm = tp.detach().clone(); pm[i, t] -= h
            fd.append((float(P.EnufEnergy.apply(pp, tq, plan, True))
                       - float(P.EnufEnergy.apply(pm, tq, plan, True))) / (2 * h))
            an.append(grad[i, t])
            ik.append(dpos_ik[i, t])
            if len(fd) == 20:
                break
        if len(fd) == 20:
            break
    fd, an, ik = np.array(fd), np.array(an), np.array(ik)
    assert len(fd) == 20
    scale = np.abs(an).max()
    assert np.abs(fd - an).max() < 1e-7 * scale
    assert np.abs(fd - ik).max() > 1e-5 * scale
