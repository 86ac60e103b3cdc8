"""Probe runs of the learned selector on held-out systems: the parameters it
picks are run through the library on the GPU, their RMS force error is
measured against converged direct Ewald (oracle) on sampled particles, and
their measured time is compared with the grid-searched optimum's."""
import math

import numpy as np
import pytest

import oracle as O
import workloads as W

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2004_12484_b300 as P  # noqa: E402
from paper_2004_12484_b300 import learned as Lr  # noqa: E402
from paper_2004_12484_b300 import selector as S  # noqa: E402

DEV = torch.device("cuda", 0)


def realise(sys_, seed):
    pos, q, L = W.random_neutral(sys_.N, sys_.L[1], seed, charged_fraction=sys_.charged_fraction,
                                 anisotropy=sys_.L[0] / sys_.L[1])
    return W.as_fp32(pos, q) + (L,)


def run_time(prm, pos, q, L, reps=10):
    plan = P.Plan(L=L, N=len(q), alpha=prm.alpha, r_c=prm.r_c, M=prm.M, p=prm.p, device=DEV)
    tp = torch.tensor(pos, dtype=torch.float32, device=DEV)
    tq = torch.tensor(q, dtype=torch.float32, device=DEV)
    F = torch.empty((len(q), 3), device=DEV)
    out = torch.empty(16, dtype=torch.float64, device=DEV)
    for _ in range(3):
        plan.compute(tp, tq, F=F, out=out)
    s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    s.record()
    for _ in range(reps):
        plan.compute(tp, tq, F=F, out=out)
    e.record()
    torch.cuda.synchronize()
    return s.elapsed_time(e) / reps, F


@pytest.fixture(scope="module")
def model():
    return Lr.MLP.load(device=DEV)


def test_probe_errors_meet_targets(model):
    held = [h for h in Lr.sample_systems(500, 6) if h[0].N <= 12000][:5]
    picks = Lr.select(model, held)
    for k, ((s, tgt), (prm, fell_back)) in enumerate(zip(held, picks)):
        pos, q, L = realise(s, 100 + k)
        _, F = run_time(prm, pos, q, L, reps=1)
        F = F.cpu().double().numpy()
        idx = np.random.default_rng(k).choice(len(q), 48, replace=False)
        a_ref = 6.5 / (0.5 * min(L))
        ref = O.direct_ewald(pos, q, L, a_ref, 0.5 * min(L), nmax=int(a_ref * max(L) / math.pi * 6.5) + 1,
                             sphere=True, idx=idx)
        sysd = S.System(N=len(q), L=tuple(L), Q=float((q * q).sum()), charged_fraction=s.charged_fraction)
        meas = np.sqrt(((F[idx] - ref.F) ** 2).sum(1).mean()) / sysd.force_scale
        assert meas <= 2.0 * tgt, (k, prm, tgt, meas)


def test_probe_measured_time_near_grid_optimum(model):
    held = [h for h in Lr.sample_systems(500, 6) if 20000 <= h[0].N <= 1_500_000][:10]
    picks = Lr.select(model, held)
    ratios = []
    for k, ((s, tgt), (prm, _)) in enumerate(zip(held, picks)):
        opt = S.grid_search(s, tgt)[0]
        pos, q, L = realise(s, 200 + k)
        t_net, _ = run_time(prm, pos, q, L)
        t_opt, _ = run_time(opt, pos, q, L)
        ratios.append(t_net / t_opt)
    ratios = np.array(ratios)
    print("measured time ratio network/grid-optimum:", np.round(ratios, 3))
    assert np.median(ratios) <= 1.10


def converged_forces(pos, q, L, idx):
    a_ref = 6.5 / (0.5 * min(L))
    return O.direct_ewald(pos, q, L, a_ref, 0.5 * min(L), nmax=int(a_ref * max(L) / math.pi * 6.5) + 1,
                          sphere=True, idx=idx).F


def test_learned_selector_gain_over_the_paper_recipe(model):
    """What the trained network gains over the method without it, measured:
    on 20 held-out systems, the network's parameters against the best the
    paper's recipe (Eq. 31-32) offers at equal or better measured accuracy.
    The recipe leaves the user three inputs, all searched here against
    measured errors: the window width p in {6, 8, 10}, r_c in {1, 1.25, 1.5,
    2} x the network's r_c, and for each pair the loosest accuracy delta in
    {target, /3, /10, /30} whose measured RMS force error is no worse than
    the network's (or the target); the fastest such setting is the recipe's
    time.  Every run is timed on the GPU (full step, real space included)
    and its error measured against converged direct Ewald on 48 sampled
    particles."""
    held = [h for h in Lr.sample_systems(500, 6) if 3000 <= h[0].N <= 40000][:20]
    assert len(held) == 20
    picks = Lr.select(model, held)
    rows = []
    for k, ((s, tgt), (prm, _)) in enumerate(zip(held, picks)):
        pos, q, L = realise(s, 300 + k)
        sysd = S.System(N=len(q), L=tuple(L), Q=float((q * q).sum()), charged_fraction=s.charged_fraction)
        idx = np.random.default_rng(300 + k).choice(len(q), 48, replace=False)
        ref = converged_forces(pos, q, L, idx)

        def err(F):
            F = F.cpu().double().numpy()
            return float(np.sqrt(((F[idx] - ref) ** 2).sum(1).mean()) / sysd.force_scale)

        t_net, F = run_time(prm, pos, q, L)
        e_net = err(F)
        best = None
        for pw in (6, 8, 10):
            for f_rc in (1.0, 1.25, 1.5, 2.0):
                rc = min(f_rc * prm.r_c, 0.5 * min(L))
                for delta in (tgt, tgt / 3, tgt / 10, tgt / 30):
                    pp = S.legal(S.paper_procedure(s, delta, rc), s)
                    pp = S.Params(pp.alpha, pp.r_c, pp.M, min(pw, pp.M))
                    t_pap, Fp = run_time(pp, pos, q, L, reps=5)
                    e_pap = err(Fp)
                    if e_pap <= max(e_net, tgt):
                        if best is None or t_pap < best[0]:
                            best = (t_pap, e_pap)
                        break
        rows.append((s.N, tgt, t_net, e_net) + (best if best else (np.inf, np.nan)))
    rows = np.array(rows)
    gain = rows[:, 4] / rows[:, 2]
    print("N, target, t_net ms, err_net, t_paper ms, err_paper, paper/network time")
    for r, g in zip(rows, gain):
        print(f"{int(r[0]):7d} {r[1]:.0e} {r[2]:.4f} {r[3]:.2e} {r[4]:.4f} {r[5]:.2e} {g:.2f}")
    print("median time gain of the network over the paper's recipe:", float(np.median(gain)),
          "; systems where the recipe reached the accuracy:", int(np.isfinite(rows[:, 4]).sum()))
    # the network meets its targets; where the recipe reaches the same
    # accuracy, the network's one 5-us prediction lands near the best of the
    # recipe's 48 measured settings
    assert (rows[:, 3] <= 2.0 * rows[:, 1]).all()
    assert np.isfinite(rows[:, 4]).sum() >= 15
    assert np.median(gain[np.isfinite(gain)]) >= 0.9
