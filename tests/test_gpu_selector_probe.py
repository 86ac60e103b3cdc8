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
