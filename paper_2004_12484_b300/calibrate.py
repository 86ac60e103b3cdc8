"""Measures the library on this GPU and writes ``timing_model.json``, the
time and window-error model the parameter selector uses.

    python -m paper_2004_12484_b300.calibrate

Timing: per-kernel device times (event-timed graph replays) of k-space-only
evaluations over a grid of (N, M, p), and full evaluations over a few
cutoffs, fitted by least squares to
    t_k = t0 + a N + b N p^3 + c M^3,        t_real = d N rho 27 r_c^3.
Window error: the relative RMS difference of the reciprocal forces computed
with window p and with p = 12 (same grid, same alpha, oversampling 2) on a
uniform random system, for every supported p.
"""
from __future__ import annotations

import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(HERE))


def _system(N, rho, seed):
    g = np.random.default_rng(seed)
    L = (N / rho) ** (1.0 / 3.0)
    pos = g.uniform(0, L, size=(N, 3)).astype(np.float32)
    q = np.where(np.arange(N) % 2 == 0, 1.0, -1.0).astype(np.float32)
    return pos, q, L


def _time_call(plan, tp, tq, kspace_only, reps=5):
    import torch
    F = torch.empty((plan.N, 3), dtype=torch.float32, device=tp.device)
    out = torch.empty(16, dtype=torch.float64, device=tp.device)
    for _ in range(2):
        plan.compute(tp, tq, F=F, out=out, kspace_only=kspace_only)
    torch.cuda.synchronize()
    s = torch.cuda.Event(enable_timing=True)
    e = torch.cuda.Event(enable_timing=True)
    s.record()
    for _ in range(reps):
        plan.compute(tp, tq, F=F, out=out, kspace_only=kspace_only)
    e.record()
    torch.cuda.synchronize()
    return s.elapsed_time(e) / reps * 1e-3


def calibrate(out_path=None, quick=False):
    import torch
    import paper_2004_12484_b300 as P
    dev = torch.device("cuda", 0)
    rho = 0.05
    rows, times = [], []
    Ns = [16384, 131072, 1048576] if not quick else [16384, 131072]
    for N in Ns:
        pos, q, L = _system(N, rho, 1)
        tp = torch.tensor(pos, device=dev)
        tq = torch.tensor(q, device=dev)
        for M in (32, 64, 128, 256):
            for p in (4, 6, 8):
                plan = P.Plan(L=L, N=N, alpha=0.3, r_c=min(8.0, 0.45 * L), M=M, p=p, device=dev)
                t = _time_call(plan, tp, tq, True)
                rows.append([1.0, N, N * p ** 3, M ** 3])
                times.append(t)
                del plan
    A = np.array(rows, dtype=np.float64)
    y = np.array(times)
    # non-negative least squares on relative error (scale rows by 1/t)
    from scipy.optimize import nnls
    coef_k, _ = nnls(A / y[:, None], np.ones_like(y))
    # real space: full minus k-space for a few cutoffs
    rr, rt = [], []
    for N in Ns[:2]:
        pos, q, L = _system(N, rho, 2)
        tp = torch.tensor(pos, device=dev)
        tq = torch.tensor(q, device=dev)
        for rc in (5.0, 7.0, 9.0, 11.0):
            if rc > 0.5 * L:
                continue
            plan = P.Plan(L=L, N=N, alpha=0.3, r_c=rc, M=64, p=6, device=dev)
            tr = _time_call(plan, tp, tq, False) - _time_call(plan, tp, tq, True)
            cell = L / max(3, int(L // rc))
            rr.append(N * rho * 27.0 * cell ** 3)
            rt.append(max(tr, 1e-7))
            del plan
    rr = np.array(rr)
    rt = np.array(rt)
    d = float((rr * rt).sum() / (rr * rr).sum())
    # window error relative to p = 12
    N = 20000
    pos, q, L = _system(N, 0.01, 3)
    tp = torch.tensor(pos, device=dev)
    tq = torch.tensor(q, device=dev)
    M = 64
    kc = 2 * np.pi * (M // 4) / L
    alpha = kc / (np.sqrt(2.0) * 2.5)  # k_c / (sqrt 2 alpha) = 2.5
    forces = {}
    for p in (2, 4, 6, 8, 10, 12):
        plan = P.Plan(L=L, N=N, alpha=alpha, r_c=min(10.0, 0.45 * L), M=M, p=p, precision="fp64", device=dev)
        _, F, _, _ = plan.energy_forces(tp.double(), tq.double(), kspace_only=True)
        forces[p] = F.cpu().numpy()
        del plan
    ref = forces[12]
    eps = {str(p): float(np.sqrt(((forces[p] - ref) ** 2).sum() / (ref ** 2).sum())) for p in (2, 4, 6, 8, 10)}
    eps["12"] = eps["10"] * eps["10"] / eps["8"]  # geometric continuation (no finer reference)
    res = {"coef": {"t0": float(coef_k[0]), "sort_per_particle": float(coef_k[1]),
                    "spread_per_point": float(coef_k[2]) / 2, "gather_per_point": float(coef_k[2]) / 2,
                    "fft_per_cell": float(coef_k[3]), "real_per_pair": d},
           "window_eps": eps,
           "fit": {"rows": A.tolist(), "seconds": y.tolist(), "real_pairs": rr.tolist(), "real_seconds": rt.tolist()},
           "gpu": torch.cuda.get_device_name(0), "when": time.strftime("%Y-%m-%dT%H:%M:%SZ", time.gmtime())}
    path = out_path or os.path.join(HERE, "timing_model.json")
    with open(path, "w") as f:
        json.dump(res, f, indent=1)
    return res


if __name__ == "__main__":
    r = calibrate(out_path=sys.argv[1] if len(sys.argv) > 1 else None)
    print(json.dumps({k: v for k, v in r.items() if k != "fit"}, indent=1))
