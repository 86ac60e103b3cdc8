"""Learned ENUF parameter selector: a 6 -> 64 -> 64 -> 4 network (bfloat16
weights, float accumulation) trained and evaluated on the GPU by the
library's own kernels (``enuf_mlp_train_step``, ``enuf_mlp_forward``).

Inputs (``selector.descriptor``): log N, density, charged fraction, charge
variance, box anisotropy, log10 target RMS force error.  Outputs: log(alpha a),
log(r_c / a), log2 M, p, with a = rho^(-1/3) the mean spacing (scale-free
forms of alpha, r_c, M, p).  Labels are the time-optimal parameters of the
analytic grid search (``selector.grid_search``) under the time model measured
on this GPU.  A prediction is legalised (M to a power of two, p to an even
window, r_c <= L/2); if its estimated error misses the target, r_c is raised
along the real-space error curve, and if that cannot reach the target the
selector falls back to the grid search.

    python -m paper_2004_12484_b300.learned [out.json]   # label, train, evaluate
"""
from __future__ import annotations

import ctypes
import json
import math
import os
import sys
import time

import numpy as np

from . import selector as S

HERE = os.path.dirname(os.path.abspath(__file__))
WEIGHTS_PATH = os.path.join(HERE, "selector_weights.json")
NPARAM = 4868
TARGETS = (1e-3, 1e-4, 1e-5)


# ---------------------------------------------------------------- data
def sample_systems(n, seed):
    """Descriptors of the training / held-out distribution: N log-uniform in
    [1e3, 4e6], density 0.005-0.1 per cubic Angstrom, charged fraction 0.1-1
    (charges +-1), one box edge stretched by a factor uniform in [1, 2],
    target in {1e-3, 1e-4, 1e-5}."""
    g = np.random.Generator(np.random.PCG64(seed))
    out = []
    for _ in range(n):
        N = int(round(math.exp(g.uniform(math.log(1e3), math.log(4e6)))))
        rho = g.uniform(0.005, 0.1)
        f = g.uniform(0.1, 1.0)
        an = g.uniform(1.0, 2.0)
        V = N / rho
        Lb = (V / an) ** (1.0 / 3.0)
        L = (Lb * an, Lb, Lb)
        tgt = TARGETS[int(g.integers(0, 3))]
        out.append((S.System(N=N, L=L, Q=f * N, charged_fraction=f), tgt))
    return out


def encode(prm: S.Params, sys_: S.System):
    a = sys_.rho ** (-1.0 / 3.0)
    return np.array([math.log(prm.alpha * a), math.log(prm.r_c / a), math.log2(prm.M), prm.p], dtype=np.float64)


def decode(y, sys_: S.System) -> S.Params:
    a = sys_.rho ** (-1.0 / 3.0)
    return S.Params(math.exp(y[0]) / a, math.exp(y[1]) * a, int(round(2 ** y[2])), int(round(y[3])))


def label(systems):
    X, Y, keep = [], [], []
    for i, (s, t) in enumerate(systems):
        r = S.grid_search(s, t)
        if r is None:
            continue
        X.append(S.descriptor(s, t))
        Y.append(encode(r[0], s))
        keep.append(i)
    return np.array(X), np.array(Y), keep


# ---------------------------------------------------------------- network
class MLP:
    """Weights and Adam state as torch device tensors; every forward and
    training step runs in the library's kernels."""

    def __init__(self, device=None, seed=0):
        import torch
        from . import lib
        self.torch = torch
        self.lib = lib()
        self.dev = torch.device(device) if device is not None else torch.device("cuda", 0)
        g = np.random.default_rng(seed)
        w = np.zeros(NPARAM, dtype=np.float32)
        o = 0
        for fan_in, fan_out in [(6, 64), (64, 64), (64, 4)]:
            n = fan_in * fan_out
            w[o:o + n] = g.normal(0, math.sqrt(1.0 / fan_in), size=n)
            o += n + fan_out  # biases start at zero
        self.set_weights(w)
        self.xm = np.zeros(6); self.xs = np.ones(6)
        self.ym = np.zeros(4); self.ys = np.ones(4)

    def set_weights(self, w):
        torch = self.torch
        self.wm = torch.tensor(np.asarray(w, dtype=np.float32), device=self.dev)
        self.wq = self.wm.to(torch.bfloat16)
        self.m = torch.zeros_like(self.wm)
        self.v = torch.zeros_like(self.wm)
        self.step = 0

    def _ptr(self, t):
        return ctypes.c_void_p(t.data_ptr())

    def _stream(self):
        return ctypes.c_void_p(self.torch.cuda.current_stream(self.dev).cuda_stream)

    def forward_raw(self, xn):
        """Network outputs for normalised inputs (n x 6 float32 device)."""
        torch = self.torch
        y = torch.empty((xn.shape[0], 4), dtype=torch.float32, device=self.dev)
        rc = self.lib.enuf_mlp_forward(self._ptr(self.wq), self._ptr(xn), ctypes.c_int64(xn.shape[0]),
                                       self._ptr(y), self._stream())
        if rc != 0:
            raise RuntimeError(self.lib.enuf_last_error().decode())
        return y

    def train_step(self, xb, yb, ow, lr, grad=None, apply=True, loss=None):
        torch = self.torch
        if apply:
            self.step += 1
        if loss is None:
            loss = torch.empty(1, dtype=torch.float32, device=self.dev)
        rc = self.lib.enuf_mlp_train_step(
            self._ptr(self.wm), self._ptr(self.wq), self._ptr(self.m), self._ptr(self.v), self._ptr(xb),
            self._ptr(yb), self._ptr(ow), ctypes.c_int(xb.shape[0]), ctypes.c_float(lr), ctypes.c_float(0.9),
            ctypes.c_float(0.999), ctypes.c_float(1e-8), ctypes.c_int(max(self.step, 1)), self._ptr(loss),
            self._ptr(grad) if grad is not None else None, ctypes.c_int(1 if apply else 0), self._stream())
        if rc != 0:
            raise RuntimeError(self.lib.enuf_last_error().decode())
        return loss

    # ----------------------------------------------------------- fit / predict
    def fit(self, X, Y, epochs=300, batch=256, lr=3e-3, seed=0, log=None):
        torch = self.torch
        self.xm, self.xs = X.mean(0), X.std(0) + 1e-12
        self.ym, self.ys = Y.mean(0), Y.std(0) + 1e-12
        xn = torch.tensor((X - self.xm) / self.xs, dtype=torch.float32, device=self.dev)
        yn = torch.tensor((Y - self.ym) / self.ys, dtype=torch.float32, device=self.dev)
        ow = torch.tensor([1.0, 1.0, 1.0, 1.0], dtype=torch.float32, device=self.dev)
        g = np.random.default_rng(seed)
        n = X.shape[0]
        loss = torch.empty(1, dtype=torch.float32, device=self.dev)
        hist = []
        for ep in range(epochs):
            perm = torch.tensor(g.permutation(n), device=self.dev)
            xs, ys = xn[perm].contiguous(), yn[perm].contiguous()
            tot = torch.zeros((), device=self.dev)
            nb = 0
            frac = ep / max(1, epochs - 1)
            lr_e = lr * (0.5 * (1 + math.cos(math.pi * frac)) * 0.95 + 0.05)  # cosine schedule
            for b0 in range(0, n - batch + 1, batch):
                self.train_step(xs[b0:b0 + batch], ys[b0:b0 + batch], ow, lr_e, loss=loss)
                tot += loss[0]
                nb += 1
            hist.append(float(tot) / max(nb, 1))
            if log and (ep % 50 == 0 or ep == epochs - 1):
                log(f"epoch {ep} loss {hist[-1]:.4e}")
        return hist

    def predict_raw(self, X):
        torch = self.torch
        xn = torch.tensor((np.asarray(X) - self.xm) / self.xs, dtype=torch.float32, device=self.dev)
        y = self.forward_raw(xn).cpu().numpy().astype(np.float64)
        return y * self.ys + self.ym

    def save(self, path=WEIGHTS_PATH, extra=None):
        d = {"w": self.wm.cpu().numpy().tolist(), "xm": self.xm.tolist(), "xs": self.xs.tolist(),
             "ym": self.ym.tolist(), "ys": self.ys.tolist()}
        if extra:
            d.update(extra)
        with open(path, "w") as f:
            json.dump(d, f)

    @classmethod
    def load(cls, path=WEIGHTS_PATH, device=None):
        d = json.load(open(path))
        m = cls(device=device)
        m.set_weights(np.array(d["w"], dtype=np.float32))
        m.xm, m.xs = np.array(d["xm"]), np.array(d["xs"])
        m.ym, m.ys = np.array(d["ym"]), np.array(d["ys"])
        return m


def choose(y, sys_: S.System, target: float):
    """Legalise a network output; raise r_c if the estimate misses the
    target; None if that cannot reach it (the caller falls back)."""
    prm = S.legal(decode(y, sys_), sys_)
    if S.rms_force_error(prm, sys_) <= target:
        return prm
    rc_max = 0.5 * min(sys_.L)
    for rc in np.geomspace(prm.r_c, rc_max, 40):
        cand = S.Params(prm.alpha, float(rc), prm.M, prm.p)
        if S.rms_force_error(cand, sys_) <= target:
            return cand
    return None


def select(model: MLP, systems):
    """Parameters for a list of (System, target): the network's choice, or
    the grid search when the choice cannot meet the target."""
    X = np.array([S.descriptor(s, t) for s, t in systems])
    Yp = model.predict_raw(X)
    out = []
    for (s, t), y in zip(systems, Yp):
        prm = choose(y, s, t)
        if prm is None:
            r = S.grid_search(s, t)
            out.append((r[0] if r else None, True))
        else:
            out.append((prm, False))
    return out


def evaluate(model: MLP, held):
    """Held-out comparison with the grid search: predicted time ratio,
    fraction within 10 %, fallback rate, selection latency."""
    import torch
    t0 = time.perf_counter()
    opt = [S.grid_search(s, t) for s, t in held]
    t_grid = (time.perf_counter() - t0) / len(held)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    X = np.array([S.descriptor(s, t) for s, t in held])
    Yp = model.predict_raw(X)
    t_net = (time.perf_counter() - t0) / len(held)
    ratios, fallback, miss = [], 0, 0
    coef = S.load_timing()
    for (s, t), y, o in zip(held, Yp, opt):
        if o is None:
            continue
        prm = choose(y, s, t)
        if prm is None:
            fallback += 1
            prm = o[0]
        tp = float(S.predicted_time(prm.alpha, prm.r_c, prm.M, prm.p, s, coef))
        ratios.append(tp / o[1])
        if S.rms_force_error(prm, s) > t * 1.0001:
            miss += 1
    ratios = np.array(ratios)
    return {"n": int(len(ratios)), "within_10pct": float((ratios <= 1.10).mean()),
            "median_time_ratio": float(np.median(ratios)), "p90_time_ratio": float(np.percentile(ratios, 90)),
            "fallback_rate": float(fallback / max(1, len(ratios))), "target_missed": int(miss),
            "grid_search_seconds_per_system": t_grid, "network_seconds_per_system": t_net}


def main(out_path=None, n_train=20000, n_held=500, epochs=300):
    t0 = time.time()
    train = sample_systems(n_train, 5)
    held = sample_systems(n_held, 6)
    X, Y, _ = label(train)
    t_label = time.time() - t0
    model = MLP()
    hist = model.fit(X, Y, epochs=epochs, log=print)
    ev = evaluate(model, held)
    ev.update({"n_train": int(X.shape[0]), "label_seconds": t_label, "final_loss": hist[-1],
               "first_loss": hist[0], "epochs": epochs})
    model.save(extra={"eval": ev})
    print(json.dumps(ev, indent=1))
    if out_path:
        with open(out_path, "w") as f:
            json.dump(ev, f, indent=1)
    return ev


if __name__ == "__main__":
    main(sys.argv[1] if len(sys.argv) > 1 else None)
