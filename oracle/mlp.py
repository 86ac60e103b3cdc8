"""FP64 reference of the learned selector's network -- TEST INFRASTRUCTURE
ONLY (used by the tests to check the CUDA forward, gradient and Adam
kernels; shares no code with them).

Network 6 -> 64 -> 64 -> 4, SiLU activations, parameters packed row-major as
W1[64][6], b1[64], W2[64][64], b2[64], W3[4][64], b3[4].  Loss
L = 1/(4B) sum_s sum_c w_c (y_sc - t_sc)^2.  The gradient is the chain rule
written out layer by layer; it is pinned by central finite differences in
tests/test_mlp_oracle.py.
"""
import numpy as np

NI, NH, NO = 6, 64, 4
SIZES = [("W1", (NH, NI)), ("b1", (NH,)), ("W2", (NH, NH)), ("b2", (NH,)), ("W3", (NO, NH)), ("b3", (NO,))]
NPARAM = sum(int(np.prod(s)) for _, s in SIZES)


def unpack(w):
    w = np.asarray(w, dtype=np.float64)
    out, o = {}, 0
    for name, shape in SIZES:
        n = int(np.prod(shape))
        out[name] = w[o:o + n].reshape(shape)
        o += n
    return out


def silu(z):
    return z / (1.0 + np.exp(-z))


def silu_grad(z):
    s = 1.0 / (1.0 + np.exp(-z))
    return s * (1.0 + z * (1.0 - s))


def forward(w, x):
    p = unpack(w)
    x = np.asarray(x, dtype=np.float64)
    a1 = x @ p["W1"].T + p["b1"]
    h1 = silu(a1)
    a2 = h1 @ p["W2"].T + p["b2"]
    h2 = silu(a2)
    return h2 @ p["W3"].T + p["b3"], (x, a1, h1, a2, h2)


def loss_and_grad(w, x, t, ow):
    p = unpack(w)
    y, (x, a1, h1, a2, h2) = forward(w, x)
    B = x.shape[0]
    ow = np.asarray(ow, dtype=np.float64)
    e = y - t
    L = (ow * e * e).sum() / (B * NO)
    dy = 2.0 * ow * e / (B * NO)
    g = {"W3": dy.T @ h2, "b3": dy.sum(0)}
    d2 = (dy @ p["W3"]) * silu_grad(a2)
    g["W2"] = d2.T @ h1
    g["b2"] = d2.sum(0)
    d1 = (d2 @ p["W2"]) * silu_grad(a1)
    g["W1"] = d1.T @ x
    g["b1"] = d1.sum(0)
    return L, np.concatenate([g[name].reshape(-1) for name, _ in SIZES])


def adam(w, m, v, g, step, lr, b1=0.9, b2=0.999, eps=1e-8):
    m = b1 * m + (1 - b1) * g
    v = b2 * v + (1 - b2) * g * g
    mh = m / (1 - b1 ** step)
    vh = v / (1 - b2 ** step)
    return w - lr * mh / (np.sqrt(vh) + eps), m, v
