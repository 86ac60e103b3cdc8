"""Pins of the FP64 network reference: its gradient equals central finite
differences of its loss; Adam's first step moves each weight by lr in the
direction opposite to the gradient's sign (bias-corrected moments)."""
import numpy as np

from oracle import mlp as R


def test_gradient_matches_finite_differences():
    g = np.random.default_rng(0)
    w = g.normal(0, 0.3, size=R.NPARAM)
    x = g.normal(size=(9, 6))
    t = g.normal(size=(9, 4))
    ow = np.array([1.0, 2.0, 0.5, 1.5])
    L, grad = R.loss_and_grad(w, x, t, ow)
    h = 1e-6
    for k in list(range(0, R.NPARAM, 97)) + [R.NPARAM - 1]:
        wp = w.copy(); wp[k] += h
        wm = w.copy(); wm[k] -= h
        fd = (R.loss_and_grad(wp, x, t, ow)[0] - R.loss_and_grad(wm, x, t, ow)[0]) / (2 * h)
        assert abs(fd - grad[k]) < 1e-7 * (1 + abs(grad[k]))


def test_adam_first_step():
    g = np.random.default_rng(1).normal(size=50)
    w = np.zeros(50)
    w1, m, v = R.adam(w, np.zeros(50), np.zeros(50), g, 1, 0.01)
    assert np.allclose(w1, -0.01 * np.sign(g), atol=1e-9)
