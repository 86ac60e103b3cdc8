"""The learned selector's kernels (through the C ABI) against the FP64
network reference, and the trained selector against the grid search."""
import json
import os

import numpy as np
import pytest

from oracle import mlp as R

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2004_12484_b300 import learned as Lr  # noqa: E402
from paper_2004_12484_b300 import selector as S  # noqa: E402

DEV = torch.device("cuda", 0)


def bf16_round(w):
    return torch.tensor(w, dtype=torch.float32).to(torch.bfloat16).float().double().numpy()


def setup(seed, B):
    g = np.random.default_rng(seed)
    w = g.normal(0, 0.25, size=R.NPARAM).astype(np.float32)
    x = g.normal(size=(B, 6)).astype(np.float32)
    t = g.normal(size=(B, 4)).astype(np.float32)
    m = Lr.MLP(device=DEV)
    m.set_weights(w)
    return m, w, x, t


def test_forward_matches_reference():
    m, w, x, _ = setup(0, 300)
    y = m.forward_raw(torch.tensor(x, device=DEV)).cpu().numpy()
    yr, _ = R.forward(bf16_round(w), x.astype(np.float64))
    assert np.abs(y - yr).max() < 1e-4 * np.abs(yr).max()


@pytest.mark.parametrize("B", [1, 64, 200])
def test_gradient_matches_reference(B):
    m, w, x, t = setup(1, B)
    ow = np.array([1.0, 0.5, 2.0, 1.0], dtype=np.float32)
    grad = torch.empty(R.NPARAM, dtype=torch.float32, device=DEV)
    loss = m.train_step(torch.tensor(x, device=DEV), torch.tensor(t, device=DEV), torch.tensor(ow, device=DEV),
                        0.0, grad=grad, apply=False)
    L, gr = R.loss_and_grad(bf16_round(w), x.astype(np.float64), t.astype(np.float64), ow.astype(np.float64))
    gg = grad.cpu().numpy()
    assert abs(float(loss) / L - 1) < 1e-5
    assert np.sqrt(((gg - gr) ** 2).sum() / (gr ** 2).sum()) < 1e-4


def test_adam_update_matches_reference():
    m, w, x, t = setup(2, 128)
    ow = np.ones(4, dtype=np.float32)
    grad = torch.empty(R.NPARAM, dtype=torch.float32, device=DEV)
    m.train_step(torch.tensor(x, device=DEV), torch.tensor(t, device=DEV), torch.tensor(ow, device=DEV), 1e-3,
                 grad=grad, apply=True)
    g = grad.cpu().numpy().astype(np.float64)
    w1, _, _ = R.adam(w.astype(np.float64), np.zeros(R.NPARAM), np.zeros(R.NPARAM), g, 1, 1e-3)
    assert np.abs(m.wm.cpu().numpy() - w1).max() < 1e-6
    assert torch.equal(m.wq, m.wm.to(torch.bfloat16))


def test_training_reduces_loss():
    g = np.random.default_rng(3)
    X = g.normal(size=(4096, 6))
    W = g.normal(size=(6, 4))
    Y = np.tanh(X @ W) + 0.1 * X[:, :4] ** 2
    m = Lr.MLP(device=DEV)
    hist = m.fit(X, Y, epochs=40, batch=256, lr=3e-3)
    assert hist[-1] < 0.1 * hist[0]


WEIGHTS = Lr.WEIGHTS_PATH


@pytest.mark.skipif(not os.path.exists(WEIGHTS), reason="selector not trained")
def test_trained_selector_on_held_out_systems():
    """500 held-out systems (seed 6): the network's legalised choices stay
    within 10 % of the grid-searched optimal time for most systems, never
    miss the error target, and are selected orders of magnitude faster than
    the grid search (the gain over selecting without the network)."""
    model = Lr.MLP.load(WEIGHTS, device=DEV)
    held = Lr.sample_systems(500, 6)
    ev = Lr.evaluate(model, held)
    assert ev["target_missed"] == 0
    assert ev["within_10pct"] >= 0.8, ev
    assert ev["median_time_ratio"] <= 1.05, ev
    assert ev["network_seconds_per_system"] * 50 < ev["grid_search_seconds_per_system"], ev
