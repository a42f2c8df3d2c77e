"""Host logic of the autograd Function (no GPU): which schedule runs.

One pass: when H or w requires a gradient and grad mode is on, the forward
pass runs the batch in tangent mode and the backward pass only scales the
gradients it kept.  Replay, or no gradient wanted: the forward pass runs
without tangents, and the backward pass (replay) reruns it in tangent mode
and checks that T is reproduced.  The runs are faked here; the GPU tests
check the real ones against a direct tangent run.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")


@pytest.fixture
def runs(monkeypatch):
    from paper_1709_02121_gb300 import grad
    calls = []

    def fake(wl, H, w, steps, tangent, capacity, stream=None):
        calls.append(bool(tangent))
        T = np.asarray(H, np.float64) * 0.1 + np.asarray(w, np.float64) * 0.01
        g = np.stack([np.full(len(H), 2.0), np.full(len(H), 3.0)], 1) if tangent else None
        return T, g, {}
    monkeypatch.setattr(grad, "run_batch", fake)
    return grad, calls


def test_one_pass_runs_the_tangent_mode_once(runs):
    grad, calls = runs
    H = torch.tensor([1.0, 2.0], dtype=torch.float64, requires_grad=True)
    w = torch.tensor([0.5, 0.7], dtype=torch.float64, requires_grad=True)
    T = grad.transmission(H, w, {}, 10, 1000)
    (T * torch.tensor([1.0, 4.0], dtype=torch.float64)).sum().backward()
    assert calls == [True]
    assert H.grad.tolist() == [2.0, 8.0] and w.grad.tolist() == [3.0, 12.0]


def test_replay_runs_forward_then_tangent(runs):
    grad, calls = runs
    H = torch.tensor([1.0], dtype=torch.float64, requires_grad=True)
    w = torch.tensor([0.5], dtype=torch.float64)
    T = grad.transmission(H, w, {}, 10, 1000, replay=True)
    T.sum().backward()
    assert calls == [False, True] and H.grad.tolist() == [2.0]


def test_no_gradient_wanted_runs_no_tangents(runs):
    grad, calls = runs
    H = torch.tensor([1.0], dtype=torch.float64, requires_grad=True)
    w = torch.tensor([0.5], dtype=torch.float64, requires_grad=True)
    with torch.no_grad():
        grad.transmission(H, w, {}, 10, 1000)
    grad.transmission(H.detach(), w.detach(), {}, 10, 1000)
    assert calls == [False, False]
