"""Pins of the FP64 Adam oracle (RoGs Sec. 4.2 optimiser; Adam's update rule), CPU only."""
import numpy as np
import pytest

import oracle


def test_first_step_is_signed_learning_rate():
    """At t = 1 the bias-corrected moments are g and g^2, so the step is
    -lr g / (|g| + eps)."""
    rng = np.random.default_rng(0)
    p, g = rng.normal(size=50), rng.normal(size=50)
    q, m, v = oracle.adam_step(p, g, np.zeros(50), np.zeros(50), lr=0.01, t=1)
    np.testing.assert_allclose(q - p, -0.01 * g / (np.abs(g) + 1e-8), rtol=1e-12, atol=0)
    np.testing.assert_allclose(m, 0.1 * g, rtol=1e-12)
    np.testing.assert_allclose(v, 0.001 * g * g, rtol=1e-12)


def test_constant_gradient_keeps_a_constant_step():
    """With the same g every step the bias-corrected moments stay g and g^2."""
    g = np.array([0.5, -2.0, 1e-3])
    p, m, v = np.zeros(3), np.zeros(3), np.zeros(3)
    for t in range(1, 30):
        q, m, v = oracle.adam_step(p, g, m, v, lr=1e-3, t=t)
        np.testing.assert_allclose(q - p, -1e-3 * g / (np.abs(g) + 1e-8), rtol=1e-9)
        p = q


def test_matches_a_library_adam():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(1)
    p0 = rng.normal(size=200)
    w = torch.tensor(p0.copy(), dtype=torch.float64, requires_grad=True)
    opt = torch.optim.Adam([w], lr=0.02, betas=(0.9, 0.999), eps=1e-8)
    p, m, v = p0.copy(), np.zeros(200), np.zeros(200)
    for t in range(1, 8):
        g = rng.normal(size=200)
        w.grad = torch.tensor(g)
        opt.step()
        p, m, v = oracle.adam_step(p, g, m, v, lr=0.02, t=t)
    np.testing.assert_allclose(w.detach().numpy(), p, rtol=1e-12, atol=1e-14)


def test_z_learning_rate_schedule_ends():
    assert oracle.z_learning_rate(0, 100, 10.0) == pytest.approx(1.6e-3)
    assert oracle.z_learning_rate(100, 100, 10.0) == pytest.approx(1.6e-5)
    assert oracle.z_learning_rate(50, 100, 1.0) == pytest.approx(1.6e-5)
