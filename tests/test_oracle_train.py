"""Pins of the oracle's loss and Adam step against closed forms."""
import numpy as np

from oracle import train as TR


def test_l2_loss_closed_form():
    g = np.random.default_rng(0)
    t = g.uniform(0, 1, 3000)
    d = g.normal(0, 0.1, 3000)
    loss, grad = TR.l2_loss(t + d, t)
    assert np.isclose(loss, 0.5 * np.sum(d * d), rtol=1e-12)
    np.testing.assert_allclose(grad, d, atol=1e-15)
    assert TR.l2_loss(t, t)[0] == 0.0


def test_adam_first_step_is_lr_times_sign():
    """At t = 1 the bias-corrected moments are g and g^2, so the step is
    lr g / (|g| + eps): lr sign(g) up to eps."""
    g = np.random.default_rng(1).normal(0, 1, 1000)
    p, m, v = TR.adam_step(np.zeros(1000), g, np.zeros(1000), np.zeros(1000), 1, lr=0.01, eps=1e-15)
    np.testing.assert_allclose(p, -0.01 * np.sign(g), rtol=1e-9)
    np.testing.assert_allclose(m, 0.1 * g, rtol=1e-12)
    np.testing.assert_allclose(v, 0.001 * g * g, rtol=1e-12)


def test_adam_constant_gradient_keeps_unit_steps():
    """For a constant gradient the bias-corrected moments stay g and g^2 at
    every step, so every step moves p by lr sign(g)."""
    g = np.array([2.0, -0.5, 1e-3])
    p, m, v = np.zeros(3), np.zeros(3), np.zeros(3)
    for t in range(1, 51):
        p, m, v = TR.adam_step(p, g, m, v, t, lr=0.1, beta1=0.8, beta2=0.95, eps=0.0)
    np.testing.assert_allclose(p, -50 * 0.1 * np.sign(g), rtol=1e-10)


def test_adam_minimises_a_quadratic():
    """Adam on f(p) = 1/2 |p - a|^2 ends near a."""
    a = np.array([1.0, -2.0, 0.5])
    p, m, v = np.zeros(3), np.zeros(3), np.zeros(3)
    for t in range(1, 2001):
        p, m, v = TR.adam_step(p, p - a, m, v, t, lr=0.01)
    np.testing.assert_allclose(p, a, atol=1e-3)
