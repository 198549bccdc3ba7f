"""Pins of the oracle's Adam ascent (App. C.1 names Adam with a decaying rate).

The update is Kingma & Ba's (Adam: a method for stochastic optimization,
ICLR 2015, Algorithm 1) applied as ascent: m <- b1 m + (1-b1) g,
v <- b2 v + (1-b2) g^2, x <- x + lr_t * (m / (1-b1^t)) / (sqrt(v / (1-b2^t)) + eps),
then the projection onto Theorem 3.1's domain. The tests below do not retype
that rule; they check consequences of it that hold for any correct
implementation:

  * from zero moments, step 1 moves each coordinate by lr * g / (|g| + eps)
    (the bias corrections make m-hat = g and v-hat = g^2 exactly);
  * under a constant gradient g, every step t = 0, 1, ... moves by
    lr * decay^t * g / (|g| + eps) (m-hat = g, v-hat = g^2 at every t);
  * a gradient g followed by 0 moves the second step by
    lr * decay * (b1 / (1 + b1)) g / (sqrt(b2 / (1 + b2)) |g| + eps);
  * on the hand-derived one-neuron instance (tests/golden/one_neuron_z_cut.txt,
    dg/dgamma = 0.5 for 0 <= gamma < 1) a few Adam steps from gamma = 0 land
    on gamma = sum_t lr decay^t 0.5 / (0.5 + eps) and the bound on
    -1 + gamma / 2.
A planted bias-correction error is caught by the constant-gradient pin.
"""
import os

import numpy as np
import pytest

from oracle import gcp_oracle as O
from paper_2208_05740_gb300 import synth

from test_oracle_pins import _one_neuron_instance, tiny

B1, B2, EPS = 0.9, 0.999, 1e-8


def _constant_gradient(P, value):
    """A stand-in for O.gradient that returns the same gradient every call."""
    D0 = O.default_duals(P)

    def grad(P_, D):
        g = np.zeros(P_.R)
        G = O.Duals([np.full_like(a, value) for a in D0.alpha], np.full_like(D0.beta, value),
                    np.full_like(D0.gamma, value))
        return g, G
    return grad


def _sequence_gradient(P, values):
    D0 = O.default_duals(P)
    calls = []

    def grad(P_, D):
        v = values[len(calls)]
        calls.append(v)
        G = O.Duals([np.full_like(a, v) for a in D0.alpha], np.full_like(D0.beta, v), np.full_like(D0.gamma, v))
        return np.zeros(P_.R), G
    return grad


def _problem():
    return O.build_problem(tiny(3, n_sub=2, n_cuts=4))


def test_first_step_from_zero_moments(monkeypatch):
    """Step 1: x_1 = proj(x_0 + lr * g / (|g| + eps)) for every coordinate with g != 0."""
    P = _problem()
    D0 = O.default_duals(P)
    rng = np.random.default_rng(0)
    # start strictly inside the domain so the projection does not act on a small step
    D0.alpha = [np.full_like(a, 0.5) for a in D0.alpha]
    D0.beta = np.full_like(D0.beta, 0.5)
    D0.gamma = np.full_like(D0.gamma, 0.5)
    for g in (rng.normal(size=3).tolist() + [1e-9, -3e-9, 7.0]):
        monkeypatch.setattr(O, "gradient", _constant_gradient(P, g))
        lr_a, lr_b, lr_g = 0.01, 0.02, 0.03
        _, D1 = O.optimize(P, D0, 1, lr_a, lr_b, lr_g, optimizer="adam", lr_decay=0.9)
        monkeypatch.undo()
        unit = g / (abs(g) + EPS)
        for a in D1.alpha:
            np.testing.assert_allclose(a, 0.5 + lr_a * unit, rtol=0, atol=1e-15)
        np.testing.assert_allclose(D1.beta, 0.5 + lr_b * unit, rtol=0, atol=1e-15)
        np.testing.assert_allclose(D1.gamma, 0.5 + lr_g * unit, rtol=0, atol=1e-15)


@pytest.mark.parametrize("decay", [1.0, 0.9, 0.98])
def test_constant_gradient_moves_lr_decay_t_per_step(monkeypatch, decay):
    """Constant g: m-hat_t = g and v-hat_t = g^2 exactly, so step t moves lr decay^t g / (|g| + eps)."""
    P = _problem()
    D0 = O.default_duals(P)
    D0.alpha = [np.full_like(a, 0.25) for a in D0.alpha]
    D0.beta = np.full_like(D0.beta, 0.25)
    D0.gamma = np.full_like(D0.gamma, 0.25)
    g = 0.37
    lr = 0.01
    monkeypatch.setattr(O, "gradient", _constant_gradient(P, g))
    for T in (1, 2, 5, 12):
        _, DT = O.optimize(P, D0, T, lr, lr, lr, optimizer="adam", lr_decay=decay)
        moved = sum(lr * decay ** t * g / (g + EPS) for t in range(T))
        for a in DT.alpha:
            np.testing.assert_allclose(a, 0.25 + moved, rtol=0, atol=1e-14)
        np.testing.assert_allclose(DT.gamma, 0.25 + moved, rtol=0, atol=1e-14)
        np.testing.assert_allclose(DT.beta, 0.25 + moved, rtol=0, atol=1e-14)


def test_gradient_then_zero_second_step(monkeypatch):
    """g then 0: m-hat_2 = b1 g / (1 + b1), v-hat_2 = b2 g^2 / (1 + b2)."""
    P = _problem()
    D0 = O.default_duals(P)
    D0.gamma = np.full_like(D0.gamma, 0.5)
    g, lr, decay = -0.8, 0.01, 0.9
    monkeypatch.setattr(O, "gradient", _sequence_gradient(P, [g, 0.0]))
    _, D2 = O.optimize(P, D0, 2, lr, lr, lr, optimizer="adam", lr_decay=decay)
    step1 = lr * g / (abs(g) + EPS)
    step2 = lr * decay * (B1 / (1 + B1)) * g / (np.sqrt(B2 / (1 + B2)) * abs(g) + EPS)
    np.testing.assert_allclose(D2.gamma, 0.5 + step1 + step2, rtol=0, atol=1e-15)


def test_projection_after_adam_step(monkeypatch):
    """A step that leaves Theorem 3.1's domain lands on its boundary (alpha in [0,1], beta, gamma >= 0)."""
    P = _problem()
    D0 = O.default_duals(P)
    D0.alpha = [np.full_like(a, 0.995) for a in D0.alpha]
    D0.gamma = np.full_like(D0.gamma, 0.004)
    D0.beta = np.full_like(D0.beta, 0.004)
    monkeypatch.setattr(O, "gradient", _constant_gradient(P, 1.0))
    _, D1 = O.optimize(P, D0, 1, 0.01, 0.01, 0.01, optimizer="adam")
    for a in D1.alpha:
        assert np.all(a == 1.0)
    monkeypatch.setattr(O, "gradient", _constant_gradient(P, -1.0))
    _, D1 = O.optimize(P, D0, 1, 0.01, 0.01, 0.01, optimizer="adam")
    assert np.all(D1.gamma == 0.0) and np.all(D1.beta == 0.0)


@pytest.mark.parametrize("lr,decay,T", [(0.1, 0.9, 5), (0.05, 0.98, 8), (0.1, 1.0, 6)])
def test_golden_one_neuron_adam_trajectory(lr, decay, T):
    """The worked example's g(gamma) = -1 + gamma/2 on [0, 1): Adam from gamma = 0 (real gradients)."""
    P = O.build_problem(_one_neuron_instance())
    D0 = O.Duals([np.array([[0.5]])], np.zeros((1, 0)), np.array([[0.0]]))
    gT, DT = O.optimize(P, D0, T, lr, lr, lr, optimizer="adam", lr_decay=decay)
    gamma = sum(lr * decay ** t * 0.5 / (0.5 + EPS) for t in range(T))
    assert gamma < 1.0
    assert abs(DT.gamma[0, 0] - gamma) < 1e-14
    assert abs(gT[0] - (-1.0 + gamma / 2)) < 1e-14
    # alpha has zero gradient here (nuhat = 1 > 0): Adam leaves it where it was
    assert DT.alpha[0][0, 0] == 0.5


def test_planted_bias_correction_error_is_caught(monkeypatch):
    """An oracle whose Adam bias correction uses t - 1 instead of t (planted here) fails the constant-gradient pin."""
    def wrong_step(x, gx, mx, vx, lr, t, b1, b2, eps):
        mx *= b1
        mx += (1 - b1) * gx
        vx *= b2
        vx += (1 - b2) * gx * gx
        c1, c2 = 1.0 - b1 ** max(t - 1, 1), 1.0 - b2 ** max(t - 1, 1)
        x += lr * (mx / c1) / (np.sqrt(vx / c2) + eps)
    P = _problem()
    D0 = O.default_duals(P)
    D0.gamma = np.full_like(D0.gamma, 0.25)
    g, lr = 0.37, 0.01
    monkeypatch.setattr(O, "gradient", _constant_gradient(P, g))
    good = O.optimize(P, D0, 3, lr, lr, lr, optimizer="adam")[1].gamma
    monkeypatch.setattr(O, "adam_step", wrong_step)
    bad = O.optimize(P, D0, 3, lr, lr, lr, optimizer="adam")[1].gamma
    expect = 0.25 + 3 * lr * g / (g + EPS)
    assert np.allclose(good, expect, rtol=0, atol=1e-14)
    assert not np.allclose(bad, expect, rtol=0, atol=1e-6)
