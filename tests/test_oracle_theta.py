"""Pins of the oracle's directly optimised ReLU duals pi = theta * [nuhat]_+ (R12).

App. A closes by noting that Lemma A.1's closed form sets pi (and gamma_r = C - pi)
per neuron without regard to nu, so optimising pi as well is what reaches the
LP optimum. Any pi in [0, C] is a feasible dual, so:

* theta = pi* / C reproduces the closed-form bound exactly (pins the theta
  path against the closed form, which has its own pins);
* the bound at random theta never exceeds the LP optimum of Eq. 16 (weak
  duality over the whole theta box), with cuts and splits;
* on a one-hidden-layer network with a point input box and no cuts, where
  g(theta) separates by neuron, no theta beats the closed form;
* dg/dtheta matches central differences;
* a planted sign error in dh/dtheta is caught by the differences.
"""
import numpy as np
import pytest

from oracle import gcp_oracle as O
from paper_2208_05740_gb300 import synth
from tests.test_oracle_pins import tiny


def _rand(P, seed):
    rng = np.random.default_rng(seed)
    return O.Duals([rng.random(a.shape) for a in O.default_duals(P).alpha], rng.exponential(0.3, (P.R, P.max_splits)),
                   rng.exponential(0.3, (P.R, P.N)))


@pytest.mark.parametrize("seed", [101, 102, 103])
def test_closed_form_theta_reproduces_the_closed_form_bound(seed):
    inst = tiny(seed, n_sub=3, n_cuts=8, splits=(0, 2))
    P = O.build_problem(inst)
    for D in (O.default_duals(P), _rand(P, seed)):
        g = O.evaluate(P, D)
        Dt = D.copy()
        Dt.theta = O.theta_closed_form(P, D)
        assert all(np.all((t >= 0) & (t <= 1)) for t in Dt.theta)
        np.testing.assert_allclose(O.evaluate(P, Dt), g, rtol=1e-13, atol=1e-13)


@pytest.mark.parametrize("seed", [111, 112])
def test_any_theta_stays_below_the_lp(seed):
    inst = tiny(seed, n_sub=2, n_cuts=6)
    P = O.build_problem(inst)
    rng = np.random.default_rng(seed)
    lps = [O.lp_value(P, r // P.K, r % P.K) for r in range(P.R)]
    checked = 0
    for _ in range(4):
        D = _rand(P, int(rng.integers(1 << 30)))
        D.theta = [rng.random(a.shape) for a in D.alpha]
        g = O.evaluate(P, D)
        for r, lp in enumerate(lps):
            if lp is None:
                continue
            assert g[r] <= lp + 1e-7 * max(1.0, abs(lp)), (r, g[r], lp)
            checked += 1
    # and after joint ascent on theta with the other duals
    D = O.default_duals(P)
    D.theta = O.theta_closed_form(P, D)
    g, D = O.optimize(P, D, 40, 0.05, 0.05, 0.05, optimizer="adam")
    for r, lp in enumerate(lps):
        if lp is not None:
            assert g[r] <= lp + 1e-7 * max(1.0, abs(lp))
    assert checked > 0


def test_closed_form_is_best_for_a_separable_unstable_term():
    """One hidden layer, no cuts, a point input box x0 (eps = 0) and widened
    bounds l < x_j < u: then g(theta) = sum_j h_j(pi_j) - pi_j x_j + const with
    x_j = W_j x0 + b_j, and h_j(pi) - pi x_j rises with slope u - x_j >= 0 below
    Lemma A.1's pi* = u C / (u - l) and falls with slope l - x_j <= 0 above it,
    so the closed form is the maximum over theta."""
    rng = np.random.default_rng(121)
    net = synth.make_mlp(rng, [4, 12, 3])
    x0 = rng.random(4)
    inst = synth._finish("one_layer", rng, net, x0, 0.0, 2, 2, (0, 0),
                         dict(n_cuts=0, min_vars=2, max_vars=3, hidden_only=True))
    # a point box leaves no unstable neuron; widen the intermediate bounds instead
    inst.inter_lo[0] = inst.inter_lo[0] - 1.0
    inst.inter_hi[0] = inst.inter_hi[0] + 1.0
    P = O.build_problem(inst)
    D = _rand(P, 121)
    best = O.evaluate(P, D)
    for _ in range(200):
        Dt = D.copy()
        Dt.theta = [rng.random(a.shape) for a in D.alpha]
        assert np.all(O.evaluate(P, Dt) <= best + 1e-12)


def _fd_check(P, D, G, rng, n=16):
    h = 1e-6
    checked = 0
    for _ in range(n):
        li = int(rng.integers(0, P.L - 1))
        r, j = int(rng.integers(0, P.R)), int(rng.integers(0, P.dims[li + 1]))
        vals = []
        for e in (h, -h, h / 2, -h / 2):
            Dx = D.copy()
            Dx.theta[li][r, j] += e
            vals.append(O.evaluate(P, Dx)[r])
        f1 = (vals[0] - vals[1]) / (2 * h)
        f2 = (vals[2] - vals[3]) / h
        if abs(f1 - f2) < 1e-6:           # away from kinks
            assert abs(f1 - G.theta[li][r, j]) < 1e-5, (li, r, j, f1, G.theta[li][r, j])
            checked += 1
    return checked


def test_theta_gradient_matches_central_differences():
    inst = tiny(131, n_sub=3, n_cuts=8, splits=(1, 2))
    P = O.build_problem(inst)
    rng = np.random.default_rng(131)
    D = _rand(P, 131)
    D.theta = [np.clip(rng.random(a.shape), 0.05, 0.95) for a in D.alpha]
    g, G = O.gradient(P, D)
    assert _fd_check(P, D, G, rng, 40) >= 10
    # the other duals' gradients still match with theta set
    for _ in range(6):
        r, k = int(rng.integers(0, P.R)), int(rng.integers(0, P.N))
        Dp, Dm = D.copy(), D.copy()
        Dp.gamma[r, k] += 1e-6
        Dm.gamma[r, k] -= 1e-6
        f = (O.evaluate(P, Dp)[r] - O.evaluate(P, Dm)[r]) / 2e-6
        assert abs(f - G.gamma[r, k]) < 1e-4 * max(1.0, abs(f))


def test_planted_theta_gradient_sign_is_caught(monkeypatch):
    inst = tiny(141, n_sub=2, n_cuts=6, splits=(1, 2))
    P = O.build_problem(inst)
    rng = np.random.default_rng(141)
    D = _rand(P, 141)
    D.theta = [np.clip(rng.random(a.shape), 0.05, 0.95) for a in D.alpha]
    g, G = O.gradient(P, D)
    G.theta = [-t for t in G.theta]          # the planted mistake
    with pytest.raises(AssertionError):
        _fd_check(P, D, G, np.random.default_rng(141), 40)
