"""Pins of the oracle's CROWN root bounds (crown_root_bounds).

The method takes sound pre-activation bounds l, u as input (Sec. 2, Eq. 1);
the measured workloads take them from CROWN, which the oracle computes by
composing its Theorem 3.1 over truncated networks. Pinned here from outside
that composition:
  * hidden layer 1 equals the exact interval image of the box (corners);
  * every bound is sound: sampled inputs' pre-activations lie inside;
  * every bound is at most as tight as the LP of the same truncated network
    over the same lower-layer bounds (weak duality, Eq. 16, HiGHS);
  * a network whose first hidden layer is stable and active everywhere is
    linear up to layer 2, so its layer-2 bounds are the exact box extrema;
  * the bounds are contained in interval bound propagation's.
"""
import itertools

import numpy as np
import pytest

from oracle import gcp_oracle as O
from paper_2208_05740_gb300 import synth

crown_root_bounds = O.crown_root_bounds


def _net(seed, dims):
    rng = np.random.default_rng(seed)
    net = synth.make_mlp(rng, list(dims))
    x0 = rng.random(dims[0])
    return net, x0 - 0.1, x0 + 0.1


def test_layer_one_is_the_exact_interval_image():
    net, lo, hi = _net(1, (4, 6, 5, 2))
    L, H = crown_root_bounds(net, lo, hi)
    W, b = net.layers[0].W, net.layers[0].b
    corners = np.array(list(itertools.product(*zip(lo, hi))))
    z = corners @ W.T + b
    np.testing.assert_allclose(L[0], z.min(0), atol=1e-12)
    np.testing.assert_allclose(H[0], z.max(0), atol=1e-12)


@pytest.mark.parametrize("seed", [2, 3, 4])
def test_bounds_are_sound_on_sampled_inputs(seed):
    net, lo, hi = _net(seed, (8, 16, 16, 16, 3))
    L, H = crown_root_bounds(net, lo, hi)
    X = synth.sample_box(np.random.default_rng(seed), lo, hi, 20000)
    for i, z in enumerate(synth.forward_all(net, X)[:-1]):
        assert np.all(z >= L[i] - 1e-12) and np.all(z <= H[i] + 1e-12), f"layer {i + 1}"


@pytest.mark.parametrize("seed", [5, 6])
def test_bounds_do_not_beat_the_lp_of_the_truncated_network(seed):
    net, lo, hi = _net(seed, (6, 10, 10, 3))
    L, H = crown_root_bounds(net, lo, hi)
    empty = synth.Subdomains(np.zeros(2, np.int32), np.zeros(0, np.int16), np.zeros(0, np.int32),
                             np.zeros(0, np.int8))
    ly = net.layers[1]
    for j in range(ly.d_out):
        last = synth.Layer(synth.DENSE, ly.W[[j]], ly.b[[j]], ly.in_shape, (1,))
        tr = synth.Instance("prefix", synth.Network([net.layers[0], last]), lo, hi,
                            np.array([[1.0], [-1.0]]), L[:1], H[:1], empty, synth.Cuts.empty())
        P = O.build_problem(tr)
        lp_min = O.lp_value(P, 0, 0, with_cuts=False)
        lp_max = -O.lp_value(P, 0, 1, with_cuts=False)
        assert L[1][j] <= lp_min + 1e-7 * max(1.0, abs(lp_min))
        assert H[1][j] >= lp_max - 1e-7 * max(1.0, abs(lp_max))


def test_stable_first_layer_gives_exact_box_extrema():
    rng = np.random.default_rng(7)
    d0, d1, d2 = 3, 5, 4
    W1 = rng.normal(size=(d1, d0))
    b1 = np.abs(W1).sum(1) * 2.0 + 1.0          # x^(1) > 0 on the whole box [-0.5, 0.5]^3
    W2 = rng.normal(size=(d2, d1))
    b2 = rng.normal(size=d2)
    W3 = rng.normal(size=(2, d2))
    net = synth.Network([synth.Layer(synth.DENSE, W1, b1, (d0,), (d1,)),
                         synth.Layer(synth.DENSE, W2, b2, (d1,), (d2,)),
                         synth.Layer(synth.DENSE, W3, np.zeros(2), (d2,), (2,))])
    lo, hi = -0.5 * np.ones(d0), 0.5 * np.ones(d0)
    L, H = crown_root_bounds(net, lo, hi)
    assert np.all(L[0] > 0)
    corners = np.array(list(itertools.product(*zip(lo, hi))))
    z2 = (corners @ W1.T + b1) @ W2.T + b2            # linear on the box: extrema at corners
    np.testing.assert_allclose(L[1], z2.min(0), rtol=0, atol=1e-10)
    np.testing.assert_allclose(H[1], z2.max(0), rtol=0, atol=1e-10)


def test_inside_interval_bounds():
    net, lo, hi = _net(8, (8, 16, 16, 16, 3))
    L, H = crown_root_bounds(net, lo, hi)
    IL, IH = synth.interval_bounds(net, lo, hi)
    for a, b, c, d in zip(L, H, IL, IH):
        assert np.all(a >= c - 1e-12) and np.all(b <= d + 1e-12)
    # strictly tighter somewhere past the first layer
    assert sum(float(np.sum(b - a)) for a, b in zip(L[1:], H[1:])) < \
        sum(float(np.sum(d - c)) for c, d in zip(IL[1:], IH[1:]))


# ---- residual networks (a skip connection into a truncated layer, R11)

def _res_net(seed):
    inst = synth.mlp_residual(seed=seed, width=12, d0=6, blocks=2, d_out=3, eps=0.1, n_sub=1, n_cuts=0)
    return inst.net, inst.x_lo, inst.x_hi


@pytest.mark.parametrize("seed", [11, 12])
def test_residual_bounds_are_sound_on_sampled_inputs(seed):
    net, lo, hi = _res_net(seed)
    L, H = crown_root_bounds(net, lo, hi)
    X = synth.sample_box(np.random.default_rng(seed), lo, hi, 20000)
    for i, z in enumerate(synth.forward_all(net, X)[:-1]):
        assert np.all(z >= L[i] - 1e-12) and np.all(z <= H[i] + 1e-12), f"layer {i + 1}"


def test_residual_bounds_inside_interval_bounds():
    net, lo, hi = _res_net(13)
    L, H = crown_root_bounds(net, lo, hi)
    IL, IH = synth.interval_bounds(net, lo, hi)
    for a, b, c, d in zip(L, H, IL, IH):
        assert np.all(a >= c - 1e-12) and np.all(b <= d + 1e-12)
    assert sum(float(np.sum(b - a)) for a, b in zip(L[1:], H[1:])) < \
        sum(float(np.sum(d - c)) for c, d in zip(IL[1:], IH[1:]))


def test_residual_skip_layer_bounds_do_not_beat_the_lp():
    """Layer 3 carries the first block's skip (it adds xhat^(1)): its bounds are
    at most as tight as the LP of the network truncated there with the skip."""
    net, lo, hi = _res_net(14)
    L, H = crown_root_bounds(net, lo, hi)
    ly = net.layers[2]
    assert int(ly.skip) == 2
    empty = synth.Subdomains(np.zeros(2, np.int32), np.zeros(0, np.int16), np.zeros(0, np.int32),
                             np.zeros(0, np.int8))
    for j in range(0, ly.d_out, 3):
        # the skip's identity restricted to row j: a one-row projection shortcut
        sel = synth.Layer(synth.DENSE, np.eye(ly.d_out)[[j]], np.zeros(1), ly.in_shape, (1,))
        import dataclasses
        last = dataclasses.replace(ly, W=ly.W[[j]], b=ly.b[[j]], out_shape=(1,), shortcut=sel)
        tr = synth.Instance("prefix", synth.Network(list(net.layers[:2]) + [last]), lo, hi,
                            np.array([[1.0], [-1.0]]), L[:2], H[:2], empty, synth.Cuts.empty())
        P = O.build_problem(tr)
        lp_min = O.lp_value(P, 0, 0, with_cuts=False)
        lp_max = -O.lp_value(P, 0, 1, with_cuts=False)
        assert L[2][j] <= lp_min + 1e-7 * max(1.0, abs(lp_min))
        assert H[2][j] >= lp_max - 1e-7 * max(1.0, abs(lp_max))
