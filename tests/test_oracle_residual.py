"""Pins of the oracle's skip connections (residual networks, R11).

A skip x^(k) = W^(k) xhat^(k-1) + b^(k) + S xhat^(m) (S the identity or a
projection shortcut) changes no arithmetic of Theorem 3.1 other than adding
S^T nu^(k) to the coefficient of xhat^(m). The pins below hold the oracle to
facts written without that code path:

* the same function as a plain feed-forward network: xhat^(m) >= 0 rides
  through the layers in between on extra neurons with identity rows and zero
  bias, whose pre-activation bounds [max(l,0), max(u,0)] make them stable
  (active, or inactive where xhat^(m) = 0), so Theorem 3.1 treats them
  exactly and the bound, its gradient and the LP optimum of Eq. 16 are the
  plain network's (S on the carried columns of layer k); a skip from the
  layer's own input is W^(k) + S;
* weak duality against the LP and MIP of the residual network;
* soundness on sampled inputs pushed through the network's forward pass;
* central differences of the bound.
"""
import dataclasses

import numpy as np
import pytest

from oracle import gcp_oracle as O
from paper_2208_05740_gb300 import synth


def _dense(ly):
    if ly.kind == synth.DENSE:
        return np.array(ly.W, np.float64)        # a copy: the plain network is edited in place
    return O.conv_matrix(np.asarray(ly.W, np.float64), ly.in_shape, ly.out_shape, ly.stride, ly.pad).toarray()


def plain_equivalent(inst):
    """The residual instance as a plain network: (instance, per-layer original widths).

    Passthrough neurons are appended after the original ones, so split and cut
    indices stay valid. Skips from the input need m = 0 only at k = 1."""
    net = inst.net
    L = net.L
    Ws = [_dense(ly) for ly in net.layers]
    bs = [np.asarray(ly.b, np.float64) for ly in net.layers]
    lo = [np.asarray(a, np.float64) for a in inst.inter_lo]
    hi = [np.asarray(a, np.float64) for a in inst.inter_hi]
    widths = [W.shape[0] for W in Ws]
    for k in range(1, L + 1):
        s = net.layers[k - 1].skip
        if not s:
            continue
        m = s - 1
        sc = net.layers[k - 1].shortcut
        d_m = widths[m - 1] if m >= 1 else net.layers[0].d_in
        S = np.eye(widths[k - 1], d_m) if sc is None else _dense(sc)
        if sc is not None:
            bs[k - 1] = bs[k - 1] + np.asarray(sc.b, np.float64)
        if m == k - 1:
            Ws[k - 1][:, :S.shape[1]] += S
            continue
        assert m >= 1, "a skip from the input is only exact as W + I"
        d = widths[m - 1]
        src_off = None            # column of xhat^(m) in the input of layer m+1: its first d entries
        for t in range(m + 1, k):
            row_off = Ws[t - 1].shape[0]
            # identity rows: from xhat^(m) itself (t = m+1) or from the previous passthrough
            col = 0 if t == m + 1 else src_off
            R_ = np.zeros((d, Ws[t - 1].shape[1]))
            R_[np.arange(d), col + np.arange(d)] = 1.0
            Ws[t - 1] = np.vstack([Ws[t - 1], R_])
            bs[t - 1] = np.concatenate([bs[t - 1], np.zeros(d)])
            # the next layer sees the new rows as extra input columns
            if t < L:
                Ws[t] = np.hstack([Ws[t], np.zeros((Ws[t].shape[0], d))])
            lo[t - 1] = np.concatenate([lo[t - 1], np.maximum(inst.inter_lo[m - 1], 0.0)])
            hi[t - 1] = np.concatenate([hi[t - 1], np.maximum(inst.inter_hi[m - 1], 0.0)])
            src_off = row_off
        Ws[k - 1][:, src_off:src_off + d] += S
    layers = [synth.Layer(synth.DENSE, W, b, (W.shape[1],), (W.shape[0],)) for W, b in zip(Ws, bs)]
    plain = dataclasses.replace(inst, net=synth.Network(layers), inter_lo=lo, inter_hi=hi)
    return plain, widths


def _lift(P_plain, D):
    """Residual duals -> plain duals (zero slopes on passthrough neurons)."""
    al = []
    for i, a in enumerate(D.alpha):
        pad = P_plain.dims[i + 1] - a.shape[1]
        al.append(np.hstack([a, np.zeros((a.shape[0], pad))]))
    return O.Duals(al, D.beta.copy(), D.gamma.copy())


def _random_duals(rng, P):
    return O.Duals([rng.random(a.shape) for a in O.default_duals(P).alpha],
                   rng.exponential(0.5, (P.R, P.max_splits)), rng.exponential(0.3, (P.R, P.N)))


def _with_skip(inst, k, s, scale=1.0):
    layers = list(inst.net.layers)
    ly = layers[k - 1]
    layers[k - 1] = dataclasses.replace(ly, W=scale * ly.W, skip=s)
    net = synth.Network(layers)
    lo, hi = synth.interval_bounds(net, inst.x_lo, inst.x_hi)
    return dataclasses.replace(inst, net=net, inter_lo=lo, inter_hi=hi)


def _proj(rng, d_out, d_in):
    return synth.Layer(synth.DENSE, rng.normal(0, 0.3, (d_out, d_in)), rng.normal(0, 0.1, d_out), (d_in,), (d_out,))


def _cases():
    yield "blocks", synth.mlp_residual(n_sub=4, n_cuts=8)
    yield "wide_blocks", synth.mlp_residual(seed=synth.SEED_BASE + 61, width=12, d0=6, blocks=3, n_sub=3,
                                            n_cuts=10, max_splits=3)
    base = synth.mlp_residual(seed=synth.SEED_BASE + 62, blocks=1, n_sub=3, n_cuts=6)
    # a skip from the layer's own input (W + I); xhat^(1) then feeds two skips
    yield "self_and_shared_source", _with_skip(base, 2, 2, 0.5)
    rng = np.random.default_rng(synth.SEED_BASE + 64)
    net = synth.make_mlp(rng, [8, 16, 16, 16, 16, 3])
    net.layers[3] = dataclasses.replace(net.layers[3], W=0.5 * net.layers[3].W, skip=2)   # x^(4) += xhat^(1)
    yield "three_back", synth._finish("three_back", rng, net, rng.random(8), 0.1, 2, 3, (0, 2),
                                      dict(n_cuts=8, min_vars=2, max_vars=4, hidden_only=True))
    # dense projection shortcuts between layers of different widths
    rng = np.random.default_rng(synth.SEED_BASE + 65)
    net = synth.make_mlp(rng, [8, 16, 12, 10, 3])
    net.layers[0] = dataclasses.replace(net.layers[0], skip=1, shortcut=_proj(rng, 16, 8))    # x^(1) += S x
    net.layers[1] = dataclasses.replace(net.layers[1], skip=2, shortcut=_proj(rng, 12, 16))   # x^(2) += S xhat^(1)
    net.layers[2] = dataclasses.replace(net.layers[2], skip=2, shortcut=_proj(rng, 10, 16))   # x^(3) += S xhat^(1)
    yield "projections", synth._finish("proj", rng, net, rng.random(8), 0.1, 2, 3, (0, 2),
                                       dict(n_cuts=8, min_vars=2, max_vars=4, hidden_only=True))
    # a residual CNN with a 1x1 stride-2 convolution shortcut (the resnet2b block structure, small)
    yield "resnet_small", synth.cnn_resnet(hw=8, stem=4, blocks=((8, 2), (8, 1)), fc=16, n_spec=2, n_sub=2,
                                           n_cuts=6, max_splits=2)


@pytest.mark.parametrize("name,inst", list(_cases()))
def test_residual_bound_equals_its_plain_network(name, inst):
    P = O.build_problem(inst)
    plain, widths = plain_equivalent(inst)
    Q = O.build_problem(plain)
    assert any(P.skip) and not any(Q.skip)
    rng = np.random.default_rng(5)
    for D in (O.default_duals(P), _random_duals(rng, P), _random_duals(rng, P)):
        g, G = O.gradient(P, D)
        h, H = O.gradient(Q, _lift(Q, D))
        np.testing.assert_allclose(g, h, rtol=1e-12, atol=1e-10)
        for i, (ga, ha) in enumerate(zip(G.alpha, H.alpha)):
            np.testing.assert_allclose(ga, ha[:, :widths[i]], rtol=1e-10, atol=1e-10)
        np.testing.assert_allclose(G.beta, H.beta, rtol=1e-10, atol=1e-10)
        np.testing.assert_allclose(G.gamma, H.gamma, rtol=1e-10, atol=1e-10)


@pytest.mark.parametrize("projection", [False, True])
def test_skip_from_the_input_and_into_the_spec_layer(projection):
    """m = 0 on layer 1 (x^(1) = (W + S) x + b) and a skip on the last layer."""
    rng = np.random.default_rng(synth.SEED_BASE + 63)
    if projection:
        net = synth.make_mlp(rng, [6, 8, 8, 8, 5])
        net.layers[0] = dataclasses.replace(net.layers[0], skip=1, shortcut=_proj(rng, 8, 6))
        net.layers[3] = dataclasses.replace(net.layers[3], skip=3, shortcut=_proj(rng, 5, 8))
    else:
        net = synth.make_mlp(rng, [6, 6, 8, 8, 8])
        net.layers[0] = dataclasses.replace(net.layers[0], skip=1)
        net.layers[3] = dataclasses.replace(net.layers[3], skip=3)       # adds xhat^(2) to the output layer
    x0 = rng.random(6)
    inst = synth._finish("skip_io", rng, net, x0, 0.1, 2, 3, (0, 2),
                         dict(n_cuts=6, min_vars=2, max_vars=3, hidden_only=True))
    P = O.build_problem(inst)
    plain, widths = plain_equivalent(inst)
    Q = O.build_problem(plain)
    for D in (O.default_duals(P), _random_duals(rng, P)):
        g, G = O.gradient(P, D)
        h, H = O.gradient(Q, _lift(Q, D))
        np.testing.assert_allclose(g, h, rtol=1e-12, atol=1e-10)
        np.testing.assert_allclose(G.gamma, H.gamma, rtol=1e-10, atol=1e-10)
    for r in range(P.R):
        a, b = O.lp_value(P, r // P.K, r % P.K), O.lp_value(Q, r // P.K, r % P.K)
        assert (a is None) == (b is None)
        if a is not None:
            assert abs(a - b) <= 1e-7 * max(1.0, abs(a))


def _duality_cases():
    yield "blocks0", synth.mlp_residual(seed=synth.SEED_BASE + 70, n_sub=3, n_cuts=6)
    yield "blocks1", synth.mlp_residual(seed=synth.SEED_BASE + 71, n_sub=3, n_cuts=6)
    cases = dict(_cases())
    yield "projections", cases["projections"]
    yield "resnet_small", cases["resnet_small"]


@pytest.mark.parametrize("name,inst", list(_duality_cases()))
def test_residual_weak_duality_and_lp_of_the_plain_network(name, inst):
    P = O.build_problem(inst)
    Q = O.build_problem(plain_equivalent(inst)[0])
    g, _ = O.optimize(P, O.default_duals(P), 20, 0.1, 0.1, 0.1)
    checked = 0
    for r in range(P.R):
        s, k = r // P.K, r % P.K
        lp = O.lp_value(P, s, k)
        lq = O.lp_value(Q, s, k)
        assert (lp is None) == (lq is None)
        if lp is None:
            continue
        assert abs(lp - lq) <= 1e-7 * max(1.0, abs(lp))
        assert g[r] <= lp + 1e-7 * max(1.0, abs(lp))
        mip = O.lp_value(P, s, k, integral=True)
        assert mip is None or mip >= lp - 1e-7 * max(1.0, abs(lp))
        checked += 1
    assert checked > 0


def test_residual_bound_is_sound_on_sampled_inputs():
    """Without cuts the bound holds for every input of the box in each subdomain."""
    inst = synth.mlp_residual(seed=synth.SEED_BASE + 72, n_sub=4, n_cuts=0)
    P = O.build_problem(inst)
    g, _ = O.optimize(P, O.default_duals(P), 20, 0.1, 0.1, 0.1)
    rng = np.random.default_rng(72)
    xs = synth.sample_box(rng, inst.x_lo, inst.x_hi, 20000)
    pre = synth.forward_all(inst.net, xs)
    checked = 0
    for s in range(inst.sub.n):
        ok = np.ones(len(xs), bool)
        for e in range(inst.sub.ptr[s], inst.sub.ptr[s + 1]):
            i, j, sg = inst.sub.layer[e], inst.sub.index[e], inst.sub.sign[e]
            ok &= (pre[i - 1][:, j] >= 0) if sg > 0 else (pre[i - 1][:, j] <= 0)
        if ok.any():
            f = pre[-1][ok] @ inst.spec.T
            for k in range(P.K):
                assert g[s * P.K + k] <= f[:, k].min() + 1e-9
                checked += 1
    assert checked > 0
    # the interval bounds of the generator contain every sampled pre-activation
    for i, (lo, hi) in enumerate(zip(inst.inter_lo, inst.inter_hi)):
        assert np.all(pre[i] >= lo - 1e-12) and np.all(pre[i] <= hi + 1e-12)


def test_residual_gradient_matches_central_differences():
    inst = synth.mlp_residual(seed=synth.SEED_BASE + 73, n_sub=2, n_cuts=5)
    P = O.build_problem(inst)
    rng = np.random.default_rng(3)
    D = _random_duals(rng, P)
    g, G = O.gradient(P, D)
    h = 1e-6

    def fd(get):
        out = []
        for _ in range(6):
            arr = get(D)
            idx = tuple(int(rng.integers(0, n)) for n in arr.shape)
            E1, E2 = D.copy(), D.copy()
            get(E1)[idx] += h
            get(E2)[idx] -= h
            out.append((idx, (O.evaluate(P, E1) - O.evaluate(P, E2)) / (2 * h)))
        return out
    for li in range(len(D.alpha)):
        for (r, j), d in fd(lambda X, li=li: X.alpha[li]):
            assert abs(d[r] - G.alpha[li][r, j]) <= 1e-5 * max(1.0, abs(d[r])), (li, r, j)
    for (r, j), d in fd(lambda X: X.gamma):
        assert abs(d[r] - G.gamma[r, j]) <= 1e-5 * max(1.0, abs(d[r]))


def test_planted_missing_skip_multiplier_is_caught(monkeypatch):
    """An oracle that forgets nu^(k) in y^(m) no longer matches the plain network."""
    inst = synth.mlp_residual(n_sub=2, n_cuts=4)
    P = O.build_problem(inst)
    Q = O.build_problem(plain_equivalent(inst)[0])
    D = O.default_duals(P)
    ref = O.evaluate(Q, _lift(Q, D))
    P.skip = [0] * len(P.skip)          # the LP rows and the bound both lose the skip
    assert np.max(np.abs(O.evaluate(P, D) - ref)) > 1e-3
