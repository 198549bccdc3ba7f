"""Pins of the FP64 oracle against facts fixed outside the oracle itself.

Each test checks the oracle against the LP/MIP of the same relaxation
(Eq. 16, Eq. 2-10), an independently written primal CROWN (Prop. 3.2),
closed forms (L = 1; Lemma A.1 by brute force), a hand-derived worked
example, invariances of the dual, finite differences, and soundness on
sampled network inputs.
"""
import dataclasses
import itertools
import os

import numpy as np
import pytest

from oracle import gcp_oracle as O
from paper_2208_05740_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def tiny(seed, n_sub=4, n_cuts=8, dims=(8, 16, 16, 3), splits=(0, 2), hidden_only=True, p_input=0.0):
    rng = np.random.default_rng(seed)
    net = synth.make_mlp(rng, list(dims))
    x0 = rng.random(dims[0])
    return synth._finish("tiny", rng, net, x0, 0.1, min(2, dims[-1] - 1), n_sub, splits,
                         dict(n_cuts=n_cuts, min_vars=2, max_vars=4, hidden_only=hidden_only,
                              p_input=p_input))


# --------------------------------------------------------------------------- P2
def test_lemma_a1_closed_form_matches_bruteforce_max():
    """Lemma A.1: h = max_{pi in [0,C]} l pi - relu(u (C - pi) + l pi - s)."""
    rng = np.random.default_rng(1)
    n = 20000
    l = -rng.exponential(1.0, n) - 1e-3
    u = rng.exponential(1.0, n) + 1e-3
    nu_hat = rng.normal(0, 1.5, n)
    s = rng.normal(0, 1.5, n)
    C = np.maximum(nu_hat, 0)
    pi, tau, h = O.unstable_closed_form(nu_hat, s, l, u, np.full(n, 0.3))

    def phi(p):
        return l * p - np.maximum(0.0, u * (C - p) + l * p - s)
    # the objective is piecewise linear in pi: its maximum sits at 0, C or the kink
    kink = np.clip((u * C - s) / (u - l), 0, C)
    brute = np.maximum(np.maximum(phi(np.zeros(n)), phi(C)), phi(kink))
    grid = np.max(np.stack([phi(C * t) for t in np.linspace(0, 1, 201)]), axis=0)
    assert np.all(brute >= grid - 1e-12)
    np.testing.assert_allclose(h, brute, rtol=0, atol=1e-12)
    assert np.all(pi >= 0) and np.all(pi <= C + 1e-15)
    np.testing.assert_allclose(phi(pi), h, atol=1e-12)
    # the printed numerator "+beta^T Q" would exceed the true maximum (unsound) for some s < 0
    p_pr = np.clip((u * C + s) / (u - l), 0, C)
    mid = (l * s <= 0)  # any
    h_printed = np.where((l * C <= s) & (s <= u * C), l * p_pr, np.where(s >= u * C, 0.0, s))
    assert np.any(h_printed > brute + 1e-9)
    assert mid.any()


# --------------------------------------------------------------------------- golden
def _one_neuron_instance(with_cut=True):
    W1 = np.array([[1.0]])
    W2 = np.array([[-1.0]])
    net = synth.Network([synth.Layer(synth.DENSE, W1, np.zeros(1), (1,), (1,)),
                         synth.Layer(synth.DENSE, W2, np.zeros(1), (1,), (1,))])
    sub = synth.Subdomains(np.array([0, 0], np.int32), np.zeros(0, np.int16), np.zeros(0, np.int32),
                           np.zeros(0, np.int8))
    if with_cut:
        cuts = synth.Cuts(np.array([0, 1], np.int64), np.array([1], np.int16), np.array([synth.KIND_Z], np.int8),
                          np.array([0], np.int32), np.array([1.0]), np.array([0.5]))
    else:
        cuts = synth.Cuts.empty()
    return synth.Instance("one_neuron", net, np.array([-1.0]), np.array([1.0]), np.array([[1.0]]),
                          [np.array([-1.0])], [np.array([1.0])], sub, cuts)


def test_golden_one_neuron_z_cut():
    rows, lp = [], {}
    for line in open(os.path.join(GOLDEN, "one_neuron_z_cut.txt")):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        parts = line.split()
        if parts[0].startswith("LP_"):
            lp[parts[0]] = float(parts[1])
        else:
            rows.append([float(v) for v in parts])
    P = O.build_problem(_one_neuron_instance())
    for gam, g_exp, dg_exp in rows:
        D = O.Duals([np.array([[0.5]])], np.zeros((1, 0)), np.array([[gam]]))
        g, G = O.gradient(P, D)
        assert abs(g[0] - g_exp) < 1e-14
        assert abs(G.gamma[0, 0] - dg_exp) < 1e-14
    assert abs(O.lp_value(P, 0, 0) - lp["LP_CUT"]) < 1e-9
    P0 = O.build_problem(_one_neuron_instance(with_cut=False))
    assert abs(O.lp_value(P0, 0, 0) - lp["LP_NOCUT"]) < 1e-9
    # optimising gamma reaches the LP-with-cut optimum on this instance
    gopt, _ = O.optimize(P, O.default_duals(P), 60, 0.1, 0.1, 0.1)
    assert abs(gopt[0] - lp["LP_CUT"]) < 1e-6


# --------------------------------------------------------------------------- P1
def test_single_linear_layer_is_exact_box_minimum():
    rng = np.random.default_rng(5)
    for _ in range(5):
        d0, dL = 6, 3
        W = rng.normal(size=(dL, d0))
        b = rng.normal(size=dL)
        net = synth.Network([synth.Layer(synth.DENSE, W, b, (d0,), (dL,))])
        x0 = rng.random(d0)
        sub = synth.Subdomains(np.array([0, 0], np.int32), np.zeros(0, np.int16), np.zeros(0, np.int32),
                               np.zeros(0, np.int8))
        C = rng.normal(size=(2, dL))
        inst = synth.Instance("lin", net, x0 - 0.2, x0 + 0.2, C, [], [], sub, synth.Cuts.empty())
        P = O.build_problem(inst)
        g = O.evaluate(P, O.default_duals(P))
        corners = np.array(list(itertools.product(*[(lo, hi) for lo, hi in zip(x0 - 0.2, x0 + 0.2)])))
        vals = (corners @ W.T + b) @ C.T
        np.testing.assert_allclose(g, vals.min(axis=0), rtol=0, atol=1e-12)


# --------------------------------------------------------------------------- P3
def primal_crown(inst, alpha_list, rows_sub, rows_spec):
    """Textbook CROWN (Zhang et al. 2018), primal form, written independently.

    Lower-bounds c^T f(x): keep the linear coefficient lam on xhat^(i); use
    xhat >= alpha x where lam >= 0 and the chord xhat <= u (x - l)/(u - l) where
    lam < 0; then pass lam through x^(i) = W xhat^(i-1) + b.
    """
    net = inst.net
    out = []
    for r, (s, k) in enumerate(zip(rows_sub, rows_spec)):
        c = inst.spec[k]
        lam = c @ net.layers[-1].W
        const = float(c @ net.layers[-1].b)
        for i in range(net.L - 1, 0, -1):
            lo, hi = inst.inter_lo[i - 1], inst.inter_hi[i - 1]
            lam_x = np.zeros_like(lam)
            for j in range(len(lam)):
                if hi[j] <= 0:
                    continue
                if lo[j] >= 0:
                    lam_x[j] = lam[j]
                elif lam[j] >= 0:
                    lam_x[j] = alpha_list[i - 1][r, j] * lam[j]
                else:
                    slope = hi[j] / (hi[j] - lo[j])
                    lam_x[j] = lam[j] * slope
                    const += -lam[j] * slope * lo[j]
            const += float(lam_x @ net.layers[i - 1].b)
            lam = lam_x @ net.layers[i - 1].W
        const += float(np.sum(np.minimum(lam * inst.x_lo, lam * inst.x_hi)))
        out.append(const)
    return np.array(out)


@pytest.mark.parametrize("seed", [11, 12, 13])
def test_no_cuts_no_splits_reduces_to_crown(seed):
    inst = tiny(seed, n_sub=3, n_cuts=0, splits=(0, 0))
    P = O.build_problem(inst)
    rng = np.random.default_rng(seed)
    D = O.default_duals(P)
    D.alpha = [rng.random(a.shape) for a in D.alpha]
    g = O.evaluate(P, D)
    ref = primal_crown(inst, D.alpha, O.row_sub(P), O.row_spec(P))
    np.testing.assert_allclose(g, ref, rtol=0, atol=1e-12)


# --------------------------------------------------------------------------- P4 / P5
@pytest.mark.parametrize("seed", [21, 22, 23, 24])
def test_weak_duality_against_lp_and_mip(seed):
    inst = tiny(seed)
    P = O.build_problem(inst)
    rng = np.random.default_rng(seed)
    Ds = [O.default_duals(P)]
    for _ in range(3):
        a, b, gm = synth.random_duals(rng, inst, 1.0, 1.0)
        Ds.append(O.Duals(a, b, gm))
    Ds.append(O.optimize(P, O.default_duals(P), 20, 0.1, 0.1, 0.1)[1])
    checked = 0
    for D in Ds:
        g = O.evaluate(P, D)
        for r in range(P.R):
            s, k = r // P.K, r % P.K
            lp = O.lp_value(P, s, k)
            if lp is None:
                continue
            assert g[r] <= lp + 1e-7 * max(1.0, abs(lp)), (r, g[r], lp)
            # sample-fitted cuts need not be MIP-valid, so the MIP may be infeasible
            mip = O.lp_value(P, s, k, integral=True)
            assert mip is None or mip >= lp - 1e-7 * max(1.0, abs(lp))
            checked += 1
    assert checked > 0


def test_optimised_bound_improves_and_stays_below_lp():
    inst = tiny(31, n_sub=2, n_cuts=6)
    P = O.build_problem(inst)
    g0 = O.evaluate(P, O.default_duals(P))
    g1, D = O.optimize(P, O.default_duals(P), 40, 0.1, 0.1, 0.1)
    assert np.mean(g1 - g0) > 0
    for r in range(P.R):
        lp = O.lp_value(P, r // P.K, r % P.K)
        if lp is not None:
            assert g1[r] <= lp + 1e-7 * max(1, abs(lp))


@pytest.mark.parametrize("seed", [41, 42])
def test_valid_cuts_bound_never_exceeds_true_minimum(seed):
    """With MIP-valid offsets d (App. C: cuts of the root MIP), g <= min f over the subdomain."""
    inst = tiny(seed, n_sub=3, n_cuts=5, dims=(4, 6, 5, 3))
    P = O.build_problem(inst)
    P.d = O.valid_cut_offsets(P)
    inst = dataclasses.replace(inst, cuts=dataclasses.replace(inst.cuts, d=P.d))
    g, D = O.optimize(P, O.default_duals(P), 30, 0.1, 0.1, 0.1)
    for r in range(P.R):
        s, k = r // P.K, r % P.K
        true_min = O.lp_value(P, s, k, integral=True, with_cuts=False)
        if true_min is None:
            continue
        assert g[r] <= true_min + 1e-7 * max(1, abs(true_min))
    # and on sampled network inputs lying in each subdomain
    rng = np.random.default_rng(seed)
    xs = synth.sample_box(rng, inst.x_lo, inst.x_hi, 4000)
    pre = synth.forward_all(inst.net, xs)
    for s in range(inst.sub.n):
        ok = np.ones(len(xs), bool)
        for e in range(inst.sub.ptr[s], inst.sub.ptr[s + 1]):
            i, j, sg = inst.sub.layer[e], inst.sub.index[e], inst.sub.sign[e]
            ok &= (pre[i - 1][:, j] >= 0) if sg > 0 else (pre[i - 1][:, j] <= 0)
        if not ok.any():
            continue
        f = pre[-1][ok] @ inst.spec.T
        for k in range(P.K):
            assert g[s * P.K + k] <= f[:, k].min() + 1e-9


def test_sampled_soundness_with_sample_fitted_cuts():
    """Inputs that satisfy every cut and split are feasible for Eq. 16: g <= f(x) there."""
    inst = tiny(51, n_sub=4, n_cuts=8)
    P = O.build_problem(inst)
    g, _ = O.optimize(P, O.default_duals(P), 20, 0.1, 0.1, 0.1)
    rng = np.random.default_rng(51)
    xs = synth.sample_box(rng, inst.x_lo, inst.x_hi, 20000)
    pre = synth.forward_all(inst.net, xs)
    lhs = np.zeros((len(xs), inst.cuts.n))
    for kk in range(inst.cuts.n):
        for e in range(inst.cuts.ptr[kk], inst.cuts.ptr[kk + 1]):
            i, kind, j, c = inst.cuts.layer[e], inst.cuts.kind[e], inst.cuts.index[e], inst.cuts.coef[e]
            x = xs[:, j] if i == 0 else pre[i - 1][:, j]
            val = x if (i == 0 or kind == synth.KIND_X) else (np.maximum(x, 0) if kind == synth.KIND_XHAT
                                                              else (x > 0).astype(float))
            lhs[:, kk] += c * val
    feas = np.all(lhs <= inst.cuts.d[None, :] + 1e-12, axis=1)
    n_checked = 0
    for s in range(inst.sub.n):
        ok = feas.copy()
        for e in range(inst.sub.ptr[s], inst.sub.ptr[s + 1]):
            i, j, sg = inst.sub.layer[e], inst.sub.index[e], inst.sub.sign[e]
            ok &= (pre[i - 1][:, j] >= 0) if sg > 0 else (pre[i - 1][:, j] <= 0)
        if ok.any():
            f = pre[-1][ok] @ inst.spec.T
            for k in range(P.K):
                assert g[s * P.K + k] <= f[:, k].min() + 1e-9
                n_checked += 1
    assert n_checked > 0


# --------------------------------------------------------------------------- P7
def test_invariants_zero_gamma_scaling_permutation():
    inst = tiny(61, n_sub=3, n_cuts=6)
    P = O.build_problem(inst)
    rng = np.random.default_rng(61)
    a, b, gm = synth.random_duals(rng, inst, 0.7, 0.7)
    D = O.Duals(a, b, gm)
    g = O.evaluate(P, D)
    # a cut whose multiplier is 0 can be removed without any change
    k0 = 2
    D0 = D.copy()
    D0.gamma[:, k0] = 0.0
    g0 = O.evaluate(P, D0)
    c = inst.cuts
    keep = [k for k in range(c.n) if k != k0]
    ptr, lay, knd, idx, cf = [0], [], [], [], []
    for k in keep:
        e0, e1 = c.ptr[k], c.ptr[k + 1]
        lay += list(c.layer[e0:e1]); knd += list(c.kind[e0:e1]); idx += list(c.index[e0:e1]); cf += list(c.coef[e0:e1])
        ptr.append(len(lay))
    cuts2 = synth.Cuts(np.array(ptr, np.int64), np.array(lay, np.int16), np.array(knd, np.int8),
                       np.array(idx, np.int32), np.array(cf), c.d[keep])
    P2 = O.build_problem(dataclasses.replace(inst, cuts=cuts2))
    D2 = O.Duals(D0.alpha, D0.beta, D0.gamma[:, keep])
    np.testing.assert_allclose(O.evaluate(P2, D2), g0, rtol=0, atol=1e-13)
    # scaling a cut row by 4 and its multiplier by 1/4 leaves g unchanged
    k1 = 1
    cs = dataclasses.replace(c, coef=c.coef.copy(), d=c.d.copy())
    cs.coef[c.ptr[k1]:c.ptr[k1 + 1]] *= 4.0
    cs.d[k1] *= 4.0
    P3 = O.build_problem(dataclasses.replace(inst, cuts=cs))
    D3 = D.copy()
    D3.gamma[:, k1] /= 4.0
    np.testing.assert_allclose(O.evaluate(P3, D3), g, rtol=0, atol=1e-12)
    # permuting the cuts together with their multipliers leaves g unchanged
    perm = rng.permutation(c.n)
    ptr, lay, knd, idx, cf = [0], [], [], [], []
    for k in perm:
        e0, e1 = c.ptr[k], c.ptr[k + 1]
        lay += list(c.layer[e0:e1]); knd += list(c.kind[e0:e1]); idx += list(c.index[e0:e1]); cf += list(c.coef[e0:e1])
        ptr.append(len(lay))
    cp = synth.Cuts(np.array(ptr, np.int64), np.array(lay, np.int16), np.array(knd, np.int8),
                    np.array(idx, np.int32), np.array(cf), c.d[perm])
    P4 = O.build_problem(dataclasses.replace(inst, cuts=cp))
    D4 = O.Duals(D.alpha, D.beta, D.gamma[:, perm])
    np.testing.assert_allclose(O.evaluate(P4, D4), g, rtol=0, atol=1e-12)


def test_split_rows_equal_general_cut_rows():
    """beta-CROWN splits are GCP cuts with H_jj = +-1, d = 0 (Sec. 3.1)."""
    inst = tiny(71, n_sub=1, n_cuts=0, splits=(3, 3))
    P = O.build_problem(inst)
    rng = np.random.default_rng(71)
    D = O.default_duals(P)
    D.alpha = [rng.random(a.shape) for a in D.alpha]
    D.beta = rng.random(D.beta.shape)
    g = O.evaluate(P, D)
    sb = inst.sub
    n = sb.ptr[1]
    cuts = synth.Cuts(np.arange(n + 1, dtype=np.int64), sb.layer[:n].copy(), np.zeros(n, np.int8),
                      sb.index[:n].copy(), -sb.sign[:n].astype(np.float64), np.zeros(n))
    # the clamped bounds stay; the split multipliers move to gamma
    Pc = O.build_problem(dataclasses.replace(inst, cuts=cuts))
    Pc.split_ptr = np.zeros(2, np.int32)
    Pc.max_splits = 0
    Dc = O.Duals(D.alpha, np.zeros((P.R, 0)), D.beta.copy())
    np.testing.assert_allclose(O.evaluate(Pc, Dc), g, rtol=0, atol=1e-13)


# --------------------------------------------------------------------------- P8
def test_gradient_matches_central_differences():
    inst = tiny(81, n_sub=3, n_cuts=8, splits=(1, 2))
    P = O.build_problem(inst)
    rng = np.random.default_rng(81)
    a, b, gm = synth.random_duals(rng, inst, 0.5, 0.5)
    D = O.Duals(a, b, gm)
    g, G = O.gradient(P, D)
    h = 1e-6
    checked = 0

    def fd(setter):
        Dp, Dm, Dp2, Dm2 = D.copy(), D.copy(), D.copy(), D.copy()
        setter(Dp, h); setter(Dm, -h); setter(Dp2, h / 2); setter(Dm2, -h / 2)
        f1 = (O.evaluate(P, Dp) - O.evaluate(P, Dm)) / (2 * h)
        f2 = (O.evaluate(P, Dp2) - O.evaluate(P, Dm2)) / h
        return f1, f2
    for _ in range(12):
        li = int(rng.integers(0, P.L - 1))
        r, j = int(rng.integers(0, P.R)), int(rng.integers(0, P.dims[li + 1]))

        def sa(Dx, e, li=li, r=r, j=j):
            Dx.alpha[li][r, j] += e
        f1, f2 = fd(sa)
        if abs(f1[r] - f2[r]) < 1e-6:
            assert abs(f1[r] - G.alpha[li][r, j]) < 1e-5
            checked += 1
    for _ in range(12):
        r, k = int(rng.integers(0, P.R)), int(rng.integers(0, P.N))

        def sg(Dx, e, r=r, k=k):
            Dx.gamma[r, k] += e
        f1, f2 = fd(sg)
        if abs(f1[r] - f2[r]) < 1e-6:
            assert abs(f1[r] - G.gamma[r, k]) < 1e-5
            checked += 1
    for r in range(P.R):
        for m in range(P.max_splits):
            def sb(Dx, e, r=r, m=m):
                Dx.beta[r, m] += e
            f1, f2 = fd(sb)
            if abs(f1[r] - f2[r]) < 1e-6:
                assert abs(f1[r] - G.beta[r, m]) < 1e-5
                checked += 1
    assert checked >= 15


def test_conv_matrix_matches_direct_convolution():
    rng = np.random.default_rng(91)
    W = rng.normal(size=(4, 3, 3, 3))
    x = rng.normal(size=(2, 3, 9, 9))
    y = synth.conv2d_forward(x, W, 2, 1)
    M = O.conv_matrix(W, (3, 9, 9), (4, 5, 5), 2, 1)
    np.testing.assert_allclose((M @ x.reshape(2, -1).T).T, y.reshape(2, -1), atol=1e-12)


def test_planted_printed_sign_is_caught_by_lp_pin(monkeypatch):
    """Planting the printed pi* numerator (+beta^T Q) into the oracle breaks weak duality.

    One ReLU neuron, cut -z <= -0.5: the LP optimum stays -1, the corrected
    closed form gives g = -1 - gamma/2 and the printed one g = -1 + 1.5 gamma.
    """
    def printed(nu_hat, s, l, u, alpha):
        C = np.maximum(nu_hat, 0.0)
        pi = np.minimum(np.maximum((u * C + s) / (u - l), 0.0), C)
        h = np.where((l * C <= s) & (s <= u * C), l * pi, np.where(s >= u * C, 0.0, s))
        return pi, alpha * np.maximum(-nu_hat, 0.0), h
    inst = _one_neuron_instance()
    inst.cuts.coef[:] = -1.0
    inst.cuts.d[:] = -0.5
    P = O.build_problem(inst)
    lp = O.lp_value(P, 0, 0)
    assert abs(lp - (-1.0)) < 1e-9
    for gam in (0.25, 0.5, 1.0):
        D = O.Duals([np.array([[0.5]])], np.zeros((1, 0)), np.array([[gam]]))
        g = O.evaluate(P, D)
        assert abs(g[0] - (-1.0 - gam / 2)) < 1e-14 and g[0] <= lp
        monkeypatch.setattr(O, "unstable_closed_form", printed)
        gp = O.evaluate(P, D)
        monkeypatch.undo()
        assert abs(gp[0] - (-1.0 + 1.5 * gam)) < 1e-14 and gp[0] > lp
