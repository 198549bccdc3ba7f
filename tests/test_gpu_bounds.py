"""Root intermediate bounds by the library's own bound propagation
(gcp_intermediate_bounds): hidden layer 1 by interval arithmetic, every later
hidden layer by bounding the truncated network with spec rows +e_j / -e_j
(CROWN at the default slopes, alpha-CROWN with ascent steps), certified.

Checked against the FP64 oracle on the same truncated networks, for soundness
on sampled inputs, and for tightness against interval bound propagation.
"""
import numpy as np
import pytest

from oracle import gcp_oracle as O
from paper_2208_05740_gb300 import gcp, synth
from tests.helpers import assert_rel

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from paper_2208_05740_gb300 import build
    build.build()
    c = gcp.Context(0)
    yield c
    c.close()


def _rows(ly, idx):
    """Rows idx of a layer's linear map as dense [len(idx), d_in] (convolutions materialised)."""
    if ly.kind == synth.DENSE:
        return ly.W[idx]
    E = np.eye(ly.d_in)
    return synth.layer_apply(ly, E).T[idx]


def _oracle_layer(inst, lo, hi, i, idx):
    """The oracle's bound of +-x^(i)_j on the network truncated after layer i."""
    ly = inst.net.layers[i - 1]
    Wr = _rows(ly, idx)
    last = synth.Layer(synth.DENSE, Wr, ly.b[idx], ly.in_shape, (len(idx),))
    net = synth.Network(inst.net.layers[:i - 1] + [last])
    spec = np.concatenate([np.eye(len(idx)), -np.eye(len(idx))])
    sub = synth.Subdomains(np.zeros(2, np.int32), np.zeros(0, np.int16), np.zeros(0, np.int32), np.zeros(0, np.int8))
    tr = synth.Instance("prefix", net, inst.x_lo, inst.x_hi, spec, lo[:i - 1], hi[:i - 1], sub, synth.Cuts.empty())
    P = O.build_problem(tr)
    g = O.evaluate(P, O.default_duals(P))
    return g[:len(idx)], -g[len(idx):]


def _sampled_preacts(inst, n, seed):
    rng = np.random.default_rng(seed)
    X = synth.sample_box(rng, inst.x_lo, inst.x_hi, n)
    return synth.forward_all(inst.net, X)[:-1]


@pytest.mark.parametrize("make", [synth.mlp_small, lambda: synth.mlp_256x6(n_sub=1, n_cuts=0)],
                         ids=["mlp_8_16_16_3", "mlp_784_256x6_10"])
def test_crown_bounds_match_oracle_and_are_sound(ctx, make):
    inst = make()
    lo, hi = ctx.intermediate_bounds(inst.net.layers, inst.x_lo, inst.x_hi)
    # hidden layer 1: the exact interval image of the box (outward rounded)
    ly = inst.net.layers[0]
    c0, r0 = (inst.x_hi + inst.x_lo) / 2, (inst.x_hi - inst.x_lo) / 2
    z = ly.W @ c0 + ly.b
    rad = np.abs(ly.W) @ r0
    assert_rel(lo[0], z - rad, 1e-12, "layer 1 lower")
    assert_rel(hi[0], z + rad, 1e-12, "layer 1 upper")
    assert np.all(lo[0] <= z - rad + 1e-12 * np.maximum(1, np.abs(z))) and np.all(hi[0] >= z + rad - 1e-12 * np.maximum(1, np.abs(z)))
    # later layers: the certified bound of the truncated network, as the oracle evaluates it
    rng = np.random.default_rng(3)
    for i in range(2, inst.net.L):
        d = inst.net.dims[i]
        idx = np.sort(rng.choice(d, size=min(d, 24), replace=False))
        olo, ohi = _oracle_layer(inst, lo, hi, i, idx)
        assert_rel(lo[i - 1][idx], olo, 1e-9, f"layer {i} lower vs oracle")
        assert_rel(hi[i - 1][idx], ohi, 1e-9, f"layer {i} upper vs oracle")
    # sound: every sampled input's pre-activations lie inside
    for i, z in enumerate(_sampled_preacts(inst, 2000, 5)):
        assert np.all(z >= lo[i] - 1e-9 * np.maximum(1, np.abs(z))), f"layer {i + 1} below the lower bound"
        assert np.all(z <= hi[i] + 1e-9 * np.maximum(1, np.abs(z))), f"layer {i + 1} above the upper bound"
    # and no wider than interval bound propagation in total (each layer)
    ilo, ihi = synth.interval_bounds(inst.net, inst.x_lo, inst.x_hi)
    for i in range(len(lo)):
        assert np.sum(hi[i] - lo[i]) <= np.sum(ihi[i] - ilo[i]) * (1 + 1e-9), f"layer {i + 1} wider than IBP"


def test_alpha_crown_bounds_are_sound_and_tighter(ctx):
    inst = synth.mlp_256x6(n_sub=1, n_cuts=0)
    lo, hi = ctx.intermediate_bounds(inst.net.layers, inst.x_lo, inst.x_hi)
    p = gcp.opt_params(20, gcp.GCP_ADAM, gcp.GCP_FP32, 1, 0.1, 0.02, 0.02, 0.98)
    alo, ahi = ctx.intermediate_bounds(inst.net.layers, inst.x_lo, inst.x_hi, p)
    for i, z in enumerate(_sampled_preacts(inst, 2000, 7)):
        assert np.all(z >= alo[i] - 1e-9 * np.maximum(1, np.abs(z))) and np.all(z <= ahi[i] + 1e-9 * np.maximum(1, np.abs(z)))
    np.testing.assert_array_equal(alo[0], lo[0])   # layer 1 is exact either way
    for i in range(1, len(lo)):
        assert np.sum(ahi[i] - alo[i]) < np.sum(hi[i] - lo[i]), f"layer {i + 1}: ascent did not tighten"


def test_cnn_bounds_sound_and_match_oracle_on_the_fc_layer(ctx):
    inst = synth.cnn_cifar(n_sub=1, n_cuts=0)
    lo, hi = ctx.intermediate_bounds(inst.net.layers, inst.x_lo, inst.x_hi)
    assert [len(a) for a in lo] == inst.net.dims[1:-1]
    for i, z in enumerate(_sampled_preacts(inst, 300, 9)):
        assert np.all(z >= lo[i] - 1e-9 * np.maximum(1, np.abs(z))) and np.all(z <= hi[i] + 1e-9 * np.maximum(1, np.abs(z)))
    idx = np.arange(0, 512, 37)
    olo, ohi = _oracle_layer(inst, lo, hi, 3, idx)
    assert_rel(lo[2][idx], olo, 1e-9, "fc layer lower vs oracle")
    assert_rel(hi[2][idx], ohi, 1e-9, "fc layer upper vs oracle")


def test_bounds_feed_a_network_and_tighten_its_certified_bound(ctx):
    """The MLP workload's subdomains bounded with GPU CROWN root bounds instead
    of interval bounds: certified bounds (the oracle's evaluation at the
    reached duals) are higher."""
    inst = synth.mlp_256x6(n_sub=8, n_cuts=20)
    lo, hi = ctx.intermediate_bounds(inst.net.layers, inst.x_lo, inst.x_hi)
    p = gcp.opt_params(10, gcp.GCP_ADAM, gcp.GCP_FP32, 1, 0.1, 0.02, 0.02, 0.98)
    certs = []
    for ilo, ihi in ((inst.inter_lo, inst.inter_hi), (lo, hi)):
        tr = synth.Instance(inst.name, inst.net, inst.x_lo, inst.x_hi, inst.spec, ilo, ihi, inst.sub, inst.cuts)
        net_id, cs = ctx.load_instance(tr)
        D = ctx.duals_create(net_id, cs, tr.sub, gcp.GCP_FP32)
        _, cert, _ = ctx.optimize_batch(D, p)
        A, B, G = ctx.duals_export(D)
        from tests.helpers import oracle_duals
        assert_rel(cert, O.evaluate(O.build_problem(tr), oracle_duals(tr, A, B, G)), 1e-9, "certified vs oracle")
        certs.append(cert)
        ctx.duals_free(D)
    assert np.mean(certs[1]) > np.mean(certs[0])


def _net_with_valid_cuts(seed=synth.SEED_BASE + 90):
    """MLP 8-16-16-16-3 with 24 random cuts over the input and hidden layers,
    offsets d set to each cut's maximum over the root MIP (valid for every
    input of the box)."""
    rng = np.random.default_rng(seed)
    net = synth.make_mlp(rng, [8, 16, 16, 16, 3])
    inst = synth._finish("mlp_cuts", rng, net, rng.random(8), 0.15, 2, 1, (0, 0),
                         dict(n_cuts=24, min_vars=2, max_vars=4, p_input=0.5))
    P = O.build_problem(inst)
    d = O.valid_cut_offsets(P)
    import dataclasses
    return dataclasses.replace(inst, cuts=dataclasses.replace(inst.cuts, d=d))


def test_bounds_with_valid_cuts_are_sound_and_reduce_to_crown(ctx):
    """Each layer's bounds take the cuts over the layers below it: with
    gamma = 0 (no ascent) the result is the cut-free CROWN; with ascent the
    bounds stay sound for sampled inputs (the cuts hold for all of them) and
    are at least as tight as alpha-CROWN's without cuts, up to the ascent's
    noise."""
    inst = _net_with_valid_cuts()
    c = inst.cuts
    tops = [int(np.max(c.layer[c.ptr[k]:c.ptr[k + 1]])) for k in range(c.n)]
    assert min(tops) <= 2 < inst.net.L      # some cut is usable below the last hidden layer
    lo0, hi0 = ctx.intermediate_bounds(inst.net.layers, inst.x_lo, inst.x_hi)
    loc, hic = ctx.intermediate_bounds(inst.net.layers, inst.x_lo, inst.x_hi, cuts=c)
    for a, b in zip(lo0 + hi0, loc + hic):
        np.testing.assert_array_equal(a, b)
    p = gcp.opt_params(40, gcp.GCP_ADAM, gcp.GCP_FP32, 1, 0.1, 0.1, 0.1, 1.0)
    la, ha = ctx.intermediate_bounds(inst.net.layers, inst.x_lo, inst.x_hi, p)
    lc, hc = ctx.intermediate_bounds(inst.net.layers, inst.x_lo, inst.x_hi, p, cuts=c)
    pre = _sampled_preacts(inst, 20000, 90)
    for i, (x, l, h) in enumerate(zip(pre, lc, hc)):
        assert np.all(x >= l[None, :]) and np.all(x <= h[None, :]), f"layer {i + 1} not sound with cuts"
    wa = sum(float(np.sum(h - l)) for l, h in zip(la, ha))
    wc = sum(float(np.sum(h - l)) for l, h in zip(lc, hc))
    assert wc <= wa * (1 + 1e-3), (wc, wa)


@pytest.mark.parametrize("make", [lambda: synth.mlp_residual(n_sub=1, n_cuts=0),
                                  lambda: synth.cnn_resnet(n_sub=1, n_cuts=0)],
                         ids=["mlp_residual", "resnet2b_shape"])
def test_residual_crown_bounds_match_the_oracle(ctx, make):
    """Skip connections (identity and 1x1 projection shortcuts) in the root
    bounds: every hidden layer's certified CROWN bounds against the oracle's
    CROWN (its truncated networks keep the skip, restricted to the bounded
    rows), and sound on sampled inputs."""
    inst = make()
    lo, hi = ctx.intermediate_bounds(inst.net.layers, inst.x_lo, inst.x_hi)
    olo, ohi = O.crown_root_bounds(inst.net, inst.x_lo, inst.x_hi)
    for i, (a, b, c, d) in enumerate(zip(lo, hi, olo, ohi)):
        assert_rel(a, c, 1e-9, f"layer {i + 1} lower vs oracle")
        assert_rel(b, d, 1e-9, f"layer {i + 1} upper vs oracle")
    for i, z in enumerate(_sampled_preacts(inst, 2000, 7)):
        assert np.all(z >= lo[i] - 1e-9 * np.maximum(1, np.abs(z))), f"layer {i + 1} below the lower bound"
        assert np.all(z <= hi[i] + 1e-9 * np.maximum(1, np.abs(z))), f"layer {i + 1} above the upper bound"
