"""Residual networks (skip connections) through the C ABI against the oracle.

Tolerances as in the other parity tests: FP64 chain 1e-12 (bound) and 1e-10
(gradient), FP32 chain 1e-5, BF16 chain 1e-3 at the same duals, certified
1e-9 against the oracle's float64 evaluation at the duals the GPU holds.
"""
import dataclasses

import numpy as np
import pytest

from oracle import gcp_oracle as O
from paper_2208_05740_gb300 import gcp, synth
from tests.helpers import assert_rel, join_alpha, oracle_duals, rows_of, select

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from paper_2208_05740_gb300 import build
    build.build()
    c = gcp.Context(0)
    yield c
    c.close()


def _load(ctx, inst, seed, scale=0.05, fp64=False):
    net_id, cs = ctx.load_instance(inst)
    D = ctx.duals_create(net_id, cs, inst.sub, gcp.GCP_FP64 if fp64 else gcp.GCP_FP32)
    rng = np.random.default_rng(seed)
    a, b, g = synth.random_duals(rng, inst, scale, scale)
    ctx.duals_import(D, join_alpha(a), b, g)
    return D, ctx.duals_export(D)


def _net_with_skips(seed, dims, skips, name, n_sub=24, n_cuts=40, eps=0.02, projections=()):
    """MLP of the given widths; skips maps a 1-based layer to its skip s; the
    layers in projections add their source through a dense shortcut
    N(0, 1/(4 d_m)) instead of the identity."""
    rng = np.random.default_rng(seed)
    net = synth.make_mlp(rng, list(dims))
    for k, s in skips.items():
        ly = net.layers[k - 1]
        sc = None
        if k in projections:
            dm = dims[s - 1]
            sc = synth.Layer(synth.DENSE, rng.normal(0, 0.5 / np.sqrt(dm), (ly.d_out, dm)), np.zeros(ly.d_out),
                             (dm,), (ly.d_out,))
        net.layers[k - 1] = dataclasses.replace(ly, W=0.5 * ly.W, skip=s, shortcut=sc)
    return synth._finish(name, rng, net, rng.random(dims[0]), eps, 4, n_sub, (0, 4),
                         dict(n_cuts=n_cuts, min_vars=2, max_vars=6, span_layers=True, need_z=True, p_input=0.5))


def _cases():
    # several 128-row tiles and a ragged tail (24 x 4 = 96 rows, 40 x 9 = 360 rows), widths on the tensor cores
    yield "blocks", synth.mlp_residual(seed=synth.SEED_BASE + 80, width=256, d0=784, blocks=2, d_out=10, eps=0.015,
                                       n_spec=9, n_sub=40, n_cuts=60, max_splits=6)
    yield "input_and_spec_layer", _net_with_skips(synth.SEED_BASE + 81, [256, 256, 256, 256, 256], {1: 1, 4: 3},
                                                  "skips_io")
    yield "own_input_of_last", _net_with_skips(synth.SEED_BASE + 82, [128, 256, 256, 256], {2: 2, 3: 3}, "skips_self")
    yield "three_back", _net_with_skips(synth.SEED_BASE + 83, [300, 256, 256, 256, 256, 10], {4: 2}, "skips_far")
    # dense projections: from the layer's own input, from the input two layers back, into the spec layer
    yield "projections", _net_with_skips(synth.SEED_BASE + 84, [200, 256, 192, 256, 10], {2: 2, 3: 1, 4: 3},
                                         "proj", projections=(2, 3, 4))
    yield "projection_into_last", _net_with_skips(synth.SEED_BASE + 85, [128, 256, 128, 10], {3: 3}, "proj_last",
                                                  projections=(3,))


CASES = list(_cases())


@pytest.mark.parametrize("name,inst", CASES, ids=[c[0] for c in CASES])
def test_residual_fp32_bf16_and_certified_at_same_duals(ctx, name, inst):
    P = O.build_problem(inst)
    assert any(P.skip)
    D, (A, B, G) = _load(ctx, inst, 5)
    ref = O.evaluate(P, oracle_duals(inst, A, B, G))
    g, cert = ctx.bound_batch(D, gcp.GCP_FP32, certify=True)
    assert_rel(g, ref, 1e-5, f"{name} fp32 bound")
    assert_rel(cert, ref, 1e-9, f"{name} certified")
    g16, _ = ctx.bound_batch(D, gcp.GCP_BF16)
    assert_rel(g16, ref, 1e-3, f"{name} bf16 bound")
    _, RG = O.gradient(P, oracle_duals(inst, A, B, G))
    _, ga, gb, gg = ctx.grad_batch(D, gcp.GCP_FP32)
    for got, want, nm in ((ga, join_alpha(RG.alpha), "alpha"), (gb, RG.beta, "beta"), (gg, RG.gamma, "gamma")):
        scale = max(1.0, float(np.max(np.abs(want)))) if want.size else 1.0
        assert np.max(np.abs(got - want), initial=0.0) <= 1e-4 * scale, (name, nm)
    ctx.duals_free(D)


FP64_CASES = [c for c in CASES if c[0] in ("blocks", "input_and_spec_layer", "projections")]


@pytest.mark.parametrize("name,inst", FP64_CASES, ids=[c[0] for c in FP64_CASES])
def test_residual_fp64_chain_bound_and_gradient(ctx, name, inst):
    P = O.build_problem(inst)
    D, (A, B, G) = _load(ctx, inst, 6, fp64=True)
    ref, RG = O.gradient(P, oracle_duals(inst, A, B, G))
    g, ga, gb, gg = ctx.grad_batch(D, gcp.GCP_FP64)
    assert_rel(g, ref, 1e-12, "fp64 bound")
    assert_rel(ga, join_alpha(RG.alpha), 1e-10, "dg/dalpha")
    assert_rel(gb, RG.beta, 1e-10, "dg/dbeta")
    assert_rel(gg, RG.gamma, 1e-10, "dg/dgamma")
    _, cert = ctx.bound_batch(D, gcp.GCP_FP64, certify=True)
    assert_rel(cert, ref, 1e-9, "certified (fp64 duals)")
    ctx.duals_free(D)


def test_residual_optimisation_improves_and_certifies(ctx):
    inst = CASES[0][1]
    P = O.build_problem(inst)
    net_id, cs = ctx.load_instance(inst)
    D = ctx.duals_create(net_id, cs, inst.sub, gcp.GCP_FP32)
    g0, _ = ctx.bound_batch(D, gcp.GCP_FP32)
    for prec in (gcp.GCP_FP32, gcp.GCP_BF16):
        ctx.duals_import(D)
        bound, cert, _ = ctx.optimize_batch(D, gcp.opt_params(20, gcp.GCP_ADAM, prec, 1, 0.1, 0.02, 0.02, 0.9))
        A, B, G = ctx.duals_export(D)
        ref = O.evaluate(P, oracle_duals(inst, A, B, G))
        assert_rel(cert, ref, 1e-9, "certified after ascent")
        assert np.mean(cert) > np.mean(g0)
    ctx.duals_free(D)


# ----------------------------------------------------------------------------- residual CNN
RESNETS = {
    # resnet2b's block structure at 16 x 16: a 1x1 stride-2 convolution shortcut, then an identity block
    "resnet2b_16": dict(hw=16, stem=8, blocks=((16, 2), (16, 1)), fc=64),
    # resnet4b's: both blocks downsample through projections
    "resnet4b_16": dict(hw=16, stem=8, blocks=((16, 2), (16, 2)), fc=64),
}


@pytest.fixture(scope="module", params=list(RESNETS))
def resnet_case(ctx, request):
    inst = synth.cnn_resnet(n_sub=3, n_cuts=60, **RESNETS[request.param])
    assert any(ly.shortcut is not None for ly in inst.net.layers)
    P = O.build_problem(inst)
    D, duals = _load(ctx, inst, 9)
    return inst, P, D, duals


def test_resnet_fp32_bf16_and_certify(ctx, resnet_case):
    inst, P, D, (A, B, G) = resnet_case
    ref = O.evaluate(P, oracle_duals(inst, A, B, G))
    g, cert = ctx.bound_batch(D, gcp.GCP_FP32, certify=True)
    assert_rel(g, ref, 1e-5, "resnet fp32")
    assert_rel(cert, ref, 1e-9, "resnet certified")
    g16, _ = ctx.bound_batch(D, gcp.GCP_BF16)
    assert_rel(g16, ref, 1e-3, "resnet bf16")


def test_resnet_gradient(ctx, resnet_case):
    inst, P, D, (A, B, G) = resnet_case
    _, RG = O.gradient(P, oracle_duals(inst, A, B, G))
    _, ga, gb, gg = ctx.grad_batch(D, gcp.GCP_FP32)
    for got, want, nm in ((ga, join_alpha(RG.alpha), "alpha"), (gb, RG.beta, "beta"), (gg, RG.gamma, "gamma")):
        scale = max(1.0, float(np.max(np.abs(want)))) if want.size else 1.0
        assert np.max(np.abs(got - want), initial=0.0) <= 1e-4 * scale, nm


# ----------------------------------------------------------------------------- root bounds
def _oracle_rows(inst, lo, hi, i, idx):
    """The oracle's bound of +-x^(i)_j (j in idx) on the network truncated after layer i."""
    ly = inst.net.layers[i - 1]
    n = ly.d_out
    spec = np.zeros((2 * len(idx), n))
    spec[np.arange(len(idx)), idx] = 1.0
    spec[len(idx) + np.arange(len(idx)), idx] = -1.0
    net = synth.Network(inst.net.layers[:i])
    sub = synth.Subdomains(np.zeros(2, np.int32), np.zeros(0, np.int16), np.zeros(0, np.int32), np.zeros(0, np.int8))
    tr = synth.Instance("prefix", net, inst.x_lo, inst.x_hi, spec, lo[:i - 1], hi[:i - 1], sub, synth.Cuts.empty())
    P = O.build_problem(tr)
    g = O.evaluate(P, O.default_duals(P))
    return g[:len(idx)], -g[len(idx):]


@pytest.mark.parametrize("make", [lambda: CASES[1][1], lambda: dict(CASES)["projections"],
                                  lambda: synth.cnn_resnet(n_sub=1, n_cuts=0, **RESNETS["resnet2b_16"]),
                                  lambda: synth.cnn_resnet(n_sub=1, n_cuts=0, **RESNETS["resnet4b_16"])],
                         ids=["mlp_input_and_spec_skips", "mlp_projections", "resnet2b_16", "resnet4b_16"])
def test_root_bounds_of_residual_networks(ctx, make):
    inst = make()
    lo, hi = ctx.intermediate_bounds(inst.net.layers, inst.x_lo, inst.x_hi)
    rng = np.random.default_rng(0)
    X = synth.sample_box(rng, inst.x_lo, inst.x_hi, 2000)
    pre = synth.forward_all(inst.net, X)[:-1]
    for i, (p, l, h) in enumerate(zip(pre, lo, hi)):
        assert np.all(p >= l[None, :]) and np.all(p <= h[None, :]), f"layer {i + 1} not sound"
    for i in range(2, inst.net.L):
        idx = rng.choice(len(lo[i - 1]), size=min(6, len(lo[i - 1])), replace=False)
        olo, ohi = _oracle_rows(inst, lo, hi, i, idx)
        assert_rel(lo[i - 1][idx], olo, 1e-9, f"layer {i} lower vs oracle")
        assert_rel(hi[i - 1][idx], ohi, 1e-9, f"layer {i} upper vs oracle")
    # tighter than the interval bounds the generator uses
    ilo, ihi = synth.interval_bounds(inst.net, inst.x_lo, inst.x_hi)
    assert sum(float(np.sum(h - l)) for l, h in zip(lo, hi)) < sum(float(np.sum(h - l)) for l, h in zip(ilo, ihi))


def test_bad_skips_are_rejected(ctx):
    inst = CASES[0][1]
    layers = list(inst.net.layers)
    bad_width = layers[:]
    bad_width[1] = dataclasses.replace(layers[1], skip=1)            # xhat^(0) has 784 entries, layer 2 has 256
    shared = layers[:]
    shared[3] = dataclasses.replace(layers[3], skip=2)               # xhat^(1) already feeds layer 3
    later = layers[:]
    later[1] = dataclasses.replace(layers[1], skip=3)                # not an earlier layer
    wrong_proj = layers[:]
    wrong_proj[2] = dataclasses.replace(layers[2], shortcut=synth.Layer(synth.DENSE, np.ones((256, 100)), np.zeros(256),
                                                                        (100,), (256,)))   # xhat^(1) has 256 entries
    for net in (bad_width, shared, later, wrong_proj):
        with pytest.raises(gcp.GCPError) as e:
            ctx.init_net(net, inst.x_lo, inst.x_hi, inst.spec, inst.inter_lo, inst.inter_hi)
        assert e.value.status == -1          # GCP_EINVAL
    biased = layers[:]
    biased[2] = dataclasses.replace(layers[2], shortcut=synth.Layer(synth.DENSE, np.eye(256), np.ones(256),
                                                                    (256,), (256,)))
    with pytest.raises(ValueError):
        ctx.init_net(biased, inst.x_lo, inst.x_hi, inst.spec, inst.inter_lo, inst.inter_hi)


def test_full_size_resnet_sampled_rows(ctx):
    """The residual CNN (resnet2b shape) at the bench's size: 2048 subdomains x
    9 rows, 500 cuts, BF16 ascent steps (tensor-core convolutions, a 1x1 stride-2
    projection shortcut and an identity block), FP64 certification; 4 sampled
    subdomains checked row by row against the oracle at the reached duals."""
    inst = synth.cnn_resnet()
    net_id, cs = ctx.load_instance(inst)
    D = ctx.duals_create(net_id, cs, inst.sub, gcp.GCP_FP32)
    bound, cert, _ = ctx.optimize_batch(D, gcp.opt_params(5, gcp.GCP_ADAM, gcp.GCP_BF16, 1, 0.1, 0.02, 0.02, 0.98))
    A, B, G = ctx.duals_export(D)
    idx = [0, 1, 1023, 2047]
    rows = rows_of(inst, idx)
    sub_inst = select(inst, idx)
    P = O.build_problem(sub_inst)
    ref = O.evaluate(P, oracle_duals(sub_inst, A[rows], B[rows][:, :P.max_splits], G[rows]))
    assert_rel(bound[rows], ref, 1e-3, "sampled bf16")
    assert_rel(cert[rows], ref, 1e-9, "sampled certified")
    assert np.all(np.isfinite(bound)) and np.all(np.isfinite(cert))
    ctx.duals_free(D)


def test_serving_a_residual_network_alone_and_in_a_mix():
    """The serving loop on residual networks (the resnet2b-shaped CNN with its
    projection shortcut and a residual MLP with opt_pi): each request's result
    is the same alone and in a mix with another network's request."""
    rn = synth.cnn_resnet(hw=16, stem=8, blocks=((16, 2), (16, 1)), fc=64, n_sub=6, n_cuts=40)
    mlp = CASES[0][1]
    p = gcp.opt_params(10, gcp.GCP_ADAM, gcp.GCP_BF16, 1, 0.1, 0.02, 0.02, 0.98)
    q = gcp.opt_params(10, gcp.GCP_ADAM, gcp.GCP_BF16, 1, 0.1, 0.02, 0.02, 0.98, opt_pi=1)
    with gcp.Context(0) as c:
        nr, cr = c.load_instance(rn)
        nm, cm = c.load_instance(mlp)
        c.serve_start(8)
        r1, alone_r = c.serve_wait(c.serve_submit(nr, cr, rn.sub, p, 3, 11), rn.n_rows + 64)
        r2, alone_m = c.serve_wait(c.serve_submit(nm, cm, mlp.sub, q, 3, 12), mlp.n_rows + 64)
        t1 = c.serve_submit(nr, cr, rn.sub, p, 3, 11)
        t2 = c.serve_submit(nm, cm, mlp.sub, q, 3, 12)
        s1, mixed_r = c.serve_wait(t1, rn.n_rows + 64)
        s2, mixed_m = c.serve_wait(t2, mlp.n_rows + 64)
        c.serve_stop()
    for r in (r1, r2, s1, s2):
        assert r.status == 0
    assert_rel(mixed_r[:r1.rows], alone_r[:r1.rows], 1e-9, "resnet alone vs mixed")
    assert_rel(mixed_m[:r2.rows], alone_m[:r2.rows], 1e-9, "residual MLP (opt_pi) alone vs mixed")
    assert np.all(np.isfinite(alone_r[:r1.rows])) and np.all(np.isfinite(alone_m[:r2.rows]))
