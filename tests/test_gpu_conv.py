"""Tensor-core implicit-GEMM convolution of the BF16 chain.

The BF16 chain runs both convolution directions on the tensor cores (the
backward step y = W^T nu as a transposed convolution of three-term bf16
operands, the reverse-mode step W a as a convolution). Without the tensor
cores the backward step runs in float on the SIMT units and the reverse-mode
step on the same bf16 operands. Here the two are compared with the FP64
oracle (the tensor-core chain at the bf16 tolerance, the float one at the
fp32 tolerance) and with each other, on the CIFAR-shaped CNN (tiles that
straddle rows, a ragged last tile) and on a CNN with odd shapes: 5 input
channels (padded to 8 in the GEMM's K), 7x9 maps, a stride-2 padded and a
stride-1 unpadded convolution, 12 and 20 channels; and on kernels 5 and 4 with
strides 3 and 2 (nine and four phases of the transposed convolution). The
same three networks run through the FP32 chain, whose convolutions are all
float SIMT kernels, against the oracle.
"""
import math
import os

import numpy as np
import pytest

from oracle import gcp_oracle as O
from paper_2208_05740_gb300 import gcp, synth
from tests.helpers import assert_rel, join_alpha, oracle_duals

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from paper_2208_05740_gb300 import build
    build.build()
    c = gcp.Context(0)
    yield c
    c.close()


def _odd_cnn():
    rng = np.random.default_rng(synth.SEED_BASE + 31)
    c1 = synth.make_conv(rng, (5, 9, 7), 12, 3, 2, 1)       # -> 12 x 5 x 4
    c2 = synth.make_conv(rng, c1.out_shape, 20, 3, 1, 0)    # -> 20 x 3 x 2
    d2 = c2.d_out
    W3 = rng.normal(0.0, math.sqrt(1.0 / d2), size=(16, d2))
    b3 = rng.normal(0.0, math.sqrt(0.1), size=16)
    W4 = rng.normal(0.0, math.sqrt(1.0 / 16), size=(3, 16))
    b4 = rng.normal(0.0, math.sqrt(0.1), size=3)
    net = synth.Network([c1, c2, synth.Layer(synth.DENSE, W3, b3, (d2,), (16,)),
                         synth.Layer(synth.DENSE, W4, b4, (16,), (3,))])
    x0 = rng.random(c1.d_in)
    return synth._finish("cnn_odd", rng, net, x0, 0.05, 2, 23, (0, 3),
                         dict(n_cuts=30, min_vars=2, max_vars=6, span_layers=True, need_z=True, p_input=0.5))


def _odd_cnn2():
    """Kernel 5 stride 3 pad 2, then kernel 4 stride 2 pad 1 (nine and four
    phases in the transposed direction)."""
    rng = np.random.default_rng(synth.SEED_BASE + 32)
    c1 = synth.make_conv(rng, (3, 11, 10), 5, 5, 3, 2)      # -> 5 x 4 x 4
    c2 = synth.make_conv(rng, c1.out_shape, 8, 4, 2, 1)     # -> 8 x 2 x 2
    d2 = c2.d_out
    W3 = rng.normal(0.0, math.sqrt(1.0 / d2), size=(12, d2))
    b3 = rng.normal(0.0, math.sqrt(0.1), size=12)
    W4 = rng.normal(0.0, math.sqrt(1.0 / 12), size=(2, 12))
    b4 = rng.normal(0.0, math.sqrt(0.1), size=2)
    net = synth.Network([c1, c2, synth.Layer(synth.DENSE, W3, b3, (d2,), (12,)),
                         synth.Layer(synth.DENSE, W4, b4, (12,), (2,))])
    x0 = rng.random(c1.d_in)
    return synth._finish("cnn_odd2", rng, net, x0, 0.05, 2, 41, (0, 2),
                         dict(n_cuts=20, min_vars=2, max_vars=5, span_layers=True, need_z=True, p_input=0.5))


CASES = {
    "cifar": lambda: synth.cnn_cifar(n_sub=7, n_cuts=60),
    "odd": _odd_cnn,
    "odd2": _odd_cnn2,
}


def _batch(ctx, net_id, cs, inst, tc: bool):
    old = os.environ.get("GCP_TC")
    if not tc:
        os.environ["GCP_TC"] = "0"
    try:
        return ctx.duals_create(net_id, cs, inst.sub, gcp.GCP_FP32)
    finally:
        if old is None:
            os.environ.pop("GCP_TC", None)
        else:
            os.environ["GCP_TC"] = old


@pytest.mark.parametrize("case", sorted(CASES))
def test_conv_tc_matches_simt_and_oracle(ctx, case):
    inst = CASES[case]()
    net_id, cs = ctx.load_instance(inst)
    Dt = _batch(ctx, net_id, cs, inst, True)
    Ds = _batch(ctx, net_id, cs, inst, False)
    rng = np.random.default_rng(5)
    a, b, g = synth.random_duals(rng, inst, 0.05, 0.05)
    for D in (Dt, Ds):
        ctx.duals_import(D, join_alpha(a), b, g)
    A, B, G = ctx.duals_export(Dt)
    ref = O.evaluate(O.build_problem(inst), oracle_duals(inst, A, B, G))
    gt, _ = ctx.bound_batch(Dt, gcp.GCP_BF16)
    gs, _ = ctx.bound_batch(Ds, gcp.GCP_BF16)
    assert_rel(gt, ref, 1e-3, f"{case}: bf16 chain (three-term tensor-core products) vs oracle")
    assert_rel(gs, ref, 1e-5, f"{case}: bf16 chain without tensor cores (float products) vs oracle")
    assert_rel(gt, gs, 1e-4, f"{case}: tensor-core vs SIMT convolution")
    # reverse mode: the forward convolution on the tensor cores. The reverse
    # pass rounds each layer's operand a to bf16, so a last-bit difference of
    # the fp32 sums upstream can flip one rounding (a 2^-8 relative change of
    # that operand): the two chains agree to the bf16 tolerance, not tighter.
    _, at, bt, ct = ctx.grad_batch(Dt, gcp.GCP_BF16)
    _, as_, bs, cs_ = ctx.grad_batch(Ds, gcp.GCP_BF16)
    for x, y, nm in ((at, as_, "alpha"), (bt, bs, "beta"), (ct, cs_, "gamma")):
        scale = max(1.0, float(np.max(np.abs(y))))
        assert np.max(np.abs(x - y)) <= 1e-3 * scale, f"{case}: gradient {nm}, tensor-core vs SIMT"
    # (The BF16 gradient is not compared with the FP64 oracle element by
    # element: the local derivatives switch case at kinks of Lemma A.1, and a
    # bf16-propagated nuhat can sit on the other side of a kink than the
    # float64 one, so single entries jump. The bound is the BF16 contract;
    # the FP32 chain's gradient is pinned to the oracle in the parity tests.)
    for D in (Dt, Ds):
        ctx.duals_free(D)


def test_conv_tc_optimisation_certifies_like_simt(ctx):
    """A few BF16 Adam steps with each convolution, then FP64 certification:
    both trajectories stay within the bf16 tolerance of each other and the
    certified values match the oracle at the reached duals."""
    inst = synth.cnn_cifar(n_sub=5, n_cuts=40)
    net_id, cs = ctx.load_instance(inst)
    P = O.build_problem(inst)
    p = gcp.opt_params(5, gcp.GCP_ADAM, gcp.GCP_BF16, 1, 0.1, 0.02, 0.02, 0.98)
    out = []
    for tc in (True, False):
        D = _batch(ctx, net_id, cs, inst, tc)
        bound, cert, _ = ctx.optimize_batch(D, p)
        A, B, G = ctx.duals_export(D)
        assert_rel(cert, O.evaluate(P, oracle_duals(inst, A, B, G)), 1e-9, f"certified (tc={tc})")
        out.append(cert)
        ctx.duals_free(D)
    assert_rel(out[0], out[1], 1e-3, "certified after bf16 steps, tensor-core vs SIMT")


@pytest.mark.parametrize("case", sorted(CASES))
def test_fp32_chain_convolutions_match_oracle(ctx, case):
    """The FP32 chain runs both convolution directions in float on the SIMT
    units: row-staged kernels with two or four output pixels per work item
    (chosen per layer from its item count), channel tiles fastest across
    lanes, and the tap loops unrolled at compile time for 3x3 kernels (the
    cifar and odd cases) but not for 5x5 and 4x4 (odd2). The bound and the
    certified bound at the same duals match the oracle (1e-5, 1e-9), and so
    does the gradient, which runs the forward convolution in the adjoint."""
    inst = CASES[case]()
    net_id, cs = ctx.load_instance(inst)
    D = ctx.duals_create(net_id, cs, inst.sub, gcp.GCP_FP32)
    rng = np.random.default_rng(7)
    a, b, g = synth.random_duals(rng, inst, 0.05, 0.05)
    ctx.duals_import(D, join_alpha(a), b, g)
    A, B, G = ctx.duals_export(D)
    P = O.build_problem(inst)
    od = oracle_duals(inst, A, B, G)
    ref = O.evaluate(P, od)
    g32, cert = ctx.bound_batch(D, gcp.GCP_FP32, certify=True)
    assert_rel(g32, ref, 1e-5, f"{case}: fp32 chain vs oracle")
    assert_rel(cert, ref, 1e-9, f"{case}: certified vs oracle")
    _, RG = O.gradient(P, od)
    _, ga, gb, gg = ctx.grad_batch(D, gcp.GCP_FP32)
    for got, want, nm in ((ga, join_alpha(RG.alpha), "alpha"), (gb, RG.beta, "beta"), (gg, RG.gamma, "gamma")):
        scale = max(1.0, float(np.max(np.abs(want))))
        assert np.max(np.abs(got - want)) <= 1e-4 * scale, f"{case}: gradient {nm}"
    ctx.duals_free(D)
