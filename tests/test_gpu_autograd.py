"""The adjoint behind torch.autograd: gcp_bound_device / gcp_grad_device.

The forward of the autograd function is the bound of every row at the duals
given as CUDA tensors (export layouts); its backward runs the hand-written
adjoint. Checked against the C-ABI host entry points and the FP64 oracle's
gradient (reverse mode of Theorem 3.1), with a weighted sum of the rows as
the loss so that grad_out reaches the adjoint as a per-row seed.
"""
import numpy as np
import pytest

from oracle import gcp_oracle as O
from paper_2208_05740_gb300 import gcp, synth
from tests.helpers import assert_rel, join_alpha, oracle_duals

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def ctx():
    from paper_2208_05740_gb300 import build
    build.build()
    c = gcp.Context(0)
    yield c
    c.close()


@pytest.mark.parametrize("make", [lambda: synth.mlp_256x6(n_sub=5, n_cuts=40),
                                  lambda: synth.cnn_cifar(n_sub=2, n_cuts=30)], ids=["mlp", "cnn"])
def test_autograd_forward_backward(ctx, make):
    inst = make()
    net_id, cs = ctx.load_instance(inst)
    D = ctx.duals_create(net_id, cs, inst.sub, gcp.GCP_FP32)
    rng = np.random.default_rng(12)
    a, b, g = synth.random_duals(rng, inst, 0.05, 0.05)
    ctx.duals_import(D, join_alpha(a), b, g)
    A, B, G = ctx.duals_export(D)
    host_bound, _ = ctx.bound_batch(D, gcp.GCP_FP32)

    dev = torch.device("cuda:0")
    ta = torch.tensor(A, dtype=torch.float32, device=dev, requires_grad=True)
    tb = torch.tensor(B, dtype=torch.float32, device=dev, requires_grad=True)
    tg = torch.tensor(G, dtype=torch.float32, device=dev, requires_grad=True)
    fn = gcp.make_bound_function()
    out = fn.apply(ta, tb, tg, ctx, D, gcp.GCP_FP32)
    got = out.detach().cpu().numpy().astype(np.float64)
    assert_rel(got, host_bound, 1e-6, "autograd forward vs gcp_bound_batch")

    P = O.build_problem(inst)
    ref, RG = O.gradient(P, oracle_duals(inst, A, B, G))
    assert_rel(got, ref, 1e-5, "autograd forward vs oracle")

    w = rng.normal(size=D.rows)
    (out * torch.tensor(w, dtype=torch.float32, device=dev)).sum().backward()
    ga = ta.grad.cpu().numpy()
    gb = tb.grad.cpu().numpy()
    gg = tg.grad.cpu().numpy()
    # each row's bound depends on its own duals only: d(sum_r w_r g_r)/d(duals of r) = w_r dg_r
    for got_g, ref_g, nm in ((ga, join_alpha(RG.alpha), "alpha"), (gb, RG.beta, "beta"), (gg, RG.gamma, "gamma")):
        ref_w = w[:, None] * ref_g[:, :got_g.shape[1]]
        scale = max(1.0, float(np.max(np.abs(ref_w))))
        assert np.max(np.abs(got_g - ref_w)) <= 1e-4 * scale, f"autograd backward {nm} vs oracle"
    # and against the host gradient entry point
    _, ha, hb, hg = ctx.grad_batch(D, gcp.GCP_FP32)
    for got_g, h, nm in ((ga, ha, "alpha"), (gb, hb, "beta"), (gg, hg, "gamma")):
        hw = w[:, None] * h
        scale = max(1.0, float(np.max(np.abs(hw))))
        assert np.max(np.abs(got_g - hw)) <= 1e-5 * scale, f"autograd backward {nm} vs gcp_grad_batch"
    ctx.duals_free(D)


def test_autograd_ascent_step_raises_the_bound(ctx):
    """A small step along the gradient of the summed bound, computed through
    torch, raises the summed bound (first-order ascent; every coordinate moves
    by at most 1e-4 of its gradient scale)."""
    inst = synth.mlp_256x6(n_sub=3, n_cuts=20)
    net_id, cs = ctx.load_instance(inst)
    D = ctx.duals_create(net_id, cs, inst.sub, gcp.GCP_FP32)
    A, B, G = ctx.duals_export(D)
    dev = torch.device("cuda:0")
    ta = torch.tensor(A, dtype=torch.float32, device=dev, requires_grad=True)
    tb = torch.tensor(B, dtype=torch.float32, device=dev, requires_grad=True)
    tg = torch.tensor(G, dtype=torch.float32, device=dev, requires_grad=True)
    fn = gcp.make_bound_function()
    g0 = fn.apply(ta, tb, tg, ctx, D, gcp.GCP_FP32)
    g0.sum().backward()
    with torch.no_grad():
        scale = max(float(t.grad.abs().max()) for t in (ta, tb, tg) if t.grad.numel())
        lr = 1e-4 / scale
        na = (ta + lr * ta.grad).clamp(0.0, 1.0)
        nb = (tb + lr * tb.grad).clamp(min=0.0)
        ng = (tg + lr * tg.grad).clamp(min=0.0)
        g1 = fn.apply(na, nb, ng, ctx, D, gcp.GCP_FP32)
    assert float(g1.double().sum()) > float(g0.detach().double().sum())
    ctx.duals_free(D)


@pytest.mark.parametrize("prec", [gcp.GCP_FP32, gcp.GCP_BF16], ids=["fp32", "bf16"])
def test_bound_and_gradient_calls_leave_the_duals_unchanged(ctx, prec):
    """Evaluations and gradients read the duals; only ascent steps may change
    them (regression: the tail threads of the gather's last block once
    stepped beta during a gradient call)."""
    inst = synth.mlp_256x6(n_sub=7, n_cuts=33)
    net_id, cs = ctx.load_instance(inst)
    D = ctx.duals_create(net_id, cs, inst.sub, gcp.GCP_FP32)
    rng = np.random.default_rng(3)
    a, b, g = synth.random_duals(rng, inst, 0.1, 0.1)
    ctx.duals_import(D, join_alpha(a), b, g)
    before = ctx.duals_export(D)
    ctx.bound_batch(D, prec, certify=True)
    ctx.grad_batch(D, prec)
    _, ga, gb, gg = ctx.grad_batch(D, prec)
    after = ctx.duals_export(D)
    for x, y, nm in zip(before, after, ("alpha", "beta", "gamma")):
        np.testing.assert_array_equal(x, y, err_msg=f"{nm} changed by a bound or gradient call")
    ctx.duals_free(D)
