"""Directly optimised ReLU duals (opt_pi: pi = theta * [nuhat]_+) against the oracle.

Tolerances as in the other parity tests: FP64 chain 1e-10 (trajectory, gradient),
FP32 chain 1e-5 at the same duals, certified 1e-9 against the oracle's float64
evaluation at the duals (alpha, beta, gamma, theta) the GPU holds.
"""
import numpy as np
import pytest

from oracle import gcp_oracle as O
from paper_2208_05740_gb300 import gcp, synth
from tests.helpers import assert_rel, join_alpha, oracle_duals, split_alpha

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from paper_2208_05740_gb300 import build
    build.build()
    c = gcp.Context(0)
    yield c
    c.close()


def _unstable_mask(P):
    """[R, sum d_i]: neurons unstable in their row's subdomain (theta matters only there)."""
    rs = O.row_sub(P)
    return np.concatenate([(lo[rs] < 0) & (hi[rs] > 0) for lo, hi in zip(P.sub_lo, P.sub_hi)], axis=1)


def _with_theta(inst, A, B, G, T):
    D = oracle_duals(inst, A, B, G)
    D.theta = split_alpha(inst, T)
    return D


@pytest.mark.parametrize("optimizer,iters", [(gcp.GCP_PGA, 5), (gcp.GCP_ADAM, 10)])
def test_fp64_trajectory_with_theta_matches_oracle(ctx, optimizer, iters):
    """From an imported theta: at the closed form itself every 'inside' neuron
    sits on the kink of h (u (C - pi*) + l pi* - s = 0), where rounding picks
    the side of the derivative, so trajectories started there are compared by
    their bounds only (next test)."""
    inst = synth.mlp_small(n_sub=4, n_cuts=8)
    P = O.build_problem(inst)
    net_id, cs = ctx.load_instance(inst)
    D = ctx.duals_create(net_id, cs, inst.sub, gcp.GCP_FP64)
    T0 = np.random.default_rng(8).uniform(0.05, 0.95, (D.rows, D.n_alpha))
    ctx.duals_theta(D, T0)
    p = gcp.opt_params(iters, optimizer, gcp.GCP_FP64, 1, 0.1, 0.05, 0.05, 0.95, opt_pi=1)
    bound, cert, _ = ctx.optimize_batch(D, p)
    D0 = O.default_duals(P)
    D0.theta = split_alpha(inst, T0)
    ref, Dr = O.optimize(P, D0, iters, 0.1, 0.05, 0.05, optimizer="pga" if optimizer == gcp.GCP_PGA else "adam",
                         lr_decay=0.95)
    assert_rel(bound, ref, 1e-10, "bound after the trajectory")
    assert_rel(cert, ref, 1e-9, "certified after the trajectory")
    A, B, G = ctx.duals_export(D)
    T = ctx.duals_theta(D)
    assert_rel(A, join_alpha(Dr.alpha), 1e-10, "alpha")
    assert_rel(G, Dr.gamma, 1e-10, "gamma")
    m = _unstable_mask(P)
    assert_rel(T[m], join_alpha(Dr.theta)[m], 1e-10, "theta on unstable neurons")
    assert np.all((T >= 0) & (T <= 1))
    ctx.duals_free(D)


def test_closed_form_start_never_lowers_the_bound(ctx):
    """Started at the closed form, the opt_pi ascent's certified bounds match
    the oracle at the reached duals, and the first evaluation equals the
    closed-form bound (theta = pi*/C reproduces it)."""
    inst = synth.mlp_small(n_sub=4, n_cuts=8)
    P = O.build_problem(inst)
    net_id, cs = ctx.load_instance(inst)
    D = ctx.duals_create(net_id, cs, inst.sub, gcp.GCP_FP64)
    b0, _, _ = ctx.optimize_batch(D, gcp.opt_params(0, gcp.GCP_PGA, gcp.GCP_FP64, 1, opt_pi=1))
    assert_rel(b0, O.evaluate(P, O.default_duals(P)), 1e-12, "closed-form start")
    ctx.duals_import(D)
    bound, cert, _ = ctx.optimize_batch(D, gcp.opt_params(20, gcp.GCP_ADAM, gcp.GCP_FP64, 1, 0.05, 0.05, 0.05,
                                                          opt_pi=1))
    A, B, G = ctx.duals_export(D)
    ref = O.evaluate(P, _with_theta(inst, A, B, G, ctx.duals_theta(D)))
    assert_rel(bound, ref, 1e-12, "bound at the reached duals")
    assert_rel(cert, ref, 1e-9, "certified at the reached duals")
    ctx.duals_free(D)


def test_fp64_bound_and_gradient_at_imported_theta(ctx):
    inst = synth.mlp_small(seed=synth.SEED_BASE + 12, n_sub=5, n_cuts=8)
    P = O.build_problem(inst)
    net_id, cs = ctx.load_instance(inst)
    D = ctx.duals_create(net_id, cs, inst.sub, gcp.GCP_FP64)
    rng = np.random.default_rng(3)
    a, b, g = synth.random_duals(rng, inst, 0.3, 0.3)
    ctx.duals_import(D, join_alpha(a), b, g)
    with pytest.raises(gcp.GCPError):
        ctx.duals_theta(D)                         # closed form: no theta yet
    T = rng.random((D.rows, D.n_alpha))
    ctx.duals_theta(D, T)
    Dr = _with_theta(inst, join_alpha(a), b, g, T)
    ref, RG = O.gradient(P, Dr)
    gb, ga, gbe, gg = ctx.grad_batch(D, gcp.GCP_FP64)
    assert_rel(gb, ref, 1e-12, "bound at theta")
    assert_rel(ga, join_alpha(RG.alpha), 1e-10, "dg/dalpha at theta")
    assert_rel(gbe, RG.beta, 1e-10, "dg/dbeta at theta")
    assert_rel(gg, RG.gamma, 1e-10, "dg/dgamma at theta")
    _, cert = ctx.bound_batch(D, gcp.GCP_FP64, certify=True)
    assert_rel(cert, ref, 1e-9, "certified at theta")
    # importing duals returns to the closed form
    ctx.duals_import(D, join_alpha(a), b, g)
    g0, _ = ctx.bound_batch(D, gcp.GCP_FP64)
    assert_rel(g0, O.evaluate(P, oracle_duals(inst, join_alpha(a), b, g)), 1e-12, "closed form again")
    ctx.duals_free(D)


@pytest.mark.parametrize("prec", [gcp.GCP_FP32, gcp.GCP_BF16])
def test_fp32_bf16_opt_pi_certifies_against_oracle(ctx, prec):
    # 40 subdomains x 9 rows: several tiles and a ragged tail on the tensor-core path
    inst = synth.mlp_256x6(n_sub=40, n_cuts=100)
    P = O.build_problem(inst)
    net_id, cs = ctx.load_instance(inst)
    D = ctx.duals_create(net_id, cs, inst.sub, gcp.GCP_FP32)
    p = gcp.opt_params(10, gcp.GCP_ADAM, prec, 1, 0.1, 0.02, 0.02, 0.98, opt_pi=1)
    bound, cert, _ = ctx.optimize_batch(D, p)
    A, B, G = ctx.duals_export(D)
    T = ctx.duals_theta(D)
    ref = O.evaluate(P, _with_theta(inst, A, B, G, T))
    assert_rel(cert, ref, 1e-9, "certified at the reached duals")
    assert_rel(bound, ref, 1e-5 if prec == gcp.GCP_FP32 else 1e-3, "chain bound at the reached duals")
    # the FP32 chain at the same duals through bound_batch (theta kept)
    g32, _ = ctx.bound_batch(D, gcp.GCP_FP32)
    assert_rel(g32, ref, 1e-5, "fp32 bound at theta")
    ctx.duals_free(D)


def test_opt_pi_on_a_residual_network(ctx):
    inst = synth.mlp_residual(seed=synth.SEED_BASE + 80, width=256, d0=784, blocks=2, d_out=10, eps=0.015,
                              n_spec=9, n_sub=24, n_cuts=60, max_splits=6)
    P = O.build_problem(inst)
    net_id, cs = ctx.load_instance(inst)
    D = ctx.duals_create(net_id, cs, inst.sub, gcp.GCP_FP32)
    bound, cert, _ = ctx.optimize_batch(D, gcp.opt_params(10, gcp.GCP_ADAM, gcp.GCP_FP32, 1, 0.1, 0.02, 0.02, 0.98,
                                                          opt_pi=1))
    A, B, G = ctx.duals_export(D)
    ref = O.evaluate(P, _with_theta(inst, A, B, G, ctx.duals_theta(D)))
    assert_rel(cert, ref, 1e-9, "residual certified with theta")
    assert_rel(bound, ref, 1e-5, "residual fp32 bound with theta")
    ctx.duals_free(D)


def test_zero_iterations_reproduce_the_closed_form(ctx):
    inst = synth.mlp_256x6(n_sub=12, n_cuts=50)
    net_id, cs = ctx.load_instance(inst)
    D = ctx.duals_create(net_id, cs, inst.sub, gcp.GCP_FP32)
    b0, c0, _ = ctx.optimize_batch(D, gcp.opt_params(0, gcp.GCP_ADAM, gcp.GCP_FP32, 1))
    b1, c1, _ = ctx.optimize_batch(D, gcp.opt_params(0, gcp.GCP_ADAM, gcp.GCP_FP32, 1, opt_pi=1))
    # theta = pi*/C is held in float32 (FP32 duals): pi = theta C moves by its
    # rounding (2^-24 relative), and so does the bound, certified or not
    assert_rel(b1, b0, 1e-6, "theta at the closed form: same chain bound")
    assert_rel(c1, c0, 1e-6, "theta at the closed form: same certified bound")
    T = ctx.duals_theta(D)
    assert np.all((T >= 0) & (T <= 1))
    ctx.duals_free(D)


def test_full_size_mlp_opt_pi_sampled_rows(ctx):
    """The benchmark's MLP at its full batch (1024 subdomains x 9 rows, 200
    cuts) with opt_pi in the FP32 chain, 20 Adam steps, FP64 certification;
    four sampled subdomains checked row by row against the oracle at the
    reached duals, theta included."""
    from tests.helpers import rows_of, select
    inst = synth.mlp_256x6()
    net_id, cs = ctx.load_instance(inst)
    D = ctx.duals_create(net_id, cs, inst.sub, gcp.GCP_FP32)
    bound, cert, _ = ctx.optimize_batch(D, gcp.opt_params(20, gcp.GCP_ADAM, gcp.GCP_FP32, 1, 0.1, 0.02, 0.02, 0.98,
                                                          opt_pi=1))
    A, B, G = ctx.duals_export(D)
    T = ctx.duals_theta(D)
    idx = [0, 1, 511, 1023]
    rows = rows_of(inst, idx)
    sub_inst = select(inst, idx)
    P = O.build_problem(sub_inst)
    Dr = oracle_duals(sub_inst, A[rows], B[rows][:, :P.max_splits], G[rows])
    Dr.theta = split_alpha(sub_inst, T[rows])
    ref = O.evaluate(P, Dr)
    assert_rel(bound[rows], ref, 1e-5, "sampled fp32 with theta")
    assert_rel(cert[rows], ref, 1e-9, "sampled certified with theta")
    assert np.all(np.isfinite(bound)) and np.all(np.isfinite(cert))
    ctx.duals_free(D)
