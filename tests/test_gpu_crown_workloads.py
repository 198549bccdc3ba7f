"""The measured workloads on CROWN root bounds (Sec. 2 takes l, u from a bound
propagation such as CROWN; App. C.1 uses alpha-CROWN).

The root bounds here come from the oracle alone (tests/helpers.py,
oracle_crown_bounds) and are fed to both sides. At the launch shapes the
benchmark times -- MLP 784-256x6-10 with 1024 subdomains x 9 rows and 200
cuts, 100 Adam steps in the FP32 chain; CNN 3x32x32 with 4096 subdomains x 9
rows and 1000 cuts, 50 Adam steps in the BF16 chain; the resnet2b-shaped residual CNN with
2048 subdomains x 9 rows and 500 cuts, 20 Adam steps in the BF16 chain -- sampled subdomains are
checked row by row against the oracle at the duals the GPU reached: the
chain's bound (FP32 1e-5, BF16 1e-3) and the certified FP64 bound (1e-9).
"""
import numpy as np
import pytest

from oracle import gcp_oracle as O
from paper_2208_05740_gb300 import gcp, synth
from tests.helpers import assert_rel, oracle_crown_bounds, oracle_duals, rows_of, select

pytestmark = pytest.mark.gpu

ADAM = dict(lr_alpha=0.1, lr_beta=0.02, lr_gamma=0.02, lr_decay=0.98)


@pytest.fixture(scope="module")
def ctx():
    from paper_2208_05740_gb300 import build
    build.build()
    c = gcp.Context(0)
    yield c
    c.close()


def _check_sampled(ctx, inst, D, bound, cert, idx, chain_tol, other_prec, other_tol):
    A, B, G = ctx.duals_export(D)
    rows = rows_of(inst, idx)
    sub_inst = select(inst, idx)
    P = O.build_problem(sub_inst)
    ref = O.evaluate(P, oracle_duals(sub_inst, A[rows], B[rows][:, :P.max_splits], G[rows]))
    assert_rel(bound[rows], ref, chain_tol, "sampled chain bound")
    assert_rel(cert[rows], ref, 1e-9, "sampled certified")
    assert np.all(np.isfinite(bound)) and np.all(np.isfinite(cert))
    # the other chain precision at the same duals
    b2, _ = ctx.bound_batch(D, other_prec, certify=False)
    assert_rel(b2[rows], ref, other_tol, "sampled bound, other chain precision")


def test_gpu_crown_root_bounds_equal_the_oracles_on_the_mlp(ctx):
    inst = synth.mlp_256x6(n_sub=1, n_cuts=0)
    lo, hi = ctx.intermediate_bounds(inst.net.layers, inst.x_lo, inst.x_hi)
    olo, ohi = oracle_crown_bounds(inst.net, inst.x_lo, inst.x_hi)
    for i, (a, b, c, d) in enumerate(zip(lo, hi, olo, ohi)):
        assert_rel(a, c, 1e-9, f"layer {i + 1} lower")
        assert_rel(b, d, 1e-9, f"layer {i + 1} upper")
        # certified: never tighter than the exact FP64 value by more than rounding
        assert np.all(a <= c + 1e-12 * np.maximum(1, np.abs(c))) and np.all(b >= d - 1e-12 * np.maximum(1, np.abs(d)))


def test_full_size_mlp_on_crown_root_bounds_sampled_rows(ctx):
    inst = synth.mlp_256x6(root_bounds=oracle_crown_bounds)
    net_id, cs = ctx.load_instance(inst)
    D = ctx.duals_create(net_id, cs, inst.sub, gcp.GCP_FP32)
    bound, cert, err = ctx.optimize_batch(D, gcp.opt_params(100, gcp.GCP_ADAM, gcp.GCP_FP32, 1, **ADAM))
    _check_sampled(ctx, inst, D, bound, cert, [0, 3, 400, 777, 1023], 1e-5, gcp.GCP_BF16, 1e-3)
    assert np.all(cert <= bound + 1e-5 * np.maximum(1, np.abs(bound)))
    ctx.duals_free(D)


def test_full_size_cnn_on_crown_root_bounds_sampled_rows(ctx):
    inst = synth.cnn_cifar(root_bounds=oracle_crown_bounds)
    net_id, cs = ctx.load_instance(inst)
    D = ctx.duals_create(net_id, cs, inst.sub, gcp.GCP_FP32)
    bound, cert, err = ctx.optimize_batch(D, gcp.opt_params(50, gcp.GCP_ADAM, gcp.GCP_BF16, 1, **ADAM))
    _check_sampled(ctx, inst, D, bound, cert, [0, 2047, 4095], 1e-3, gcp.GCP_FP32, 1e-5)
    ctx.duals_free(D)


def test_full_size_resnet_on_crown_root_bounds_sampled_rows(ctx):
    """The residual CNN (resnet2b shape) the benchmark's --workload resnet
    times: 2048 subdomains x 9 rows, 500 cuts, 20 Adam steps in the BF16 chain,
    on the oracle's CROWN root bounds through its skip connections."""
    inst = synth.cnn_resnet(root_bounds=oracle_crown_bounds)
    net_id, cs = ctx.load_instance(inst)
    D = ctx.duals_create(net_id, cs, inst.sub, gcp.GCP_FP32)
    bound, cert, err = ctx.optimize_batch(D, gcp.opt_params(20, gcp.GCP_ADAM, gcp.GCP_BF16, 1, **ADAM))
    _check_sampled(ctx, inst, D, bound, cert, [0, 1000, 2047], 1e-3, gcp.GCP_FP32, 1e-5)
    ctx.duals_free(D)
