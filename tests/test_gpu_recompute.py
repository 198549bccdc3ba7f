"""The adjoint with each layer's nuhat recomputed from the top instead of
stored by the evaluation (GCP_NUHAT=recompute; chosen by the memory budget
otherwise). The kernels and their order of operations are the same, so the
bound, its gradients and a whole ascent trajectory must come out bit-identical,
with less device memory held."""
import numpy as np
import pytest

from paper_2208_05740_gb300 import gcp, synth
from tests.helpers import join_alpha

pytestmark = pytest.mark.gpu


def _run(monkeypatch, mode, inst, prec, dual_prec):
    monkeypatch.setenv("GCP_NUHAT", mode)
    from paper_2208_05740_gb300 import build
    build.build()
    with gcp.Context(0) as ctx:
        net_id, cs = ctx.load_instance(inst)
        D = ctx.duals_create(net_id, cs, inst.sub, dual_prec)
        rng = np.random.default_rng(4)
        a, b, g = synth.random_duals(rng, inst, 0.1, 0.1)
        ctx.duals_import(D, join_alpha(a), b, g)
        used0 = ctx.mem_used()
        grads = ctx.grad_batch(D, prec)
        used1 = ctx.mem_used()
        ctx.duals_import(D)
        opt = ctx.optimize_batch(D, gcp.opt_params(8, gcp.GCP_ADAM, prec, 1, 0.1, 0.02, 0.02, 0.98))
        duals = ctx.duals_export(D)
        ctx.duals_free(D)
    return grads, opt, duals, used1 - used0


CASES = [
    ("mlp_fp64", lambda: synth.mlp_small(n_sub=5), gcp.GCP_FP64, gcp.GCP_FP64),
    ("mlp_fp32", lambda: synth.mlp_256x6(n_sub=40, n_cuts=60), gcp.GCP_FP32, gcp.GCP_FP32),
    ("mlp_bf16", lambda: synth.mlp_256x6(n_sub=40, n_cuts=60), gcp.GCP_BF16, gcp.GCP_FP32),
    ("cnn_bf16", lambda: synth.cnn_cifar(n_sub=3, n_cuts=60), gcp.GCP_BF16, gcp.GCP_FP32),
]


@pytest.mark.parametrize("name,make,prec,dual_prec", CASES, ids=[c[0] for c in CASES])
def test_recomputed_nuhat_gives_identical_gradients_and_trajectory(monkeypatch, name, make, prec, dual_prec):
    inst = make()
    g_s, o_s, d_s, mem_s = _run(monkeypatch, "store", inst, prec, dual_prec)
    g_r, o_r, d_r, mem_r = _run(monkeypatch, "recompute", inst, prec, dual_prec)
    for a, b in zip(g_s, g_r):
        np.testing.assert_array_equal(a, b)
    for a, b in zip(o_s, o_r):
        np.testing.assert_array_equal(a, b)
    for a, b in zip(d_s, d_r):
        np.testing.assert_array_equal(a, b)
    if name.startswith("mlp_fp32"):
        # six 256-wide hidden layers: the stored copies (R x 1536) against three
        # recompute buffers of the widest layer (R x 3 x 256)
        assert mem_r < mem_s


def test_budget_chooses_recompute_by_itself(monkeypatch):
    """With GCP_NUHAT unset and a budget that holds the three widest-layer
    buffers of the recomputing adjoint but not every layer's stored nuhat,
    the library recomputes on its own: no GCP_EBUDGET, and the gradients equal
    the stored run's bit for bit."""
    inst = synth.mlp_256x6(n_sub=40, n_cuts=60)
    g_s, _, _, mem_s = _run(monkeypatch, "store", inst, gcp.GCP_FP32, gcp.GCP_FP32)
    g_r, _, _, mem_r = _run(monkeypatch, "recompute", inst, gcp.GCP_FP32, gcp.GCP_FP32)
    monkeypatch.delenv("GCP_NUHAT", raising=False)
    with gcp.Context(0) as probe:
        net_id, cs = probe.load_instance(inst)
        D = probe.duals_create(net_id, cs, inst.sub, gcp.GCP_FP32)
        base = probe.mem_used()
        probe.duals_free(D)
    # everything the batch needs before the adjoint, plus the recomputing
    # adjoint's workspace and half of what storing would add on top of it
    budget = base + mem_r + (mem_s - mem_r) // 2
    with gcp.Context(0, hbm_budget_bytes=budget) as ctx:
        net_id, cs = ctx.load_instance(inst)
        D = ctx.duals_create(net_id, cs, inst.sub, gcp.GCP_FP32)
        rng = np.random.default_rng(4)
        a, b, g = synth.random_duals(rng, inst, 0.1, 0.1)
        ctx.duals_import(D, join_alpha(a), b, g)
        grads = ctx.grad_batch(D, gcp.GCP_FP32)      # raises on GCP_EBUDGET
        assert ctx.mem_used() <= budget
        ctx.duals_free(D)
    for x, y in zip(g_s, grads):
        np.testing.assert_array_equal(x, y)
