"""Launch accounting with repeated launches (gcp_profile_repeat): the
tensor-core GEMMs recompute their output from inputs they do not write, so
issuing each of their launches twice must leave every result bit-identical,
count each launch once, and cost extra device time."""
import numpy as np
import pytest

from paper_2208_05740_gb300 import gcp, synth

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("prec,name", [(gcp.GCP_FP32, "gemm_tc_tf32x3"), (gcp.GCP_BF16, "gemm_tc_bf16")])
def test_repeated_gemm_launches_change_nothing(prec, name):
    inst = synth.mlp_256x6(n_sub=64, n_cuts=40)
    p = gcp.opt_params(4, gcp.GCP_ADAM, prec, 1, 0.1, 0.02, 0.02, 0.98)
    with gcp.Context(0) as ctx:
        net_id, cs = ctx.load_instance(inst)
        D = ctx.duals_create(net_id, cs, inst.sub, gcp.GCP_FP32)
        runs = []
        for repeat in (None, name):
            ctx.duals_import(D)
            gcp.profile_start(None)
            if repeat:
                gcp.profile_repeat(repeat)
            b, c, _ = ctx.optimize_batch(D, p)
            n, _, _, _ = gcp.profile_query(name)
            gcp.profile_stop()
            runs.append((b, c, ctx.duals_export(D), n))
        (b0, c0, d0, n0), (b1, c1, d1, n1) = runs
        np.testing.assert_array_equal(b0, b1)
        np.testing.assert_array_equal(c0, c1)
        for x, y in zip(d0, d1):
            np.testing.assert_array_equal(x, y)
        assert n0 == n1 > 0
        ctx.duals_free(D)


def test_repeat_is_cleared_by_profile_stop():
    gcp.profile_start(None)
    gcp.profile_repeat("gemm_tc")
    gcp.profile_stop()
    inst = synth.mlp_256x6(n_sub=16, n_cuts=20)
    with gcp.Context(0) as ctx:
        net_id, cs = ctx.load_instance(inst)
        D = ctx.duals_create(net_id, cs, inst.sub, gcp.GCP_FP32)
        gcp.profile_start("gemm_tc_tf32x3")
        ctx.bound_batch(D, gcp.GCP_FP32)
        n, ms, _, _ = gcp.profile_query("gemm_tc_tf32x3")
        gcp.profile_stop()
        assert n > 0 and ms > 0
        ctx.duals_free(D)
