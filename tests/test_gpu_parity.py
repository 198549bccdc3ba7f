"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Tolerances (|gpu - oracle| <= tol * max(|oracle|, 1)):
  FP64 chain  1e-9  (same arithmetic, different summation order)
  FP32 chain  1e-5  at the same duals
  BF16 chain  1e-3  at the same duals (GEMM operands rounded to bfloat16)
  certified   1e-9  against the oracle's float64 evaluation at the GPU's duals
"""
import numpy as np
import pytest

from oracle import gcp_oracle as O
from paper_2208_05740_gb300 import gcp, synth
from tests.helpers import assert_rel, join_alpha, oracle_duals, rel_close, rows_of, select

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from paper_2208_05740_gb300 import build
    build.build()
    c = gcp.Context(0)
    yield c
    c.close()


def _rand_duals(inst, seed, scale=0.3):
    rng = np.random.default_rng(seed)
    a, b, g = synth.random_duals(rng, inst, scale, scale)
    return join_alpha(a), b, g


# ----------------------------------------------------------------------------- FP64, small MLP
def test_fp64_small_mlp_bound_gradient_and_trajectory(ctx):
    inst = synth.mlp_small()
    P = O.build_problem(inst)
    net_id, cs = ctx.load_instance(inst)
    D = ctx.duals_create(net_id, cs, inst.sub, gcp.GCP_FP64)
    g, _ = ctx.bound_batch(D, gcp.GCP_FP64)
    assert_rel(g, O.evaluate(P, O.default_duals(P)), 1e-12, "default duals")
    A, B, G = _rand_duals(inst, 3)
    ctx.duals_import(D, A, B, G)
    Dr = oracle_duals(inst, A, B, G)
    g, ga, gb, gg = ctx.grad_batch(D, gcp.GCP_FP64)
    ref, RG = O.gradient(P, Dr)
    assert_rel(g, ref, 1e-12, "bound at random duals")
    assert_rel(ga, join_alpha(RG.alpha), 1e-10, "dg/dalpha")
    assert_rel(gb, RG.beta, 1e-10, "dg/dbeta")
    assert_rel(gg, RG.gamma, 1e-10, "dg/dgamma")
    # 20 projected-gradient steps, lr 0.1, from the default duals. Each GPU step
    # is compared with one oracle step taken from the GPU's own duals, then the
    # whole trajectory with the oracle's own ascent.
    ctx.duals_import(D)
    p1 = gcp.opt_params(1, gcp.GCP_PGA, gcp.GCP_FP64, 1, 0.1, 0.1, 0.1)
    for t in range(20):
        A0, B0, G0 = ctx.duals_export(D)
        bound, cert, err = ctx.optimize_batch(D, p1)
        ref, Dref = O.optimize(P, oracle_duals(inst, A0, B0, G0), 1, 0.1, 0.1, 0.1)
        A1, B1, G1 = ctx.duals_export(D)
        assert_rel(A1, join_alpha(Dref.alpha), 1e-10, f"alpha after step {t}")
        assert_rel(B1, Dref.beta, 1e-10, f"beta after step {t}")
        assert_rel(G1, Dref.gamma, 1e-10, f"gamma after step {t}")
        assert_rel(bound, ref, 1e-10, f"bound after step {t}")
        assert_rel(cert, ref, 1e-9, f"certified after step {t}")
        assert np.all(cert <= bound + 1e-12 * np.maximum(1, np.abs(bound)))
        np.testing.assert_allclose(err, np.abs(bound - cert))
    traj, _ = O.optimize(P, O.default_duals(P), 20, 0.1, 0.1, 0.1)
    assert_rel(bound, traj, 1e-9, "20-step trajectory")
    ctx.duals_free(D)


def test_fp64_adam_with_decay_matches_oracle(ctx):
    inst = synth.mlp_small(seed=77)
    P = O.build_problem(inst)
    net_id, cs = ctx.load_instance(inst)
    D = ctx.duals_create(net_id, cs, inst.sub, gcp.GCP_FP64)
    bound, cert, _ = ctx.optimize_batch(D, gcp.opt_params(20, gcp.GCP_ADAM, gcp.GCP_FP64, 1, 0.1, 0.02, 0.02, 0.9))
    traj, _ = O.optimize(P, O.default_duals(P), 20, 0.1, 0.02, 0.02, optimizer="adam", lr_decay=0.9)
    assert_rel(bound, traj, 1e-9, "adam trajectory")
    A, B, G = ctx.duals_export(D)
    ref = O.evaluate(P, oracle_duals(inst, A, B, G))
    assert_rel(bound, ref, 1e-12, "adam bound at final duals")
    assert_rel(cert, ref, 1e-9, "adam certified")


# ----------------------------------------------------------------------------- FP32 / BF16 MLP
@pytest.fixture(scope="module")
def mlp_case(ctx):
    # 40 subdomains x 9 spec rows = 360 rows: several 128-row tiles and a ragged tail
    inst = synth.mlp_256x6(n_sub=40)
    P = O.build_problem(inst)
    net_id, cs = ctx.load_instance(inst)
    D = ctx.duals_create(net_id, cs, inst.sub, gcp.GCP_FP32)
    A, B, G = _rand_duals(inst, 5, 0.05)
    ctx.duals_import(D, A, B, G)
    A, B, G = ctx.duals_export(D)          # the float32 values the GPU holds
    return inst, P, D, (A, B, G)


def test_fp32_mlp_bound_and_certify_at_same_duals(ctx, mlp_case):
    inst, P, D, (A, B, G) = mlp_case
    ref = O.evaluate(P, oracle_duals(inst, A, B, G))
    g, cert = ctx.bound_batch(D, gcp.GCP_FP32, certify=True)
    assert_rel(g, ref, 1e-5, "fp32 bound")
    assert_rel(cert, ref, 1e-9, "certified")


def test_bf16_mlp_bound_at_same_duals(ctx, mlp_case):
    inst, P, D, (A, B, G) = mlp_case
    ref = O.evaluate(P, oracle_duals(inst, A, B, G))
    g, _ = ctx.bound_batch(D, gcp.GCP_BF16)
    assert_rel(g, ref, 1e-3, "bf16 bound")


def test_fp32_mlp_gradient(ctx, mlp_case):
    inst, P, D, (A, B, G) = mlp_case
    _, RG = O.gradient(P, oracle_duals(inst, A, B, G))
    g, ga, gb, gg = ctx.grad_batch(D, gcp.GCP_FP32)
    for got, ref, nm in ((ga, join_alpha(RG.alpha), "alpha"), (gb, RG.beta, "beta"), (gg, RG.gamma, "gamma")):
        scale = max(1.0, float(np.max(np.abs(ref))))
        assert np.max(np.abs(got - ref)) <= 1e-4 * scale, nm


def test_fp32_optimised_duals_certify_against_oracle(ctx, mlp_case):
    inst, P, D, _ = mlp_case
    ctx.duals_import(D)
    bound, cert, err = ctx.optimize_batch(D, gcp.opt_params(10, gcp.GCP_PGA, gcp.GCP_FP32, 1, 0.1, 0.01, 0.01))
    A, B, G = ctx.duals_export(D)
    ref = O.evaluate(P, oracle_duals(inst, A, B, G))
    assert_rel(bound, ref, 1e-5, "fp32 bound at final duals")
    assert_rel(cert, ref, 1e-9, "certified at final duals")
    assert np.all(A >= 0) and np.all(A <= 1) and np.all(B >= 0) and np.all(G >= 0)


# ----------------------------------------------------------------------------- CNN
@pytest.fixture(scope="module")
def cnn_case(ctx):
    inst = synth.cnn_cifar(n_sub=3, n_cuts=100)
    P = O.build_problem(inst)
    net_id, cs = ctx.load_instance(inst)
    D = ctx.duals_create(net_id, cs, inst.sub, gcp.GCP_FP32)
    A, B, G = _rand_duals(inst, 9, 0.05)
    ctx.duals_import(D, A, B, G)
    A, B, G = ctx.duals_export(D)
    return inst, P, D, (A, B, G)


def test_cnn_fp32_bf16_and_certify(ctx, cnn_case):
    inst, P, D, (A, B, G) = cnn_case
    ref = O.evaluate(P, oracle_duals(inst, A, B, G))
    g32, cert = ctx.bound_batch(D, gcp.GCP_FP32, certify=True)
    assert_rel(g32, ref, 1e-5, "cnn fp32")
    assert_rel(cert, ref, 1e-9, "cnn certified")
    g16, _ = ctx.bound_batch(D, gcp.GCP_BF16)
    assert_rel(g16, ref, 1e-3, "cnn bf16")


def test_cnn_fp32_gradient(ctx, cnn_case):
    inst, P, D, (A, B, G) = cnn_case
    _, RG = O.gradient(P, oracle_duals(inst, A, B, G))
    _, ga, gb, gg = ctx.grad_batch(D, gcp.GCP_FP32)
    for got, ref, nm in ((ga, join_alpha(RG.alpha), "alpha"), (gb, RG.beta, "beta"), (gg, RG.gamma, "gamma")):
        scale = max(1.0, float(np.max(np.abs(ref))))
        assert np.max(np.abs(got - ref)) <= 1e-4 * scale, nm


# ----------------------------------------------------------------------------- gradient check
def test_adjoint_vs_oracle_and_central_differences(ctx):
    """MLP 784-1024x4-10: adjoint vs the oracle gradient and central differences
    (h = 1e-4, float64) at 32 random coordinates."""
    q = synth.mlp_1024x4_queries(sizes=(2, 3, 2), cut_counts=(0, 50, 300))[2]
    P = O.build_problem(q)
    net_id, cs = ctx.load_instance(q)
    D = ctx.duals_create(net_id, cs, q.sub, gcp.GCP_FP64)
    A, B, G = _rand_duals(q, 13, 0.2)
    ctx.duals_import(D, A, B, G)
    g, ga, gb, gg = ctx.grad_batch(D, gcp.GCP_FP64)
    ref, RG = O.gradient(P, oracle_duals(q, A, B, G))
    assert_rel(g, ref, 1e-9, "bound")
    assert_rel(ga, join_alpha(RG.alpha), 1e-9, "alpha grad")
    assert_rel(gb, RG.beta, 1e-9, "beta grad")
    assert_rel(gg, RG.gamma, 1e-9, "gamma grad")
    rng = np.random.default_rng(17)
    h = 1e-4
    checked = 0
    groups = [("a", ga), ("b", gb), ("g", gg)]

    def bound_at(which, r, j, delta):
        AA, BB, GG = A.copy(), B.copy(), G.copy()
        {"a": AA, "b": BB, "g": GG}[which][r, j] += delta
        ctx.duals_import(D, AA, BB, GG)
        return ctx.bound_batch(D, gcp.GCP_FP64)[0][r]
    tries = 0
    while checked < 32 and tries < 400:
        tries += 1
        which, arr = groups[int(rng.integers(0, 3))]
        if arr.shape[1] == 0:
            continue
        r, j = int(rng.integers(0, arr.shape[0])), int(rng.integers(0, arr.shape[1]))
        if which == "a" and arr[r, j] == 0:
            continue     # stable neuron or nuhat >= 0: alpha has no effect
        f0 = bound_at(which, r, j, 0.0)
        fp, fm = bound_at(which, r, j, h), bound_at(which, r, j, -h)
        fp2, fm2 = bound_at(which, r, j, h / 2), bound_at(which, r, j, -h / 2)
        c1, c2 = (fp - fm) / (2 * h), (fp2 - fm2) / h
        fwd, bwd = (fp - f0) / h, (f0 - fm) / h
        tol = 1e-6 * max(1.0, abs(c1))
        if abs(fwd - bwd) > tol or abs(c1 - c2) > tol:
            continue     # a kink of the piecewise-linear bound inside the stencil
        assert abs(c1 - arr[r, j]) <= tol, (which, r, j, c1, arr[r, j])
        checked += 1
    assert checked == 32


# ----------------------------------------------------------------------------- edge cases
def test_empty_batch_and_no_cuts(ctx):
    inst = synth.mlp_small()
    net_id, _ = ctx.load_instance(inst)
    empty = synth.Subdomains(np.zeros(1, np.int32), np.zeros(0, np.int16), np.zeros(0, np.int32), np.zeros(0, np.int8))
    D = ctx.duals_create(net_id, -1, empty, gcp.GCP_FP32)
    assert D.rows == 0
    g, cert = ctx.bound_batch(D, gcp.GCP_FP32, certify=True)
    assert g.shape == (0,)
    b, c, e = ctx.optimize_batch(D, gcp.opt_params(3))
    assert b.shape == (0,)
    ctx.duals_free(D)
    # no cut set at all: plain beta-CROWN rows
    import dataclasses
    inst2 = dataclasses.replace(inst, cuts=synth.Cuts.empty())
    P = O.build_problem(inst2)
    D = ctx.duals_create(net_id, -1, inst.sub, gcp.GCP_FP64)
    g, cert = ctx.bound_batch(D, gcp.GCP_FP64, certify=True)
    ref = O.evaluate(P, O.default_duals(P))
    assert_rel(g, ref, 1e-12, "no cuts")
    assert_rel(cert, ref, 1e-9, "no cuts certified")


def test_all_stable_layers_and_max_splits(ctx):
    import dataclasses
    inst = synth.mlp_small(seed=5)
    # layer 1 all active, layer 2 all inactive (parity only needs consistent inputs)
    lo = [np.full(16, 0.1), -np.abs(inst.inter_lo[1]) - 1.0]
    hi = [0.1 + np.abs(inst.inter_hi[0]) + 1.0, np.full(16, -0.1)]
    inst2 = dataclasses.replace(inst, inter_lo=lo, inter_hi=hi)
    P = O.build_problem(inst2)
    with gcp.Context(0) as c2:
        net_id, cs = c2.load_instance(inst2)
        D = c2.duals_create(net_id, cs, inst2.sub, gcp.GCP_FP64)
        A, B, G = _rand_duals(inst2, 1)
        c2.duals_import(D, A, B, G)
        g, cert = c2.bound_batch(D, gcp.GCP_FP64, certify=True)
        ref = O.evaluate(P, oracle_duals(inst2, A, B, G))
        assert_rel(g, ref, 1e-12, "all stable")
        assert_rel(cert, ref, 1e-9, "all stable certified")
    # the largest split sets: every hidden neuron of a 2x16 net split in one subdomain
    rng = np.random.default_rng(2)
    inst3 = synth.mlp_small(seed=6)
    n = 32
    sub = synth.Subdomains(np.array([0, n], np.int32), np.array([1] * 16 + [2] * 16, np.int16),
                           np.array(list(range(16)) * 2, np.int32), rng.choice([-1, 1], n).astype(np.int8))
    inst3 = dataclasses.replace(inst3, sub=sub)
    P3 = O.build_problem(inst3)
    with gcp.Context(0) as c3:
        net_id, cs = c3.load_instance(inst3)
        D = c3.duals_create(net_id, cs, sub, gcp.GCP_FP64)
        A, B, G = _rand_duals(inst3, 4)
        c3.duals_import(D, A, B, G)
        g, ga, gb, gg = c3.grad_batch(D, gcp.GCP_FP64)
        ref, RG = O.gradient(P3, oracle_duals(inst3, A, B, G))
        assert_rel(g, ref, 1e-12, "max splits")
        assert_rel(gb, RG.beta, 1e-10, "max splits beta grad")


def test_invalid_arguments_are_rejected(ctx):
    inst = synth.mlp_small()
    net_id, cs = ctx.load_instance(inst)
    bad = synth.Subdomains(np.array([0, 2], np.int32), np.array([1, 1], np.int16), np.array([3, 3], np.int32),
                           np.array([1, -1], np.int8))
    with pytest.raises(gcp.GCPError) as e:
        ctx.duals_create(net_id, cs, bad, gcp.GCP_FP32)
    assert e.value.status == -1
    with pytest.raises(gcp.GCPError):
        ctx.add_cuts(net_id, [0, 1], [1], [2], [99], [1.0], [0.0])        # index out of range
    with pytest.raises(gcp.GCPError):
        ctx.add_cuts(net_id, [0, 1], [0], [2], [0], [1.0], [0.0])         # z on an input variable
    D = ctx.duals_create(net_id, cs, inst.sub, gcp.GCP_FP32)
    with pytest.raises(gcp.GCPError):
        ctx.bound_batch(D, gcp.GCP_FP64)                                  # FP64 chain on FP32 duals
    with gcp.Context(0, hbm_budget_bytes=1 << 16) as small:
        with pytest.raises(gcp.GCPError) as e:
            small.load_instance(synth.mlp_256x6(n_sub=1))
        assert e.value.status == -5


def test_cuts_are_append_only(ctx):
    inst = synth.mlp_small()
    P = O.build_problem(inst)
    net_id = ctx.init_net(inst.net.layers, inst.x_lo, inst.x_hi, inst.spec, inst.inter_lo, inst.inter_hi)
    c = inst.cuts
    h = 4
    cs, first = ctx.add_cuts(net_id, c.ptr[:h + 1], c.layer[:c.ptr[h]], c.kind[:c.ptr[h]], c.index[:c.ptr[h]],
                             c.coef[:c.ptr[h]], c.d[:h])
    assert first == 0
    p2 = c.ptr[h:] - c.ptr[h]
    cs2, first2 = ctx.add_cuts(net_id, p2, c.layer[c.ptr[h]:], c.kind[c.ptr[h]:], c.index[c.ptr[h]:],
                               c.coef[c.ptr[h]:], c.d[h:], cutset_id=cs)
    assert cs2 == cs and first2 == h
    D = ctx.duals_create(net_id, cs, inst.sub, gcp.GCP_FP64)
    A, B, G = _rand_duals(inst, 8)
    ctx.duals_import(D, A, B, G)
    g, _ = ctx.bound_batch(D, gcp.GCP_FP64)
    assert_rel(g, O.evaluate(P, oracle_duals(inst, A, B, G)), 1e-12, "appended cuts")


# ----------------------------------------------------------------------------- full size, sampled
def test_full_size_mlp_sampled_rows(ctx):
    """1024 subdomains x 9 rows, 200 cuts, FP32, certify: the launch shape of the
    benchmark; 6 sampled subdomains checked row by row against the oracle."""
    inst = synth.mlp_256x6()
    net_id, cs = ctx.load_instance(inst)
    D = ctx.duals_create(net_id, cs, inst.sub, gcp.GCP_FP32)
    bound, cert, err = ctx.optimize_batch(D, gcp.opt_params(20, gcp.GCP_PGA, gcp.GCP_FP32, 1, 0.1, 0.01, 0.01))
    A, B, G = ctx.duals_export(D)
    idx = [0, 1, 511, 777, 1022, 1023]
    rows = rows_of(inst, idx)
    sub_inst = select(inst, idx)
    P = O.build_problem(sub_inst)
    Bs = B[rows][:, :P.max_splits]
    ref = O.evaluate(P, oracle_duals(sub_inst, A[rows], Bs, G[rows]))
    assert_rel(bound[rows], ref, 1e-5, "sampled fp32")
    assert_rel(cert[rows], ref, 1e-9, "sampled certified")
    assert np.all(np.isfinite(bound)) and np.all(np.isfinite(cert))
    assert np.all(cert <= bound + 1e-5 * np.maximum(1, np.abs(bound)))


def test_full_size_cnn_sampled_rows(ctx):
    """CNN 3x32x32-c32-c64-fc512-fc10 at its full batch: 4096 subdomains x 9
    rows, 1000 cuts, BF16 ascent steps (tensor-core convolutions), then FP64
    certification; 4 sampled subdomains checked row by row against the oracle
    at the reached duals."""
    inst = synth.cnn_cifar()
    net_id, cs = ctx.load_instance(inst)
    D = ctx.duals_create(net_id, cs, inst.sub, gcp.GCP_FP32)
    bound, cert, _ = ctx.optimize_batch(D, gcp.opt_params(5, gcp.GCP_ADAM, gcp.GCP_BF16, 1, 0.1, 0.02, 0.02, 0.98))
    A, B, G = ctx.duals_export(D)
    idx = [0, 1, 2047, 4095]
    rows = rows_of(inst, idx)
    sub_inst = select(inst, idx)
    P = O.build_problem(sub_inst)
    ref = O.evaluate(P, oracle_duals(sub_inst, A[rows], B[rows][:, :P.max_splits], G[rows]))
    assert_rel(bound[rows], ref, 1e-3, "sampled bf16")
    assert_rel(cert[rows], ref, 1e-9, "sampled certified")
    assert np.all(np.isfinite(bound)) and np.all(np.isfinite(cert))
    ctx.duals_free(D)


def test_full_size_three_queries_sampled_rows(ctx):
    """MLP 784-1024x4-10, three queries of 64, 700 and 2048 subdomains with 0,
    500 and 3000 cuts in one batch (shared launches), FP32 ascent steps and
    FP64 certification; sampled subdomains of each query checked against the
    oracle at the reached duals."""
    qs = synth.mlp_1024x4_queries()
    q0 = qs[0]
    net_id = ctx.init_net(q0.net.layers, q0.x_lo, q0.x_hi, q0.spec, q0.inter_lo, q0.inter_hi)
    cs_ids = []
    for q in qs:
        c = q.cuts
        cs_ids.append(ctx.add_cuts(net_id, c.ptr, c.layer, c.kind, c.index, c.coef, c.d)[0] if c.n else -1)
    M = ctx.duals_create_multi(net_id, cs_ids, [q.sub for q in qs], gcp.GCP_FP32)
    assert M.rows == 9 * (64 + 700 + 2048) and M.n_cuts == 3500
    bound, cert, _ = ctx.optimize_batch(M, gcp.opt_params(5, gcp.GCP_ADAM, gcp.GCP_FP32, 1, 0.1, 0.02, 0.02, 0.98))
    A, B, G = ctx.duals_export(M)
    r0, c0 = 0, 0
    for q, idx in zip(qs, ([0, 63], [0, 350, 699], [0, 1024, 2047])):
        n = q.sub.n * 9
        Aq, Bq, Gq = A[r0:r0 + n], B[r0:r0 + n], G[r0:r0 + n, c0:c0 + q.cuts.n]
        mask = np.ones(M.n_cuts, bool)
        mask[c0:c0 + q.cuts.n] = False
        assert np.all(G[r0:r0 + n][:, mask] == 0)          # other queries' cuts stay at zero
        rows = rows_of(q, idx)
        sub_q = select(q, idx)
        P = O.build_problem(sub_q)
        ref = O.evaluate(P, oracle_duals(sub_q, Aq[rows], Bq[rows][:, :P.max_splits], Gq[rows]))
        assert_rel(bound[r0 + rows], ref, 1e-5, f"query of {q.sub.n}: sampled fp32")
        assert_rel(cert[r0 + rows], ref, 1e-9, f"query of {q.sub.n}: sampled certified")
        r0 += n
        c0 += q.cuts.n
    assert np.all(np.isfinite(bound)) and np.all(np.isfinite(cert))
    ctx.duals_free(M)


def test_certify_by_slices_matches_simt_float64(ctx):
    """The certification's dense products on the tensor cores (exact bf16
    slices) against the SIMT float64 products (GCP_TC=0): the two certified
    bounds differ only by their rounding-error terms, and both lie within
    1e-9 of the oracle at the same duals."""
    import os
    inst = synth.mlp_256x6(n_sub=40, n_cuts=60)
    P = O.build_problem(inst)
    net_id, cs = ctx.load_instance(inst)
    A, B, G = _rand_duals(inst, 23, 0.2)
    certs = []
    for tc in ("1", "0"):
        old = os.environ.get("GCP_TC")
        os.environ["GCP_TC"] = tc
        try:
            D = ctx.duals_create(net_id, cs, inst.sub, gcp.GCP_FP32)
        finally:
            if old is None:
                os.environ.pop("GCP_TC", None)
            else:
                os.environ["GCP_TC"] = old
        ctx.duals_import(D, A, B, G)
        _, cert = ctx.bound_batch(D, gcp.GCP_FP32, certify=True)
        certs.append(cert)
        Ae, Be, Ge = ctx.duals_export(D)
        assert_rel(cert, O.evaluate(P, oracle_duals(inst, Ae, Be, Ge)), 1e-9, f"certified (GCP_TC={tc})")
        ctx.duals_free(D)
    assert_rel(certs[0], certs[1], 1e-11, "slices vs SIMT float64")


def test_degenerate_box_gives_the_exact_output(ctx):
    """A zero-width input box (x_lo = x_hi = x0): the interval bounds are exact,
    no neuron is unstable, and the certified bound of every spec row equals
    c^T f(x0) (within the FP64 certification's rounding), in every chain."""
    inst = synth.mlp_256x6(n_sub=3, n_cuts=0)
    x0 = (inst.x_lo + inst.x_hi) / 2
    lo, hi = synth.interval_bounds(inst.net, x0, x0)
    sub = synth.Subdomains(np.arange(4, dtype=np.int32) * 0, np.zeros(0, np.int16), np.zeros(0, np.int32),
                           np.zeros(0, np.int8))
    net_id = ctx.init_net(inst.net.layers, x0, x0, inst.spec, lo, hi)
    exact = inst.spec @ synth.forward_all(inst.net, x0[None, :])[-1][0]
    for prec in (gcp.GCP_FP32, gcp.GCP_BF16):
        D = ctx.duals_create(net_id, -1, sub, gcp.GCP_FP32)
        g, cert = ctx.bound_batch(D, prec, certify=True)
        assert_rel(cert, np.tile(exact, 3), 1e-9, "certified at a point")
        ex = np.tile(exact, 3)
        assert np.all(cert <= ex + 1e-12 * np.maximum(1, np.abs(ex)))   # sound: never above
        ctx.duals_free(D)
