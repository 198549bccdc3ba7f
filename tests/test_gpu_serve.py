"""Uneven batching (several queries in one launch) and the serving loop."""
import dataclasses
import time

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


def _queries():
    return synth.mlp_1024x4_queries(sizes=(2, 3, 4), cut_counts=(0, 40, 120))


def test_three_queries_in_one_batch_match_separate_batches(ctx):
    """Queries of 2, 3 and 4 subdomains with 0, 40 and 120 cuts in one batch."""
    qs = _queries()
    net_id = ctx.init_net(qs[0].net.layers, qs[0].x_lo, qs[0].x_hi, qs[0].spec, qs[0].inter_lo, qs[0].inter_hi)
    cs_ids = []
    for q in qs:
        c = q.cuts
        cs_ids.append(ctx.add_cuts(net_id, c.ptr, c.layer, c.kind, c.index, c.coef, c.d)[0] if c.n else -1)
    rng = np.random.default_rng(4)
    sep, duals = [], []
    for q, cs in zip(qs, cs_ids):
        D = ctx.duals_create(net_id, cs, q.sub, gcp.GCP_FP32)
        a, b, g = synth.random_duals(rng, q, 0.2, 0.2)
        ctx.duals_import(D, join_alpha(a), b, g)
        duals.append(ctx.duals_export(D))
        sep.append((D, ctx.bound_batch(D, gcp.GCP_FP32, certify=True)))
    M = ctx.duals_create_multi(net_id, cs_ids, [q.sub for q in qs], gcp.GCP_FP32)
    assert M.rows == sum(d.rows for d, _ in sep) and M.n_cuts == sum(q.cuts.n for q in qs)
    A = np.concatenate([d[0] for d in duals])
    B = np.zeros((M.rows, M.max_splits))
    G = np.zeros((M.rows, M.n_cuts))
    r0, c0 = 0, 0
    for (a, b, g), q in zip(duals, qs):
        B[r0:r0 + a.shape[0], :b.shape[1]] = b
        G[r0:r0 + a.shape[0], c0:c0 + g.shape[1]] = g
        r0 += a.shape[0]
        c0 += q.cuts.n
    ctx.duals_import(M, A, B, G)
    bm, cm = ctx.bound_batch(M, gcp.GCP_FP32, certify=True)
    r0 = 0
    for (D, (b1, c1)) in sep:
        assert_rel(bm[r0:r0 + D.rows], b1, 1e-6, "fp32 bound in the mix")
        assert_rel(cm[r0:r0 + D.rows], c1, 1e-12, "certified in the mix")
        r0 += D.rows
    # optimise the mix and each query alone: duals and bounds agree
    p = gcp.opt_params(5, gcp.GCP_ADAM, gcp.GCP_FP32, 1, 0.1, 0.02, 0.02, 0.98)
    bm, cm, _ = ctx.optimize_batch(M, p)
    Am, Bm, Gm = ctx.duals_export(M)
    r0, c0 = 0, 0
    for (D, _), q in zip(sep, qs):
        b1, c1, _ = ctx.optimize_batch(D, p)
        a1, bb1, g1 = ctx.duals_export(D)
        np.testing.assert_array_equal(Am[r0:r0 + D.rows], a1)
        np.testing.assert_array_equal(Gm[r0:r0 + D.rows, c0:c0 + q.cuts.n], g1)
        mask = np.ones(M.n_cuts, bool)
        mask[c0:c0 + q.cuts.n] = False
        assert np.all(Gm[r0:r0 + D.rows][:, mask] == 0)        # other queries' cuts untouched
        assert_rel(bm[r0:r0 + D.rows], b1, 1e-6, "optimised bound in the mix")
        assert_rel(cm[r0:r0 + D.rows], c1, 1e-12, "optimised certified in the mix")
        r0 += D.rows
        c0 += q.cuts.n
    # and the mix agrees with the oracle at its duals, query by query
    r0, c0 = 0, 0
    for (D, _), q in zip(sep, qs):
        P = O.build_problem(q)
        ref = O.evaluate(P, oracle_duals(q, Am[r0:r0 + D.rows], Bm[r0:r0 + D.rows, :P.max_splits],
                                         Gm[r0:r0 + D.rows, c0:c0 + q.cuts.n]))
        assert_rel(cm[r0:r0 + D.rows], ref, 1e-9, "mix certified vs oracle")
        r0 += D.rows
        c0 += q.cuts.n


def _submit(ctx, net_id, cs, sub, rounds, seed, iters=10):
    p = gcp.opt_params(iters, gcp.GCP_ADAM, gcp.GCP_BF16, 1, 0.1, 0.02, 0.02, 0.98)
    return ctx.serve_submit(net_id, cs, sub, p, rounds, seed)


def test_serving_result_is_the_same_alone_and_in_the_mix():
    a = synth.mlp_small(n_sub=6)
    b = synth.mlp_small(seed=synth.SEED_BASE + 11, n_sub=5)
    c = synth.mlp_256x6(n_sub=12, n_cuts=30)
    with gcp.Context(0) as ctx:
        na, csa = ctx.load_instance(a)
        cb = b.cuts                      # a second cut set on the same network
        csb, _ = ctx.add_cuts(na, cb.ptr, cb.layer, cb.kind, cb.index, cb.coef, cb.d)
        nc, csc = ctx.load_instance(c)
        ctx.serve_start(8)
        t = _submit(ctx, na, csa, a.sub, 3, 99)
        res, alone = ctx.serve_wait(t, a.n_rows + 64)
        assert res.status == 0 and res.rows == a.n_rows and res.latency_ms > 0
        # the same request again, now in a mix: another query on the same network
        # (shared launches), a query on another network (concurrent stream)
        t1 = _submit(ctx, na, csa, a.sub, 3, 99)
        t2 = _submit(ctx, na, csb, b.sub, 2, 7)
        t3 = _submit(ctx, nc, csc, c.sub, 3, 5)
        r1, mixed = ctx.serve_wait(t1, a.n_rows + 64)
        r2, out2 = ctx.serve_wait(t2, b.n_rows + 64)
        r3, out3 = ctx.serve_wait(t3, c.n_rows + 64)
        ctx.serve_stop()
    assert r1.status == 0 and r2.status == 0 and r3.status == 0
    assert_rel(mixed, alone, 1e-9, "same request alone and in the mix")
    assert np.all(np.isfinite(out2)) and np.all(np.isfinite(out3))
    assert r3.rows == c.n_rows and r3.max_err_vs_fp64 >= 0


def test_serving_admits_by_memory_budget_and_rejects_oversize():
    a = synth.mlp_256x6(n_sub=30, n_cuts=20)
    with gcp.Context(0, hbm_budget_bytes=256 << 20) as ctx:
        na, csa = ctx.load_instance(a)
        ctx.serve_start(4)
        tickets = [_submit(ctx, na, csa, a.sub, 2, s) for s in range(3)]
        for t in tickets:
            res, out = ctx.serve_wait(t, a.n_rows + 16)
            assert res.status == 0 and res.rows == a.n_rows and np.all(np.isfinite(out))
        big = synth.mlp_256x6(n_sub=1024, n_cuts=20)
        with pytest.raises(gcp.GCPError) as e:
            _submit(ctx, na, csa, big.sub, 2, 1)
        assert e.value.status == -5
        ctx.serve_stop()


def test_requests_arriving_during_a_round_join_later():
    a = synth.mlp_256x6(n_sub=64, n_cuts=40)
    s = synth.mlp_small(n_sub=3)
    with gcp.Context(0) as ctx:
        na, csa = ctx.load_instance(a)
        ns, css = ctx.load_instance(s)
        ctx.serve_start(4)
        t_long = _submit(ctx, na, csa, a.sub, 12, 1, iters=40)
        time.sleep(0.05)
        t_short = _submit(ctx, ns, css, s.sub, 1, 2, iters=5)
        r_short, _ = ctx.serve_wait(t_short, s.n_rows + 8)
        r_long, _ = ctx.serve_wait(t_long, a.n_rows + 8)
        ctx.serve_stop()
    assert r_short.status == 0 and r_long.status == 0
    # the short request was admitted while the long one was running and
    # finished without waiting for all of its rounds
    assert r_short.latency_ms < r_long.latency_ms


def _oracle_final(inst, sub, A, B, G):
    """The oracle's bound of a finished request at its last round's subdomains and duals."""
    fin = dataclasses.replace(inst, sub=sub)
    P = O.build_problem(fin)
    return O.evaluate(P, oracle_duals(fin, A, B[:, :P.max_splits], G))


def test_serving_results_match_the_oracle_alone_and_in_a_three_network_mix():
    """Every finished request's certified bounds equal the oracle's evaluation
    (1e-9) at the request's last-round subdomains (App. B children) and duals,
    for requests of three networks served together and for one served alone;
    the BF16 chain's error against the certified FP64 bound stays within 1e-3."""
    a = synth.mlp_small(n_sub=6)
    c = synth.mlp_256x6(n_sub=10, n_cuts=40)
    n = synth.cnn_cifar(n_sub=3, n_cuts=60)
    rounds = 3
    with gcp.Context(0) as ctx:
        ids = [ctx.load_instance(x) for x in (a, c, n)]
        ctx.serve_start(8)
        t_alone = ctx.serve_submit(ids[1][0], ids[1][1], c.sub,
                                   gcp.opt_params(10, gcp.GCP_ADAM, gcp.GCP_BF16, 1, 0.1, 0.02, 0.02, 0.98),
                                   rounds, 17, keep_final=True)
        r_alone, cert_alone = ctx.serve_wait(t_alone, c.n_rows)
        final_alone = ctx.serve_final(t_alone)
        tickets = [ctx.serve_submit(nid, cs, x.sub,
                                    gcp.opt_params(10, gcp.GCP_ADAM, gcp.GCP_BF16, 1, 0.1, 0.02, 0.02, 0.98),
                                    rounds, seed, keep_final=True)
                   for x, (nid, cs), seed in zip((a, c, n), ids, (30, 17, 31))]
        results = [ctx.serve_wait(t, x.n_rows) for t, x in zip(tickets, (a, c, n))]
        finals = [ctx.serve_final(t) for t in tickets]
        with pytest.raises(gcp.GCPError):
            ctx.serve_final(tickets[0])             # taken once
        ctx.serve_stop()
    checks = [(c, r_alone, cert_alone, final_alone)] + [(x, r, cert, f) for x, (r, cert), f in
                                                         zip((a, c, n), results, finals)]
    for inst, res, cert, (sub, A, B, G) in checks:
        assert res.status == 0 and res.rows == inst.n_rows
        # the last round's subdomains are children of the submitted ones
        for s in range(inst.sub.n):
            p0, p1 = int(inst.sub.ptr[s]), int(inst.sub.ptr[s + 1])
            q0, q1 = int(sub.ptr[s]), int(sub.ptr[s + 1])
            assert p1 - p0 <= q1 - q0 <= p1 - p0 + rounds - 1
            np.testing.assert_array_equal(sub.layer[q0:q0 + p1 - p0], inst.sub.layer[p0:p1])
            np.testing.assert_array_equal(sub.index[q0:q0 + p1 - p0], inst.sub.index[p0:p1])
            np.testing.assert_array_equal(sub.sign[q0:q0 + p1 - p0], inst.sub.sign[p0:p1])
        ref = _oracle_final(inst, sub, A, B, G)
        assert_rel(cert, ref, 1e-9, f"{inst.name}: served certified bound vs oracle")
        assert res.max_rel_err_vs_fp64 <= 1e-3, (inst.name, res.max_rel_err_vs_fp64)
        assert abs(res.min_certified - float(np.min(cert))) == 0.0
    # the request served alone and the same request (same seed) in the mix
    # took the same children; both are anchored to the oracle above
    np.testing.assert_array_equal(final_alone[0].index, finals[1][0].index)
    assert_rel(results[1][1], cert_alone, 1e-9, "same request alone and in the mix")
