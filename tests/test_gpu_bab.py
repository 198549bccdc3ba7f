"""Branch and bound over ReLU splits with the library's bounding
(gcp_bab_verify, Sec. 3.2 / App. B).

On the MLP 8-16-16-3 with one spec row, the last layer's bias is shifted so
that the exact minimum of c^T f(x) over the box (the oracle's MILP) is +0.05
or -0.05. The root bound is below zero in both cases; branch and bound must
prove the first property and must not prove the second.
"""
import dataclasses

import numpy as np
import pytest

from oracle import gcp_oracle as O
from paper_2208_05740_gb300 import gcp, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from paper_2208_05740_gb300 import build
    build.build()
    c = gcp.Context(0)
    yield c
    c.close()


def _shifted(margin):
    inst = synth.mlp_small()
    c = inst.spec[:1]
    root = synth.Subdomains(np.zeros(2, np.int32), np.zeros(0, np.int16), np.zeros(0, np.int32),
                            np.zeros(0, np.int8))
    base = dataclasses.replace(inst, spec=c, sub=root, cuts=synth.Cuts.empty())
    m = O.lp_value(O.build_problem(base), 0, 0, integral=True, with_cuts=False)
    last = inst.net.layers[-1]
    b = last.b - (m - margin) * c[0] / float(c[0] @ c[0])
    net = synth.Network(inst.net.layers[:-1] + [dataclasses.replace(last, b=b)])
    out = dataclasses.replace(base, net=net)
    m2 = O.lp_value(O.build_problem(out), 0, 0, integral=True, with_cuts=False)
    assert abs(m2 - margin) < 1e-6
    return out


PARAMS = dict(iters=20, optimizer=gcp.GCP_ADAM, prec=gcp.GCP_FP32, certify=1, lr_alpha=0.1, lr_beta=0.05,
              lr_gamma=0.02, lr_decay=0.98)


def _load(ctx, inst):
    if inst.cuts.n == 0:
        return ctx.init_net(inst.net.layers, inst.x_lo, inst.x_hi, inst.spec, inst.inter_lo, inst.inter_hi), -1
    return ctx.load_instance(inst)


@pytest.mark.parametrize("margin", [0.05, -0.05])
def test_bab_proves_true_and_rejects_false_properties(ctx, margin):
    inst = _shifted(margin)
    net_id, cs = _load(ctx, inst)
    # the root alone does not decide it
    D = ctx.duals_create(net_id, cs, inst.sub, gcp.GCP_FP32)
    _, root_cert, _ = ctx.optimize_batch(D, gcp.opt_params(**PARAMS))
    ctx.duals_free(D)
    assert root_cert[0] < 0
    r = ctx.bab_verify(net_id, cs, gcp.opt_params(**PARAMS), batch=64, max_rounds=400, max_domains=1 << 15)
    if margin > 0:
        assert r["verified"] == 1, r
        assert r["domains_left"] == 0 and r["min_bound"] > 0, r
        assert r["domains_verified"] >= 2
    else:
        assert r["verified"] == 0, r       # sound: a false property is never proven
        assert r["min_bound"] <= 0, r
    r1 = ctx.bab_verify(net_id, cs, gcp.opt_params(**PARAMS), batch=64, max_rounds=1)
    assert r1["verified"] == 0 and r1["rounds"] == 1 and r1["domains_left"] == 2, r1


def test_bab_with_cuts(ctx):
    """Cuts valid at the root hold in every subdomain: with MIP-valid cuts the
    property is still proven, with no more subdomains than without them."""
    inst = _shifted(0.05)
    P = O.build_problem(dataclasses.replace(inst, cuts=synth.mlp_small().cuts))
    cuts = synth.mlp_small().cuts
    d_valid = O.valid_cut_offsets(P)   # MIP-valid offsets: the cuts hold at every feasible point
    inst = dataclasses.replace(inst, cuts=dataclasses.replace(cuts, d=d_valid))
    net_id, cs = _load(ctx, inst)
    # the static branching order: the same tree with and without the cuts
    r = ctx.bab_verify(net_id, cs, gcp.opt_params(**PARAMS), batch=64, max_rounds=400, branching=1)
    assert r["verified"] == 1, r
    plain = _shifted(0.05)
    n0, _ = _load(ctx, plain)
    r0 = ctx.bab_verify(n0, -1, gcp.opt_params(**PARAMS), batch=64, max_rounds=400, branching=1)
    assert r0["verified"] == 1 and r["domains_bounded"] <= r0["domains_bounded"], (r, r0)


def _two_labels(m0, m1):
    """MLP 8-16-16-3 with its two spec rows e_y - e_a, e_y - e_b; the biases of
    classes a and b shifted so that the exact minima (the oracle's MILP) are
    m0 and m1."""
    inst = synth.mlp_small()
    C = inst.spec
    root = synth.Subdomains(np.zeros(2, np.int32), np.zeros(0, np.int16), np.zeros(0, np.int32),
                            np.zeros(0, np.int8))
    base = dataclasses.replace(inst, sub=root, cuts=synth.Cuts.empty())
    P = O.build_problem(base)
    m = [O.lp_value(P, 0, k, integral=True, with_cuts=False) for k in range(2)]
    last = inst.net.layers[-1]
    b = last.b.copy()
    for k, target in enumerate((m0, m1)):
        other = int(np.argmin(C[k]))            # the -1 entry: class a (row 0) or b (row 1)
        b[other] += m[k] - target              # raising f_a lowers f_y - f_a
    net = synth.Network(inst.net.layers[:-1] + [dataclasses.replace(last, b=b)])
    out = dataclasses.replace(base, net=net)
    P2 = O.build_problem(out)
    for k, target in enumerate((m0, m1)):
        assert abs(O.lp_value(P2, 0, k, integral=True, with_cuts=False) - target) < 1e-6
    return out


def test_bab_label_by_label_easiest_first(ctx):
    """Label 0's minimum is +0.05 (provable), label 1's -0.05 (false): the
    labels are settled in the order of their root bounds closest to zero, the
    first is proved and the second is not; with stop_at_failure the labels
    after a failure are not attempted. Every label's verdict matches
    gcp_bab_verify on that label alone."""
    inst = _two_labels(0.05, -0.05)
    net_id, cs = _load(ctx, inst)
    p = gcp.opt_params(**PARAMS)
    D = ctx.duals_create(net_id, cs, inst.sub, gcp.GCP_FP32)
    _, root, _ = ctx.optimize_batch(D, p)
    ctx.duals_free(D)
    r, order, ver = ctx.bab_verify_labels(net_id, cs, 2, p, batch=64, max_rounds=400, max_domains=1 << 15)
    pos = [k for k in range(2) if root[k] > 0]
    neg = sorted([k for k in range(2) if root[k] <= 0], key=lambda k: -root[k])
    assert list(order) == pos + neg
    assert list(ver) == [1, 0] and r["verified"] == 0
    for k in range(2):
        one = dataclasses.replace(inst, spec=inst.spec[k:k + 1])
        nk, ck = _load(ctx, one)
        rk = ctx.bab_verify(nk, ck, p, batch=64, max_rounds=400, max_domains=1 << 15)
        assert rk["verified"] == ver[k]
    r2, order2, ver2 = ctx.bab_verify_labels(net_id, cs, 2, p, batch=64, max_rounds=400, max_domains=1 << 15,
                                             stop_at_failure=True)
    seen_fail = False
    for k in order2:
        if seen_fail:
            assert ver2[k] == -1
        seen_fail = seen_fail or ver2[k] == 0
    proved = _two_labels(0.05, 0.1)
    n2, c2 = _load(ctx, proved)
    r3, _, ver3 = ctx.bab_verify_labels(n2, c2, 2, p, batch=64, max_rounds=400, max_domains=1 << 15)
    assert list(ver3) == [1, 1] and r3["verified"] == 1 and r3["min_bound"] > 0


def _oracle_scores(inst, A, B, G):
    """The branching score of every (subdomain, layer, neuron) from the oracle's
    nuhat at the given duals: w_j * sum_k [nuhat_j]_+ over the subdomain's rows,
    w_j = -l u / (u - l) on root-unstable neurons the subdomain has not split."""
    from tests.helpers import oracle_duals
    P = O.build_problem(inst)
    _, T = O.evaluate(P, oracle_duals(inst, A, B[:, :P.max_splits], G), trace=True)
    K = inst.spec.shape[0]
    S = inst.sub.n
    out = []
    for s in range(S):
        split = {(int(inst.sub.layer[e]), int(inst.sub.index[e])) for e in range(inst.sub.ptr[s], inst.sub.ptr[s + 1])}
        sc = {}
        for i, (lo, hi) in enumerate(zip(inst.inter_lo, inst.inter_hi), start=1):
            nh = T.nu_hat[i - 1][s * K:(s + 1) * K]
            w = np.where((lo < 0) & (hi > 0), -lo * hi / np.where(hi - lo > 0, hi - lo, 1.0), 0.0)
            tot = w * np.maximum(nh, 0.0).sum(axis=0)
            for j in np.nonzero(tot > 0)[0]:
                if (i, int(j)) not in split:
                    sc[(i, int(j))] = float(tot[j])
        out.append(sc)
    return out


@pytest.mark.parametrize("prec", [gcp.GCP_FP32, gcp.GCP_BF16])
def test_branch_picks_maximise_the_oracle_score(ctx, prec):
    """gcp_branch_picks: for every subdomain the pick's score (computed by the
    oracle) is the largest up to the chain's tolerance, is never a split
    neuron, and is the oracle's argmax wherever the best two are apart."""
    inst = synth.mlp_256x6(n_sub=24, n_cuts=30)
    net_id, cs = ctx.load_instance(inst)
    D = ctx.duals_create(net_id, cs, inst.sub, gcp.GCP_FP32)
    ctx.optimize_batch(D, gcp.opt_params(10, gcp.GCP_ADAM, gcp.GCP_FP32, 0, 0.1, 0.02, 0.02, 0.98))
    A, B, G = ctx.duals_export(D)
    lay, idx = ctx.branch_picks(D, prec, inst.sub.n)
    ctx.duals_free(D)
    scores = _oracle_scores(inst, A, B, G)
    tol = 1e-5 if prec == gcp.GCP_FP32 else 1e-3
    exact = 0
    for s, sc in enumerate(scores):
        if not sc:
            assert lay[s] == -1
            continue
        best = max(sc.values())
        got = sc.get((int(lay[s]), int(idx[s])))
        assert got is not None, (s, lay[s], idx[s])          # an unsplit root-unstable neuron with a score
        assert got >= best * (1 - 10 * tol), (s, got, best)
        top = sorted(sc.values(), reverse=True)
        if len(top) == 1 or top[0] > top[1] * (1 + 100 * tol):
            assert got == best
            exact += 1
    if prec == gcp.GCP_FP32:
        assert exact >= len(scores) // 2


@pytest.mark.parametrize("margin", [0.05, -0.05])
def test_bab_branching_by_duals_and_static_order_agree_on_verdicts(ctx, margin):
    inst = _shifted(margin)
    net_id, cs = _load(ctx, inst)
    rd = ctx.bab_verify(net_id, cs, gcp.opt_params(**PARAMS), batch=64, max_rounds=400, max_domains=1 << 15,
                        branching=0)
    rs = ctx.bab_verify(net_id, cs, gcp.opt_params(**PARAMS), batch=64, max_rounds=400, max_domains=1 << 15,
                        branching=1)
    assert rd["verified"] == rs["verified"] == (1 if margin > 0 else 0), (rd, rs)
