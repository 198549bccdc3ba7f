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
    r = ctx.bab_verify(net_id, cs, gcp.opt_params(**PARAMS), batch=64, max_rounds=400)
    assert r["verified"] == 1, r
    plain = _shifted(0.05)
    n0, _ = _load(ctx, plain)
    r0 = ctx.bab_verify(n0, -1, gcp.opt_params(**PARAMS), batch=64, max_rounds=400)
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
