"""Shared helpers of the GPU parity tests (no bound arithmetic here)."""
import dataclasses

import numpy as np

from oracle import gcp_oracle as O
from paper_2208_05740_gb300 import synth


def rel_close(a, b, tol):
    """|a - b| <= tol * max(|b|, 1) elementwise (relative, absolute near 0)."""
    a, b = np.asarray(a, np.float64), np.asarray(b, np.float64)
    return np.abs(a - b) <= tol * np.maximum(np.abs(b), 1.0)


def assert_rel(a, b, tol, what=""):
    ok = rel_close(a, b, tol)
    if not ok.all():
        i = int(np.argmin(ok.ravel()))
        raise AssertionError(f"{what}: {int((~ok).sum())} of {ok.size} off; e.g. {np.ravel(a)[i]!r} vs "
                             f"{np.ravel(b)[i]!r} (tol {tol})")


def split_alpha(inst, A):
    """[R, sum d_i] -> list of [R, d_i] (hidden layers in order)."""
    out, off = [], 0
    for d in inst.net.dims[1:-1]:
        out.append(A[:, off:off + d].copy())
        off += d
    return out


def join_alpha(alist):
    return np.concatenate(alist, axis=1) if alist else np.zeros((0, 0))


def oracle_duals(inst, A, B, G):
    return O.Duals(split_alpha(inst, A), B.copy(), G.copy())


def select(inst, idx):
    """Instance restricted to the subdomains idx (same net, spec, cuts)."""
    s = inst.sub
    ptr, lay, ind, sg = [0], [], [], []
    for q in idx:
        a, b = int(s.ptr[q]), int(s.ptr[q + 1])
        lay += s.layer[a:b].tolist(); ind += s.index[a:b].tolist(); sg += s.sign[a:b].tolist()
        ptr.append(len(lay))
    sub = synth.Subdomains(np.asarray(ptr, np.int32), np.asarray(lay, np.int16), np.asarray(ind, np.int32),
                           np.asarray(sg, np.int8))
    return dataclasses.replace(inst, sub=sub)


def rows_of(inst, sub_idx):
    K = inst.spec.shape[0]
    return np.concatenate([np.arange(s * K, (s + 1) * K) for s in sub_idx])


def _layer_rows(ly, idx):
    """Rows idx of a layer's linear map as dense [len(idx), d_in] (convolutions materialised)."""
    if ly.kind == synth.DENSE:
        return ly.W[idx]
    return O.conv_matrix(ly.W, ly.in_shape, ly.out_shape, ly.stride, ly.pad)[idx].toarray()


def oracle_crown_bounds(net, x_lo, x_hi, block=512):
    """Root intermediate bounds l, u (Sec. 2) computed by the oracle alone.

    Hidden layer 1: the interval image of the box under W^(1) x + b^(1).
    Hidden layer i > 1: the network truncated after layer i's linear map,
    with spec rows +e_j and -e_j, bounded by the oracle's Theorem 3.1 at the
    default duals (no cuts, no splits) over the bounds already found for the
    layers below: l_j = g(+e_j), u_j = -g(-e_j) -- CROWN with the adaptive
    lower slope. Plain feed-forward networks only (no skip connections).
    """
    if any(getattr(ly, "skip", 0) for ly in net.layers):
        raise ValueError("oracle_crown_bounds: skip connections are not handled here")
    ly = net.layers[0]
    W = _layer_rows(ly, np.arange(ly.d_out))
    c0, r0 = (x_hi + x_lo) / 2, (x_hi - x_lo) / 2
    z = W @ c0 + ly.b
    rad = np.abs(W) @ r0
    lo, hi = [z - rad], [z + rad]
    empty = synth.Subdomains(np.zeros(2, np.int32), np.zeros(0, np.int16), np.zeros(0, np.int32),
                             np.zeros(0, np.int8))
    for i in range(2, net.L):
        ly = net.layers[i - 1]
        d = ly.d_out
        li, hi_ = np.empty(d), np.empty(d)
        for a in range(0, d, block):
            idx = np.arange(a, min(d, a + block))
            last = synth.Layer(synth.DENSE, _layer_rows(ly, idx), ly.b[idx], ly.in_shape, (len(idx),))
            tr = synth.Instance("prefix", synth.Network(net.layers[:i - 1] + [last]), x_lo, x_hi,
                                np.concatenate([np.eye(len(idx)), -np.eye(len(idx))]), lo, hi, empty,
                                synth.Cuts.empty())
            P = O.build_problem(tr)
            g = O.evaluate(P, O.default_duals(P))
            li[idx], hi_[idx] = g[:len(idx)], -g[len(idx):]
        lo.append(li)
        hi.append(hi_)
    return lo, hi
