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


def oracle_crown_bounds(net, x_lo, x_hi):
    """Root intermediate bounds by CROWN, computed by the oracle alone (Sec. 2)."""
    return O.crown_root_bounds(net, x_lo, x_hi)
