"""FP64 CPU oracle of the GCP-CROWN bound -- TEST INFRASTRUCTURE ONLY.

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this module. The CUDA library never calls it and it
never calls the CUDA library; the two share nothing but the seeded input
arrays of ``paper_2208_05740_gb300.synth``.

It is a plain, slow restatement, in float64 and in the paper's notation, of

  * Theorem 3.1 (Sec. 3.1; restated and proved in App. A): the bound
    g(alpha, beta) obtained by propagating nu^(L) = -1 (the spec row folded
    into the last layer) backwards through every layer, with the per-neuron
    closed form of Lemma A.1 (App. A) for unstable neurons;
  * beta-CROWN's neuron splits as special cut rows (Sec. 3.1, "Connection to
    CROWN-like bound propagation methods");
  * the bound with the ReLU duals pi (and gamma_r = C - pi) of every unstable
    neuron optimised directly instead of set by Lemma A.1's closed form: the
    closed form maximises each neuron's own term but ignores pi's effect on
    nu and hence on the layers below, so optimising pi too is what reaches
    the LP optimum (the remark closing App. A); pi = theta * [nuhat]_+ with
    theta in [0, 1];
  * reverse-mode differentiation of that bound with respect to the
    optimisable duals (the paper optimises them by gradient ascent, Sec. 3.1
    after Theorem 3.1; App. C.1 names Adam with 20 iterations);
  * the LP of Eq. 16 and its MIP counterpart (Eq. 2-10 plus cuts), solved by
    SciPy/HiGHS, used only to pin the bound from outside;
  * residual (skip) connections, x^(k) = W^(k) xhat^(k-1) + b^(k) + S xhat^(m)
    with m < k and S the identity or a projection shortcut (a 1x1 convolution
    where a block changes channels or size): the residual CIFAR models of
    Sec. 4 / App. C.1 (ResBlock(a, b)); the skip term is one more linear map,
    whose multiplier nu^(k) adds S^T nu^(k) to the coefficient of xhat^(m).

Readings of the paper (each is listed with its reason in the design notes):
  R1 concretisation is the minimum of the linear input term over the box,
     sum_j min(c0_j lo_j, c0_j hi_j) with c0 = -W1^T nu1 + H0^T gamma
     (App. A explains the l1 term as that minimum; the printed
     "-eps||nu1^T W1 x0||_1" drops the linear term nu1^T W1 x0).
  R2 the layer equalities enter the Lagrangian as nu^T(x - W xhat - b),
     which is what yields the printed objective term -sum nu^T b.
  R3 the numerator of pi* is u[nuhat]_+ - beta^T Q (Lemma A.1 with
     q = -beta^T Q); the printed "+" makes h exceed the true maximum over pi
     for negative beta^T Q, i.e. it would be unsound.
  R4 tau = alpha * max(-nuhat, 0) >= 0 and nu = pi* - tau - beta^T H, so a
     negative nuhat gives nu = alpha * nuhat (the CROWN lower slope).
  R5 z of a stable neuron is fixed (1 if active, 0 if inactive); a cut term
     Q z on an active neuron therefore adds s = beta^T Q to the objective.
  R6 cuts may contain input variables (layer 0, kind x): their coefficients
     are added to c0 before concretisation (App. C.2 reports that almost all
     generated cuts involve input neurons although Eq. 15 starts at i = 1).
  R7 neuron classes: inactive if u <= 0, else active if l >= 0, else
     unstable (the printed sets overlap at 0).
  R8 every row (subdomain x spec row) has its own alpha, beta, gamma.
  R9 derivative conventions at kinks: d max(a,0)/da = 1 only for a > 0;
     clip(p, 0, C) passes d/dp only strictly inside (0, C) and d/dC for
     p >= C; at nuhat = 0 exactly every local derivative is 0.
 R10 default initial duals: alpha = 1 if u >= -l else 0, beta = gamma = 0.
 R11 a skip connection enters the Lagrangian like the layer's weight matrix:
     the equality x^(k) - W^(k) xhat^(k-1) - b^(k) - S xhat^(m) - b_S = 0 with
     multiplier nu^(k) adds S^T nu^(k) to y^(m), the coefficient of xhat^(m)
     (xhat^(0) = x, so m = 0 adds it to the input term before concretisation);
     the shortcut's bias b_S joins b^(k).
 R12 optimised pi (App. A's closing remark) is parametrised as
     pi = theta * C, C = [nuhat]_+, theta in [0, 1] per row and neuron, so it
     stays feasible (0 <= pi <= C) whatever the other duals do; its start is
     Lemma A.1's pi* (theta = pi* / C, u / (u - l) where C = 0) and its step
     uses alpha's learning rate.

Layouts (float64 numpy): rows r = s * K + k for subdomain s and spec row k;
alpha is a list over hidden layers of [R, d_i]; beta is [R, max_splits]
(slot m = m-th split of the row's subdomain); gamma is [R, N].

Parity of the optimisation trajectory in reduced precision is not pinned here:
the oracle pins the bound, its gradient and the trajectory in float64.
"""
from __future__ import annotations

import dataclasses
from typing import List, Optional

import numpy as np
import scipy.sparse as sp

KIND_X, KIND_XHAT, KIND_Z = 0, 1, 2
DENSE, CONV2D = 0, 1


# ----------------------------------------------------------------------------
# linear operators written out from their definitions
# ----------------------------------------------------------------------------

def conv_matrix(W: np.ndarray, in_shape, out_shape, stride: int, pad: int) -> sp.csr_matrix:
    """The matrix M with (M x)[o,oh,ow] = sum_{c,kh,kw} W[o,c,kh,kw] x[c, oh*s+kh-p, ow*s+kw-p]."""
    c_in, H, Wd = in_shape
    c_out, Ho, Wo = out_shape
    k = W.shape[2]
    rows, cols, vals = [], [], []
    oh, ow = np.meshgrid(np.arange(Ho), np.arange(Wo), indexing="ij")
    oh = oh.ravel()
    ow = ow.ravel()
    for o in range(c_out):
        for c in range(c_in):
            for kh in range(k):
                for kw in range(k):
                    ih = oh * stride + kh - pad
                    iw = ow * stride + kw - pad
                    ok = (ih >= 0) & (ih < H) & (iw >= 0) & (iw < Wd)
                    rows.append(o * Ho * Wo + oh[ok] * Wo + ow[ok])
                    cols.append(c * H * Wd + ih[ok] * Wd + iw[ok])
                    vals.append(np.full(int(ok.sum()), W[o, c, kh, kw]))
    r = np.concatenate(rows)
    cc = np.concatenate(cols)
    v = np.concatenate(vals)
    return sp.csr_matrix((v, (r, cc)), shape=(c_out * Ho * Wo, c_in * H * Wd))


def _rmul(A: np.ndarray, M) -> np.ndarray:
    """A @ M for a dense A and a dense or sparse M."""
    if sp.issparse(M):
        return np.asarray((M.T @ A.T).T)
    return A @ M


@dataclasses.dataclass
class Problem:
    """Everything the bound needs, in float64, built from an instance."""
    L: int
    dims: List[int]
    Wm: list                 # per layer: [d_i, d_{i-1}] dense ndarray or csr
    b: List[np.ndarray]
    x_lo: np.ndarray
    x_hi: np.ndarray
    spec: np.ndarray         # [K, d_L]
    root_lo: List[np.ndarray]
    root_hi: List[np.ndarray]
    # per subdomain split-clamped bounds, per hidden layer [S, d_i]
    sub_lo: List[np.ndarray]
    sub_hi: List[np.ndarray]
    split_ptr: np.ndarray
    split_layer: np.ndarray
    split_index: np.ndarray
    split_sign: np.ndarray
    max_splits: int
    # cut matrices [N, d_i] per layer (index 0 = input, only H used there)
    H: list
    G: list
    Q: list
    d: np.ndarray
    # per layer (index i-1 for layer i): 0, or s >= 1 when layer i adds xhat^(s-1)
    skip: List[int] = dataclasses.field(default_factory=list)
    # per layer: the shortcut S [d_i, d_{s-1}] (dense or csr), None for the identity
    skip_map: list = dataclasses.field(default_factory=list)

    @property
    def K(self) -> int:
        return self.spec.shape[0]

    @property
    def S(self) -> int:
        return len(self.split_ptr) - 1

    @property
    def R(self) -> int:
        return self.S * self.K

    @property
    def N(self) -> int:
        return self.d.shape[0]


def build_problem(inst) -> Problem:
    """Turn the synthetic instance arrays into the oracle's matrices."""
    net = inst.net
    L = net.L
    dims = [net.layers[0].d_in] + [ly.d_out for ly in net.layers]
    Wm, b = [], []
    skip = [int(getattr(ly, "skip", 0)) for ly in net.layers]
    skip_map = []
    for i, (s_, ly) in enumerate(zip(skip, net.layers)):
        sc = getattr(ly, "shortcut", None) if s_ else None
        assert 0 <= s_ <= i + 1, "skip source must precede the layer"
        if sc is None:
            assert s_ == 0 or dims[s_ - 1] == dims[i + 1], "an identity skip needs equal widths"
            skip_map.append(None)
        else:
            assert sc.d_in == dims[s_ - 1] and sc.d_out == dims[i + 1], "shortcut shape"
            skip_map.append(np.asarray(sc.W, np.float64) if sc.kind == DENSE else
                            conv_matrix(np.asarray(sc.W, np.float64), sc.in_shape, sc.out_shape, sc.stride, sc.pad))
    for ly in net.layers:
        if ly.kind == DENSE:
            Wm.append(np.asarray(ly.W, np.float64))
        else:
            Wm.append(conv_matrix(np.asarray(ly.W, np.float64), ly.in_shape, ly.out_shape, ly.stride, ly.pad))
        b.append(np.asarray(ly.b, np.float64))
        sc = getattr(ly, "shortcut", None) if getattr(ly, "skip", 0) else None
        if sc is not None:
            b[-1] = b[-1] + np.asarray(sc.b, np.float64)
    sub = inst.sub
    S = sub.n
    sub_lo = [np.repeat(np.asarray(lo, np.float64)[None, :], S, 0) for lo in inst.inter_lo]
    sub_hi = [np.repeat(np.asarray(hi, np.float64)[None, :], S, 0) for hi in inst.inter_hi]
    for s in range(S):
        for e in range(int(sub.ptr[s]), int(sub.ptr[s + 1])):
            i, j, sg = int(sub.layer[e]), int(sub.index[e]), int(sub.sign[e])
            if sg > 0:       # x >= 0 branch
                sub_lo[i - 1][s, j] = max(sub_lo[i - 1][s, j], 0.0)
            else:            # x <= 0 branch
                sub_hi[i - 1][s, j] = min(sub_hi[i - 1][s, j], 0.0)
    cuts = inst.cuts
    N = cuts.n
    H = [None] * L
    G = [None] * L
    Q = [None] * L
    for i in range(L):
        for mats, kind in ((H, KIND_X), (G, KIND_XHAT), (Q, KIND_Z)):
            rows, cols, vals = [], [], []
            for k in range(N):
                for e in range(int(cuts.ptr[k]), int(cuts.ptr[k + 1])):
                    if int(cuts.layer[e]) == i and int(cuts.kind[e]) == kind:
                        rows.append(k)
                        cols.append(int(cuts.index[e]))
                        vals.append(float(cuts.coef[e]))
            mats[i] = sp.csr_matrix((vals, (rows, cols)), shape=(N, dims[i]))
    return Problem(L, dims, Wm, b, np.asarray(inst.x_lo, np.float64), np.asarray(inst.x_hi, np.float64),
                   np.asarray(inst.spec, np.float64), [np.asarray(a, np.float64) for a in inst.inter_lo],
                   [np.asarray(a, np.float64) for a in inst.inter_hi], sub_lo, sub_hi,
                   np.asarray(sub.ptr), np.asarray(sub.layer), np.asarray(sub.index), np.asarray(sub.sign),
                   sub.max_splits if S else 0, H, G, Q, np.asarray(cuts.d, np.float64), skip, skip_map)


# ----------------------------------------------------------------------------
# duals
# ----------------------------------------------------------------------------

@dataclasses.dataclass
class Duals:
    alpha: List[np.ndarray]   # per hidden layer [R, d_i]
    beta: np.ndarray          # [R, max_splits]
    gamma: np.ndarray         # [R, N]
    # per hidden layer [R, d_i]: pi = theta * [nuhat]_+ on unstable neurons
    # (R12); None: Lemma A.1's closed-form pi
    theta: Optional[List[np.ndarray]] = None

    def copy(self) -> "Duals":
        return Duals([a.copy() for a in self.alpha], self.beta.copy(), self.gamma.copy(),
                     None if self.theta is None else [t.copy() for t in self.theta])


def _through_skip(P: Problem, layer: int, nu: np.ndarray) -> np.ndarray:
    """S^T nu of the skip of `layer` (nu itself for the identity), as rows [R, d_m]."""
    S = P.skip_map[layer - 1] if P.skip_map else None
    return nu.copy() if S is None else _rmul(nu, S)


def _skip_forward(P: Problem, layer: int, a: np.ndarray) -> np.ndarray:
    """S a of the skip of `layer` as rows [R, d_layer] (a itself for the identity)."""
    S = P.skip_map[layer - 1] if P.skip_map else None
    if S is None:
        return a
    return np.asarray(S @ a.T).T if sp.issparse(S) else a @ S.T


def row_sub(P: Problem) -> np.ndarray:
    return np.arange(P.R) // P.K


def row_spec(P: Problem) -> np.ndarray:
    return np.arange(P.R) % P.K


def default_duals(P: Problem) -> Duals:
    """R10: alpha = 1 where u >= -l (else 0), beta = gamma = 0."""
    rs = row_sub(P)
    alpha = [(P.sub_hi[i][rs] >= -P.sub_lo[i][rs]).astype(np.float64) for i in range(P.L - 1)]
    return Duals(alpha, np.zeros((P.R, P.max_splits)), np.zeros((P.R, P.N)))


def _split_terms(P: Problem, beta: np.ndarray, layer: int):
    """(row, neuron, coefficient-of-beta, beta slot) for splits in `layer`.

    A split x_j >= 0 is the cut row -x_j <= 0 and x_j <= 0 is x_j <= 0
    (beta-CROWN as a special case, Sec. 3.1): its H entry is -sign.
    """
    rr, jj, hh, mm = [], [], [], []
    for s in range(P.S):
        a, e_end = int(P.split_ptr[s]), int(P.split_ptr[s + 1])
        for e in range(a, e_end):
            if int(P.split_layer[e]) != layer:
                continue
            for k in range(P.K):
                rr.append(s * P.K + k)
                jj.append(int(P.split_index[e]))
                hh.append(-float(P.split_sign[e]))
                mm.append(e - a)
    return (np.asarray(rr, np.int64), np.asarray(jj, np.int64),
            np.asarray(hh, np.float64), np.asarray(mm, np.int64))


# ----------------------------------------------------------------------------
# Lemma A.1 for one unstable neuron
# ----------------------------------------------------------------------------

def unstable_closed_form(nu_hat, s, l, u, alpha):
    """Per unstable neuron (l < 0 < u): returns (pi*, tau, h).

    Lemma A.1 maximises l*pi - ReLU(u*gam + l*pi + q) over pi + gam = C,
    pi, gam >= 0, with C = [nuhat]_+ and q = -s (s = beta^T Q[:, j]):
    pi* = clip((u C - s) / (u - l), 0, C) and h = l pi* - max(0, u (C - pi*) + l pi* - s).
    tau = alpha * max(-nuhat, 0) is the share of [nuhat]_- carried by the lower
    relaxation xhat >= x (R4).
    """
    C = np.maximum(nu_hat, 0.0)
    p0 = (u * C - s) / (u - l)
    pi = np.minimum(np.maximum(p0, 0.0), C)
    h = l * pi - np.maximum(0.0, u * (C - pi) + l * pi - s)
    tau = alpha * np.maximum(-nu_hat, 0.0)
    return pi, tau, h


# ----------------------------------------------------------------------------
# the bound (Theorem 3.1) and its gradient
# ----------------------------------------------------------------------------

@dataclasses.dataclass
class Trace:
    """Per-layer intermediates of one evaluation (index = hidden layer i-1)."""
    nu: List[np.ndarray]
    nu_hat: List[np.ndarray]
    t: List[np.ndarray]
    s: List[np.ndarray]
    lo: List[np.ndarray]
    hi: List[np.ndarray]
    c0: np.ndarray
    g: np.ndarray


def evaluate(P: Problem, D: Duals, trace: bool = False):
    """g(alpha, beta, gamma) for every row, Theorem 3.1 with R1-R8."""
    rs, rk = row_sub(P), row_spec(P)
    R = P.R
    gam = D.gamma
    # nu^(L) = -c (spec folded as the last layer, Sec. 2); its bias term.
    nu = -P.spec[rk]                                  # [R, d_L]
    obj = -(nu @ P.b[P.L - 1]) - gam @ P.d
    # R11: multipliers of skip terms waiting for the layer they skip to
    carry = {}
    if P.skip and P.skip[P.L - 1]:
        carry[P.skip[P.L - 1] - 1] = _through_skip(P, P.L, nu)
    T = Trace([None] * (P.L - 1), [None] * (P.L - 1), [None] * (P.L - 1), [None] * (P.L - 1),
              [None] * (P.L - 1), [None] * (P.L - 1), None, None)
    for i in range(P.L - 1, 0, -1):
        y = _rmul(nu, P.Wm[i])                        # nu^(i+1)^T W^(i+1)
        if i in carry:
            y = y + carry.pop(i)                      # + nu^(k) of the layer k that adds xhat^(i)
        t = np.asarray((P.H[i].T @ gam.T).T) if P.N else np.zeros((R, P.dims[i]))
        gg = np.asarray((P.G[i].T @ gam.T).T) if P.N else np.zeros((R, P.dims[i]))
        s = np.asarray((P.Q[i].T @ gam.T).T) if P.N else np.zeros((R, P.dims[i]))
        rr, jj, hh, mm = _split_terms(P, D.beta, i)
        if len(rr):
            np.add.at(t, (rr, jj), hh * D.beta[rr, mm])
        nu_hat = y - gg
        lo = P.sub_lo[i - 1][rs]
        hi = P.sub_hi[i - 1][rs]
        inactive = hi <= 0
        active = (~inactive) & (lo >= 0)
        unstable = ~(inactive | active)
        den_l = np.where(unstable, lo, -1.0)
        den_u = np.where(unstable, hi, 1.0)
        pi, tau, h = unstable_closed_form(nu_hat, s, den_l, den_u, D.alpha[i - 1])
        if D.theta is not None:     # R12: pi = theta * C, h at that pi (Lemma A.1's objective)
            C = np.maximum(nu_hat, 0.0)
            pi = np.clip(D.theta[i - 1], 0.0, 1.0) * C
            h = den_l * pi - np.maximum(0.0, den_u * (C - pi) + den_l * pi - s)
        nu_i = np.where(active, nu_hat - t, np.where(inactive, -t, pi - tau - t))
        obj = obj + np.sum(np.where(unstable, h, 0.0), axis=1) + np.sum(np.where(active, s, 0.0), axis=1)
        obj = obj - nu_i @ P.b[i - 1]
        if trace:
            T.nu[i - 1], T.nu_hat[i - 1], T.t[i - 1], T.s[i - 1] = nu_i, nu_hat, t, s
            T.lo[i - 1], T.hi[i - 1] = lo, hi
        nu = nu_i
        if P.skip and P.skip[i - 1]:
            m = P.skip[i - 1] - 1
            v = _through_skip(P, i, nu_i)
            carry[m] = carry[m] + v if m in carry else v
    y0 = _rmul(nu, P.Wm[0])
    if 0 in carry:
        y0 = y0 + carry.pop(0)
    c0 = -y0 + (np.asarray((P.H[0].T @ gam.T).T) if P.N else 0.0)
    obj = obj + np.sum(np.minimum(c0 * P.x_lo[None, :], c0 * P.x_hi[None, :]), axis=1)
    if trace:
        T.c0, T.g = c0, obj
        return obj, T
    return obj


def gradient(P: Problem, D: Duals):
    """g and dg/d(alpha, beta, gamma) by reverse mode through Theorem 3.1.

    The adjoint of y^(i-1) = W^(i)^T nu^(i) is a forward pass: with
    a = dg/dy^(i-1), nubar^(i) = W^(i) a - b^(i) = dg/dnu^(i) (plus dg/dy^(m)
    when layer i adds xhat^(m), R11). Starting value
    a = -x*, the box corner minimising c0^T x (R1, R9: the centre where
    c0 = 0). dg/dgamma_k is then the violation H x + G xhat + Q z - d of cut k
    at the primal point implied by the duals (x = -nubar, xhat = -dg/dnuhat,
    z = dg/ds).
    """
    g, T = evaluate(P, D, trace=True)
    R = P.R
    xc = 0.5 * (P.x_lo + P.x_hi)
    xstar = np.where(T.c0 > 0, P.x_lo[None, :], np.where(T.c0 < 0, P.x_hi[None, :], xc[None, :]))
    a = -xstar
    sources = {s_ - 1 for s_ in P.skip[:P.L - 1] if s_}
    a_saved = {0: a} if 0 in sources else {}
    g_gamma = -np.repeat(P.d[None, :], R, 0) + (np.asarray((P.H[0] @ xstar.T).T) if P.N else 0.0)
    g_beta = np.zeros_like(D.beta)
    g_alpha = [np.zeros_like(x) for x in D.alpha]
    g_theta = None if D.theta is None else [np.zeros_like(x) for x in D.theta]
    for i in range(1, P.L):
        Wi = P.Wm[i - 1]
        nubar = (np.asarray(Wi @ a.T).T if sp.issparse(Wi) else a @ Wi.T) - P.b[i - 1][None, :]
        if P.skip and P.skip[i - 1]:
            nubar = nubar + _skip_forward(P, i, a_saved[P.skip[i - 1] - 1])
        nu_hat, s, lo, hi = T.nu_hat[i - 1], T.s[i - 1], T.lo[i - 1], T.hi[i - 1]
        al = D.alpha[i - 1]
        inactive = hi <= 0
        active = (~inactive) & (lo >= 0)
        unstable = ~(inactive | active)
        ul = np.where(unstable, hi - lo, 1.0)
        C = np.maximum(nu_hat, 0.0)
        p0 = (hi * C - s) / ul
        pos = nu_hat > 0
        inside = pos & (p0 > 0) & (p0 < C)
        upper = pos & (p0 >= C) & ~inside          # pi* = C  (s <= l C)
        # d nu / d nuhat, d h / d nuhat, d nu / d s, d h / d s per case (R9)
        dnu_dnh = np.where(pos, np.where(inside, hi / ul, np.where(upper, 1.0, 0.0)),
                           np.where(nu_hat < 0, al, 0.0))
        dh_dnh = np.where(inside, lo * hi / ul, 0.0)
        dnu_ds = np.where(inside, -1.0 / ul, 0.0)
        # h = min(s, 0) when C = 0; h = s when pi* = C with l C - s > 0
        dh_ds = np.where(pos, np.where(inside, -lo / ul, np.where(upper & (lo * C - s > 0), 1.0, 0.0)),
                         np.where(s < 0, 1.0, 0.0))
        if D.theta is not None:
            # R12: pi = th C, q = u (C - pi) + l pi - s, h = l pi - max(q, 0), nu = pi - tau - t
            th = np.clip(D.theta[i - 1], 0.0, 1.0)
            q = hi * (C - th * C) + lo * th * C - s
            act = q > 0
            dnu_dnh = np.where(pos, th, np.where(nu_hat < 0, al, 0.0))
            dh_dnh = np.where(pos, lo * th - np.where(act, hi * (1.0 - th) + lo * th, 0.0), 0.0)
            dnu_ds = np.zeros_like(nu_hat)
            dh_ds = np.where(act, 1.0, 0.0)
            g_theta[i - 1] = np.where(unstable, C * (nubar + lo + np.where(act, hi - lo, 0.0)), 0.0)
        dnu_dnh = np.where(unstable, dnu_dnh, np.where(active, 1.0, 0.0))
        dh_dnh = np.where(unstable, dh_dnh, 0.0)
        dnu_ds = np.where(unstable, dnu_ds, 0.0)
        dh_ds = np.where(unstable, dh_ds, np.where(active, 1.0, 0.0))
        dg_dnh = nubar * dnu_dnh + dh_dnh
        dg_ds = nubar * dnu_ds + dh_ds
        dg_dt = -nubar
        g_alpha[i - 1] = np.where(unstable, nubar * (-np.maximum(-nu_hat, 0.0)), 0.0)
        if P.N:
            g_gamma = g_gamma + np.asarray((P.H[i] @ dg_dt.T).T) - np.asarray((P.G[i] @ dg_dnh.T).T) \
                + np.asarray((P.Q[i] @ dg_ds.T).T)
        rr, jj, hh, mm = _split_terms(P, D.beta, i)
        if len(rr):
            np.add.at(g_beta, (rr, mm), hh * dg_dt[rr, jj])
        a = dg_dnh
        if i in sources:
            a_saved[i] = a
    return g, Duals(g_alpha, g_beta, g_gamma, g_theta)


def theta_closed_form(P: Problem, D: Duals) -> List[np.ndarray]:
    """theta with theta * C = Lemma A.1's pi* at the duals D (R12's start);
    u / (u - l) where C = 0 and on stable neurons (where it is unused)."""
    _, T = evaluate(P, D, trace=True)
    out = []
    for i in range(1, P.L):
        nu_hat, s, lo, hi = T.nu_hat[i - 1], T.s[i - 1], T.lo[i - 1], T.hi[i - 1]
        unstable = (hi > 0) & (lo < 0)
        den_l = np.where(unstable, lo, -1.0)
        den_u = np.where(unstable, hi, 1.0)
        pi, _, _ = unstable_closed_form(nu_hat, s, den_l, den_u, D.alpha[i - 1])
        C = np.maximum(nu_hat, 0.0)
        out.append(np.where(C > 0, pi / np.where(C > 0, C, 1.0), den_u / (den_u - den_l)))
    return out


def project(P: Problem, D: Duals) -> None:
    """0 <= alpha <= 1, beta >= 0, gamma >= 0 (Theorem 3.1's domain)."""
    for a in D.alpha + (D.theta or []):
        np.clip(a, 0.0, 1.0, out=a)
    np.maximum(D.beta, 0.0, out=D.beta)
    np.maximum(D.gamma, 0.0, out=D.gamma)


def optimize(P: Problem, D: Duals, iters: int, lr_alpha: float, lr_beta: float, lr_gamma: float,
             optimizer: str = "pga", lr_decay: float = 1.0, adam_b1: float = 0.9,
             adam_b2: float = 0.999, adam_eps: float = 1e-8):
    """Gradient ascent on (alpha, beta, gamma) with projection after each step.

    'pga': x <- proj(x + lr_t * grad). 'adam': Adam (Kingma & Ba) ascent with
    moments 0.9 / 0.999 and eps 1e-8 (the paper names Adam but not its
    moments, App. C.1). lr_t = lr * lr_decay**t at iteration t = 0, 1, ...
    With D.theta set, theta (R12) is optimised too, at alpha's rate.
    Returns the bound at the final duals (one more evaluation) and the duals.
    """
    D = D.copy()
    if optimizer == "adam":
        m = Duals([np.zeros_like(a) for a in D.alpha], np.zeros_like(D.beta), np.zeros_like(D.gamma),
                  None if D.theta is None else [np.zeros_like(t) for t in D.theta])
        v = m.copy()
    for it in range(iters):
        _, G = gradient(P, D)
        f = lr_decay ** it
        lrs = (lr_alpha * f, lr_beta * f, lr_gamma * f)
        if optimizer == "pga":
            for a, ga in zip(D.alpha + (D.theta or []), G.alpha + (G.theta or [])):
                a += lrs[0] * ga
            D.beta += lrs[1] * G.beta
            D.gamma += lrs[2] * G.gamma
        else:
            tt = it + 1
            for a, ga, ma, va in zip(D.alpha + (D.theta or []), G.alpha + (G.theta or []),
                                     m.alpha + (m.theta or []), v.alpha + (v.theta or [])):
                adam_step(a, ga, ma, va, lrs[0], tt, adam_b1, adam_b2, adam_eps)
            adam_step(D.beta, G.beta, m.beta, v.beta, lrs[1], tt, adam_b1, adam_b2, adam_eps)
            adam_step(D.gamma, G.gamma, m.gamma, v.gamma, lrs[2], tt, adam_b1, adam_b2, adam_eps)
        project(P, D)
    return evaluate(P, D), D


def adam_step(x, gx, mx, vx, lr, t, b1, b2, eps):
    """One Adam ascent step in place (Kingma & Ba 2015, Algorithm 1), step number t >= 1.

    m <- b1 m + (1-b1) g; v <- b2 v + (1-b2) g^2; x <- x + lr m-hat / (sqrt(v-hat) + eps)
    with the bias corrections m-hat = m / (1 - b1^t), v-hat = v / (1 - b2^t).
    """
    mx *= b1
    mx += (1 - b1) * gx
    vx *= b2
    vx += (1 - b2) * gx * gx
    c1, c2 = 1.0 - b1 ** t, 1.0 - b2 ** t
    x += lr * (mx / c1) / (np.sqrt(vx / c2) + eps)


def crown_root_bounds(net, x_lo, x_hi, block: int = 512):
    """Root intermediate bounds l, u of every hidden layer (Sec. 2, Eq. 1: the
    method takes them from a bound propagation such as CROWN or IBP).

    Hidden layer 1: the interval image of the box under its affine map (W^(1),
    plus the shortcut of a skip from the input). Hidden layer i > 1: the
    network truncated after layer i's linear map, with spec rows +e_j and
    -e_j over its neurons, bounded by this module's Theorem 3.1 at the
    default duals (no cuts, no splits; R10's adaptive slope) over the bounds
    already found for the layers below: l_j = g(+e_j), u_j = -g(-e_j). That is
    CROWN. A skip connection into layer i (R11) stays in the truncated network,
    restricted to the same rows j (the identity shortcut becomes the selection
    of those rows).
    """
    layers = net.layers
    L = len(layers)
    dims = [layers[0].d_in] + [ly.d_out for ly in layers]

    def lin(ly):
        return (np.asarray(ly.W, np.float64) if ly.kind == DENSE else
                conv_matrix(np.asarray(ly.W, np.float64), ly.in_shape, ly.out_shape, ly.stride, ly.pad))
    mats = [lin(ly) for ly in layers]
    skip = [int(getattr(ly, "skip", 0)) for ly in layers]
    smap, bias = [], []
    for ly, s_ in zip(layers, skip):
        sc = getattr(ly, "shortcut", None) if s_ else None
        smap.append(None if sc is None else lin(sc))
        bias.append(np.asarray(ly.b, np.float64) + (np.asarray(sc.b, np.float64) if sc is not None else 0.0))

    def rows_of(M, idx):
        r = M[idx]
        return r.toarray() if sp.issparse(r) else r

    x_lo = np.asarray(x_lo, np.float64)
    x_hi = np.asarray(x_hi, np.float64)
    c0, r0 = (x_hi + x_lo) / 2, (x_hi - x_lo) / 2
    M1 = mats[0]
    if skip[0]:
        # layer 1 may only add the input itself (xhat^(0) = x)
        M1 = (M1.toarray() if sp.issparse(M1) else M1) + (np.eye(dims[0]) if smap[0] is None else
                                                         (smap[0].toarray() if sp.issparse(smap[0]) else smap[0]))
    z = np.asarray(M1 @ c0).ravel() + bias[0]
    rad = np.asarray(abs(M1) @ r0).ravel()
    lo, hi = [z - rad], [z + rad]
    for i in range(2, L):
        li, ui = np.empty(dims[i]), np.empty(dims[i])
        for a in range(0, dims[i], block):
            idx = np.arange(a, min(dims[i], a + block))
            n = len(idx)
            dt = dims[:i] + [n]
            s_i = skip[i - 1]
            last_map = None
            if s_i:
                last_map = (np.eye(dims[i])[idx] if smap[i - 1] is None else rows_of(smap[i - 1], idx))
            none = [sp.csr_matrix((0, d)) for d in dt[:-1]]
            P = Problem(i, dt, mats[:i - 1] + [rows_of(mats[i - 1], idx)], bias[:i - 1] + [bias[i - 1][idx]],
                        x_lo, x_hi, np.concatenate([np.eye(n), -np.eye(n)]), lo, hi,
                        [l[None, :] for l in lo], [h[None, :] for h in hi],
                        np.zeros(2, np.int64), np.zeros(0, np.int64), np.zeros(0, np.int64), np.zeros(0, np.int64),
                        0, none, list(none), list(none), np.zeros(0), skip[:i - 1] + [s_i],
                        smap[:i - 1] + [last_map])
            g = evaluate(P, default_duals(P))
            li[idx], ui[idx] = g[:n], -g[n:]
        lo.append(li)
        hi.append(ui)
    return lo, hi


# ----------------------------------------------------------------------------
# LP / MIP of the same relaxation (Eq. 2-10, Eq. 16), via SciPy HiGHS
# ----------------------------------------------------------------------------

def _lp_model(P: Problem, s: int, k: int, cut_d: Optional[np.ndarray] = None, with_cuts: bool = True):
    """Variables, constraints and objective of Eq. 16 for subdomain s, spec row k.

    Variables: x0, then per hidden layer i: x^(i), xhat^(i), z^(i). A skip
    connection adds -S xhat^(m) to its layer's equality rows (R11). Stable
    neurons keep their equalities (Eq. 9-10) and fixed z (R5); unstable ones
    get Eq. 4-7 and 0 <= z <= 1. Split rows are extra constraints
    (-x <= 0 for x >= 0, x <= 0 for x <= 0). The objective is
    c^T (W^(L) xhat^(L-1) + b^(L)), plus c^T S xhat^(m) when the last layer
    adds S xhat^(m).
    """
    dims = P.dims
    off = [0]
    off.append(dims[0])
    for i in range(1, P.L):
        off.append(off[-1] + 3 * dims[i])
    nvar = off[-1]

    def vx(i, j):
        return off[i] + j if i == 0 else off[i] + j

    def vxh(i, j):
        return off[i] + dims[i] + j

    def vz(i, j):
        return off[i] + 2 * dims[i] + j

    lb = np.full(nvar, -np.inf)
    ub = np.full(nvar, np.inf)
    integ = np.zeros(nvar, np.int8)
    lb[:dims[0]] = P.x_lo
    ub[:dims[0]] = P.x_hi
    Aeq_r, Aeq_c, Aeq_v, beq = [], [], [], []
    Aub_r, Aub_c, Aub_v, bub = [], [], [], []
    neq = [0]
    nub = [0]

    def eq(entries, rhs):
        for c, v in entries:
            Aeq_r.append(neq[0])
            Aeq_c.append(c)
            Aeq_v.append(v)
        beq.append(rhs)
        neq[0] += 1

    def le(entries, rhs):
        for c, v in entries:
            Aub_r.append(nub[0])
            Aub_c.append(c)
            Aub_v.append(v)
        bub.append(rhs)
        nub[0] += 1

    for i in range(1, P.L):
        Wi = P.Wm[i - 1]
        Wd = Wi.toarray() if sp.issparse(Wi) else Wi
        prev = (lambda j: vx(0, j)) if i == 1 else (lambda j, i=i: vxh(i - 1, j))
        m = P.skip[i - 1] - 1 if P.skip and P.skip[i - 1] else -1
        src = None if m < 0 else ((lambda j: vx(0, j)) if m == 0 else (lambda j, m=m: vxh(m, j)))
        Sk = P.skip_map[i - 1] if src is not None and P.skip_map else None
        Sd = None if Sk is None else (Sk.toarray() if sp.issparse(Sk) else Sk)
        lo = P.sub_lo[i - 1][s]
        hi = P.sub_hi[i - 1][s]
        for j in range(dims[i]):
            row = [(vx(i, j), 1.0)]
            nz = np.nonzero(Wd[j])[0]
            row += [(prev(q), -Wd[j, q]) for q in nz]
            if src is not None and Sd is None:
                row.append((src(j), -1.0))
            elif src is not None:
                row += [(src(q), -Sd[j, q]) for q in np.nonzero(Sd[j])[0]]
            eq(row, P.b[i - 1][j])
            if hi[j] <= 0:                       # inactive: xhat = 0, z = 0
                lb[vxh(i, j)] = ub[vxh(i, j)] = 0.0
                lb[vz(i, j)] = ub[vz(i, j)] = 0.0
            elif lo[j] >= 0:                     # active: xhat = x, z = 1
                eq([(vxh(i, j), 1.0), (vx(i, j), -1.0)], 0.0)
                lb[vz(i, j)] = ub[vz(i, j)] = 1.0
            else:                                # unstable: Eq. 4-7, 0 <= z <= 1
                lb[vxh(i, j)] = 0.0
                lb[vz(i, j)], ub[vz(i, j)] = 0.0, 1.0
                integ[vz(i, j)] = 1
                le([(vx(i, j), 1.0), (vxh(i, j), -1.0)], 0.0)
                le([(vxh(i, j), 1.0), (vz(i, j), -hi[j])], 0.0)
                le([(vxh(i, j), 1.0), (vx(i, j), -1.0), (vz(i, j), -lo[j])], -lo[j])
    for e in range(int(P.split_ptr[s]), int(P.split_ptr[s + 1])):
        i, j, sg = int(P.split_layer[e]), int(P.split_index[e]), int(P.split_sign[e])
        le([(vx(i, j), -float(sg))], 0.0)
    if with_cuts and P.N:
        dvec = P.d if cut_d is None else cut_d
        for kk in range(P.N):
            row = []
            for i in range(P.L):
                for mat, fn in ((P.H[i], vx), (P.G[i], vxh), (P.Q[i], vz)):
                    if i == 0 and fn is not vx:
                        continue
                    rw = mat.getrow(kk)
                    for j, v in zip(rw.indices, rw.data):
                        row.append((fn(i, int(j)), float(v)))
            if row:
                le(row, float(dvec[kk]))
            elif dvec[kk] < 0:
                le([(0, 0.0)], float(dvec[kk]))
    # objective c^T (W^(L) xhat^(L-1) + b^(L) [+ xhat^(m)])
    cvec = np.zeros(nvar)
    WL = P.Wm[P.L - 1]
    WLd = WL.toarray() if sp.issparse(WL) else WL
    coef = P.spec[k] @ WLd
    for j in range(dims[P.L - 1]):
        cvec[vxh(P.L - 1, j) if P.L > 1 else vx(0, j)] += coef[j]
    if P.skip and P.skip[P.L - 1]:
        m = P.skip[P.L - 1] - 1
        sc = _through_skip(P, P.L, P.spec[k][None, :])[0]       # c^T S
        for j in range(dims[m]):
            cvec[vxh(m, j) if m > 0 else vx(0, j)] += sc[j]
    const = float(P.spec[k] @ P.b[P.L - 1])
    Aeq = sp.csr_matrix((Aeq_v, (Aeq_r, Aeq_c)), shape=(neq[0], nvar)) if neq[0] else None
    Aub = sp.csr_matrix((Aub_v, (Aub_r, Aub_c)), shape=(nub[0], nvar)) if nub[0] else None
    return cvec, const, Aub, np.asarray(bub), Aeq, np.asarray(beq), lb, ub, integ, (vx, vxh, vz)


def lp_value(P: Problem, s: int, k: int, integral: bool = False, with_cuts: bool = True,
             cut_d: Optional[np.ndarray] = None):
    """Optimum of Eq. 16 (integral=False) or of the MIP with cuts (True).

    Returns None when the program is infeasible (possible with synthetic cuts
    combined with splits).
    """
    from scipy.optimize import linprog, milp, LinearConstraint, Bounds
    cvec, const, Aub, bub, Aeq, beq, lb, ub, integ, _ = _lp_model(P, s, k, cut_d, with_cuts)
    if not integral:
        res = linprog(cvec, A_ub=Aub, b_ub=bub if Aub is not None else None, A_eq=Aeq,
                      b_eq=beq if Aeq is not None else None, bounds=list(zip(lb, ub)), method="highs")
        if res.status == 2:
            return None
        assert res.status == 0, res.message
        return float(res.fun) + const
    cons = []
    if Aub is not None:
        cons.append(LinearConstraint(Aub, -np.inf, bub))
    if Aeq is not None:
        cons.append(LinearConstraint(Aeq, beq, beq))
    res = milp(cvec, constraints=cons, integrality=integ, bounds=Bounds(lb, ub))
    if res.status == 2:
        return None
    assert res.status == 0, res.message
    return float(res.fun) + const


def valid_cut_offsets(P: Problem) -> np.ndarray:
    """d_k = max of cut k's left-hand side over the root MIP (no cuts, no splits).

    Such cuts remove no integer-feasible point of the root problem, so they
    are valid cutting planes for every subdomain (Sec. 3.2).
    """
    from scipy.optimize import milp, LinearConstraint, Bounds
    saved = (P.split_ptr, P.sub_lo, P.sub_hi)
    P.split_ptr = np.zeros(2, np.int64)
    P.sub_lo = [r[None, :] for r in P.root_lo]
    P.sub_hi = [r[None, :] for r in P.root_hi]
    try:
        _, _, Aub, bub, Aeq, beq, lb, ub, integ, (vx, vxh, vz) = _lp_model(P, 0, 0, with_cuts=False)
        out = np.zeros(P.N)
        for kk in range(P.N):
            cvec = np.zeros(len(lb))
            for i in range(P.L):
                for mat, fn in ((P.H[i], vx), (P.G[i], vxh), (P.Q[i], vz)):
                    if i == 0 and fn is not vx:
                        continue
                    rw = mat.getrow(kk)
                    for j, v in zip(rw.indices, rw.data):
                        cvec[fn(i, int(j))] -= float(v)     # maximise
            cons = []
            if Aub is not None:
                cons.append(LinearConstraint(Aub, -np.inf, bub))
            if Aeq is not None:
                cons.append(LinearConstraint(Aeq, beq, beq))
            res = milp(cvec, constraints=cons, integrality=integ, bounds=Bounds(lb, ub))
            assert res.status == 0, res.message
            out[kk] = -float(res.fun)
        return out
    finally:
        P.split_ptr, P.sub_lo, P.sub_hi = saved
