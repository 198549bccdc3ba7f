"""Seeded synthetic verification instances (inputs only).

This module produces the *inputs* of the bounding problem of GCP-CROWN
(Zhang et al., arXiv 2208.05740): ReLU networks (Sec. 2, network model),
an L-infinity input box (Sec. 2, Eq. 1), spec rows c = e_y - e_j folded in as
the last linear layer (Sec. 2), sound intermediate pre-activation bounds
l <= x <= u (Sec. 2, "we assume that we know sound pre-activation bounds"),
branch-and-bound subdomains given as neuron split sets (Sec. 3.1,
connection to beta-CROWN; App. B), and general cutting planes
sum_i H x + G xhat + Q z <= d (Sec. 3.1, Eq. 15).

It holds none of the bound-propagation arithmetic of the method: the
intermediate bounds are interval bounds (IBP, which Sec. 2 names as one
admissible source of l and u), the cut offsets d come from plain network
forward passes at sampled inputs, and everything else is random draws.
Both the FP64 oracle and the CUDA library consume these arrays; neither
imports the other.

Shapes follow Table 4 of the paper (batch sizes 1024-4096), its cut case
study (App. C.2: hundreds to thousands of cuts, almost all touching a ReLU
indicator z and an input variable, most spanning several layers) and the
five workload descriptions this library is measured on. Seeds: workload k
uses ``SEED_BASE + k`` with NumPy's PCG64.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional, Sequence

import numpy as np

SEED_BASE = 2208057400

KIND_X, KIND_XHAT, KIND_Z = 0, 1, 2
DENSE, CONV2D = 0, 1


@dataclasses.dataclass
class Layer:
    """One affine layer x_out = W x_in + b (dense or 2-D convolution).

    dense : W is [d_out, d_in] row-major.
    conv2d: W is [c_out, c_in, k, k] (OIHW), input/output tensors are CHW
            flattened; ``b`` is always the full per-output-element bias of
            length d_out (a per-channel bias is broadcast over positions).
    """
    kind: int
    W: np.ndarray
    b: np.ndarray
    in_shape: tuple
    out_shape: tuple
    stride: int = 1
    pad: int = 0
    skip: int = 0      # 0: none; s >= 1: the layer adds xhat^(s-1) (s = 1: the input x) to W x + b
    # the map applied to xhat^(s-1) before it is added (a projection shortcut,
    # S xhat^(s-1) + b_S); None: the identity
    shortcut: Optional["Layer"] = None

    @property
    def d_in(self) -> int:
        return int(np.prod(self.in_shape))

    @property
    def d_out(self) -> int:
        return int(np.prod(self.out_shape))


@dataclasses.dataclass
class Network:
    layers: List[Layer]

    @property
    def L(self) -> int:
        return len(self.layers)

    @property
    def dims(self) -> List[int]:
        return [self.layers[0].d_in] + [ly.d_out for ly in self.layers]


@dataclasses.dataclass
class Subdomains:
    """Split sets in CSR form: subdomain s owns entries ptr[s]:ptr[s+1].

    layer is 1..L-1, index is the neuron, sign +1 means x >= 0 and -1 means
    x <= 0 (the two branches of a ReLU split, App. B).
    """
    ptr: np.ndarray      # int32 [S+1]
    layer: np.ndarray    # int16 [nnz]
    index: np.ndarray    # int32 [nnz]
    sign: np.ndarray     # int8  [nnz]

    @property
    def n(self) -> int:
        return len(self.ptr) - 1

    @property
    def max_splits(self) -> int:
        return int(np.max(np.diff(self.ptr))) if self.n else 0


@dataclasses.dataclass
class Cuts:
    """N cuts in CSR form by cut: sum_e coef[e] * var(layer, kind, index) <= d.

    layer 0 is the input x (kind must be X); layers 1..L-1 are hidden.
    """
    ptr: np.ndarray      # int64 [N+1]
    layer: np.ndarray    # int16 [nnz]
    kind: np.ndarray     # int8  [nnz]
    index: np.ndarray    # int32 [nnz]
    coef: np.ndarray     # float64 [nnz]
    d: np.ndarray        # float64 [N]

    @property
    def n(self) -> int:
        return len(self.ptr) - 1

    @staticmethod
    def empty() -> "Cuts":
        return Cuts(np.zeros(1, np.int64), np.zeros(0, np.int16), np.zeros(0, np.int8),
                    np.zeros(0, np.int32), np.zeros(0, np.float64), np.zeros(0, np.float64))


@dataclasses.dataclass
class Instance:
    name: str
    net: Network
    x_lo: np.ndarray          # [d0]
    x_hi: np.ndarray          # [d0]
    spec: np.ndarray          # [K, d_L]
    inter_lo: List[np.ndarray]  # per hidden layer 1..L-1
    inter_hi: List[np.ndarray]
    sub: Subdomains
    cuts: Cuts

    @property
    def n_rows(self) -> int:
        return self.sub.n * self.spec.shape[0]


# ----------------------------------------------------------------------------
# network construction and plain forward evaluation
# ----------------------------------------------------------------------------

def conv2d_forward(x: np.ndarray, W: np.ndarray, stride: int, pad: int) -> np.ndarray:
    """Plain cross-correlation, x [B, C, H, W] -> [B, O, Ho, Wo] (no bias)."""
    B, C, H, Wd = x.shape
    O, C2, k, k2 = W.shape
    assert C == C2 and k == k2
    Ho = (H + 2 * pad - k) // stride + 1
    Wo = (Wd + 2 * pad - k) // stride + 1
    xp = np.zeros((B, C, H + 2 * pad, Wd + 2 * pad), dtype=x.dtype)
    xp[:, :, pad:pad + H, pad:pad + Wd] = x
    out = np.zeros((B, O, Ho, Wo), dtype=np.result_type(x, W))
    for kh in range(k):
        for kw in range(k):
            patch = xp[:, :, kh:kh + stride * (Ho - 1) + 1:stride, kw:kw + stride * (Wo - 1) + 1:stride]
            out += np.einsum("bchw,oc->bohw", patch, W[:, :, kh, kw], optimize=True)
    return out


def layer_apply(ly: Layer, x: np.ndarray, W: Optional[np.ndarray] = None) -> np.ndarray:
    """x [B, d_in] -> W x (no bias), with an optional replacement weight."""
    Wm = ly.W if W is None else W
    if ly.kind == DENSE:
        return x @ Wm.T
    B = x.shape[0]
    y = conv2d_forward(x.reshape((B,) + tuple(ly.in_shape)), Wm, ly.stride, ly.pad)
    return y.reshape(B, -1)


def forward_all(net: Network, x: np.ndarray):
    """Return pre-activations [x^(1..L)] for a batch of inputs x [B, d0]."""
    pre = []
    post = [x]            # xhat^(0) = x, xhat^(i) = ReLU(x^(i))
    for i, ly in enumerate(net.layers):
        z = layer_apply(ly, post[-1]) + ly.b[None, :]
        if ly.skip:
            src = post[ly.skip - 1]
            z = z + (src if ly.shortcut is None else layer_apply(ly.shortcut, src) + ly.shortcut.b[None, :])
        pre.append(z)
        post.append(np.maximum(z, 0.0))
    return pre


def make_mlp(rng, dims: Sequence[int]) -> Network:
    layers = []
    for i in range(1, len(dims)):
        W = rng.normal(0.0, math.sqrt(1.0 / dims[i - 1]), size=(dims[i], dims[i - 1]))
        b = rng.normal(0.0, math.sqrt(0.1), size=dims[i])
        layers.append(Layer(DENSE, W, b, (dims[i - 1],), (dims[i],)))
    return Network(layers)


def make_conv(rng, in_shape, c_out, k, stride, pad) -> Layer:
    c_in, H, Wd = in_shape
    Ho = (H + 2 * pad - k) // stride + 1
    Wo = (Wd + 2 * pad - k) // stride + 1
    fan_in = c_in * k * k
    W = rng.normal(0.0, math.sqrt(1.0 / fan_in), size=(c_out, c_in, k, k))
    bc = rng.normal(0.0, math.sqrt(0.1), size=c_out)
    b = np.repeat(bc, Ho * Wo)
    return Layer(CONV2D, W, b, (c_in, H, Wd), (c_out, Ho, Wo), stride, pad)


def make_cnn(rng) -> Network:
    """3x32x32 -> conv32 3x3 s2 p1 -> conv64 3x3 s2 p1 -> FC512 -> FC10."""
    c1 = make_conv(rng, (3, 32, 32), 32, 3, 2, 1)
    c2 = make_conv(rng, c1.out_shape, 64, 3, 2, 1)
    d2 = c2.d_out
    W3 = rng.normal(0.0, math.sqrt(1.0 / d2), size=(512, d2))
    b3 = rng.normal(0.0, math.sqrt(0.1), size=512)
    W4 = rng.normal(0.0, math.sqrt(1.0 / 512), size=(10, 512))
    b4 = rng.normal(0.0, math.sqrt(0.1), size=10)
    return Network([c1, c2, Layer(DENSE, W3, b3, (d2,), (512,)), Layer(DENSE, W4, b4, (512,), (10,))])


# ----------------------------------------------------------------------------
# input region, spec rows, interval bounds
# ----------------------------------------------------------------------------

def spec_rows(net: Network, x0: np.ndarray, n_rows: int) -> np.ndarray:
    """Rows e_y - e_j with y = argmax f(x0), j != y, for the first n_rows j."""
    out = forward_all(net, x0[None, :])[-1][0]
    y = int(np.argmax(out))
    dL = out.shape[0]
    others = [j for j in range(dL) if j != y][:n_rows]
    C = np.zeros((len(others), dL))
    for r, j in enumerate(others):
        C[r, y] = 1.0
        C[r, j] = -1.0
    return C


def interval_bounds(net: Network, x_lo: np.ndarray, x_hi: np.ndarray):
    """Interval (IBP) pre-activation bounds for hidden layers 1..L-1."""
    c = 0.5 * (x_lo + x_hi)
    r = 0.5 * (x_hi - x_lo)
    cs, rs = [c], [r]     # centre and radius of xhat^(0..)
    lo_list, hi_list = [], []
    for i, ly in enumerate(net.layers[:-1]):
        cc = layer_apply(ly, c[None, :])[0] + ly.b
        rr = layer_apply(ly, r[None, :], np.abs(ly.W))[0]
        if ly.skip and ly.shortcut is None:
            cc = cc + cs[ly.skip - 1]
            rr = rr + rs[ly.skip - 1]
        elif ly.skip:
            sc = ly.shortcut
            cc = cc + layer_apply(sc, cs[ly.skip - 1][None, :])[0] + sc.b
            rr = rr + layer_apply(sc, rs[ly.skip - 1][None, :], np.abs(sc.W))[0]
        lo, hi = cc - rr, cc + rr
        lo_list.append(lo)
        hi_list.append(hi)
        c = 0.5 * (np.maximum(lo, 0) + np.maximum(hi, 0))
        r = 0.5 * (np.maximum(hi, 0) - np.maximum(lo, 0))
        cs.append(c)
        rs.append(r)
    return lo_list, hi_list


# ----------------------------------------------------------------------------
# subdomains and cuts
# ----------------------------------------------------------------------------

def make_subdomains(rng, inter_lo, inter_hi, n_sub: int, min_splits: int, max_splits: int) -> Subdomains:
    """Each subdomain splits distinct root-unstable neurons with random sides."""
    unstable = [(i + 1, j) for i, (lo, hi) in enumerate(zip(inter_lo, inter_hi))
                for j in np.nonzero((lo < 0) & (hi > 0))[0]]
    ptr = [0]
    lay, idx, sgn = [], [], []
    for _ in range(n_sub):
        k = int(rng.integers(min_splits, max_splits + 1)) if max_splits > 0 else 0
        k = min(k, len(unstable))
        if k:
            pick = rng.choice(len(unstable), size=k, replace=False)
            for p in pick:
                lay.append(unstable[p][0])
                idx.append(unstable[p][1])
                sgn.append(1 if rng.random() < 0.5 else -1)
        ptr.append(len(lay))
    return Subdomains(np.asarray(ptr, np.int32), np.asarray(lay, np.int16),
                      np.asarray(idx, np.int32), np.asarray(sgn, np.int8))


def sample_box(rng, x_lo, x_hi, n):
    return x_lo[None, :] + (x_hi - x_lo)[None, :] * rng.random((n, x_lo.shape[0]))


def make_cuts(rng, net: Network, inter_lo, inter_hi, x_lo, x_hi, n_cuts: int,
              min_vars: int, max_vars: int, *, hidden_only: bool = False,
              span_layers: bool = False, need_z: bool = False,
              p_input: float = 0.0, n_samples: int = 64) -> Cuts:
    """Random sparse cuts whose offset d makes them hold at n_samples points.

    Each variable is (layer, kind, index); z variables are drawn among the
    root-unstable neurons of their layer (the MIP has z only there). d is the
    maximum of the cut's left-hand side over n_samples box samples evaluated
    at (x, relu(x), z = 1[x > 0]).
    """
    if n_cuts == 0:
        return Cuts.empty()
    L = net.L
    hidden = list(range(1, L))
    xs = sample_box(rng, x_lo, x_hi, n_samples)
    pre = forward_all(net, xs)
    unst = {i: np.nonzero((inter_lo[i - 1] < 0) & (inter_hi[i - 1] > 0))[0] for i in hidden}
    z_layers = [i for i in hidden if len(unst[i]) > 0]
    ptr = [0]
    lay, knd, idx, cf, dd = [], [], [], [], []
    for _ in range(n_cuts):
        m = int(rng.integers(min_vars, max_vars + 1))
        vars_ = []
        if need_z and z_layers:
            i = int(rng.choice(z_layers))
            vars_.append((i, KIND_Z, int(rng.choice(unst[i]))))
        if (not hidden_only) and rng.random() < p_input:
            vars_.append((0, KIND_X, int(rng.integers(0, net.dims[0]))))
        while len(vars_) < m:
            i = int(rng.choice(hidden))
            kind = int(rng.integers(0, 3))
            if kind == KIND_Z:
                if len(unst[i]) == 0:
                    kind = KIND_XHAT
                else:
                    vars_.append((i, kind, int(rng.choice(unst[i]))))
                    continue
            vars_.append((i, kind, int(rng.integers(0, net.dims[i]))))
        if span_layers and len({v[0] for v in vars_}) < 2 and len(vars_) >= 2:
            i0 = vars_[0][0]
            others = [i for i in hidden if i != i0] or hidden
            i = int(rng.choice(others))
            v = vars_[-1]
            if v[1] == KIND_Z and len(unst[i]) > 0:
                vars_[-1] = (i, KIND_Z, int(rng.choice(unst[i])))
            else:
                vars_[-1] = (i, KIND_XHAT if v[1] == KIND_Z else v[1], int(rng.integers(0, net.dims[i])))
        # merge duplicate variables
        seen = {}
        for v in vars_:
            seen[v] = seen.get(v, 0.0) + float(rng.normal())
        lhs = np.zeros(n_samples)
        for (i, kind, j), c in seen.items():
            if i == 0:
                val = xs[:, j]
            else:
                xv = pre[i - 1][:, j]
                val = xv if kind == KIND_X else (np.maximum(xv, 0) if kind == KIND_XHAT else (xv > 0).astype(float))
            lhs += c * val
            lay.append(i)
            knd.append(kind)
            idx.append(j)
            cf.append(c)
        dd.append(float(np.max(lhs)))
        ptr.append(len(lay))
    return Cuts(np.asarray(ptr, np.int64), np.asarray(lay, np.int16), np.asarray(knd, np.int8),
                np.asarray(idx, np.int32), np.asarray(cf, np.float64), np.asarray(dd, np.float64))


# ----------------------------------------------------------------------------
# the five workloads
# ----------------------------------------------------------------------------

def _finish(name, rng, net, x0, eps, n_spec, n_sub, split_rng, cut_args, root_bounds=None) -> Instance:
    """The instance around a network: box, spec rows, root intermediate bounds,
    subdomains (splits of root-unstable neurons) and cuts.

    root_bounds: None for interval bounds, else a callable (net, x_lo, x_hi) ->
    (lo, hi) supplied by the caller (e.g. CROWN bounds computed by the library
    or by the oracle); the random stream is the same either way, so the same
    seed gives the same network, box and spec whatever bounds are used.
    """
    x_lo, x_hi = x0 - eps, x0 + eps
    C = spec_rows(net, x0, n_spec)
    if root_bounds is None:
        lo, hi = interval_bounds(net, x_lo, x_hi)
    else:
        lo, hi = root_bounds(net, x_lo, x_hi)
        lo = [np.asarray(v, np.float64) for v in lo]
        hi = [np.asarray(v, np.float64) for v in hi]
    sub = make_subdomains(rng, lo, hi, n_sub, *split_rng)
    cuts = make_cuts(rng, net, lo, hi, x_lo, x_hi, **cut_args)
    return Instance(name, net, x_lo, x_hi, C, lo, hi, sub, cuts)


def mlp_small(seed: int = SEED_BASE + 1, n_sub: int = 4, n_cuts: int = 8, root_bounds=None) -> Instance:
    """MLP 8-16-16-3, eps 0.1, 2 spec rows, 0-2 splits, 8 hidden-layer cuts of 2-4 vars."""
    rng = np.random.default_rng(seed)
    net = make_mlp(rng, [8, 16, 16, 3])
    x0 = rng.random(8)
    return _finish("mlp_8_16_16_3", rng, net, x0, 0.1, 2, n_sub, (0, 2),
                   dict(n_cuts=n_cuts, min_vars=2, max_vars=4, hidden_only=True), root_bounds)


def mlp_256x6(seed: int = SEED_BASE + 2, n_sub: int = 1024, n_cuts: int = 200, root_bounds=None) -> Instance:
    """MLP 784-256x6-10, eps 0.015, 9 spec rows, 1-8 splits, 200 cuts of 2-8 vars."""
    rng = np.random.default_rng(seed)
    net = make_mlp(rng, [784] + [256] * 6 + [10])
    x0 = rng.random(784)
    return _finish("mlp_784_256x6_10", rng, net, x0, 0.015, 9, n_sub, (1, 8),
                   dict(n_cuts=n_cuts, min_vars=2, max_vars=8, span_layers=True, need_z=True, p_input=0.99),
                   root_bounds)


def cnn_cifar(seed: int = SEED_BASE + 3, n_sub: int = 4096, n_cuts: int = 1000, root_bounds=None) -> Instance:
    """CNN 3x32x32 -> conv32 s2 -> conv64 s2 -> FC512 -> FC10, eps 2/255, 9 rows."""
    rng = np.random.default_rng(seed)
    net = make_cnn(rng)
    x0 = rng.random(3 * 32 * 32)
    return _finish("cnn_3x32x32_c32_c64_fc512_fc10", rng, net, x0, 2.0 / 255.0, 9, n_sub, (1, 12),
                   dict(n_cuts=n_cuts, min_vars=2, max_vars=16, span_layers=True, need_z=True, p_input=0.99),
                   root_bounds)


def mlp_residual(seed: int = SEED_BASE + 6, width: int = 16, d0: int = 8, blocks: int = 2, d_out: int = 3,
                 eps: float = 0.1, n_spec: int = 2, n_sub: int = 4, n_cuts: int = 8, max_splits: int = 2) -> Instance:
    """Residual MLP: d0 -> width, then `blocks` blocks of two layers whose
    second layer adds the block input (xhat two layers back) to its
    pre-activation, then width -> d_out. Weights N(0, 1/fan_in), biases
    N(0, 0.1); the skip-carrying layers are scaled by 1/2 (residual nets keep
    the block's branch small)."""
    rng = np.random.default_rng(seed)
    dims = [d0] + [width] * (2 * blocks + 1) + [d_out]
    net = make_mlp(rng, dims)
    for q in range(blocks):
        i = 3 + 2 * q                  # 1-based index of the block's second layer
        ly = net.layers[i - 1]
        net.layers[i - 1] = dataclasses.replace(ly, W=0.5 * ly.W, skip=i - 1)   # adds xhat^(i-2)
    x0 = rng.random(d0)
    return _finish(f"mlp_residual_{d0}_{width}x{2 * blocks + 1}_{d_out}", rng, net, x0, eps, n_spec, n_sub,
                   (0, max_splits), dict(n_cuts=n_cuts, min_vars=2, max_vars=4, hidden_only=True))


def make_resnet(rng, hw: int = 32, stem: int = 8, blocks=((16, 2), (16, 1)), fc: int = 100,
                d_out: int = 10) -> Network:
    """Residual CNN shaped like the residual CIFAR models (App. C.1):
    3 x hw x hw -> conv stem 3x3 s2 p1 -> residual blocks -> FC fc -> FC d_out.
    A block (c, stride) is conv c 3x3 s(stride) p1, then conv c 3x3 s1 p1
    whose output adds the block input: through the identity when channels and
    size are unchanged, else through a 1x1 convolution with the block's stride
    (ResBlock(a, b)). The second conv of a block is scaled by 1/2. The
    defaults give the resnet2b shape (FC 1024 -> 100); stem 16 with blocks
    ((32, 2), (32, 2)) gives the resnet4b shape (FC 512 -> 100)."""
    layers = [make_conv(rng, (3, hw, hw), stem, 3, 2, 1)]
    shape = layers[0].out_shape
    for c, stride in blocks:
        n = len(layers)                       # the block adds xhat^(n), its input
        first = make_conv(rng, shape, c, 3, stride, 1)
        second = make_conv(rng, first.out_shape, c, 3, 1, 1)
        sc = None
        if c != shape[0] or stride != 1:
            sc = make_conv(rng, shape, c, 1, stride, 0)
            sc = dataclasses.replace(sc, b=np.zeros(sc.d_out))      # one bias per output (the second conv's)
        layers += [first, dataclasses.replace(second, W=0.5 * second.W, skip=n + 1, shortcut=sc)]
        shape = second.out_shape
    d = int(np.prod(shape))
    W1 = rng.normal(0.0, math.sqrt(1.0 / d), size=(fc, d))
    b1 = rng.normal(0.0, math.sqrt(0.1), size=fc)
    W2 = rng.normal(0.0, math.sqrt(1.0 / fc), size=(d_out, fc))
    b2 = rng.normal(0.0, math.sqrt(0.1), size=d_out)
    return Network(layers + [Layer(DENSE, W1, b1, (d,), (fc,)), Layer(DENSE, W2, b2, (fc,), (d_out,))])


def cnn_resnet(seed: int = SEED_BASE + 7, hw: int = 32, stem: int = 8, blocks=((16, 2), (16, 1)), fc: int = 100,
               eps: float = 2.0 / 255.0, n_spec: int = 9, n_sub: int = 2048, n_cuts: int = 500,
               max_splits: int = 12, root_bounds=None) -> Instance:
    """Residual CNN (make_resnet; resnet2b shape by default), eps 2/255, 9 spec rows, 1-12 splits, cuts of
    2-16 variables."""
    rng = np.random.default_rng(seed)
    net = make_resnet(rng, hw, stem, blocks, fc)
    x0 = rng.random(3 * hw * hw)
    tag = "_".join(f"b{c}s{st}" for c, st in blocks)
    return _finish(f"resnet_3x{hw}x{hw}_c{stem}_{tag}_fc{fc}_fc10", rng, net, x0, eps, n_spec, n_sub,
                   (1, max_splits), dict(n_cuts=n_cuts, min_vars=2, max_vars=16, span_layers=True, need_z=True,
                                         p_input=0.99), root_bounds)


def mlp_1024x4_queries(seed: int = SEED_BASE + 4, sizes=(64, 700, 2048), cut_counts=(0, 500, 3000)):
    """Three queries on one MLP 784-1024x4-10 with different batch and cut counts."""
    rng = np.random.default_rng(seed)
    net = make_mlp(rng, [784] + [1024] * 4 + [10])
    x0 = rng.random(784)
    x_lo, x_hi = x0 - 0.015, x0 + 0.015
    C = spec_rows(net, x0, 9)
    lo, hi = interval_bounds(net, x_lo, x_hi)
    out = []
    for q, (ns, nc) in enumerate(zip(sizes, cut_counts)):
        sub = make_subdomains(rng, lo, hi, ns, 0, 8)
        cuts = make_cuts(rng, net, lo, hi, x_lo, x_hi, nc, 2, 8, span_layers=True, need_z=True, p_input=0.99)
        out.append(Instance(f"mlp_784_1024x4_10_q{q}", net, x_lo, x_hi, C, lo, hi, sub, cuts))
    return out


def restrict(inst: Instance, n_sub: int) -> Instance:
    """The first n_sub subdomains of an instance (same network, spec and cuts)."""
    s = inst.sub
    e = int(s.ptr[n_sub])
    sub = Subdomains(s.ptr[:n_sub + 1].copy(), s.layer[:e].copy(), s.index[:e].copy(), s.sign[:e].copy())
    return dataclasses.replace(inst, sub=sub)


def child_subdomains(rng, inst: Instance, sub: Subdomains) -> Subdomains:
    """One branch-and-bound child per subdomain: one more split on a random
    root-unstable neuron not yet split in it, on a random side (App. B)."""
    unstable = [(i + 1, j) for i, (lo, hi) in enumerate(zip(inst.inter_lo, inst.inter_hi))
                for j in np.nonzero((lo < 0) & (hi > 0))[0]]
    ptr = [0]
    lay, idx, sgn = [], [], []
    for s in range(sub.n):
        a, b = int(sub.ptr[s]), int(sub.ptr[s + 1])
        have = set(zip(sub.layer[a:b].tolist(), sub.index[a:b].tolist()))
        lay += sub.layer[a:b].tolist()
        idx += sub.index[a:b].tolist()
        sgn += sub.sign[a:b].tolist()
        free = [u for u in unstable if u not in have]
        if free:
            u = free[int(rng.integers(0, len(free)))]
            lay.append(u[0])
            idx.append(u[1])
            sgn.append(1 if rng.random() < 0.5 else -1)
        ptr.append(len(lay))
    return Subdomains(np.asarray(ptr, np.int32), np.asarray(lay, np.int16),
                      np.asarray(idx, np.int32), np.asarray(sgn, np.int8))


def random_duals(rng, inst: Instance, scale_beta=0.5, scale_gamma=0.5):
    """Random feasible duals: alpha in [0,1] per hidden neuron, beta, gamma >= 0."""
    R = inst.n_rows
    alpha = [rng.random((R, d)) for d in inst.net.dims[1:-1]]
    beta = scale_beta * rng.random((R, max(inst.sub.max_splits, 0)))
    gamma = scale_gamma * rng.random((R, inst.cuts.n))
    return alpha, beta, gamma
