"""Python binding of libgcp (the C ABI in include/gcp.h).

Argument marshalling only: every step of the bound, its gradient, the dual
updates and the certification runs in the CUDA kernels of libgcp.so. The
library must have been built (``paper_2208_05740_gb300.build.build()``);
importing the binding without it raises, there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libgcp.so")

GCP_OK, GCP_PENDING = 0, 1
STATUS = {0: "GCP_OK", 1: "GCP_PENDING", -1: "GCP_EINVAL", -2: "GCP_ENOMEM", -3: "GCP_ECUDA",
          -4: "GCP_ETIMEOUT", -5: "GCP_EBUDGET", -6: "GCP_ENOTFOUND", -7: "GCP_EDEVICE"}
GCP_DENSE, GCP_CONV2D = 0, 1
GCP_FP64, GCP_FP32, GCP_BF16 = 0, 1, 2
GCP_PGA, GCP_ADAM = 0, 1

EXPORTED = ["gcp_create", "gcp_destroy", "gcp_last_error", "gcp_set_stream", "gcp_mem_used", "gcp_init_net",
            "gcp_intermediate_bounds", "gcp_intermediate_bounds_cuts", "gcp_bab_verify", "gcp_bab_verify_labels",
            "gcp_add_cuts", "gcp_duals_create", "gcp_duals_create_multi", "gcp_duals_shape", "gcp_duals_export", "gcp_duals_import",
            "gcp_duals_free", "gcp_duals_theta", "gcp_bound_batch", "gcp_grad_batch", "gcp_optimize_batch", "gcp_bound_device",
            "gcp_branch_picks",
            "gcp_grad_device", "gcp_bound_dense_noalloc", "gcp_selftest_gemm", "gcp_selftest_gemm_f64", "gcp_profile_start", "gcp_profile_stop", "gcp_profile_repeat", "gcp_profile_query", "gcp_profile_report",
            "gcp_serve_start", "gcp_serve_submit", "gcp_serve_poll", "gcp_serve_wait",
            "gcp_serve_final", "gcp_serve_stop"]


class GCPError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class LayerDesc(C.Structure):
    pass


LayerDesc._fields_ = [("kind", C.c_int32), ("d_in", C.c_int32), ("d_out", C.c_int32), ("c_in", C.c_int32),
                      ("h_in", C.c_int32), ("w_in", C.c_int32), ("c_out", C.c_int32), ("h_out", C.c_int32),
                      ("w_out", C.c_int32), ("k", C.c_int32), ("stride", C.c_int32), ("pad", C.c_int32),
                      ("W", C.POINTER(C.c_double)), ("b", C.POINTER(C.c_double)), ("skip", C.c_int32),
                      ("shortcut", C.POINTER(LayerDesc))]


class Subdomains(C.Structure):
    _fields_ = [("n_sub", C.c_int32), ("split_ptr", C.POINTER(C.c_int32)), ("split_layer", C.POINTER(C.c_int16)),
                ("split_index", C.POINTER(C.c_int32)), ("split_sign", C.POINTER(C.c_int8))]


class OptParams(C.Structure):
    _fields_ = [("iters", C.c_int32), ("optimizer", C.c_int32), ("prec", C.c_int32), ("certify", C.c_int32),
                ("lr_alpha", C.c_double), ("lr_beta", C.c_double), ("lr_gamma", C.c_double),
                ("lr_decay", C.c_double), ("opt_pi", C.c_int32)]


class BabParams(C.Structure):
    _fields_ = [("batch", C.c_int32), ("max_rounds", C.c_int32), ("max_domains", C.c_int64),
                ("timeout_s", C.c_double), ("p", OptParams), ("branching", C.c_int32)]


class BabResult(C.Structure):
    _fields_ = [("verified", C.c_int32), ("rounds", C.c_int32), ("domains_bounded", C.c_int64),
                ("domains_verified", C.c_int64), ("domains_left", C.c_int64), ("min_bound", C.c_double),
                ("time_ms", C.c_double)]


class Request(C.Structure):
    _fields_ = [("net_id", C.c_int32), ("cutset_id", C.c_int32), ("rounds", C.c_int32), ("seed", C.c_uint64),
                ("sub", Subdomains), ("p", OptParams), ("keep_final", C.c_int32)]


class Result(C.Structure):
    _fields_ = [("status", C.c_int32), ("rows", C.c_int32), ("certified", C.POINTER(C.c_double)),
                ("min_certified", C.c_double), ("latency_ms", C.c_double), ("max_err_vs_fp64", C.c_double),
                ("max_rel_err_vs_fp64", C.c_double)]


class Final(C.Structure):
    _fields_ = [("n_sub", C.c_int32), ("rows", C.c_int32), ("n_alpha", C.c_int32), ("max_splits", C.c_int32),
                ("n_cuts", C.c_int32), ("n_split_entries", C.c_int64), ("split_ptr", C.POINTER(C.c_int32)),
                ("split_layer", C.POINTER(C.c_int16)), ("split_index", C.POINTER(C.c_int32)),
                ("split_sign", C.POINTER(C.c_int8)), ("alpha", C.POINTER(C.c_float)), ("beta", C.POINTER(C.c_float)),
                ("gamma", C.POINTER(C.c_float))]


_lib = None


def lib():
    """Load libgcp.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with paper_2208_05740_gb300.build.build()")
        L = C.CDLL(LIB_PATH)
        P, I32, I64, U64 = C.c_void_p, C.c_int32, C.c_int64, C.c_uint64
        pd = C.POINTER(C.c_double)
        sig = {
            "gcp_create": [C.POINTER(P), I32, U64],
            "gcp_destroy": [P],
            "gcp_set_stream": [P, P],
            "gcp_mem_used": [P, C.POINTER(U64)],
            "gcp_init_net": [P, C.POINTER(LayerDesc), I32, pd, pd, pd, I32, pd, pd, C.POINTER(I32)],
            "gcp_add_cuts": [P, I32, I32, C.POINTER(I64), C.POINTER(C.c_int16), C.POINTER(C.c_int8),
                             C.POINTER(I32), pd, pd, C.POINTER(I32), C.POINTER(I32)],
            "gcp_duals_create": [P, I32, I32, C.POINTER(Subdomains), I32, C.POINTER(P)],
            "gcp_duals_create_multi": [P, I32, I32, C.POINTER(I32), C.POINTER(Subdomains), I32, C.POINTER(P)],
            "gcp_duals_shape": [P, P, C.POINTER(I64), C.POINTER(I64), C.POINTER(I32), C.POINTER(I32)],
            "gcp_duals_export": [P, P, pd, pd, pd],
            "gcp_duals_import": [P, P, pd, pd, pd],
            "gcp_duals_free": [P, P],
            "gcp_duals_theta": [P, P, pd, pd],
            "gcp_bound_batch": [P, P, I32, I32, pd, pd],
            "gcp_grad_batch": [P, P, I32, pd, pd, pd, pd],
            "gcp_branch_picks": [P, P, I32, C.POINTER(I32), C.POINTER(I32)],
            "gcp_optimize_batch": [P, P, C.POINTER(OptParams), pd, pd, pd],
            "gcp_intermediate_bounds": [P, C.POINTER(LayerDesc), I32, pd, pd, C.POINTER(OptParams), pd, pd],
            "gcp_intermediate_bounds_cuts": [P, C.POINTER(LayerDesc), I32, pd, pd, C.POINTER(OptParams), I32,
                                             C.POINTER(I64), C.POINTER(C.c_int16), C.POINTER(C.c_int8),
                                             C.POINTER(I32), pd, pd, pd, pd],
            "gcp_bab_verify": [P, I32, I32, C.POINTER(BabParams), C.POINTER(BabResult)],
            "gcp_bab_verify_labels": [P, I32, I32, C.POINTER(BabParams), I32, C.POINTER(I32), C.POINTER(I32),
                                      C.POINTER(BabResult)],
            "gcp_bound_device": [P, P, I32, P, P, P, P, P],
            "gcp_grad_device": [P, P, I32, P, P, P, P, P, P, P, P],
            "gcp_bound_dense_noalloc": [I32, C.POINTER(I32), C.POINTER(P), C.POINTER(P), C.POINTER(P),
                                        C.POINTER(P), C.POINTER(P), P, P, P, P, I32, I64, P, P],
            "gcp_selftest_gemm": [I32, I64, I32, I32, C.POINTER(C.c_float), C.POINTER(C.c_float),
                                  C.POINTER(C.c_float)],
            "gcp_selftest_gemm_f64": [I64, I32, I32, pd, pd, pd, C.POINTER(C.c_float), pd],
            "gcp_profile_start": [C.c_char_p],
            "gcp_profile_stop": [],
            "gcp_profile_repeat": [C.c_char_p],
            "gcp_profile_query": [C.c_char_p, C.POINTER(I64), pd, pd, pd],
            "gcp_profile_report": [C.c_char_p, I64],
            "gcp_serve_start": [P, I32],
            "gcp_serve_submit": [P, C.POINTER(Request), C.POINTER(U64)],
            "gcp_serve_poll": [P, U64, C.POINTER(Result)],
            "gcp_serve_wait": [P, U64, I32, C.POINTER(Result)],
            "gcp_serve_stop": [P],
        }
        for name, args in sig.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = I32
        L.gcp_last_error.argtypes = [P]
        L.gcp_last_error.restype = C.c_char_p
        _lib = L
    return _lib


def _ptr(a: Optional[np.ndarray], ct):
    if a is None:
        return None
    return a.ctypes.data_as(C.POINTER(ct))


def _c(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


def opt_params(iters, optimizer=GCP_PGA, prec=GCP_FP32, certify=1, lr_alpha=0.1, lr_beta=0.1, lr_gamma=0.1,
               lr_decay=1.0, opt_pi=0) -> OptParams:
    return OptParams(iters, optimizer, prec, certify, lr_alpha, lr_beta, lr_gamma, lr_decay, opt_pi)


class Duals:
    """Handle of a device-resident batch (duals + workspace) of a Context."""

    def __init__(self, ctx: "Context", handle, net_id, cutset_id, prec):
        self.ctx, self.handle, self.net_id, self.cutset_id, self.prec = ctx, handle, net_id, cutset_id, prec
        R, na, M, N = C.c_int64(), C.c_int64(), C.c_int32(), C.c_int32()
        ctx._check(lib().gcp_duals_shape(ctx.h, handle, C.byref(R), C.byref(na), C.byref(M), C.byref(N)))
        self.rows, self.n_alpha, self.max_splits, self.n_cuts = R.value, na.value, M.value, N.value


class Context:
    """One GB300 device context (gcp_create / gcp_destroy)."""

    def __init__(self, device: int = 0, hbm_budget_bytes: int = 0):
        self.h = C.c_void_p()
        st = lib().gcp_create(C.byref(self.h), device, hbm_budget_bytes)
        if st != GCP_OK:
            raise GCPError(st, "gcp_create failed (no CUDA device?)")

    def close(self):
        if self.h:
            lib().gcp_destroy(self.h)
            self.h = C.c_void_p()

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def last_error(self) -> str:
        return lib().gcp_last_error(self.h).decode()

    def _check(self, st):
        if st not in (GCP_OK, GCP_PENDING):
            raise GCPError(st, self.last_error())
        return st

    def set_stream(self, stream_ptr: int):
        self._check(lib().gcp_set_stream(self.h, C.c_void_p(stream_ptr)))

    def mem_used(self) -> int:
        v = C.c_uint64()
        self._check(lib().gcp_mem_used(self.h, C.byref(v)))
        return v.value

    # ------------------------------------------------------------ inputs
    @staticmethod
    def _layer_descs(layers, keep):
        def fill(d, ly, with_bias=True):
            W = _c(ly.W, np.float64)
            keep.append(W)
            d.kind = ly.kind
            d.d_in = int(np.prod(ly.in_shape))
            d.d_out = int(np.prod(ly.out_shape))
            if ly.kind == GCP_CONV2D:
                d.c_in, d.h_in, d.w_in = ly.in_shape
                d.c_out, d.h_out, d.w_out = ly.out_shape
                d.k, d.stride, d.pad = W.shape[2], ly.stride, ly.pad
            d.W = _ptr(W, C.c_double)
            if with_bias:
                b = _c(ly.b, np.float64)
                keep.append(b)
                d.b = _ptr(b, C.c_double)

        descs = (LayerDesc * len(layers))()
        for i, ly in enumerate(layers):
            d = descs[i]
            fill(d, ly)
            d.skip = int(getattr(ly, "skip", 0))
            sc = getattr(ly, "shortcut", None) if d.skip else None
            if sc is not None:
                if np.any(np.asarray(sc.b) != 0):
                    raise ValueError("a shortcut's bias belongs in the layer's own bias b")
                sd = LayerDesc()
                fill(sd, sc, with_bias=False)
                keep.append(sd)
                d.shortcut = C.pointer(sd)
        return descs

    def init_net(self, layers, x_lo, x_hi, spec_c, inter_lo, inter_hi) -> int:
        """layers: objects with kind, W, b, in_shape, out_shape, stride, pad
        and optionally skip (0, or s >= 1: the layer adds xhat^(s-1)) and
        shortcut (None, or a layer object S applied to xhat^(s-1), zero bias)."""
        keep = []
        descs = self._layer_descs(layers, keep)
        xl, xh, sc = _c(x_lo, np.float64), _c(x_hi, np.float64), _c(spec_c, np.float64)
        lo = _c(np.concatenate([np.asarray(a, np.float64) for a in inter_lo]) if len(inter_lo) else np.zeros(0), np.float64)
        hi = _c(np.concatenate([np.asarray(a, np.float64) for a in inter_hi]) if len(inter_hi) else np.zeros(0), np.float64)
        nid = C.c_int32()
        self._check(lib().gcp_init_net(self.h, descs, len(layers), _ptr(xl, C.c_double), _ptr(xh, C.c_double),
                                       _ptr(sc, C.c_double), sc.shape[0], _ptr(lo, C.c_double), _ptr(hi, C.c_double),
                                       C.byref(nid)))
        return nid.value

    def intermediate_bounds(self, layers, x_lo, x_hi, params: Optional[OptParams] = None, cuts=None):
        """Root bounds (lo, hi) of every hidden layer (list of arrays), by the
        library's own certified bound propagation: CROWN at the default
        slopes (params None) or alpha-CROWN with params.iters ascent steps.
        cuts (ptr, layer, kind, index, coef, d, as for add_cuts; valid over the
        whole box): each layer's bounds also use the cuts over the layers below
        it, with their multipliers optimised (params given)."""
        keep = []
        descs = self._layer_descs(layers, keep)
        xl, xh = _c(x_lo, np.float64), _c(x_hi, np.float64)
        dims = [int(np.prod(ly.out_shape)) for ly in layers[:-1]]
        lo, hi = np.zeros(sum(dims)), np.zeros(sum(dims))
        pp = C.byref(params) if params is not None else None
        if cuts is None:
            self._check(lib().gcp_intermediate_bounds(self.h, descs, len(layers), _ptr(xl, C.c_double),
                                                      _ptr(xh, C.c_double), pp, _ptr(lo, C.c_double),
                                                      _ptr(hi, C.c_double)))
        else:
            a = [_c(cuts.ptr, np.int64), _c(cuts.layer, np.int16), _c(cuts.kind, np.int8), _c(cuts.index, np.int32),
                 _c(cuts.coef, np.float64), _c(cuts.d, np.float64)]
            self._check(lib().gcp_intermediate_bounds_cuts(
                self.h, descs, len(layers), _ptr(xl, C.c_double), _ptr(xh, C.c_double), pp, len(a[5]),
                _ptr(a[0], C.c_int64), _ptr(a[1], C.c_int16), _ptr(a[2], C.c_int8), _ptr(a[3], C.c_int32),
                _ptr(a[4], C.c_double), _ptr(a[5], C.c_double), _ptr(lo, C.c_double), _ptr(hi, C.c_double)))
        out_lo, out_hi, o = [], [], 0
        for d in dims:
            out_lo.append(lo[o:o + d].copy())
            out_hi.append(hi[o:o + d].copy())
            o += d
        return out_lo, out_hi

    def bab_verify(self, net_id: int, cutset_id: int, params: OptParams, batch: int = 256, max_rounds: int = 100,
                   max_domains: int = 1 << 16, timeout_s: float = 0.0, branching: int = 0) -> dict:
        """Branch and bound over ReLU splits: is every spec row positive over the box?
        branching 0: by the duals (gcp_branch_picks' score), 1: static root intercept."""
        bp = BabParams(batch, max_rounds, max_domains, timeout_s, params, branching)
        r = BabResult()
        self._check(lib().gcp_bab_verify(self.h, net_id, cutset_id, C.byref(bp), C.byref(r)))
        return {f: getattr(r, f) for f, _ in BabResult._fields_}

    def bab_verify_labels(self, net_id: int, cutset_id: int, n_spec: int, params: OptParams, batch: int = 256,
                          max_rounds: int = 100, max_domains: int = 1 << 16, timeout_s: float = 0.0,
                          stop_at_failure: bool = False, branching: int = 0):
        """Branch and bound label by label, the easiest first: (result dict,
        order of the labels, per-label 1 proved / 0 not / -1 not attempted)."""
        bp = BabParams(batch, max_rounds, max_domains, timeout_s, params, branching)
        r = BabResult()
        order = np.zeros(n_spec, np.int32)
        ver = np.zeros(n_spec, np.int32)
        self._check(lib().gcp_bab_verify_labels(self.h, net_id, cutset_id, C.byref(bp), int(stop_at_failure),
                                                _ptr(order, C.c_int32), _ptr(ver, C.c_int32), C.byref(r)))
        return {f: getattr(r, f) for f, _ in BabResult._fields_}, order, ver

    def add_cuts(self, net_id: int, ptr, layer, kind, index, coef, d, cutset_id: int = -1):
        ptr = _c(ptr, np.int64)
        layer, kind, index = _c(layer, np.int16), _c(kind, np.int8), _c(index, np.int32)
        coef, d = _c(coef, np.float64), _c(d, np.float64)
        cs, first = C.c_int32(cutset_id), C.c_int32()
        self._check(lib().gcp_add_cuts(self.h, net_id, len(d), _ptr(ptr, C.c_int64), _ptr(layer, C.c_int16),
                                       _ptr(kind, C.c_int8), _ptr(index, C.c_int32), _ptr(coef, C.c_double),
                                       _ptr(d, C.c_double), C.byref(cs), C.byref(first)))
        return cs.value, first.value

    def load_instance(self, inst):
        """init_net + add_cuts for a synthetic instance; returns (net_id, cutset_id)."""
        net_id = self.init_net(inst.net.layers, inst.x_lo, inst.x_hi, inst.spec, inst.inter_lo, inst.inter_hi)
        c = inst.cuts
        cs, _ = self.add_cuts(net_id, c.ptr, c.layer, c.kind, c.index, c.coef, c.d)
        return net_id, cs

    # ------------------------------------------------------------ duals
    def duals_create(self, net_id: int, cutset_id: int, sub, dual_prec: int = GCP_FP32) -> Duals:
        arrs = [_c(sub.ptr, np.int32), _c(sub.layer, np.int16), _c(sub.index, np.int32), _c(sub.sign, np.int8)]
        sd = Subdomains(sub.n, _ptr(arrs[0], C.c_int32), _ptr(arrs[1], C.c_int16), _ptr(arrs[2], C.c_int32),
                        _ptr(arrs[3], C.c_int8))
        h = C.c_void_p()
        self._check(lib().gcp_duals_create(self.h, net_id, cutset_id, C.byref(sd), dual_prec, C.byref(h)))
        return Duals(self, h, net_id, cutset_id, dual_prec)

    def duals_create_multi(self, net_id: int, cutset_ids, subs, dual_prec: int = GCP_FP32) -> Duals:
        """Several queries on one network in one batch (rows query-major)."""
        keep = []
        arr = (Subdomains * len(subs))()
        for q, sub in enumerate(subs):
            a = [_c(sub.ptr, np.int32), _c(sub.layer, np.int16), _c(sub.index, np.int32), _c(sub.sign, np.int8)]
            keep.append(a)
            arr[q] = Subdomains(sub.n, _ptr(a[0], C.c_int32), _ptr(a[1], C.c_int16), _ptr(a[2], C.c_int32),
                                _ptr(a[3], C.c_int8))
        ids = (C.c_int32 * len(subs))(*cutset_ids)
        h = C.c_void_p()
        self._check(lib().gcp_duals_create_multi(self.h, net_id, len(subs), ids, arr, dual_prec, C.byref(h)))
        return Duals(self, h, net_id, -1, dual_prec)

    def duals_export(self, D: Duals):
        a = np.zeros((D.rows, D.n_alpha))
        b = np.zeros((D.rows, D.max_splits))
        g = np.zeros((D.rows, D.n_cuts))
        self._check(lib().gcp_duals_export(self.h, D.handle, _ptr(a, C.c_double), _ptr(b, C.c_double),
                                           _ptr(g, C.c_double)))
        return a, b, g

    def duals_theta(self, D: Duals, theta=None):
        """The directly optimised ReLU duals theta [R, n_alpha] (pi = theta *
        [nuhat]_+): sets them when theta is given, returns them otherwise."""
        if theta is not None:
            t = _c(theta, np.float64)
            self._check(lib().gcp_duals_theta(self.h, D.handle, _ptr(t, C.c_double), None))
            return None
        out = np.zeros((D.rows, D.n_alpha))
        self._check(lib().gcp_duals_theta(self.h, D.handle, None, _ptr(out, C.c_double)))
        return out

    def duals_import(self, D: Duals, alpha=None, beta=None, gamma=None):
        a = None if alpha is None else _c(alpha, np.float64)
        b = None if beta is None else _c(beta, np.float64)
        g = None if gamma is None else _c(gamma, np.float64)
        self._check(lib().gcp_duals_import(self.h, D.handle, _ptr(a, C.c_double), _ptr(b, C.c_double),
                                           _ptr(g, C.c_double)))

    def duals_free(self, D: Duals):
        self._check(lib().gcp_duals_free(self.h, D.handle))

    # ------------------------------------------------------------ bounds
    def bound_batch(self, D: Duals, prec: int, certify: bool = False):
        out = np.zeros(D.rows)
        cert = np.zeros(D.rows) if certify else None
        self._check(lib().gcp_bound_batch(self.h, D.handle, prec, int(certify), _ptr(out, C.c_double),
                                          _ptr(cert, C.c_double)))
        return out, cert

    def grad_batch(self, D: Duals, prec: int):
        out = np.zeros(D.rows)
        ga = np.zeros((D.rows, D.n_alpha))
        gb = np.zeros((D.rows, D.max_splits))
        gg = np.zeros((D.rows, D.n_cuts))
        self._check(lib().gcp_grad_batch(self.h, D.handle, prec, _ptr(out, C.c_double), _ptr(ga, C.c_double),
                                         _ptr(gb, C.c_double), _ptr(gg, C.c_double)))
        return out, ga, gb, gg

    def branch_picks(self, D: Duals, prec: int, n_sub: int):
        """The branching neuron (layer, index; -1 for none) of each of the batch's n_sub subdomains."""
        S = n_sub
        lay = np.zeros(max(S, 1), np.int32)
        idx = np.zeros(max(S, 1), np.int32)
        self._check(lib().gcp_branch_picks(self.h, D.handle, prec, _ptr(lay, C.c_int32), _ptr(idx, C.c_int32)))
        return lay[:S], idx[:S]

    def optimize_batch(self, D: Duals, params: OptParams):
        out = np.zeros(D.rows)
        cert = np.zeros(D.rows)
        err = np.zeros(D.rows)
        self._check(lib().gcp_optimize_batch(self.h, D.handle, C.byref(params), _ptr(out, C.c_double),
                                             _ptr(cert, C.c_double), _ptr(err, C.c_double)))
        return out, cert, err

    def bound_device(self, D: Duals, prec, alpha, beta, gamma, out, stream: int):
        """alpha/beta/gamma/out: float32 CUDA tensors (export layouts)."""
        self._check(lib().gcp_bound_device(self.h, D.handle, prec, _dptr(alpha), _dptr(beta), _dptr(gamma),
                                           _dptr(out), C.c_void_p(stream)))

    def grad_device(self, D: Duals, prec, alpha, beta, gamma, grad_out, ga, gb, gg, stream: int):
        self._check(lib().gcp_grad_device(self.h, D.handle, prec, _dptr(alpha), _dptr(beta), _dptr(gamma),
                                          _dptr(grad_out), _dptr(ga), _dptr(gb), _dptr(gg), C.c_void_p(stream)))

    # ------------------------------------------------------------ serving
    def serve_start(self, max_inflight: int):
        self._check(lib().gcp_serve_start(self.h, max_inflight))

    def serve_submit(self, net_id, cutset_id, sub, params: OptParams, rounds: int, seed: int,
                     keep_final: bool = False) -> int:
        arrs = [_c(sub.ptr, np.int32), _c(sub.layer, np.int16), _c(sub.index, np.int32), _c(sub.sign, np.int8)]
        sd = Subdomains(sub.n, _ptr(arrs[0], C.c_int32), _ptr(arrs[1], C.c_int16), _ptr(arrs[2], C.c_int32),
                        _ptr(arrs[3], C.c_int8))
        req = Request(net_id, cutset_id, rounds, seed, sd, params, 1 if keep_final else 0)
        t = C.c_uint64()
        self._check(lib().gcp_serve_submit(self.h, C.byref(req), C.byref(t)))
        return t.value

    def serve_wait(self, ticket: int, capacity: int, timeout_ms: int = 600000):
        buf = np.zeros(max(capacity, 1))
        res = Result(0, 0, _ptr(buf, C.c_double), 0.0, 0.0, 0.0, 0.0)
        st = lib().gcp_serve_wait(self.h, ticket, timeout_ms, C.byref(res))
        self._check(st)
        return res, buf[:res.rows].copy()

    def serve_poll(self, ticket: int, capacity: int):
        buf = np.zeros(max(capacity, 1))
        res = Result(0, 0, _ptr(buf, C.c_double), 0.0, 0.0, 0.0, 0.0)
        st = self._check(lib().gcp_serve_poll(self.h, ticket, C.byref(res)))
        if st == GCP_PENDING:
            return None, None
        return res, buf[:res.rows].copy()

    def serve_final(self, ticket: int):
        """The last round's subdomains and duals of a finished keep_final request
        (after serve_wait / serve_poll took its result): (Subdomains, alpha, beta, gamma)."""
        f = Final()
        self._check(lib().gcp_serve_final(self.h, ticket, C.byref(f)))
        ptr = np.zeros(f.n_sub + 1, np.int32)
        lay = np.zeros(max(f.n_split_entries, 1), np.int16)
        idx = np.zeros(max(f.n_split_entries, 1), np.int32)
        sgn = np.zeros(max(f.n_split_entries, 1), np.int8)
        A = np.zeros((f.rows, f.n_alpha), np.float32)
        B = np.zeros((f.rows, f.max_splits), np.float32)
        G = np.zeros((f.rows, f.n_cuts), np.float32)
        f.split_ptr, f.split_layer = _ptr(ptr, C.c_int32), _ptr(lay, C.c_int16)
        f.split_index, f.split_sign = _ptr(idx, C.c_int32), _ptr(sgn, C.c_int8)
        f.alpha = _ptr(A if A.size else np.zeros(1, np.float32), C.c_float)
        f.beta = _ptr(B if B.size else np.zeros(1, np.float32), C.c_float)
        f.gamma = _ptr(G if G.size else np.zeros(1, np.float32), C.c_float)
        self._check(lib().gcp_serve_final(self.h, ticket, C.byref(f)))
        n = int(f.n_split_entries)
        from . import synth
        sub = synth.Subdomains(ptr, lay[:n].copy(), idx[:n].copy(), sgn[:n].copy())
        return sub, A.astype(np.float64), B.astype(np.float64), G.astype(np.float64)

    def serve_stop(self):
        self._check(lib().gcp_serve_stop(self.h))


def bound_dense_noalloc(dims, WT, bias, lo, hi, alpha, x_lo, x_hi, y_last, cb, K, out, stream: int) -> int:
    """gcp_bound_dense_noalloc on float32 CUDA tensors; returns the status.

    WT, bias, lo, hi, alpha: lists over hidden layers i = 1..L-1 (entry i-1).
    """
    nl = len(dims) - 1
    dd = (C.c_int32 * len(dims))(*dims)

    def arr(ts):
        a = (C.c_void_p * max(len(ts), 1))()
        for q, t in enumerate(ts):
            a[q] = t.data_ptr()
        return a
    R = out.numel()
    return lib().gcp_bound_dense_noalloc(nl, dd, arr(WT), arr(bias), arr(lo), arr(hi), arr(alpha),
                                         C.c_void_p(x_lo.data_ptr()), C.c_void_p(x_hi.data_ptr()),
                                         C.c_void_p(y_last.data_ptr()), C.c_void_p(cb.data_ptr()), K, R,
                                         C.c_void_p(out.data_ptr()), C.c_void_p(stream))


def selftest_gemm(kind: int, A: np.ndarray, B: np.ndarray) -> np.ndarray:
    """C = A @ B.T through kind 0 (tcgen05 bf16), 1 (tcgen05 3xtf32) or 2 (SIMT fp32)."""
    A = _c(A, np.float32)
    B = _c(B, np.float32)
    M, K = A.shape
    N = B.shape[0]
    out = np.zeros((M, N), np.float32)
    st = lib().gcp_selftest_gemm(kind, M, N, K, _ptr(A, C.c_float), _ptr(B, C.c_float), _ptr(out, C.c_float))
    if st != GCP_OK:
        raise GCPError(st, "selftest gemm failed")
    return out


def selftest_gemm_f64(A: np.ndarray, B: np.ndarray):
    """(C, Cabs, cerr): C = A @ B.T in float64 on the tensor cores by exact
    slices, with |C - exact| <= cerr * Cabs."""
    A = _c(A, np.float64)
    B = _c(B, np.float64)
    M, K = A.shape
    N = B.shape[0]
    out = np.zeros((M, N), np.float64)
    cabs = np.zeros((M, N), np.float32)
    cerr = C.c_double()
    st = lib().gcp_selftest_gemm_f64(M, N, K, _ptr(A, C.c_double), _ptr(B, C.c_double), _ptr(out, C.c_double),
                                     _ptr(cabs, C.c_float), C.byref(cerr))
    if st != GCP_OK:
        raise GCPError(st, "selftest float64 gemm failed")
    return out, cabs, cerr.value


def profile_start(kernel_prefix: Optional[str] = None):
    """Count every library kernel launch; time those whose name starts with the prefix."""
    lib().gcp_profile_start(kernel_prefix.encode() if kernel_prefix else None)


def profile_stop():
    lib().gcp_profile_stop()


def profile_repeat(kernel_prefix: Optional[str] = None):
    """While profiling, issue every launch of the idempotent tensor-core GEMM
    named by the prefix twice (its in-stream cost = the extra step time over
    the launch count)."""
    lib().gcp_profile_repeat(kernel_prefix.encode() if kernel_prefix else None)


def profile_query(name: Optional[str] = None):
    """(launches, device ms of timed launches, algorithmic flops, algorithmic bytes)."""
    n, ms, fl, by = C.c_int64(), C.c_double(), C.c_double(), C.c_double()
    lib().gcp_profile_query(name.encode() if name else None, C.byref(n), C.byref(ms), C.byref(fl), C.byref(by))
    return n.value, ms.value, fl.value, by.value


def profile_report():
    """{kernel: (launches, timed launches, ms, flops, bytes)}."""
    buf = C.create_string_buffer(1 << 16)
    lib().gcp_profile_report(buf, len(buf))
    out = {}
    for line in buf.value.decode().splitlines():
        nm, n, t, ms, fl, by = line.split()
        out[nm] = (int(n), int(t), float(ms), float(fl), float(by))
    return out


def _dptr(t):
    if t is None or t.numel() == 0:
        return None
    return C.c_void_p(t.data_ptr())


def torch_stream_handle(stream=None) -> int:
    """cudaStream_t of a torch stream for the device entry points. torch's
    legacy default stream has handle 0, which the library reads as "the
    context's own stream"; it is passed as cudaStreamLegacy (1) instead so the
    work stays ordered with torch's."""
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return s.cuda_stream or 1


def make_bound_function():
    """torch.autograd.Function around gcp_bound_device / gcp_grad_device."""
    import torch

    class GCPBound(torch.autograd.Function):
        @staticmethod
        def forward(fctx, alpha, beta, gamma, ctx: Context, D: Duals, prec: int):
            alpha, beta, gamma = alpha.contiguous(), beta.contiguous(), gamma.contiguous()
            out = torch.empty(D.rows, dtype=torch.float32, device=alpha.device)
            ctx.bound_device(D, prec, alpha, beta, gamma, out, torch_stream_handle())
            fctx.save_for_backward(alpha, beta, gamma)
            fctx.gcp = (ctx, D, prec)
            return out

        @staticmethod
        def backward(fctx, grad_out):
            alpha, beta, gamma = fctx.saved_tensors
            ctx, D, prec = fctx.gcp
            ga, gb, gg = torch.empty_like(alpha), torch.zeros_like(beta), torch.empty_like(gamma)
            ctx.grad_device(D, prec, alpha, beta, gamma, grad_out.contiguous().float(), ga, gb, gg,
                            torch_stream_handle())
            return ga, gb, gg, None, None, None

    return GCPBound
