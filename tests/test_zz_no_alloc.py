"""The no-allocation bound entry point agrees with gcp_bound_batch and the oracle.

gcp_bound_dense_noalloc is for callers that cannot allocate device memory:
processes that reserve the whole GPU for their own pool up front, so that any
further cudaMalloc fails, and loops that cannot pay for the device-wide
synchronisation of cudaMalloc/cudaFree. It keeps its scratch in a fixed
device array of the library, shared by every call. Here it runs twice in a
row on the same caller-owned inputs, and each result must match the ordinary
FP32 path (gcp_bound_batch) and the FP64 oracle within the FP32 tolerance of
the parity tests; a batch whose scratch exceeds the array is refused with
GCP_EBUDGET, and a host pointer where device memory is required with
GCP_EINVAL.
"""
import dataclasses

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _outward(x, down):
    f = np.asarray(x, np.float64).astype(np.float32)
    if down:
        return np.where(f.astype(np.float64) > x, np.nextafter(f, np.float32(-np.inf)), f)
    return np.where(f.astype(np.float64) < x, np.nextafter(f, np.float32(np.inf)), f)


def test_noalloc_bound_matches_bound_batch_on_two_calls():
    torch = pytest.importorskip("torch")
    from paper_2208_05740_gb300 import build, gcp, synth
    build.build()
    inst = synth.mlp_256x6(n_sub=24, n_cuts=0)
    S = inst.sub.n
    no_splits = synth.Subdomains(np.zeros(S + 1, np.int32), np.zeros(0, np.int16), np.zeros(0, np.int32),
                                 np.zeros(0, np.int8))
    inst = dataclasses.replace(inst, sub=no_splits)
    with gcp.Context(0) as ctx:
        net_id, _ = ctx.load_instance(inst)
        D = ctx.duals_create(net_id, -1, inst.sub, gcp.GCP_FP32)
        rng = np.random.default_rng(3)
        ctx.duals_import(D, rng.random((D.rows, D.n_alpha)), None, None)
        A, _, _ = ctx.duals_export(D)
        ref, _ = ctx.bound_batch(D, gcp.GCP_FP32)
        R = D.rows
    # the oracle's float64 bound at the same slopes (Theorem 3.1; no cuts, no splits)
    from oracle import gcp_oracle as O
    P = O.build_problem(inst)
    alist, off = [], 0
    for d in inst.net.dims[1:-1]:
        alist.append(A[:, off:off + d].astype(np.float64))
        off += d
    oracle = O.evaluate(P, O.Duals(alist, np.zeros((R, 0)), np.zeros((R, 0))))
    dev = torch.device("cuda:0")
    net = inst.net
    dims, L, K = net.dims, net.L, inst.spec.shape[0]

    def f32(a):
        return torch.tensor(np.ascontiguousarray(a, np.float32), device=dev)
    WT = [f32(ly.W.T) for ly in net.layers[:-1]]
    bias = [f32(ly.b) for ly in net.layers[:-1]]
    lo = [f32(_outward(a, True)) for a in inst.inter_lo]
    hi = [f32(_outward(a, False)) for a in inst.inter_hi]
    alpha, off = [], 0
    for d in dims[1:-1]:
        alpha.append(f32(A[:, off:off + d]))
        off += d
    y_last = f32(-(inst.spec @ net.layers[-1].W))
    cb = f32(inst.spec @ net.layers[-1].b)
    x_lo, x_hi = f32(inst.x_lo), f32(inst.x_hi)
    out = torch.empty(R, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream().cuda_stream
    for call in range(2):
        out.fill_(float("nan"))
        st = gcp.bound_dense_noalloc(dims, WT, bias, lo, hi, alpha, x_lo, x_hi, y_last, cb, K, out, stream)
        assert st == 0, f"call {call}: status {st}"
        torch.cuda.synchronize()
        got = out.cpu().numpy().astype(np.float64)
        tol = 1e-5 * np.maximum(np.abs(ref), 1.0)
        assert np.all(np.abs(got - ref) <= tol), f"call {call}: max diff {np.max(np.abs(got - ref))}"
        tol = 1e-5 * np.maximum(np.abs(oracle), 1.0)
        assert np.all(np.abs(got - oracle) <= tol), f"call {call}: max diff vs oracle {np.max(np.abs(got - oracle))}"
    # a batch whose scratch exceeds the fixed array is refused (GCP_EBUDGET = -5)
    R_big = K * 4096      # 3 x R x 784 floats alone exceed 32 MiB
    alpha_big = [torch.zeros((R_big, d), dtype=torch.float32, device=dev) for d in dims[1:-1]]
    out_big = torch.empty(R_big, dtype=torch.float32, device=dev)
    st = gcp.bound_dense_noalloc(dims, WT, bias, lo, hi, alpha_big, x_lo, x_hi, y_last, cb, K, out_big, stream)
    assert st == -5, st
    # a host array where device memory is required is refused (GCP_EINVAL = -1)
    x_lo_host = torch.tensor(np.ascontiguousarray(inst.x_lo, np.float32))
    st = gcp.bound_dense_noalloc(dims, WT, bias, lo, hi, alpha, x_lo_host, x_hi, y_last, cb, K, out, stream)
    assert st == -1, st
