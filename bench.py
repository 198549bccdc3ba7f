#!/usr/bin/env python
"""Benchmark: certified subdomain-bounds per second at a fixed iteration count.

Every workload takes its root intermediate bounds from CROWN (Sec. 2),
computed by the library's own certified propagation before the timed region
(the oracle legs compute them with the oracle).

Headline (default --workload mlp): ReLU MLP 784-256x6-10, 1024
branch-and-bound subdomains (1-8 neuron splits each) x 9 spec rows, 200
sparse cuts over 2-8 variables, 100 Adam ascent iterations on (alpha, beta,
gamma) in the FP32 chain, then the FP64 outward-rounded certification pass.
One step = that whole hot path for the batch; one unit = one subdomain with
all its spec rows optimised and certified. Inputs are seeded synthetic data
of the paper's shapes.

The default run also times, under "workloads.cnn", the CNN 3x32x32 ->
conv32 3x3 s2 -> conv64 3x3 s2 -> FC512 -> FC10, 4096 subdomains (1-12
splits) x 9 spec rows, 1000 cuts over 2-16 variables, 50 Adam iterations in
the BF16 chain, FP64 certification (--workload cnn makes it the headline).

--workload resnet: residual CNN of the resnet2b shape, 3x32x32 -> conv8 3x3
s2 -> ResBlock(8,16) (conv s2, conv, 1x1 s2 shortcut) -> ResBlock(16,16)
(identity shortcut) -> FC100 -> FC10, 2048 subdomains (the residual models'
batch size) x 9 spec rows, 500 cuts over 2-16 variables, 20 Adam iterations
in the BF16 chain, FP64 certification.

value  : device-timed (CUDA events on the library's stream), inputs resident.
e2e    : the same through the public C ABI from host buffers: every step
         creates the batch from host split arrays (uploads splits and cuts),
         optimises, certifies, copies bounds back and frees the batch.
forms  : the same workload in the other chain precision (and with pi
         optimised directly), with the certified-bound quality of each form
         against the workload's own form.
serving: the continuous-batching stream at 200 requests/s (over capacity)
         and at 1 request/s (below it).
--impl reference : the FP64 CPU oracle on a bounded sample of the workload.
Multi-GPU (torchrun): every rank runs its own batch (weak scaling, no
collective on the data path); value = all ranks' subdomains / max time.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "certified subdomain-bounds/sec at fixed iters; p50/p99 latency; bound err vs FP64"
UNIT = "subdomain-bounds/s"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["gcp", "reference"], default="gcp")
    ap.add_argument("--workload", choices=sorted(WORKLOADS), default="mlp",
                    help="mlp: MLP 784-256x6-10 (the headline); cnn: the CIFAR-shaped CNN; resnet: resnet2b shape")
    ap.add_argument("--prec", choices=["fp32", "bf16"], default=None, help="chain precision (workload default)")
    ap.add_argument("--iters", type=int, default=None, help="ascent iterations (workload default)")
    ap.add_argument("--n-sub", type=int, default=None, help="subdomains per GPU (workload default)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-inter-bounds", action="store_true",
                    help="skip the GPU intermediate-bounds measurement (CROWN / alpha-CROWN root bounds)")
    ap.add_argument("--profile-all", action="store_true", help="print every kernel's share (untimed step)")
    ap.add_argument("--serve-requests", type=int, default=48, help="requests of the serving stream (0: skip)")
    ap.add_argument("--no-bf16-form", action="store_true", help="skip the BF16-chain form of the workload")
    ap.add_argument("--no-cnn", action="store_true",
                    help="skip the CNN workload that the default (mlp) run also times")
    ap.add_argument("--no-opt-pi-form", action="store_true",
                    help="skip the form with the ReLU duals pi optimised directly (opt_pi)")
    a = ap.parse_args()
    w = WORKLOADS[a.workload]
    a.prec = a.prec or w["prec"]
    a.iters = a.iters if a.iters is not None else w["iters"]
    a.n_sub = a.n_sub if a.n_sub is not None else w["n_sub"]
    return a


def _build_mlp(n_sub, root_bounds=None):
    from paper_2208_05740_gb300 import synth
    return synth.mlp_256x6(n_sub=n_sub, root_bounds=root_bounds)


def _build_cnn(n_sub, root_bounds=None):
    from paper_2208_05740_gb300 import synth
    return synth.cnn_cifar(n_sub=n_sub, root_bounds=root_bounds)


def _build_resnet(n_sub, root_bounds=None):
    from paper_2208_05740_gb300 import synth
    return synth.cnn_resnet(n_sub=n_sub, root_bounds=root_bounds)


# The workloads: name, instance builder, defaults, oracle sample size.
WORKLOADS = {
    "mlp": dict(name="mlp_784_256x6_10", cuts=200, splits="1-8", prec="fp32", iters=100, n_sub=1024, sample=4,
                build=_build_mlp),
    "cnn": dict(name="cnn_3x32x32_c32_c64_fc512_fc10", cuts=1000, splits="1-12", prec="bf16", iters=50, n_sub=4096,
                sample=2, build=_build_cnn),
    "resnet": dict(name="resnet_3x32x32_c8_b16s2_b16s1_fc100_fc10", cuts=500, splits="1-12", prec="bf16", iters=20,
                   n_sub=2048, sample=2, build=_build_resnet),
}


def workload_config(wname, n_sub, iters, prec, n_gpus, inter="CROWN"):
    w = WORKLOADS[wname]
    return {"workload": w["name"], "n_subdomains_per_gpu": n_sub, "spec_rows": 9, "rows_per_gpu": n_sub * 9,
            "cuts": w["cuts"], "splits_per_subdomain": w["splits"], "iters": iters, "optimizer": "adam",
            "lr": [0.1, 0.02, 0.02], "lr_decay": 0.98, "chain": prec, "certify": "fp64_outward_rounded",
            "intermediate_bounds": inter, "l2": "flushed between steps (256 MiB write)",
            "parallelism": f"replicas{n_gpus}" if n_gpus > 1 else "single_gpu"}


# --------------------------------------------------------------------------- clocks
class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.p = None

    def start(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.p = None

    def stop(self):
        if self.p is None:
            return None
        self.p.terminate()
        try:
            out, _ = self.p.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.p.kill()
            out, _ = self.p.communicate()
        rows = []
        for line in out.strip().splitlines():
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 8:
                continue
            try:
                rows.append((float(parts[0]), float(parts[1]), parts[4:8]))
            except ValueError:
                continue
        if not rows:
            return None
        mhz = sorted(r[0] for r in rows)
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i, v in enumerate(r[2]) if v.lower().startswith("active")})
        return {"sm_mhz": mhz[len(mhz) // 2], "sm_max_mhz": max(r[1] for r in rows), "reasons": reasons,
                "samples": len(rows)}


# --------------------------------------------------------------------------- peaks
def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0, "sm_max_mhz": 2070.0}, \
            "fallback"


def kernel_peak(name, peaks, src):
    """(bound, peak, unit, note) for a kernel class.

    FP32 SIMT contractions: 152 SMs x 128 FP32 lanes x 2 flop x max SM clock.
    FP64 SIMT contractions: 152 SMs x 2 FP64 lanes x 2 flop x max SM clock
    (the nominal 1.25 TFLOP/s of GB300's FP64 units). Per-neuron kernels: HBM.
    """
    mhz = float(peaks.get("sm_max_mhz", 2070.0))
    if name.startswith(("gemm_simt_f32", "conv_fwd_f32", "conv_T_f32")):
        return "alu", 152 * 128 * 2 * mhz * 1e6 / 1e12, "TFLOP/s", f"FFMA peak from unit counts and {mhz:.0f} MHz"
    if name.startswith(("gemm_simt_f64", "conv_T_f64", "conv_fwd_f64")):
        return "alu", 152 * 2 * 2 * mhz * 1e6 / 1e12, "TFLOP/s", f"DFMA peak from unit counts and {mhz:.0f} MHz"
    if name.startswith(("gemm_tc_bf16", "conv_tc_bf16")):
        return "tensor", float(peaks["bf16_tflops_sustained"]), "TFLOP/s", f"bf16 sustained ({src})"
    if name.startswith(("gemm_tc_tf32", "conv_tc_tf32")):
        # tf32 tensor rate = measured bf16 rate x nominal tf32/bf16 ratio (1.1/2.25);
        # the three-pass kernel's achieved flops count the product once
        tf = float(peaks["bf16_tflops_sustained"]) * 1.1 / 2.25
        return "tensor", tf / 3.0, "TFLOP/s", f"tf32 tensor (bf16 sustained x 1.1/2.25, {src}) / 3 passes"
    return "hbm", float(peaks["hbm_gbs"]), "GB/s", f"copy bandwidth ({src})"


def traffic_for(name, workload):
    """Per-launch DRAM bytes of an ncu capture, if the kernel source is unchanged since."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as f:
            tab = json.load(f)
    except (OSError, ValueError):
        return None
    ent = tab.get(f"{workload}:{name}")
    if not ent:
        return None
    src = os.path.join(ROOT, "paper_2208_05740_gb300", "csrc", ent["source"])
    try:
        h = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]
    except OSError:
        return None
    return ent["bytes_per_launch"] if h == ent["source_sha"] else None


# --------------------------------------------------------------------------- CPU oracle
def oracle_sample(inst, n_sub, iters, seconds_cap=25.0):
    """Time the FP64 oracle on the first n_sub subdomains: a few Adam steps and
    the two evaluations (final bound and certification), extrapolated to
    `iters` steps. Returns (subdomains per second, description)."""
    import numpy as np
    from oracle import gcp_oracle as O
    from paper_2208_05740_gb300 import synth
    sub = synth.restrict(inst, n_sub)
    P = O.build_problem(sub)
    D = O.default_duals(P)
    t0 = time.perf_counter()
    O.evaluate(P, D)
    t_eval = time.perf_counter() - t0
    # probe one step, then time k contiguous steps (k fits the cap); optimize()
    # ends with one evaluation, which is subtracted
    t0 = time.perf_counter()
    O.optimize(P, D, 1, 0.1, 0.02, 0.02, optimizer="adam", lr_decay=0.98)
    t1 = max(time.perf_counter() - t0 - t_eval, 1e-6)
    k = int(max(1, min(iters, seconds_cap / t1)))
    t0 = time.perf_counter()
    O.optimize(P, D, k, 0.1, 0.02, 0.02, optimizer="adam", lr_decay=0.98)
    t_it = max(time.perf_counter() - t0 - t_eval, 1e-9) / k
    per_batch = t_it * iters + 2 * t_eval
    return n_sub / per_batch, f"{inst.name}: {n_sub} subdomains x 9 rows, {k} timed Adam steps + 1 evaluation, " \
                              f"extrapolated to {iters} steps + 2 evaluations"


# --------------------------------------------------------------------------- ranks
def max_over_ranks(x: float, device) -> float:
    """The maximum of a per-rank scalar over all ranks of the job (its time is
    the slowest rank's); the value itself without a process group."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return x
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(world: int, units_per_rank: int, steps: int, seconds: float) -> float:
    """Whole-job throughput: every rank's units over the slowest rank's time."""
    return world * units_per_rank * steps / seconds


def oracle_instance(wname, n_sub):
    """The workload with CROWN root bounds computed by the oracle (CPU legs only)."""
    from oracle import gcp_oracle as O
    return WORKLOADS[wname]["build"](n_sub, O.crown_root_bounds)


def run_reference(a):
    import numpy as np
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    inst = oracle_instance(a.workload, 64)
    n_sub = WORKLOADS[a.workload]["sample"]
    cfg = workload_config(a.workload, a.n_sub, a.iters, a.prec, a.gpus)
    for _ in range(a.warmup):
        oracle_sample(inst, n_sub, a.iters, seconds_cap=2.0)
    vals = []
    for _ in range(a.steps):
        v, desc = oracle_sample(inst, n_sub, a.iters, seconds_cap=8.0)
        vals.append(v)
    value = float(np.median(vals))
    cores = os.cpu_count()
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": a.gpus, "steps": a.steps,
            "warmup": a.warmup, "ms_per_step": 1000.0 * n_sub / value, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": cfg,
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": desc},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


# --------------------------------------------------------------------------- serving stream
SERVE_SEED = 2208057405


def serving_bench(dev, n_requests, rate=200.0, rounds=10, iters=20, max_inflight=16):
    """Serving stream: Poisson arrivals (mean `rate` requests/s) mixing the
    MLP 8-16-16-3, MLP 784-256x6-10 and CNN networks; each request holds
    1-2048 subdomains (log-uniform) and one of five cut sets of 0-2000 cuts,
    admitted under a 100 GB device-memory budget, optimised for `rounds`
    branch-and-bound rounds of `iters` Adam steps in the BF16 chain and
    certified in FP64 every round."""
    import numpy as np
    from paper_2208_05740_gb300 import gcp, synth
    rng = np.random.default_rng(SERVE_SEED)
    nets = [
        (synth.mlp_small(n_sub=1, n_cuts=0), (0, 2), dict(min_vars=2, max_vars=4, hidden_only=True)),
        (synth.mlp_256x6(n_sub=1, n_cuts=0), (1, 8),
         dict(min_vars=2, max_vars=8, span_layers=True, need_z=True, p_input=0.99)),
        (synth.cnn_cifar(n_sub=1, n_cuts=0), (1, 12),
         dict(min_vars=2, max_vars=16, span_layers=True, need_z=True, p_input=0.99)),
    ]
    cut_counts = (0, 500, 1000, 1500, 2000)
    ctx = gcp.Context(dev, hbm_budget_bytes=100 << 30)
    loaded = []
    for inst, srange, cargs in nets:
        net_id = ctx.init_net(inst.net.layers, inst.x_lo, inst.x_hi, inst.spec, inst.inter_lo, inst.inter_hi)
        sets = []
        for n in cut_counts:
            if n == 0:
                sets.append(-1)
                continue
            c = synth.make_cuts(rng, inst.net, inst.inter_lo, inst.inter_hi, inst.x_lo, inst.x_hi, n, **cargs)
            sets.append(ctx.add_cuts(net_id, c.ptr, c.layer, c.kind, c.index, c.coef, c.d)[0])
        loaded.append((inst, net_id, sets, srange))
    reqs = []
    t = 0.0
    for q in range(n_requests):
        t += float(rng.exponential(1.0 / rate))
        inst, net_id, sets, srange = loaded[int(rng.integers(0, len(loaded)))]
        n_sub = int(round(float(np.exp(rng.uniform(0.0, np.log(2048.0))))))
        sub = synth.make_subdomains(rng, inst.inter_lo, inst.inter_hi, n_sub, *srange)
        reqs.append((t, inst, net_id, sets[int(rng.integers(0, len(sets)))], sub))
    params = gcp.opt_params(iters, gcp.GCP_ADAM, gcp.GCP_BF16, 1, 0.1, 0.02, 0.02, 0.98)
    ctx.serve_start(max_inflight)
    tickets = []
    t0 = time.perf_counter()
    for q, (ta, inst, net_id, cs, sub) in enumerate(reqs):
        dt = ta - (time.perf_counter() - t0)
        if dt > 0:
            time.sleep(dt)
        tickets.append(ctx.serve_submit(net_id, cs, sub, params, rounds, SERVE_SEED + q))
    lat, rows_total, subs_total, errs, rel = [], 0, 0, [], []
    for (ta, inst, net_id, cs, sub), tk in zip(reqs, tickets):
        res, out = ctx.serve_wait(tk, sub.n * inst.spec.shape[0] + 8)
        if res.status != 0:
            raise RuntimeError(f"serving request failed with status {res.status}")
        lat.append(res.latency_ms)
        rows_total += res.rows
        subs_total += sub.n
        errs.append(res.max_err_vs_fp64)
        rel.append(res.max_rel_err_vs_fp64)
    wall = time.perf_counter() - t0
    ctx.serve_stop()
    ctx.close()
    lat = np.array(lat)
    return {
        "workload": "serving stream: MLP 8-16-16-3 / MLP 784-256x6-10 / CNN 3x32x32-c32-c64-fc512-fc10 mix",
        "requests": n_requests, "arrival_rate_per_s": rate, "rounds": rounds, "iters_per_round": iters,
        "subdomains_per_request": "1-2048 log-uniform", "cuts_per_request": list(cut_counts),
        "chain": "bf16", "certify": "fp64_outward_rounded", "hbm_budget_gb": 100, "max_inflight": max_inflight,
        "certified_subdomain_bounds_per_s": subs_total * rounds / wall,
        "requests_per_s": n_requests / wall, "wall_s": wall,
        "latency_ms": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99)),
                       "max": float(lat.max())},
        "max_err_vs_fp64": float(np.max(errs)),
        "max_rel_err_vs_fp64": float(np.max(rel)),
        "note": "latency = completion - submission; max errors are over every row of every request, chain "
                "(BF16) bound against the certified FP64 bound; relative = divided by max(1, |certified|)",
    }


def inter_bounds_bench(ctx, wname, inst, params):
    """Root intermediate bounds by the library's own certified propagation:
    wall time of CROWN (default slopes) and alpha-CROWN (20 Adam steps per
    neuron row) bounds for the workload's network, the fraction of unstable
    hidden neurons under interval, CROWN and alpha-CROWN bounds, the
    workload's mean certified bound under interval and CROWN root bounds
    (same seed and schedule), and a few rounds of branch and bound from the
    root on the CROWN bounds."""
    import numpy as np
    import torch
    from paper_2208_05740_gb300 import gcp

    def unstable(lo, hi):
        n = sum(len(x) for x in lo)
        return float(sum(int(np.sum((l < 0) & (h > 0))) for l, h in zip(lo, hi)) / n)

    out = {"note": "wall time on the host clock around the whole layer-by-layer procedure (one GPU)"}
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    lo, hi = ctx.intermediate_bounds(inst.net.layers, inst.x_lo, inst.x_hi)
    out["crown_s"] = time.perf_counter() - t0
    pa = gcp.opt_params(20, gcp.GCP_ADAM, gcp.GCP_FP32, 1, 0.1, 0.02, 0.02, 0.98)
    t0 = time.perf_counter()
    alo, ahi = ctx.intermediate_bounds(inst.net.layers, inst.x_lo, inst.x_hi, pa)
    out["alpha_crown_20it_s"] = time.perf_counter() - t0
    ibp = WORKLOADS[wname]["build"](inst.sub.n)
    out["unstable_fraction"] = {"interval": unstable(ibp.inter_lo, ibp.inter_hi), "crown": unstable(lo, hi),
                                "alpha_crown": unstable(alo, ahi)}
    net_i, cs_i = ctx.load_instance(ibp)
    D = ctx.duals_create(net_i, cs_i, ibp.sub, gcp.GCP_FP32)
    _, cert_ibp, _ = ctx.optimize_batch(D, params)
    ctx.duals_free(D)
    out["mean_certified"] = {"interval_root_bounds": float(np.mean(cert_ibp))}
    # branch and bound from the root on the CROWN bounds: a few rounds of full batches
    net_id, cs = ctx.load_instance(inst)
    pb = gcp.opt_params(20, gcp.GCP_ADAM, gcp.GCP_FP32, 1, 0.1, 0.02, 0.02, 0.98)
    na = sum(inst.net.dims[1:-1]) * inst.spec.shape[0]
    batch = 1024 if na <= 50_000 else 64
    out["bab"] = {}
    for rule, name in ((0, "by_duals"), (1, "static_intercept")):
        ctx.bab_verify(net_id, cs, pb, batch=batch, max_rounds=2, branching=rule)   # warm
        torch.cuda.synchronize()
        r = ctx.bab_verify(net_id, cs, pb, batch=batch, max_rounds=12, branching=rule)
        out["bab"][name] = {"batch": batch, "iters_per_round": 20, "rounds": r["rounds"],
                            "domains_bounded": r["domains_bounded"], "domains_verified": r["domains_verified"],
                            "domains_left": r["domains_left"], "verified": r["verified"], "min_bound": r["min_bound"],
                            "time_s": r["time_ms"] / 1e3,
                            "domains_per_s": r["domains_bounded"] / max(r["time_ms"] / 1e3, 1e-9)}
    return out


def quality(cert, ref, K):
    """Certified-bound quality of a form against a reference form on the same rows."""
    import numpy as np
    ok = cert >= ref - 1e-3 * np.maximum(1.0, np.abs(ref))
    return {"mean_certified": float(np.mean(cert)),
            "rows_certified_at_least_as_high": float(np.mean(ok)),
            "rows_certified_at_least_as_high_tol": "1e-3 * max(1, |reference form's certified bound|)",
            "subdomains_verified": float(np.mean(np.all(cert.reshape(-1, K) > 0, axis=1)))}


# tensor-core GEMMs that recompute their output from inputs they do not write:
# their launches can be issued twice to measure their cost inside the stream
IDEMPOTENT = ("gemm_tc_tf32x3", "gemm_tc_bf16")


def measure_workload(ctx, stream, dev, world, wname, prec_name, iters, n_sub, steps, warmup, flush,
                     forms=("other",), profile_all=False):
    """Time one workload on CROWN root bounds computed by the library before
    the timed region: device time of `steps` steps (L2 flushed, events on the
    library's stream), the dominant kernel's per-launch time in a second pass,
    the end-to-end rate through the C ABI from host buffers, and the other
    forms of the same workload. Returns (the JSON fields, instance, certified
    bounds)."""
    import numpy as np
    import torch
    from paper_2208_05740_gb300 import gcp
    prec = gcp.GCP_FP32 if prec_name == "fp32" else gcp.GCP_BF16
    inst = WORKLOADS[wname]["build"](n_sub, lambda net, lo, hi: ctx.intermediate_bounds(net.layers, lo, hi))
    net_id, cs = ctx.load_instance(inst)
    params = gcp.opt_params(iters, gcp.GCP_ADAM, prec, 1, 0.1, 0.02, 0.02, 0.98)
    D = ctx.duals_create(net_id, cs, inst.sub, gcp.GCP_FP32)
    K = inst.spec.shape[0]

    def step():
        ctx.duals_import(D)                       # default duals: same work every step
        return ctx.optimize_batch(D, params)      # the ascent + final bound + FP64 certify

    for _ in range(warmup):
        step()
    # shares of every kernel in one untimed step, to pick the dominant one
    gcp.profile_start("*")
    step()
    rep = gcp.profile_report()
    gcp.profile_stop()
    dominant = max(rep, key=lambda k: rep[k][2])
    total_ms = sum(v[2] for v in rep.values())
    if profile_all:
        for k, v in sorted(rep.items(), key=lambda kv: -kv[1][2]):
            print(f"# {wname} {k:28s} launches {v[0]:6d} ms {v[2]:9.3f} share {100 * v[2] / total_ms:5.1f}%",
                  file=sys.stderr)

    def timed_steps(selector, repeat=None):
        gcp.profile_start(selector)
        if repeat:
            gcp.profile_repeat(repeat)
        ts = []
        for _ in range(steps):
            flush.fill_(1.0)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            out = step()
            e1.record(stream)
            e1.synchronize()
            ts.append(e0.elapsed_time(e1))
        torch.cuda.synchronize()
        q_all = gcp.profile_query(None)
        q_dom = gcp.profile_query(dominant)
        gcp.profile_stop()
        return ts, out, q_all, q_dom

    # ---- timed region: device time per step. An event recorded between two
    # launches stops the second from overlapping the first one's tail
    # (programmatic dependent launch), so the step time is taken with the
    # launches only counted, and the dominant kernel's per-launch time in a
    # second pass of the same steps with each of its launches bracketed.
    sampler = ClockSampler(dev)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    sampler.start()
    times, (bound, cert, err), (launches_all, *_), _ = timed_steps(None)
    times_instr, _, _, (n_dom, ms_dom, fl_dom, by_dom) = timed_steps(dominant)
    # an idempotent GEMM's cost inside the stream, with no event between
    # launches: a third pass of the same steps issues each of its launches
    # twice; the extra device time over the launch count
    in_stream_ms = None
    if dominant in IDEMPOTENT and n_dom > 0:
        times_rep, *_ = timed_steps(None, repeat=dominant)
        extra = (sum(times_rep) - sum(times)) / n_dom
        in_stream_ms = extra if extra > 0 else None
    clocks = sampler.stop()
    total_s = max_over_ranks(sum(times) / 1000.0, f"cuda:{dev}")
    value = job_value(world, n_sub, steps, total_s)

    # ---- end to end through the C ABI from host buffers
    sub = inst.sub
    h2d = sub.ptr.nbytes + sub.layer.nbytes + sub.index.nbytes + sub.sign.nbytes
    c = inst.cuts
    nnz = len(c.coef)
    h2d += (c.n + 1) * 4 + c.n * 12 + sum(d + 1 for d in inst.net.dims[:-1]) * 4 + nnz * (4 + 1 + 8 + 4 + 4 + 4)
    d2h = 3 * 8 * inst.n_rows
    e2e_t = []
    for _ in range(steps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        D2 = ctx.duals_create(net_id, cs, sub, gcp.GCP_FP32)
        ctx.optimize_batch(D2, params)
        ctx.duals_free(D2)
        e2e_t.append(time.perf_counter() - t0)
    e2e_s = max_over_ranks(sum(e2e_t), f"cuda:{dev}")
    e2e_value = job_value(world, n_sub, steps, e2e_s)

    peaks, src = measured_peaks()
    bound_kind, peak, unit, note = kernel_peak(dominant, peaks, src)
    bracketed_ms = ms_dom / max(n_dom, 1)
    per_launch_ms = in_stream_ms if in_stream_ms else bracketed_ms
    if unit == "TFLOP/s":
        achieved = (fl_dom / max(n_dom, 1)) / (per_launch_ms / 1e3) / 1e12
    else:
        achieved = (by_dom / max(n_dom, 1)) / (per_launch_ms / 1e3) / 1e9
    lat = np.array(times)
    dtype = "f32" if prec_name == "fp32" else "bf16"
    res = {
        "value": value, "unit": UNIT, "steps": steps, "warmup": warmup, "ms_per_step": float(np.mean(times)),
        "dtype": dtype, "config": workload_config(wname, n_sub, iters, prec_name, world),
        "latency_ms": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99))},
        "bound": {"mean_certified": float(np.mean(cert)), "max_err_vs_fp64": float(np.max(err)),
                  "max_rel_err_vs_fp64": float(np.max(err / np.maximum(1.0, np.abs(cert)))),
                  "subdomains_verified": float(np.mean(np.all(cert.reshape(-1, K) > 0, axis=1)))},
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h)},
        "gpu_launches": int(launches_all),
        "roofline": {"kernel": dominant, "bound": bound_kind, "achieved": achieved, "peak": peak, "unit": unit,
                     "frac": achieved / peak, "traffic": traffic_for(dominant, WORKLOADS[wname]["name"]),
                     "peak_source": note, "launches": int(n_dom), "ms_per_launch": per_launch_ms,
                     "ms_per_launch_bracketed": bracketed_ms, "ms_per_launch_in_stream": in_stream_ms,
                     "share_of_step": (per_launch_ms * n_dom / sum(times)) if in_stream_ms else
                     rep[dominant][2] / total_ms,
                     "timed_in": ("third pass of the timed steps issuing each launch of this (idempotent) kernel "
                                  "twice: extra device time / launches (CUDA events around each step only); the "
                                  "second pass's per-launch event brackets, which stop programmatic dependent "
                                  "launch from overlapping neighbours, give ms_per_launch_bracketed")
                     if in_stream_ms else
                     "second pass of the timed steps, each launch of this kernel bracketed by events",
                     "ms_per_step_bracketed": float(np.mean(times_instr))},
        "clocks": clocks,
    }

    def timed_form(pf, n_timed):
        """The same workload under other optimiser settings: steps timed like
        the headline's (L2 flushed, events on the library's stream)."""
        ctx.duals_import(D)
        ctx.optimize_batch(D, pf)
        tb = []
        for _ in range(n_timed):
            flush.fill_(1.0)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            ctx.duals_import(D)
            _, cert_f, err_f = ctx.optimize_batch(D, pf)
            e1.record(stream)
            e1.synchronize()
            tb.append(e0.elapsed_time(e1))
        ms = float(np.mean(tb))
        out = {"value": n_sub * 1000.0 / ms, "ms_per_step": ms, "max_err_vs_fp64": float(np.max(err_f)),
               "max_rel_err_vs_fp64": float(np.max(err_f / np.maximum(1.0, np.abs(cert_f))))}
        out.update(quality(cert_f, cert, K))
        out["quality_against"] = dtype
        return out

    fm = {dtype: dict(value=value, ms_per_step=res["ms_per_step"], **quality(cert, cert, K))}
    n_form = max(3, min(steps, 5))
    if "other" in forms:
        # the same workload with the other chain precision (BF16 tensor-core
        # chain with FP32 accumulation <-> FP32 chain) and the same FP64
        # certification: throughput and certified-bound quality side by side
        other = gcp.GCP_BF16 if prec == gcp.GCP_FP32 else gcp.GCP_FP32
        fm["bf16" if prec == gcp.GCP_FP32 else "f32"] = timed_form(
            gcp.opt_params(iters, gcp.GCP_ADAM, other, 1, 0.1, 0.02, 0.02, 0.98), n_form)
    if "opt_pi" in forms:
        # the workload's chain with the ReLU duals pi optimised directly
        # (opt_pi, App. A's closing remark) instead of Lemma A.1's closed form
        fm[dtype + "_opt_pi"] = timed_form(gcp.opt_params(iters, gcp.GCP_ADAM, prec, 1, 0.1, 0.02, 0.02, 0.98,
                                                          opt_pi=1), n_form)
    res["forms"] = fm
    ctx.duals_free(D)
    return res, inst, params


def cpu_leg(wname, iters):
    v, desc = oracle_sample(oracle_instance(wname, 64), WORKLOADS[wname]["sample"], iters)
    return {"value": v, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
            "sample": desc + "; CROWN root bounds computed by the oracle"}


# --------------------------------------------------------------------------- GPU arm
def main():
    a = parse()
    if a.impl == "reference":
        return run_reference(a)
    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    from paper_2208_05740_gb300 import build, gcp
    build.build()
    dev = local
    torch.cuda.set_device(dev)
    stream = torch.cuda.Stream(device=dev)
    ctx = gcp.Context(dev)
    ctx.set_stream(stream.cuda_stream)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=f"cuda:{dev}")
    forms = () if a.no_bf16_form else ("other",)
    forms += () if a.no_opt_pi_form else ("opt_pi",)
    head, inst, params = measure_workload(ctx, stream, dev, world, a.workload, a.prec, a.iters, a.n_sub, a.steps,
                                          a.warmup, flush, forms, a.profile_all)
    # the largest single-GPU configuration (CNN, 4096 subdomains x 9 rows,
    # 1000 cuts, 50 steps, BF16 chain + FP64 certify) beside the headline
    extra = {}
    if a.workload == "mlp" and not a.no_cnn:
        w = WORKLOADS["cnn"]
        extra["cnn"], _, _ = measure_workload(ctx, stream, dev, world, "cnn", w["prec"], w["iters"], w["n_sub"],
                                              max(3, min(a.steps, 5)), a.warmup, flush, ("other",), a.profile_all)
    if rank != 0:
        ctx.close()
        return
    line = {"metric": METRIC, "value": head["value"], "unit": UNIT, "n_gpus": world, "steps": a.steps,
            "warmup": a.warmup, "ms_per_step": head["ms_per_step"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": head["dtype"], "data": "synthetic", "config": head["config"]}
    for k in ("latency_ms", "bound", "e2e", "gpu_launches", "roofline", "clocks", "forms"):
        line[k] = head[k]
    if extra:
        line["workloads"] = extra
    if world == 1 and not a.no_inter_bounds:
        line["intermediate_bounds"] = inter_bounds_bench(ctx, a.workload, inst, params)
    if a.serve_requests > 0 and world == 1:
        line["serving"] = serving_bench(dev, a.serve_requests)
        # below the measured service rate: latency once admitted, not the backlog
        line["serving"]["below_capacity"] = serving_bench(dev, max(8, a.serve_requests // 2), rate=1.0)
    if world == 1 and not a.no_cpu_baseline:
        line["cpu_baseline"] = cpu_leg(a.workload, a.iters)
        for k, v in extra.items():
            v["cpu_baseline"] = cpu_leg(k, v["config"]["iters"])
    print(json.dumps(line))
    ctx.close()


if __name__ == "__main__":
    main()
