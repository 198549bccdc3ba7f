"""The C ABI: header/binding/library agree (no GPU needed)."""
import os
import re

import numpy as np
import pytest

from paper_2208_05740_gb300 import gcp, synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared():
    txt = open(os.path.join(ROOT, "include", "gcp.h")).read()
    return sorted(set(re.findall(r"GCP_API\s+[\w\s\*]+?\b(gcp_\w+)\s*\(", txt)))


def test_header_declares_the_boundary_calls():
    names = declared()
    for n in ["gcp_init_net", "gcp_add_cuts", "gcp_bound_batch", "gcp_optimize_batch", "gcp_serve_start",
              "gcp_serve_submit", "gcp_serve_poll", "gcp_serve_wait", "gcp_serve_stop", "gcp_grad_batch"]:
        assert n in names


def test_library_loads_and_exports_every_declared_symbol():
    if not os.path.exists(gcp.LIB_PATH):
        from paper_2208_05740_gb300 import build
        build.build()
    L = gcp.lib()
    for n in declared():
        assert hasattr(L, n), n
    assert sorted(declared()) == sorted(gcp.EXPORTED)
    syms = os.popen(f"nm -D --defined-only {gcp.LIB_PATH}").read()
    exported = set(re.findall(r"\bT (gcp_\w+)", syms))
    assert exported == set(declared())


def test_create_fails_cleanly_without_a_gpu():
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(gcp.GCPError):
        gcp.Context(0)


def test_instances_have_the_documented_shapes():
    inst = synth.mlp_small()
    assert inst.net.dims == [8, 16, 16, 3] and inst.spec.shape == (2, 3) and inst.sub.n == 4
    assert inst.cuts.n == 8 and set(np.unique(inst.cuts.layer)) <= {1, 2}
    q = synth.mlp_256x6(n_sub=8)
    assert q.net.dims == [784] + [256] * 6 + [10] and q.spec.shape == (9, 10) and q.cuts.n == 200
    nsplit = np.diff(q.sub.ptr)
    assert nsplit.min() >= 1 and nsplit.max() <= 8
    # almost every cut touches an input variable and a ReLU indicator, and spans >= 2 layers
    c = q.cuts
    has_in = [np.any(c.layer[c.ptr[k]:c.ptr[k + 1]] == 0) for k in range(c.n)]
    has_z = [np.any(c.kind[c.ptr[k]:c.ptr[k + 1]] == 2) for k in range(c.n)]
    span = [len(set(c.layer[c.ptr[k]:c.ptr[k + 1]].tolist())) >= 2 for k in range(c.n)]
    assert np.mean(has_in) > 0.9 and all(has_z) and np.mean(span) > 0.95


def test_struct_layouts_match_the_binding(tmp_path):
    """Every struct of the header has the binding's size and field offsets
    (a small C program compiled against the header prints them)."""
    import ctypes as C
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    pairs = [("gcp_layer_desc", gcp.LayerDesc), ("gcp_subdomains", gcp.Subdomains), ("gcp_opt_params", gcp.OptParams),
             ("gcp_bab_params", gcp.BabParams), ("gcp_bab_result", gcp.BabResult), ("gcp_request", gcp.Request),
             ("gcp_result", gcp.Result)]
    lines = ['#include <stddef.h>', '#include <stdio.h>', '#include "gcp.h"', "int main(void) {"]
    for cname, py in pairs:
        lines.append(f'  printf("{cname} size %zu\\n", sizeof({cname}));')
        for f, _ in py._fields_:
            lines.append(f'  printf("{cname} {f} %zu\\n", offsetof({cname}, {f}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = dict((" ".join(l.split()[:2]), int(l.split()[2]))
               for l in subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.splitlines())
    for cname, py in pairs:
        assert got[f"{cname} size"] == C.sizeof(py), cname
        for f, _ in py._fields_:
            assert got[f"{cname} {f}"] == getattr(py, f).offset, (cname, f)
