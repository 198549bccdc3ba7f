"""The host-side launch checks (csrc/prof.cu), without a GPU.

A caller-owned array registered for one call beside a library allocation at
the same base neither replaces nor removes the library's entry, and a launch
check that fails on one host thread is reported to that thread only (serving
runs groups of different networks on concurrent worker threads).
"""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_registry_keeps_library_entries_and_reports_per_thread(tmp_path):
    nvcc = shutil.which("nvcc") or ("/usr/local/cuda/bin/nvcc" if os.path.exists("/usr/local/cuda/bin/nvcc") else None)
    if nvcc is None:
        pytest.skip("nvcc not available")
    exe = tmp_path / "launch_checks"
    subprocess.run([nvcc, "-std=c++17", "-O1", "-I", os.path.join(ROOT, "include"),
                    "-I", os.path.join(ROOT, "paper_2208_05740_gb300", "csrc"),
                    os.path.join(ROOT, "tests", "launch_checks_driver.cu"),
                    os.path.join(ROOT, "paper_2208_05740_gb300", "csrc", "prof.cu"), "-o", str(exe)],
                   check=True, capture_output=True)
    r = subprocess.run([str(exe)], capture_output=True, text=True)
    assert r.returncode == 0, r.stdout + r.stderr
    assert "registry ok" in r.stdout
