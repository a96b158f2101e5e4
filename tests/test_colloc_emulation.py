"""The collocated stages of the generic (FP64 / double-float) tile kernel, run on the host.

``tests/colloc_emulation.cu`` includes the library's kernel header, runs the host-callable stage
functions of ``Colloc<D1, TT>`` in loops over the thread indices between the kernel's barriers,
and compares the tile's output with a per-element tensor-product J v (10 tile shapes, orders 1-6).
It needs nvcc (host compilation only; no GPU)."""
from __future__ import annotations

import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(ROOT, "paper_2506_00746_gb300", "csrc")


def _nvcc():
    for c in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if c and os.path.exists(c):
            return c
    return None


def test_collocated_stages_match_element_reference(tmp_path):
    nvcc = _nvcc()
    if nvcc is None:
        pytest.skip("nvcc not available")
    exe = str(tmp_path / "colloc_emulation")
    cmd = [nvcc, "-O2", "-std=c++17", "--expt-relaxed-constexpr", f"-I{CSRC}", f"-I{os.path.join(ROOT, 'include')}",
           "-o", exe, os.path.join(HERE, "colloc_emulation.cu"), os.path.join(CSRC, "rules1d.cpp")]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr[-3000:]
    run = subprocess.run([exe], capture_output=True, text=True, timeout=300)
    assert run.returncode == 0 and "ALL OK" in run.stdout, run.stdout + run.stderr
    assert run.stdout.count("slots written != once: 0") == 20
