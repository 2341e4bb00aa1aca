"""Host-side check of the row-block-tiled Gram's tile tables (no GPU): a small program built
with nvcc against the library's own gram_tiles verifies that every block of the upper
block triangle is computed exactly once, from loaded operands, within 512 accumulator
columns and two shared-memory stages."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2512_15187_gb300", "csrc")


def _nvcc():
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    return None


def test_tile_tables(tmp_path):
    nvcc = _nvcc()
    if nvcc is None:
        pytest.skip("nvcc not found")
    exe = str(tmp_path / "gram_tiles_check")
    cmd = [nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-std=c++17",
           "--expt-relaxed-constexpr", "-I", CSRC,
           os.path.join(ROOT, "tests", "native", "gram_tiles_check.cu"),
           os.path.join(CSRC, "gram_tiled.cu"), "-o", exe]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr[-2000:]
    out = subprocess.run([exe], capture_output=True, text=True, timeout=60)
    assert out.returncode == 0 and "ALL OK" in out.stdout, out.stdout
