"""CPU index checks of the step kernels' shared-memory plans (no GPU).

`tests/geometry_check.cu` replays, on the host, the index maps of every tile variant the
library registers: the Stockham stages of the row and column transforms (each element read
and written once per stage, inside the padded buffer; compile-time offsets equal to the
padded indices), the shared-memory regions (aligned, disjoint, inside the launch's bytes),
the row pass's G-tile staging (every copy aligned and inside its plane, every source chunk
inside its column's rows) and the first stage's reads of the staged tile (each slot written
by the staging).  It stands in for a bounds-checking build of the kernels.
"""
import os
import shutil
import subprocess
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _nvcc():
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    return None


def test_every_registered_tile_plan_stays_in_bounds():
    nvcc = _nvcc()
    if nvcc is None:
        pytest.skip("nvcc is not available")
    with tempfile.TemporaryDirectory() as tmp:
        exe = os.path.join(tmp, "geometry_check")
        cmd = [nvcc, "-std=c++17", "-O1", "-I" + os.path.join(ROOT, "include"),
               "-I" + os.path.join(ROOT, "paper_2304_03306_gb300", "csrc"),
               os.path.join(ROOT, "tests", "geometry_check.cu"), "-o", exe]
        r = subprocess.run(cmd, capture_output=True, text=True, timeout=600)
        assert r.returncode == 0, r.stderr[-4000:]
        r = subprocess.run([exe], capture_output=True, text=True, timeout=300)
        assert r.returncode == 0, r.stdout[-4000:]
        last = r.stdout.strip().splitlines()[-1]
        checked = int(last.split()[0])
        assert checked > 300 and last.endswith(" 0 failures"), last


def test_checker_covers_the_registered_variants():
    """The checker's variant lists are the registry's (csrc/ttsh_ops_impl.cuh), entry for
    entry, so a variant added to the library cannot escape the index checks."""
    import re
    impl = open(os.path.join(ROOT, "paper_2304_03306_gb300", "csrc", "ttsh_ops_impl.cuh")).read()
    chk = open(os.path.join(ROOT, "tests", "geometry_check.cu")).read()

    def shapes(pattern, text):
        return [s for s in re.findall(pattern, text) if not s.startswith("default")]

    rows = shapes(r"add_row_variant<T, N, ([^>]*?)>\(o\)", impl)
    cols = shapes(r"add_col_variant<T, N, ([^>]*?)>\(o\)", impl)
    assert rows and cols
    assert rows == shapes(r"check_row<T, N, ROW_STEP, ([^>]*?)>\(\)", chk)
    assert cols == shapes(r"check_col<T, N, COL_STEP, ([^>]*?)>\(\)", chk)
    # and both start from each size's default shapes
    assert "add_row_variant<T, N, default_step_rows<T, N>(), default_step_row_pe<T, N>(), default_row_cluster<T, N>()>(o)" in impl
    assert "check_row<T, N, ROW_STEP, default_step_rows<T, N>(), default_step_row_pe<T, N>(), default_row_cluster<T, N>()>()" in chk
    assert "add_col_variant<T, N, default_step_col_pe<T, N>()>(o)" in impl
    assert "check_col<T, N, COL_STEP, default_step_col_pe<T, N>()>()" in chk
