"""The bounds checks of the HMVM work tables (csrc/hbi_tables.h, run by the packer on every
operator and, in the bounds-checked build, by the product kernels on the device) compiled for
the host with the library's own table structures (CPU; needs nvcc): a valid table set passes,
and every corruption of a batch, item, task or gather index -- a segment past its stream, an x
slice past [x | t] or off its alignment, t or output rows out of range, a gather range or index
out of range, an index pair past the end, shared memory too small -- is reported."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _nvcc():
    for c in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", shutil.which("nvcc")):
        if c and os.path.exists(c):
            return c
    return None


def test_corrupted_tables_are_reported(tmp_path):
    nvcc = _nvcc()
    if nvcc is None:
        pytest.skip("nvcc not available")
    exe = str(tmp_path / "host_tables")
    r = subprocess.run([nvcc, "-O1", "-std=c++17", "-gencode", "arch=compute_103a,code=sm_103a", "-o", exe,
                        os.path.join(ROOT, "tests", "host_tables.cu")], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr[-3000:]
    out = subprocess.run([exe], capture_output=True, text=True, check=True).stdout.split("\n")
    res = dict((l.split()[0], int(l.split()[1])) for l in out if l.strip())
    assert res.pop("valid") == 0
    assert len(res) >= 15
    for name, bad in res.items():
        assert bad >= 1, name
