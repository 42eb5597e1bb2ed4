"""The CUDA path's entry functions, compiled for the host, against the oracle (CPU; needs nvcc).

The entry math of the library (hbi_entry_math.cuh: the full-space closed form and the
half-space correction with jets and Radon's rule) is __host__ __device__; tests/host_entries.cu
runs it on the host with the library's own element frames (hbi_host.cpp).  This checks the
formulas of the CUDA path on every CPU test run; the GPU tests check the same functions on the
device.  Tolerances as in the GPU entry tests: full space 1e-9 of the largest entry (closed
form against the oracle's adaptive quadrature), half space 2e-6 of each pair's largest entry
(the library's quadrature of the correction)."""
import os
import shutil
import subprocess

import numpy as np
import pytest

import oracle
from synthetic import meshes, rng

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
MU, NU = 32e9, 0.25


def _nvcc():
    for c in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", shutil.which("nvcc")):
        if c and os.path.exists(c):
            return c
    return None


@pytest.fixture(scope="module")
def harness(tmp_path_factory):
    nvcc = _nvcc()
    if nvcc is None:
        pytest.skip("nvcc not available")
    out = str(tmp_path_factory.mktemp("host_entries") / "host_entries")
    src = [os.path.join(ROOT, "tests", "host_entries.cu"),
           os.path.join(ROOT, "paper_2110_12165_gb300", "csrc", "hbi_host.cpp")]
    cmd = [nvcc, "-O2", "-std=c++17", "-gencode", "arch=compute_103a,code=sm_103a", "-o", out] + src
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr[-3000:]
    return out


def _entries(exe, tmp, m, op, recv, src, half, rake=None):
    n, nv = m.n_elem, m.verts.shape[1]
    fin, fout = os.path.join(tmp, "in.bin"), os.path.join(tmp, "out.bin")
    with open(fin, "wb") as f:
        np.array([n, nv, op, int(half), len(recv)], np.int32).tofile(f)
        np.array([MU, NU]).tofile(f)
        np.ascontiguousarray(m.verts, np.float64).tofile(f)
        np.ascontiguousarray(np.zeros(n) if rake is None else rake, np.float64).tofile(f)
        np.stack([recv, src], 1).astype(np.int32).tofile(f)
    r = subprocess.run([exe, fin, fout], capture_output=True, text=True)
    assert r.returncode == 0, r.returncode
    return np.fromfile(fout).reshape(len(recv), oracle.OP_NOUT[op], oracle.OP_NIN[op])


def _all_pairs(n):
    i, j = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    return i.ravel().astype(np.int32), j.ravel().astype(np.int32)


@pytest.mark.parametrize("kind", ["rect", "tri"])
def test_full_space_entries(harness, tmp_path, kind):
    m = meshes.planar_vertical_rect(5, 4, 250.0) if kind == "rect" else meshes.scaled_thrust_mesh(5, 3, seed=8)
    recv, src = _all_pairs(m.n_elem)
    op = oracle.OP_VEC_FULL
    E = _entries(harness, str(tmp_path), m, op, recv, src, False)
    ref = oracle.pair_entries(m, op, recv, src, MU, NU)
    assert np.abs(E - ref).max() < 1e-9 * np.abs(ref).max()


@pytest.mark.parametrize("kind,op", [("shallow-rect", 3), ("shallow-rect", 1), ("thrust-tri", 3)])
def test_half_space_entries(harness, tmp_path, kind, op):
    m = (meshes.dipping_rect(6, 4, 250.0, 40.0, origin=(0.0, 0.0, -50.0)) if kind == "shallow-rect"
         else meshes.scaled_thrust_mesh(5, 3, seed=8))
    recv, src = _all_pairs(m.n_elem)
    rake = rng.uniform(71, m.n_elem) * np.pi if op == 1 else None
    E = _entries(harness, str(tmp_path), m, op, recv, src, True, rake)
    ref = oracle.pair_entries(m, op, recv, src, MU, NU, rake=rake, half_space=True)
    full = oracle.pair_entries(m, op, recv, src, MU, NU, rake=rake)
    scale = np.abs(ref).max(axis=(1, 2), keepdims=True)
    assert (np.abs(E - ref) / scale).max() < 2e-6
    assert (np.abs(full - ref) / scale).max() > 1e-2


def test_half_space_entries_on_the_thrust_fault(harness, tmp_path):
    """2,000 sampled pairs of the 160,000-element thrust fault: most sources are far from the
    receiver's image and take the three-point rule."""
    m = meshes.scaled_thrust_mesh(400, 200, seed=3)
    n = m.n_elem
    u = rng.uniform(76, 4000)
    recv, src = (u[:2000] * n).astype(np.int32), (u[2000:] * n).astype(np.int32)
    op = oracle.OP_VEC_FULL
    E = _entries(harness, str(tmp_path), m, op, recv, src, True)
    ref = oracle.pair_entries(m, op, recv, src, MU, NU, half_space=True)
    scale = np.abs(ref).max(axis=(1, 2), keepdims=True)
    assert (np.abs(E - ref) / scale).max() < 2e-6
