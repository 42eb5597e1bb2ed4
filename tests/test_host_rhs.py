"""The CUDA path's element-wise rate-and-state arithmetic, compiled for the host, against the
oracle (CPU; needs nvcc).

hbi_ode_math.cuh holds the functions the stage kernels apply per element: V from the state
(Eq. 7 read as in the oracle), dphi/dt (Eq. 8), dsigma/dt (Eq. 10), dtau/dt (Eq. 12 with
13a-c) from the product of the slip-rate deficit (the loading of Eqs. 21-22 folded in), and
the rake-free form.  tests/host_rhs.cu runs them on the host; they are compared with the
oracle's element-wise right-hand side given the same stress rates.  Both sides evaluate the
same formulas in FP64 in a different order: agreement to 1e-11 relative."""
import os
import shutil
import subprocess

import numpy as np
import pytest

import oracle
from synthetic import friction, meshes, rng

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


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
    out = str(tmp_path_factory.mktemp("host_rhs") / "host_rhs")
    cmd = [nvcc, "-O2", "-std=c++17", "-gencode", "arch=compute_103a,code=sm_103a", "-o", out,
           os.path.join(ROOT, "tests", "host_rhs.cu")]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr[-3000:]
    return out


def _run(exe, tmp, op, vec, F, y, s):
    n = len(F.a)
    fin, fout = os.path.join(tmp, "in.bin"), os.path.join(tmp, "out.bin")
    with open(fin, "wb") as f:
        np.array([n, op, int(vec)], np.int32).tofile(f)
        np.array([F.f0, F.V0, F.Vpl, F.mu / (2 * F.cs)]).tofile(f)
        for arr in (F.a, F.b, F.dc, F.rake, y, s):
            np.ascontiguousarray(arr, np.float64).tofile(f)
    r = subprocess.run([exe, fin, fout], capture_output=True, text=True)
    assert r.returncode == 0
    out = np.fromfile(fout)
    nc = 4 if vec else 3
    return out[:nc * n], out[nc * n:]


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("op", [0, 1, 2, 3])
def test_fixed_rake_rhs(harness, tmp_path, op):
    m = meshes.scaled_thrust_mesh(12, 6, seed=5)
    F = friction.thrust_friction(m, seed=5)
    n = m.n_elem
    phi, tau = oracle.steady_state(F.V_init, F.a, F.b, F.sigma0, F.f0, F.V0)
    # slip rates from 1e-12 to about 1 m/s, so that the radiation-damping terms of Eq. 12 matter
    tau = tau + F.a * F.sigma0 * np.log(10.0) * (12.0 * rng.uniform(81, n) - 3.0)
    y = np.concatenate([phi, tau, F.sigma0])
    V_ref, _ = oracle.slip_rate(y[:n], y[n:2 * n], y[2 * n:], F.a, F.V0)
    dv = V_ref - F.Vpl
    # the product input: the deficit along the rake (one-component operators) or its strike and
    # dip components
    x = dv if oracle.OP_NIN[op] == 1 else np.concatenate([dv * np.cos(F.rake), dv * np.sin(F.rake)])
    rows = np.arange(n)
    s = oracle.dense_rows(m, op, rows, x, F.mu, F.nu, rake=F.rake)          # (n, n_out)
    ref = oracle.rhs_rows(op, F, y, rows, s)                                 # (n, 3)
    dy, V = _run(harness, str(tmp_path), op, False, F, y, s)
    assert _rel(V, V_ref) < 1e-12
    for c in range(3):
        if np.linalg.norm(ref[:, c]) == 0:
            assert np.all(dy[c * n:(c + 1) * n] == 0)
        else:
            assert _rel(dy[c * n:(c + 1) * n], ref[:, c]) < 1e-11, (op, c)


def test_rake_free_rhs(harness, tmp_path):
    m = meshes.scaled_thrust_mesh(6, 4, seed=6)
    F = friction.thrust_friction(m, seed=6)
    n = m.n_elem
    H = oracle.HMatrix(m, oracle.OP_VEC_FULL, 1e-10, 8, 1, F.mu, F.nu, rake=F.rake)
    phi, tau = oracle.steady_state(F.V_init, F.a, F.b, F.sigma0, F.f0, F.V0)
    ang = F.rake + 0.3 * (2 * rng.uniform(82, n) - 1)                         # traction off the rake
    tau = tau + F.a * F.sigma0 * np.log(10.0) * (12.0 * rng.uniform(83, n) - 3.0)
    y = np.concatenate([phi, tau * np.cos(ang), tau * np.sin(ang), F.sigma0])
    dy_ref, V_ref = H.rhs_vec(F, y)
    x = np.concatenate([V_ref[:n] - F.Vpl * np.cos(F.rake), V_ref[n:] - F.Vpl * np.sin(F.rake)])
    s = H.matvec(x).reshape(3, n).T                                          # (n, 3)
    dy, V = _run(harness, str(tmp_path), oracle.OP_VEC_FULL, True, F, y, s)
    assert _rel(V, V_ref) < 1e-12
    for c in range(4):
        assert _rel(dy[c * n:(c + 1) * n], dy_ref[c * n:(c + 1) * n]) < 1e-11, c


def test_step_control(harness, tmp_path):
    """Eqs. 14-15 as the stage kernels decide them (step_control) against the oracle's
    controller: accept/reject and the next step size, over error ratios from 1e-8 to 1e4
    (both sides of eps_RK, the clamps at dt/2 and 2 dt, err = 0), and a non-finite error (NaN
    or infinity), which must reject and halve the step."""
    eps = 1e-4
    ratios = np.concatenate([[0.0, 1.0, 1.0 + 1e-12, 1.0 - 1e-12, np.nan, np.inf], np.logspace(-8, 4, 61)])
    dts = 10.0 ** rng.uniform(84, len(ratios)) * 1e3
    fin, fout = os.path.join(str(tmp_path), "in.bin"), os.path.join(str(tmp_path), "out.bin")
    with open(fin, "wb") as f:
        np.array([len(ratios), 0, 2], np.int32).tofile(f)
        np.stack([ratios * eps, np.full(len(ratios), eps), dts], 1).tofile(f)
    assert subprocess.run([harness, fin, fout]).returncode == 0
    out = np.fromfile(fout).reshape(-1, 2)
    for (acc, dt_new), r, dt in zip(out, ratios, dts):
        acc_ref, dt_ref = oracle.controller(r * eps, eps, dt)
        assert bool(acc) == acc_ref, r
        assert dt_new == pytest.approx(dt_ref, rel=1e-14), r
        assert 0.5 * dt <= dt_new <= 2.0 * dt
        if not np.isfinite(r):
            assert not acc and dt_new == 0.5 * dt, r
