"""Failure detection without a GPU fault, and checkpoint / resume.

Device conditions become statuses read by the host, never traps: a wait that cannot
complete gives up after its time limit (HBI_ERR_TIMEOUT) and the context stays usable; a
non-finite state and a non-positive normal stress each end the run with their own status
once the step size underflows.  A storm of rejected attempts (an unreachable tolerance) is
absorbed: the embedded 5th/4th-order difference is O(dt^2) once the stages agree, so it falls
below an ulp of the state, and the step is accepted, long before the step size underflows.
A run dumped and resumed on a rebuilt handle continues bit for bit."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
import paper_2110_12165_gb300 as hbi
from synthetic import friction, meshes, rng
from gpu_util import dev, host, rel_l2

pytestmark = pytest.mark.gpu

MU, NU = 32e9, 0.25


def _small():
    m = meshes.planar_vertical_rect(16, 8, 250.0)
    n = m.n_elem
    a, b = np.full(n, 0.010), np.full(n, 0.015)
    fr = hbi.friction(dev(a), dev(b), dev(np.full(n, 0.005)), dev(np.zeros(n)), 0.6, 1e-6, 1e-9, MU, 3460.0)
    phi, tau = oracle.steady_state(np.full(n, 1e-9) * (1 + 1e-3 * rng.uniform(90, n)), a, b, np.full(n, 50e6),
                                   0.6, 1e-6)
    y = np.concatenate([phi, tau, np.full(n, 50e6), np.zeros(n)])
    h = hbi.hbi_build(m.verts, MU, NU, oracle.OP_RAKE_SHEAR, 1e-6, 16, 1, "fp64", rake=np.zeros(n))
    return m, h, fr, y


def test_stalled_device_wait_reports_timeout_and_context_survives():
    assert hbi.hbi_stalled_wait_status() == -8                    # HBI_ERR_TIMEOUT
    m, h, fr, y = _small()
    x = torch.ones(m.n_elem, dtype=torch.float64, device="cuda")
    out = torch.zeros_like(x)
    hbi.hbi_matvec(h, x, out)                                   # the context is still usable
    assert torch.isfinite(out).all()


@pytest.mark.parametrize("kind,status", [("nan", -7), ("sigma", -6)])
def test_failed_runs_stop_with_their_status(kind, status):
    m, h, fr, y = _small()
    n = m.n_elem
    if kind == "nan":
        y[5] = np.nan                                           # a non-finite state value
    else:
        y[2 * n + 7] = -1e6                                     # a tensile normal stress
    st, done, rec = hbi.hbi_step(h, fr, dev(y), dev([0.0]), dev([1e5]), 1e-4, 5)
    assert st == status and done == 0
    # the handle keeps working after the failed run
    st2, done2, _ = hbi.hbi_step(h, fr, dev(_small()[3]), dev([0.0]), dev([1e5]), 1e-4, 3)
    assert st2 == 0 and done2 == 3


@pytest.mark.parametrize("kind,status", [("nan", -7), ("sigma", -6)])
def test_failed_rake_free_runs_stop_with_their_status(kind, status):
    """The same conditions under rake-free friction (hbi_step_vector, 2 -> 2 operator)."""
    m = meshes.planar_vertical_rect(16, 8, 250.0)
    n = m.n_elem
    a, b = np.full(n, 0.010), np.full(n, 0.015)
    fr = hbi.friction(dev(a), dev(b), dev(np.full(n, 0.005)), dev(np.zeros(n)), 0.6, 1e-6, 1e-9, MU, 3460.0)
    phi, tau = oracle.steady_state(np.full(n, 1e-9) * (1 + 1e-3 * rng.uniform(91, n)), a, b, np.full(n, 50e6),
                                   0.6, 1e-6)
    y = np.concatenate([phi, tau, np.zeros(n), np.full(n, 50e6), np.zeros(2 * n)])
    h = hbi.hbi_build(m.verts, MU, NU, oracle.OP_VEC_SHEAR, 1e-6, 16, 1, "fp64", rake=np.zeros(n))
    bad = y.copy()
    if kind == "nan":
        bad[n + 3] = np.nan                                     # a non-finite traction
    else:
        bad[3 * n + 7] = -1e6                                   # a tensile normal stress
    st, done, _ = hbi.hbi_step_vector(h, fr, dev(bad), dev([0.0]), dev([1e5]), 1e-4, 5)
    assert st == status and list(done) == [0]
    st2, done2, _ = hbi.hbi_step_vector(h, fr, dev(y), dev([0.0]), dev([1e5]), 1e-4, 3)
    assert st2 == 0 and list(done2) == [3]


def test_reject_storm():
    m, h, fr, y = _small()
    n = m.n_elem
    # near steady sliding: absorbed (increments below an ulp of the state accept the step)
    st, done, rec = hbi.hbi_step(h, fr, dev(y), dev([0.0]), dev([1e5]), 1e-300, 3)
    assert st == 0 and done == 3 and rec[0, 3] >= 1
    # during fast slip (state 0.2 below steady state: V ~ 0.5 m/s) it takes a few halvings
    y2 = y.copy()
    y2[:n] -= 0.2
    st, done, rec = hbi.hbi_step(h, fr, dev(y2), dev([0.0]), dev([1e-3]), 1e-300, 3)
    assert st == 0 and done == 3 and rec[0, 3] >= 1 and 1e-12 < rec[0, 1] < 1e-3


def test_checkpoint_resume_on_a_rebuilt_handle_is_bitwise(tmp_path):
    m = meshes.scaled_thrust_mesh(24, 12, seed=3)
    F = friction.thrust_friction(m, seed=3)
    n = m.n_elem
    build = dict(aca_eps=1e-5, leaf_size=16, lattice_depth=2, storage="fp32", recompress_eps=1e-5)
    mk = lambda: hbi.hbi_build(m.verts, F.mu, F.nu, oracle.OP_VEC_FULL, build["aca_eps"], build["leaf_size"],
                               build["lattice_depth"], build["storage"], rake=F.rake,
                               recompress_eps=build["recompress_eps"])
    fr = hbi.friction(dev(F.a), dev(F.b), dev(F.dc), dev(F.rake), F.f0, F.V0, F.Vpl, F.mu, F.cs)
    phi, tau = oracle.steady_state(F.V_init, F.a, F.b, F.sigma0, F.f0, F.V0)
    y0 = np.concatenate([phi, tau, F.sigma0, np.zeros(n)])
    # one run of 40 steps
    h = mk()
    s, t, dt = dev(y0), dev([0.0]), dev([1e5])
    st, done, rec = hbi.hbi_step(h, fr, s, t, dt, 1e-4, 40)
    assert st == 0
    del h
    # 20 steps, dump, a new handle, 20 more
    h1 = mk()
    s1, t1, dt1 = dev(y0), dev([0.0]), dev([1e5])
    st, done, rec1 = hbi.hbi_step(h1, fr, s1, t1, dt1, 1e-4, 20)
    path = str(tmp_path / "run.npz")
    hbi.checkpoint_save(path, s1, t1, dt1, **build)
    del h1
    state, tc, dtc, b = hbi.checkpoint_load(path)
    assert float(b["aca_eps"]) == build["aca_eps"] and str(b["storage"]) == build["storage"]
    h2 = mk()
    s2, t2, dt2 = dev(state), dev(tc), dev(dtc)
    st, done, rec2 = hbi.hbi_step(h2, fr, s2, t2, dt2, 1e-4, 20)
    assert st == 0
    assert np.array_equal(host(s2), host(s)) and host(t2)[0] == host(t)[0] and host(dt2)[0] == host(dt)[0]
    assert np.array_equal(np.concatenate([rec1, rec2])[:, :3], rec[:, :3])


def _build_all_packers(m):
    """A build that makes every kind of device allocation of the library: entries, ACA and
    recompression, the product streams of H and H^T, and the multi-RHS panels."""
    return hbi.hbi_build(m.verts, 32e9, 0.25, oracle.OP_VEC_FULL, 1e-6, 8, 2, "mixed", recompress_eps=1e-6,
                         transpose=True, multi_rhs=True)


def test_every_failed_device_allocation_of_a_build_reports_oom_and_frees_the_rest():
    """HBI_ERR_OOM on the host side: hbi_inject_failure makes the k-th device allocation of the
    library fail as cudaMalloc would, for k = 1, 2, ... until a build no longer reaches it.
    Every failed build reports HBI_ERR_OOM and returns the device memory it had taken (the
    free memory comes back to within 2 MiB of where it started), and a build afterwards
    computes the product the oracle does."""
    m = meshes.scaled_thrust_mesh(12, 6, seed=2)            # N = 144
    x = rng.normal(9, 2 * m.n_elem)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    failed = 0
    for k in range(1, 400):
        hbi.hbi_inject_failure(hbi.HBI_INJECT_ALLOC, k)
        try:
            h = _build_all_packers(m)
        except hbi.HbiError as e:
            assert "HBI_ERR_OOM" in str(e), (k, str(e))
            failed += 1
            torch.cuda.synchronize()
            assert abs(torch.cuda.mem_get_info()[0] - free0) < 2 << 20, (k, free0 - torch.cuda.mem_get_info()[0])
            continue
        hbi.hbi_inject_failure(hbi.HBI_INJECT_NONE)
        del h
        break
    hbi.hbi_inject_failure(hbi.HBI_INJECT_NONE)
    assert failed >= 20                                      # the build allocates at many sites
    h = _build_all_packers(m)
    y = torch.zeros(3 * m.n_elem, dtype=torch.float64, device="cuda")
    hbi.hbi_matvec(h, dev(x), y)
    yd = oracle.dense_matvec(m, oracle.OP_VEC_FULL, x, 32e9, 0.25)
    assert rel_l2(host(y), yd) < 2e-3


def test_aca_failure_is_reported_and_the_next_build_works():
    """HBI_ERR_ACA_FAIL: a block's ACA reported as not converged within the rank limit (host-side
    injection) ends the build with that status and no leaked memory; the next build works."""
    m = meshes.scaled_thrust_mesh(24, 12, seed=2)            # N = 576: admissible blocks of low rank
    build = lambda: hbi.hbi_build(m.verts, 32e9, 0.25, oracle.OP_VEC_FULL, 1e-4, 16, 2, "mixed", recompress_eps=1e-4,
                                  transpose=True, multi_rhs=True)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for k in (1, 3):                                         # the first block's result, or a later one
        hbi.hbi_inject_failure(hbi.HBI_INJECT_ACA, k)
        with pytest.raises(hbi.HbiError, match="HBI_ERR_ACA_FAIL"):
            build()
        hbi.hbi_inject_failure(hbi.HBI_INJECT_NONE)
        torch.cuda.synchronize()
        assert abs(torch.cuda.mem_get_info()[0] - free0) < 2 << 20
    h = build()
    assert h.stats()["n_lowrank"] > 0
