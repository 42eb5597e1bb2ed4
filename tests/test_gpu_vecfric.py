"""GPU parity of rake-free (vector) friction against the oracle (FP64 storage on the oracle's
own factors, so only summation order differs).

The traction starts off the loading direction (up to ~0.3 rad) so that the part of the
2x2 radiation-damping solve perpendicular to the traction is exercised.  Tolerances follow
the fixed-rake parity tests: dy/dt to 1e-9 per component, one attempt to 1e-12 (state) and
1e-6 (error-controlled step size), interseismic runs with identical accept/reject decisions
to 1e-7, earthquakes (where the dynamics amplify rounding) event times to 1% and peak slip
rates to 2%."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
import paper_2110_12165_gb300 as hbi
from synthetic import friction, meshes, rng
from gpu_util import dev, host, import_oracle, rel_l2

pytestmark = pytest.mark.gpu


def _setup(kind):
    if kind == "thrust-full-N900":
        m = meshes.scaled_thrust_mesh(30, 15, seed=2)       # nonplanar, normal coupling
        F = friction.thrust_friction(m, seed=2)
        op, eps, leaf, L = oracle.OP_VEC_FULL, 1e-5, 16, 1
    else:
        m = meshes.dipping_rect(16, 8, 500.0, 40.0)         # N = 128, planar, sigma constant
        F = friction.ensemble_friction(m, seed=3)
        op, eps, leaf, L = oracle.OP_VEC_SHEAR, 1e-6, 8, 1
    H = oracle.HMatrix(m, op, eps, leaf, L, F.mu, F.nu, rake=F.rake)
    n = m.n_elem
    phi, tau = oracle.steady_state(F.V_init, F.a, F.b, F.sigma0, F.f0, F.V0)
    ang = F.rake + 0.3 * np.sin(0.7 * np.arange(n))          # traction off the loading direction
    y0 = np.concatenate([phi, tau * np.cos(ang), tau * np.sin(ang), F.sigma0])
    return m, F, H, y0


def _fric(F):
    return hbi.friction(dev(F.a), dev(F.b), dev(F.dc), dev(F.rake), F.f0, F.V0, F.Vpl, F.mu, F.cs)


KINDS = ["thrust-full-N900", "dipping-shear-N128"]


@pytest.mark.parametrize("kind", KINDS)
def test_rhs_vec_matches_oracle(kind):
    m, F, H, y0 = _setup(kind)
    n = m.n_elem
    y = y0.copy()
    y[:n] += 0.01 * rng.normal(7, n)                          # slip rates spanning decades
    dy_ref, V_ref = H.rhs_vec(F, y)
    h = import_oracle(H, "fp64")
    dy = torch.zeros(4 * n, dtype=torch.float64, device="cuda")
    V = torch.zeros(2 * n, dtype=torch.float64, device="cuda")
    hbi.hbi_rhs_vec(h, _fric(F), dev(y), dy, V)
    dy, V = host(dy), host(V)
    assert np.allclose(V, V_ref, rtol=1e-12, atol=1e-14 * np.abs(V_ref).max())
    for c in range(4):
        ref = dy_ref[c * n:(c + 1) * n]
        if np.abs(ref).max() == 0:
            assert np.abs(dy[c * n:(c + 1) * n]).max() == 0
            continue
        assert rel_l2(dy[c * n:(c + 1) * n], ref) < 1e-9, (c, rel_l2(dy[c * n:(c + 1) * n], ref))


@pytest.mark.parametrize("kind", KINDS)
def test_single_attempt_matches_oracle(kind):
    m, F, H, y0 = _setup(kind)
    n = m.n_elem
    dt0, eps_rk = 1e4, 1e-4
    y5_ref, err_ref = H.rk_attempt_vec(F, y0, dt0)
    acc_ref, dtn_ref = oracle.controller(err_ref, eps_rk, dt0)
    assert acc_ref
    h = import_oracle(H, "fp64")
    state = dev(np.concatenate([y0, np.zeros(2 * n)]))
    t, dt = dev([0.0]), dev([dt0])
    st, done, rec = hbi.hbi_step_vector(h, _fric(F), state, t, dt, eps_rk, 1)
    assert st == 0 and list(done) == [1] and rec[0][0, 3] == 0
    s = host(state)
    for c in range(4):
        assert rel_l2(s[c * n:(c + 1) * n], y5_ref[c * n:(c + 1) * n]) < 1e-12
    assert host(t)[0] == dt0
    assert host(dt)[0] == pytest.approx(dtn_ref, rel=1e-6)


@pytest.mark.parametrize("kind,nsteps", [("thrust-full-N900", 14), ("dipping-shear-N128", 40)])
def test_adaptive_steps_match_oracle(kind, nsteps):
    """Interseismic run: identical accept/reject decisions; times, step sizes, states and both
    slip components to 1e-7 / 1e-6."""
    m, F, H, y0 = _setup(kind)
    n = m.n_elem
    eps_rk, dt0 = 1e-4, 1e5
    y_ref, D_ref, t_ref, dt_ref, rec_ref = H.run_vec(F, y0, np.zeros(2 * n), 0.0, dt0, eps_rk, nsteps)
    assert rec_ref[:, 2].max() < 1e-6
    h = import_oracle(H, "fp64")
    state = dev(np.concatenate([y0, np.zeros(2 * n)]))
    t, dt = dev([0.0]), dev([dt0])
    st, done, rec = hbi.hbi_step_vector(h, _fric(F), state, t, dt, eps_rk, nsteps)
    assert st == 0 and list(done) == [nsteps]
    rec = rec[0]
    assert np.array_equal(rec[:, 3], rec_ref[:, 3])
    assert np.allclose(rec[:, 0], rec_ref[:, 0], rtol=1e-7, atol=0)
    assert np.allclose(rec[:, 1], rec_ref[:, 1], rtol=1e-7, atol=0)
    assert np.allclose(rec[:, 2], rec_ref[:, 2], rtol=1e-6, atol=0)
    s = host(state)
    assert np.allclose(s[:4 * n], y_ref, rtol=1e-7, atol=1e-9 * np.abs(y_ref[n:3 * n]).max())
    assert np.allclose(s[4 * n:], D_ref, rtol=1e-6, atol=1e-9 * np.abs(D_ref).max())


def _events(rec, vth=1e-3):
    above = rec[:, 2] > vth
    out, k = [], 0
    while k < len(rec):
        if above[k]:
            k1 = k
            while k1 + 1 < len(rec) and above[k1 + 1]:
                k1 += 1
            out.append((rec[k, 0], rec[k:k1 + 1, 2].max()))
            k = k1 + 1
        else:
            k += 1
    return out


def test_event_times_and_peak_slip_rates_match_oracle():
    """Through the first earthquakes of the thrust model with rake-free friction."""
    m, F, H, y0 = _setup("thrust-full-N900")
    n = m.n_elem
    nsteps = 160
    _, _, _, _, rec_ref = H.run_vec(F, y0, np.zeros(2 * n), 0.0, 1e5, 1e-4, nsteps)
    ev_ref = _events(rec_ref)
    assert len(ev_ref) >= 2
    h = import_oracle(H, "fp64")
    state = dev(np.concatenate([y0, np.zeros(2 * n)]))
    t, dt = dev([0.0]), dev([1e5])
    st, done, rec = hbi.hbi_step_vector(h, _fric(F), state, t, dt, 1e-4, nsteps)
    assert st == 0 and list(done) == [nsteps]
    ev = _events(rec[0])
    assert len(ev) >= len(ev_ref[:3])
    for (tg, vg), (tr, vr) in zip(ev[:3], ev_ref[:3]):
        assert tg == pytest.approx(tr, rel=1e-2)
        assert vg == pytest.approx(vr, rel=2e-2)


def test_fixed_rake_and_rake_free_share_a_handle():
    """Alternating the two friction forms on one handle (separate attempt graphs, shared
    buffers) leaves each form's results those of a fresh handle, bit for bit."""
    m, F, H, y0v = _setup("dipping-shear-N128")
    n = m.n_elem
    fr = _fric(F)
    phi, tau = oracle.steady_state(F.V_init, F.a, F.b, F.sigma0, F.f0, F.V0)
    ys = np.concatenate([phi, tau, F.sigma0, np.zeros(n)])
    yv = np.concatenate([y0v, np.zeros(2 * n)])

    def scalar(h):
        s, t, dt = dev(ys), dev([0.0]), dev([1e5])
        st, done, rec = hbi.hbi_step(h, fr, s, t, dt, 1e-4, 12)
        assert st == 0 and done == 12
        return host(s), rec

    def vector(h):
        s, t, dt = dev(yv), dev([0.0]), dev([1e5])
        st, done, rec = hbi.hbi_step_vector(h, fr, s, t, dt, 1e-4, 12)
        assert st == 0 and list(done) == [12]
        return host(s), rec[0]

    hs, hv, hm = import_oracle(H, "fp64"), import_oracle(H, "fp64"), import_oracle(H, "fp64")
    s_ref, rs_ref = scalar(hs)
    v_ref, rv_ref = vector(hv)
    for _ in range(2):
        v, rv = vector(hm)
        s, rs = scalar(hm)
        assert np.array_equal(v, v_ref) and np.array_equal(rv, rv_ref)
        assert np.array_equal(s, s_ref) and np.array_equal(rs, rs_ref)


def test_ensemble_members_equal_single_vector_runs():
    ms = [meshes.dipping_rect(16, 8, 250.0, 30.0), meshes.dipping_rect(12, 6, 250.0, 60.0)]
    Fs = [friction.ensemble_friction(mm, seed=60 + k) for k, mm in enumerate(ms)]
    rk = [F.rake for F in Fs]
    eps, leaf, L = 1e-6, 8, 2
    hE, starts = hbi.hbi_build_ensemble([mm.verts for mm in ms], 32e9, 0.25, oracle.OP_VEC_FULL, eps, leaf, L,
                                        "fp32", rakes=rk)
    cat = lambda f: np.concatenate([getattr(F, f) for F in Fs])
    F0 = Fs[0]
    frE = hbi.friction(dev(cat("a")), dev(cat("b")), dev(cat("dc")), dev(cat("rake")), F0.f0, F0.V0, F0.Vpl,
                       F0.mu, F0.cs)
    states = []
    for F in Fs:
        phi, tau = oracle.steady_state(F.V_init, F.a, F.b, F.sigma0, F.f0, F.V0)
        ang = F.rake + 0.2
        states.append(np.concatenate([phi, tau * np.cos(ang), tau * np.sin(ang), F.sigma0,
                                      np.zeros(2 * len(phi))]))
    comp = lambda s, c: s[c * (len(s) // 6):(c + 1) * (len(s) // 6)]
    sE = dev(np.concatenate([np.concatenate([comp(s, c) for s in states]) for c in range(6)]))
    dt0 = np.array([1e4, 3e4])
    tE, dtE = dev(np.zeros(2)), dev(dt0)
    st, done, recE = hbi.hbi_step_vector(hE, frE, sE, tE, dtE, 1e-4, 25)
    assert st == 0 and list(done) == [25, 25]
    sE = host(sE)
    NT = int(starts[-1])
    for k, (mm, F) in enumerate(zip(ms, Fs)):
        h1 = hbi.hbi_build(mm.verts, 32e9, 0.25, oracle.OP_VEC_FULL, eps, leaf, L, "fp32", rake=rk[k])
        f1 = _fric(F)
        s1, t1, dt1 = dev(states[k]), dev([0.0]), dev([dt0[k]])
        st1, done1, rec1 = hbi.hbi_step_vector(h1, f1, s1, t1, dt1, 1e-4, 25)
        assert st1 == 0 and list(done1) == [25]
        a, b = int(starts[k]), int(starts[k + 1])
        got = np.concatenate([sE[c * NT + a:c * NT + b] for c in range(6)])
        assert np.array_equal(got, host(s1)), f"member {k}: state differs from its single run"
        assert np.array_equal(recE[k], rec1[0])


def test_vector_step_needs_a_two_component_operator():
    m = meshes.dipping_rect(8, 4, 500.0, 40.0)
    F = friction.ensemble_friction(m, seed=3)
    h = hbi.hbi_build(m.verts, F.mu, F.nu, oracle.OP_RAKE_SHEAR_NORMAL, 1e-5, 8, 1, "fp32", rake=F.rake)
    s = dev(np.zeros(6 * m.n_elem))
    st, done, _ = hbi.hbi_step_vector(h, _fric(F), s, dev([0.0]), dev([1.0]), 1e-4, 1)
    assert st == -1 and list(done) == [0]


def test_zero_traction_elements_match_oracle():
    """Elements with no shear traction (V = 0, direction from the rake) in the right-hand side
    and in a few adaptive steps, against the oracle."""
    m, F, H, y0 = _setup("dipping-shear-N128")
    n = m.n_elem
    y = y0.copy()
    zero = [0, 17, 63, n - 1]
    y[n + np.array(zero)] = 0.0
    y[2 * n + np.array(zero)] = 0.0
    dy_ref, V_ref = H.rhs_vec(F, y)
    h = import_oracle(H, "fp64")
    dy = torch.zeros(4 * n, dtype=torch.float64, device="cuda")
    V = torch.zeros(2 * n, dtype=torch.float64, device="cuda")
    hbi.hbi_rhs_vec(h, _fric(F), dev(y), dy, V)
    dy, V = host(dy), host(V)
    assert np.all(V[zero] == 0.0) and np.all(V[n + np.array(zero)] == 0.0)
    for c in range(4):
        ref = dy_ref[c * n:(c + 1) * n]
        if np.abs(ref).max() > 0:
            assert rel_l2(dy[c * n:(c + 1) * n], ref) < 1e-9, c
    y_ref, D_ref, t_ref, _, rec_ref = H.run_vec(F, y, np.zeros(2 * n), 0.0, 1e3, 1e-4, 10)
    state = dev(np.concatenate([y, np.zeros(2 * n)]))
    t, dt = dev([0.0]), dev([1e3])
    st, done, rec = hbi.hbi_step_vector(h, _fric(F), state, t, dt, 1e-4, 10)
    assert st == 0 and list(done) == [10]
    assert np.array_equal(rec[0][:, 3], rec_ref[:, 3])
    assert np.allclose(rec[0][:, 0], rec_ref[:, 0], rtol=1e-7, atol=0)
