"""GPU parity of the rate-state right-hand side and the adaptive RK45 loop against the oracle
(FP64 storage on the oracle's own factors, so only summation order differs).

Tolerances: dy/dt relative 1e-9 per component class (the loading is folded into the HMVM
input as H (V - V_pl) on the GPU and added separately in the oracle, which changes rounding
by the cancellation factor |H V| / |H (V - V_pl)| <= 1e3 at the states used).  The RK error
estimate |y5 - y4| is a difference of numbers of size |y|, so its relative precision is
about u |y| / |y5 - y4| (1e-8 here) and step sizes, proportional to err^-0.2, inherit it:
one attempt is compared to 1e-12 (state) / 1e-6 (err, dt); an interseismic run must take
the same accept/reject decisions and agree to 1e-7; through an earthquake, where the
dynamics amplify these differences, the event time must agree to 1% and the peak slip
rate to 2%."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
import paper_2110_12165_gb300 as hbi
from synthetic import friction, meshes
from gpu_util import dev, host, import_oracle, rel_l2

pytestmark = pytest.mark.gpu


def _setup(kind):
    if kind == "planar-strike-slip-N2048":
        m = meshes.config1_mesh()
        F = friction.config1_friction(m)
        op, eps, leaf, L = oracle.OP_RAKE_SHEAR, 1e-6, 32, 0
    else:
        m = meshes.scaled_thrust_mesh(30, 15, seed=2)       # N = 900, nonplanar, normal coupling
        F = friction.thrust_friction(m, seed=2)
        op, eps, leaf, L = oracle.OP_VEC_FULL, 1e-5, 16, 1
    H = oracle.HMatrix(m, op, eps, leaf, L, F.mu, F.nu, rake=F.rake)
    td, sd = H.loading(F.rake, F.Vpl)
    phi, tau = oracle.steady_state(F.V_init, F.a, F.b, F.sigma0, F.f0, F.V0)
    y0 = np.concatenate([phi, tau, F.sigma0])
    return m, F, H, td, sd, y0


def _fric(F):
    return hbi.friction(dev(F.a), dev(F.b), dev(F.dc), dev(F.rake), F.f0, F.V0, F.Vpl, F.mu, F.cs)


KINDS = ["planar-strike-slip-N2048", "thrust-full-N900"]


def test_steady_state_matches_oracle():
    m = meshes.config1_mesh()
    F = friction.config1_friction(m)
    phi_ref, tau_ref = oracle.steady_state(F.V_init, F.a, F.b, F.sigma0, F.f0, F.V0)
    phi, tau = torch.zeros(m.n_elem, dtype=torch.float64, device="cuda"), torch.zeros(m.n_elem, dtype=torch.float64, device="cuda")
    hbi.hbi_steady_state(dev(F.V_init), dev(F.a), dev(F.b), dev(F.sigma0), F.f0, F.V0, phi, tau)
    assert np.allclose(host(phi), phi_ref, rtol=1e-14, atol=0)
    assert np.allclose(host(tau), tau_ref, rtol=1e-13, atol=0)


@pytest.mark.parametrize("kind", KINDS)
def test_rhs_matches_oracle(kind):
    m, F, H, td, sd, y0 = _setup(kind)
    n = m.n_elem
    # a state off steady state: perturb tau to get V spanning decades
    y = y0.copy()
    y[n:2 * n] += 0.02 * F.a * F.sigma0 * np.sin(np.arange(n))
    dy_ref, V_ref = H.rhs(F, y, td, sd)
    h = import_oracle(H, "fp64")
    fr = _fric(F)
    dy, V = torch.zeros(3 * n, dtype=torch.float64, device="cuda"), torch.zeros(n, dtype=torch.float64, device="cuda")
    hbi.hbi_rhs(h, fr, dev(y), dy, V)
    dy, V = host(dy), host(V)
    assert np.allclose(V, V_ref, rtol=1e-12, atol=0)
    for c in range(3):
        ref = dy_ref[c * n:(c + 1) * n]
        if np.abs(ref).max() == 0:
            assert np.abs(dy[c * n:(c + 1) * n]).max() == 0
            continue
        assert rel_l2(dy[c * n:(c + 1) * n], ref) < 1e-9, (c, rel_l2(dy[c * n:(c + 1) * n], ref))


@pytest.mark.parametrize("kind", KINDS)
def test_single_attempt_matches_oracle(kind):
    """One accepted attempt from the same state: y5 to 1e-12; the error estimate is a small
    difference of O(|y|) numbers, so err (and dt_new ~ err^-0.2) agree to 1e-6."""
    m, F, H, td, sd, y0 = _setup(kind)
    n = m.n_elem
    dt0, eps_rk = 1e4, 1e-4
    y5_ref, err_ref = H.rk_attempt(F, y0, dt0, td, sd)
    acc_ref, dtn_ref = oracle.controller(err_ref, eps_rk, dt0)
    assert acc_ref
    h = import_oracle(H, "fp64")
    state = dev(np.concatenate([y0, np.zeros(n)]))
    t = dev([0.0]); dt = dev([dt0])
    st, done, rec = hbi.hbi_step(h, _fric(F), state, t, dt, eps_rk, 1)
    assert st == 0 and done == 1 and rec[0, 3] == 0
    s_ = host(state)
    for c in range(3):
        assert rel_l2(s_[c * n:(c + 1) * n], y5_ref[c * n:(c + 1) * n]) < 1e-12
    assert host(t)[0] == dt0
    assert host(dt)[0] == pytest.approx(dtn_ref, rel=1e-6)


@pytest.mark.parametrize("kind,nsteps", [("planar-strike-slip-N2048", 40), ("thrust-full-N900", 14)])
def test_adaptive_steps_match_oracle(kind, nsteps):
    """Interseismic run (before the first instability): identical accept/reject decisions;
    times, step sizes and states to 1e-7 (the conditioning of the error estimate)."""
    m, F, H, td, sd, y0 = _setup(kind)
    n = m.n_elem
    eps_rk, dt0 = 1e-4, 1e5
    y_ref, D_ref, t_ref, dt_ref, rec_ref = H.run(F, y0, np.zeros(n), 0.0, dt0, eps_rk, nsteps, td, sd)
    assert rec_ref[:, 2].max() < 1e-6          # still interseismic
    h = import_oracle(H, "fp64")
    state = dev(np.concatenate([y0, np.zeros(n)]))
    t = dev([0.0]); dt = dev([dt0])
    st, done, rec = hbi.hbi_step(h, _fric(F), state, t, dt, eps_rk, nsteps)
    assert st == 0 and done == nsteps
    assert np.array_equal(rec[:, 3], rec_ref[:, 3])                 # same rejections
    assert np.allclose(rec[:, 0], rec_ref[:, 0], rtol=1e-7, atol=0)  # times
    assert np.allclose(rec[:, 1], rec_ref[:, 1], rtol=1e-7, atol=0)  # step sizes
    assert np.allclose(rec[:, 2], rec_ref[:, 2], rtol=1e-6, atol=0)  # max slip rate
    s = host(state)
    assert np.allclose(s[:3 * n], y_ref, rtol=1e-7, atol=0)
    assert np.allclose(s[3 * n:], D_ref, rtol=1e-6, atol=1e-20)


def _events(rec, vth=1e-3):
    """(start time, peak max slip rate) of each event: an event starts when max V exceeds
    vth and ends when it drops back below."""
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
    """Through the first three earthquakes of the thrust model: event start times within 1%,
    peak slip rates within 2% (FP64 storage on the oracle's factors)."""
    m, F, H, td, sd, y0 = _setup("thrust-full-N900")
    n = m.n_elem
    nsteps = 160
    _, _, _, _, rec_ref = H.run(F, y0, np.zeros(n), 0.0, 1e5, 1e-4, nsteps, td, sd)
    ev_ref = _events(rec_ref)
    assert len(ev_ref) >= 3
    h = import_oracle(H, "fp64")
    state = dev(np.concatenate([y0, np.zeros(n)]))
    t = dev([0.0]); dt = dev([1e5])
    st, done, rec = hbi.hbi_step(h, _fric(F), state, t, dt, 1e-4, nsteps)
    assert st == 0 and done == nsteps
    ev = _events(rec)
    assert len(ev) >= 3
    for (tg, vg), (tr, vr) in zip(ev[:3], ev_ref[:3]):
        assert tg == pytest.approx(tr, rel=1e-2)
        assert vg == pytest.approx(vr, rel=2e-2)


def test_step_can_continue_and_replays_are_noops_after_target():
    m, F, H, td, sd, y0 = _setup("planar-strike-slip-N2048")
    n = m.n_elem
    h = import_oracle(H, "fp64")
    fr = _fric(F)
    state = dev(np.concatenate([y0, np.zeros(n)]))
    t = dev([0.0]); dt = dev([1e5])
    st, done, rec1 = hbi.hbi_step(h, fr, state, t, dt, 1e-4, 7)
    st2, done2, rec2 = hbi.hbi_step(h, fr, state, t, dt, 1e-4, 13)
    assert st == 0 and st2 == 0 and done == 7 and done2 == 13
    y_ref, D_ref, t_ref, dt_ref, rec_ref = H.run(F, y0, np.zeros(n), 0.0, 1e5, 1e-4, 20, td, sd)
    assert np.allclose(np.concatenate([rec1[:, 0], rec2[:, 0]]), rec_ref[:, 0], rtol=1e-7)
    assert np.allclose(host(state)[:3 * n], y_ref, rtol=1e-7)


_C1 = {}


def _config1_oracle_run():
    if not _C1:
        m, F, H, td, sd, y0 = _setup("planar-strike-slip-N2048")
        _, _, _, _, rec = H.run(F, y0, np.zeros(m.n_elem), 0.0, 1e5, 1e-4, 2000, td, sd)
        _C1["run"] = (m, F, H, td, sd, y0, rec)
    return _C1["run"]


@pytest.mark.parametrize("build", ["oracle-factors", "gpu-built"])
def test_config1_sequence_matches_oracle(build):
    """The planar strike-slip fault (N = 2048, FP64, eps 1e-6, leaf 32) over 2000 adaptive
    steps (about 30 years, two earthquakes): the start time and peak slip rate of every
    earthquake (peak above 0.1 m/s) within 1 % / 2 % of the oracle's run.  Around the 1e-3 m/s
    threshold the maximum slip rate flickers during nucleation and afterslip, so the small
    threshold crossings there are not compared one by one.  The GPU-built operator has its
    own ACA pivots (error <= 10 eps against the dense operator), the imported one the oracle's
    factors."""
    m, F, H, td, sd, y0, rec_ref = _config1_oracle_run()
    n = m.n_elem
    nsteps = len(rec_ref)
    big = lambda ev: [(t, v) for t, v in ev if v > 0.1]
    ev_ref = big(_events(rec_ref))
    assert len(ev_ref) >= 2
    if build == "oracle-factors":
        h = import_oracle(H, "fp64")
    else:
        h = hbi.hbi_build(m.verts, F.mu, F.nu, oracle.OP_RAKE_SHEAR, 1e-6, 32, 0, "fp64", rake=F.rake)
    state = dev(np.concatenate([y0, np.zeros(n)]))
    t = dev([0.0]); dt = dev([1e5])
    st, done, rec = hbi.hbi_step(h, _fric(F), state, t, dt, 1e-4, nsteps)
    assert st == 0 and done == nsteps
    ev = big(_events(rec))
    assert len(ev) >= 2
    for (tg, vg), (tr, vr) in zip(ev, ev_ref):
        assert tg == pytest.approx(tr, rel=1e-2)
        assert vg == pytest.approx(vr, rel=2e-2)


def test_recurrence_interval_converges_under_refinement():
    """The planar fault of the 2048-element case at 250, 125 and 62.5 m (N = 2048, 8192,
    32768; FP64 storage, eps 1e-6): the mean interval between earthquakes after the first
    (which depends on the initial state) changes by less than 2 % from 125 to 62.5 m, and by
    less than a quarter of the change from 250 to 125 m.  The 250 m mesh is coarser than the
    process zone (L_b = mu d_c / (b sigma) = 213 m) and its cycle alternates; from 125 m on
    the cycle is periodic.  This runs on the GPU's FP64 path, which the sequence tests above
    pin to the oracle at N = 2048; the oracle itself would need hours at N = 32768."""
    YR = 3.15576e7
    T = []
    for k, nsteps in ((1, 7000), (2, 2500), (4, 4000)):
        m = meshes.planar_vertical_rect(64 * k, 32 * k, 250.0 / k)
        m.meta.update(length=16e3, width=8e3)
        F = friction.config1_friction(m)
        n = m.n_elem
        h = hbi.hbi_build(m.verts, F.mu, F.nu, oracle.OP_RAKE_SHEAR, 1e-6, 32, 0, "fp64", rake=F.rake)
        phi, tau = oracle.steady_state(F.V_init, F.a, F.b, F.sigma0, F.f0, F.V0)
        s = dev(np.concatenate([phi, tau, F.sigma0, np.zeros(n)]))
        st, done, rec = hbi.hbi_step(h, _fric(F), s, dev([0.0]), dev([1e5]), 1e-4, nsteps)
        assert st == 0 and done == nsteps
        ev = [t / YR for t, v in _events(rec) if v > 0.1]
        assert len(ev) >= 5, (k, ev)
        T.append(float(np.mean(np.diff(ev[1:]))))
    T250, T125, T62 = T
    assert abs(T62 - T125) < 0.02 * T62, T
    assert abs(T62 - T125) < 0.25 * abs(T125 - T250), T


@pytest.mark.parametrize("kind", KINDS)
def test_step_records_carry_the_mean_friction(kind):
    """Each step record's mean friction coefficient (mean over the elements of tau / sigma after
    the step, the diagnostic the paper plots against time, Sec. 4.3) equals the mean of the state
    the step leaves, summed on the host (the device sums in fixed point 2^-40, exactly: 1e-12);
    after an interseismic run it equals the oracle's state's mean to the run's tolerance
    (1e-7)."""
    m, F, H, td, sd, y0 = _setup(kind)
    n = m.n_elem
    h = import_oracle(H, "fp64")
    fr = _fric(F)
    state = dev(np.concatenate([y0, np.zeros(n)]))
    t = dev([0.0]); dt = dev([1e5])
    last = None
    for _ in range(6):
        st, done, rec = hbi.hbi_step(h, fr, state, t, dt, 1e-4, 1)
        assert st == 0 and done == 1
        s_ = host(state)
        mu_host = float(np.mean(s_[n:2 * n] / s_[2 * n:3 * n]))
        assert rec[0, 4] == pytest.approx(mu_host, rel=1e-12, abs=1e-12)
        last = rec[0, 4]
    y_ref, _, _, _, _ = H.run(F, y0, np.zeros(n), 0.0, 1e5, 1e-4, 6, td, sd)
    assert last == pytest.approx(float(np.mean(y_ref[n:2 * n] / y_ref[2 * n:3 * n])), rel=1e-7)
