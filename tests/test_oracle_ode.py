"""Pins of the oracle's rate-state ODE and integrator (Eqs. 7-16, 21-22): Runge-Kutta
order conditions and observed order, the step controller reading, the steady state of
Eq. 8, Eqs. 13a-c against finite differences of Eq. 7, the spring-slider stability
threshold k_c = (b-a) sigma / d_c (Ruina 1983; Rice & Ruina 1983), agreement with an
independent fixed-step RK4, and relaxation of a velocity-strengthening fault to plate
rate.  CPU only."""
import numpy as np
import pytest

import oracle
from synthetic import friction, meshes, rng

MU, NU = 32e9, 0.25


def _conditions(A, b, c):
    """The 17 rooted-tree order conditions up to order 5 for an explicit RK method."""
    Ac, Ac2, Ac3 = A @ c, A @ c ** 2, A @ c ** 3
    return [
        (b.sum(), 1.0),
        (b @ c, 1 / 2),
        (b @ c ** 2, 1 / 3), (b @ Ac, 1 / 6),
        (b @ c ** 3, 1 / 4), (b @ (c * Ac), 1 / 8), (b @ Ac2, 1 / 12), (b @ (A @ Ac), 1 / 24),
        (b @ c ** 4, 1 / 5), (b @ (c ** 2 * Ac), 1 / 10), (b @ (c * Ac2), 1 / 15),
        (b @ (c * (A @ Ac)), 1 / 30), (b @ Ac ** 2, 1 / 20), (b @ Ac3, 1 / 20),
        (b @ (A @ (c * Ac)), 1 / 40), (b @ (A @ Ac2), 1 / 60), (b @ (A @ (A @ Ac)), 1 / 120),
    ]


def test_cash_karp_order_conditions():
    c, a, b5, b4 = oracle.cash_karp_tableau()
    A = np.zeros((6, 6))
    A[:, :5] = a
    assert np.allclose(A.sum(1), c, atol=1e-15)
    for got, want in _conditions(A, b5, c):
        assert got == pytest.approx(want, abs=1e-14)
    cond4 = _conditions(A, b4, c)
    for got, want in cond4[:8]:
        assert got == pytest.approx(want, abs=1e-14)
    assert any(abs(g - w) > 1e-6 for g, w in cond4[8:])   # the embedded solution is 4th order


def test_observed_order_on_linear_decay():
    errs5, ests = [], []
    for dt in (0.2, 0.1, 0.05):
        y5, est = oracle.ck_linear_step(1.0, 1.0, dt)
        errs5.append(abs(y5 - np.exp(-dt)))
        ests.append(est)
    assert 50 < errs5[0] / errs5[1] < 80 and 50 < errs5[1] / errs5[2] < 80      # ~2^6
    assert 25 < ests[0] / ests[1] < 40 and 25 < ests[1] / ests[2] < 40          # ~2^5


@pytest.mark.parametrize("ratio,accept,factor", [
    (4.0, False, 0.9 * 4.0 ** -0.25),
    (100.0, False, 0.5),               # Eq. 14 floor at dt/2
    (1.0 / 32, True, 0.9 * 32 ** 0.2),
    (1e-6, True, 2.0),                 # Eq. 15 cap at 2 dt
    (1.0, True, 0.9),
    (float("inf"), False, 0.5),        # non-finite trial: rejected, dt halved
])
def test_controller_reading_of_eqs_14_15(ratio, accept, factor):
    eps, dt = 1e-4, 3.0
    acc, dt_new = oracle.controller(ratio * eps, eps, dt)
    assert acc == accept
    assert dt_new == pytest.approx(factor * dt, rel=1e-14)
    assert 0.5 * dt <= dt_new <= 2.0 * dt


def test_steady_state_inverts_eq7_and_zeroes_eq8():
    n = 50
    V = 1e-9 * np.exp(rng.normal(41, n) * 3)
    a = 0.008 + 0.01 * rng.uniform(42, n)
    b = 0.012 + 0.01 * rng.uniform(43, n)
    sig = 30e6 + 40e6 * rng.uniform(44, n)
    f0, V0 = 0.6, 1e-6
    phi, tau = oracle.steady_state(V, a, b, sig, f0, V0)
    V2, _ = oracle.slip_rate(phi, tau, sig, a, V0)
    assert np.allclose(V2, V, rtol=1e-9, atol=0)
    # Eq. 8 with these values: V0 exp((f0-phi)/b) - V = 0
    assert np.allclose(V0 * np.exp((f0 - phi) / b), V, rtol=1e-12, atol=0)
    # steady-state friction = f0 + (a - b) ln(V/V0) when V >> V0 e^{-phi/a}
    assert np.allclose(tau / sig, f0 + (a - b) * np.log(V / V0), rtol=0, atol=1e-12)


def test_eq13_partials_match_finite_differences_of_eq7():
    n = 20
    phi = 0.65 + 0.1 * rng.uniform(45, n)
    a = 0.008 + 0.01 * rng.uniform(46, n)
    sig = 30e6 + 40e6 * rng.uniform(47, n)
    tau = sig * (phi + 0.02 * (rng.uniform(48, n) - 0.5))
    V0 = 1e-6
    V, P = oracle.slip_rate(phi, tau, sig, a, V0)
    for k, (arr, step) in enumerate(((tau, 1e-3 * a * sig), (sig, 1e-6 * sig), (phi, 1e-5 * a))):
        hi = [phi, tau, sig]
        lo = [phi, tau, sig]
        idx = {0: 1, 1: 2, 2: 0}[k]
        hi = [x.copy() for x in hi]; lo = [x.copy() for x in lo]
        hi[idx] = hi[idx] + step; lo[idx] = lo[idx] - step
        Vh, _ = oracle.slip_rate(hi[0], hi[1], hi[2], a, V0)
        Vl, _ = oracle.slip_rate(lo[0], lo[1], lo[2], a, V0)
        fd = (Vh - Vl) / (2 * step)
        assert np.allclose(P[:, k], fd, rtol=1e-5, atol=0)


def _one_element(r, dc_scale=True, V_init=1.1e-9):
    m = meshes.planar_vertical_rect(1, 1, 250.0)
    H = oracle.HMatrix(m, oracle.OP_RAKE_SHEAR, 1e-6, 32, 0, MU, NU)
    k = -oracle.pair_entries(m, 0, [0], [0], MU, NU)[0, 0, 0]
    a, b, sig = 0.010, 0.015, 50e6
    dc = r * (b - a) * sig / k                 # k / k_c = r
    F = friction.Friction(a=np.array([a]), b=np.array([b]), dc=np.array([dc]),
                          sigma0=np.array([sig]), rake=np.zeros(1), V_init=np.array([V_init]),
                          mu=MU, nu=NU, cs=3464.0)
    td, sd = H.loading(F.rake, F.Vpl)
    phi, tau = oracle.steady_state(F.V_init, F.a, F.b, F.sigma0, F.f0, F.V0)
    y = np.concatenate([phi, tau, F.sigma0])
    return H, F, y, td, sd, k


def test_loading_is_backslip_of_self_stiffness():
    H, F, y, td, sd, k = _one_element(2.0)
    assert td[0] == pytest.approx(k * F.Vpl, rel=1e-14)     # Eq. 21 with A_11 = -k
    assert sd[0] == 0.0


@pytest.mark.parametrize("r,stable", [(2.0, True), (0.5, False)])
def test_spring_slider_stability_threshold(r, stable):
    """k > k_c: perturbations of steady sliding decay; k < k_c: stick-slip instability."""
    H, F, y, td, sd, k = _one_element(r)
    y2, D, t, dt, rec = H.run(F, y, np.zeros(1), 0.0, 1e5, 1e-8, 400, td, sd)
    lnv = np.abs(np.log(rec[:, 2] / F.Vpl))
    if stable:
        assert lnv[-50:].max() < 0.25 * np.log(1.1)
        assert rec[:, 2].max() < 1.2e-9
    else:
        assert rec[:, 2].max() > 1e-3            # an instability (seismic slip rate)


def test_adaptive_rk_matches_fixed_step_rk4():
    """Independent classical RK4 (many small steps) on the same right-hand side."""
    H, F, y0, td, sd, k = _one_element(2.0, V_init=1.5e-9)
    y1, D1, t1, _, rec = H.run(F, y0, np.zeros(1), 0.0, 1e4, 1e-9, 60, td, sd)
    def f(z):
        dy, V = H.rhs(F, z[:3], td, sd)
        return np.concatenate([dy, V])
    z = np.concatenate([y0, [0.0]])
    nst = 4000
    h = t1 / nst
    for _ in range(nst):
        k1 = f(z); k2 = f(z + 0.5 * h * k1); k3 = f(z + 0.5 * h * k2); k4 = f(z + h * k3)
        z = z + h / 6 * (k1 + 2 * k2 + 2 * k3 + k4)
    V_ad, _ = oracle.slip_rate(y1[:1], y1[1:2], y1[2:3], F.a, F.V0)
    V_rk4, _ = oracle.slip_rate(z[:1], z[1:2], z[2:3], F.a, F.V0)
    assert abs(np.log(V_ad[0] / V_rk4[0])) < 1e-6
    assert y1[0] == pytest.approx(z[0], rel=1e-8)
    assert D1[0] == pytest.approx(z[3], rel=1e-3)      # Eq. 16 is second order


def test_velocity_strengthening_fault_relaxes_to_plate_rate():
    m = meshes.planar_vertical_rect(8, 8, 250.0)
    F = friction.velocity_strengthening(m, seed=7, amp=0.3)
    H = oracle.HMatrix(m, oracle.OP_RAKE_SHEAR, 1e-6, 16, 0, F.mu, F.nu, rake=F.rake)
    td, sd = H.loading(F.rake, F.Vpl)
    phi, tau = oracle.steady_state(F.V_init, F.a, F.b, F.sigma0, F.f0, F.V0)
    y = np.concatenate([phi, tau, F.sigma0])
    y2, D, t, dt, rec = H.run(F, y, np.zeros(m.n_elem), 0.0, 1e5, 1e-6, 300, td, sd)
    V, _ = oracle.slip_rate(y2[:64], y2[64:128], y2[128:], F.a, F.V0)
    assert np.abs(V / F.Vpl - 1).max() < 1e-3
    assert np.abs(F.V_init / F.Vpl - 1).max() > 0.25


@pytest.mark.parametrize("op", [oracle.OP_RAKE_SHEAR_NORMAL, oracle.OP_VEC_FULL])
def test_rhs_at_sampled_rows_equals_the_full_rhs(op):
    """rhs_rows (the element-wise right-hand side at chosen elements, from dense operator rows
    of the slip-rate deficit) equals the full right-hand side of a near-exact H-matrix whose
    loading is added separately (Eqs. 21-22): the two routes differ only in where the
    backslip enters and in the ACA error (eps 1e-12)."""
    m = meshes.scaled_thrust_mesh(12, 6, seed=2)             # N = 144, nonplanar
    F = friction.thrust_friction(m, seed=2)
    n = m.n_elem
    H = oracle.HMatrix(m, op, 1e-12, 8, 1, F.mu, F.nu, rake=F.rake)
    td, sd = H.loading(F.rake, F.Vpl)
    phi, tau = oracle.steady_state(F.V_init, F.a, F.b, F.sigma0, F.f0, F.V0)
    y = np.concatenate([phi + 0.01 * rng.normal(21, n), tau, F.sigma0])
    dy, V = H.rhs(F, y, td, sd)
    rows = np.array([0, 5, 77, n - 1])
    dv = V - F.Vpl
    x = dv if H.nin == 1 else np.concatenate([dv * np.cos(F.rake), dv * np.sin(F.rake)])
    s = oracle.dense_rows(m, op, rows, x, F.mu, F.nu, rake=F.rake)
    got = oracle.rhs_rows(op, F, y, rows, s)
    for c in range(3):
        ref = dy[c * n + rows]
        assert np.allclose(got[:, c], ref, rtol=1e-8, atol=1e-9 * np.abs(dy[c * n:(c + 1) * n]).max())


def test_complex_step_gradient_of_a_fixed_step_run():
    """The oracle's complex-step derivative of a fixed-step loss (its reference for a discrete
    adjoint): the real part equals the same steps taken by the oracle's real Cash-Karp
    attempt (1e-12), and the derivatives with respect to a (b fixed) and d_c equal central
    differences of the loss (1e-6: truncation O(d^2) and rounding u L / d both far below)."""
    import dataclasses
    m = meshes.scaled_thrust_mesh(6, 4, seed=3)              # N = 48, nonplanar, 2 -> 3
    F = friction.thrust_friction(m, seed=3)
    n = m.n_elem
    H = oracle.HMatrix(m, oracle.OP_VEC_FULL, 1e-10, 8, 1, F.mu, F.nu, rake=F.rake)
    phi, tau = oracle.steady_state(F.V_init, F.a, F.b, F.sigma0, F.f0, F.V0)
    y0 = np.concatenate([phi + 0.02 * rng.normal(3, n), tau, F.sigma0])
    dts = np.full(8, 2e5)
    target = np.log(1e-9) + 0.1 * rng.normal(4, n)
    L, _ = H.fixed_loss(F, y0, dts, target)
    td, sd = H.loading(F.rake, F.Vpl)
    y = y0.copy()
    for dt in dts:
        y, _ = H.rk_attempt(F, y, dt, td, sd)
    V, _ = oracle.slip_rate(y[:n], y[n:2 * n], y[2 * n:], F.a, F.V0)
    assert L == pytest.approx(0.5 * np.sum((np.log(V) - target) ** 2), rel=1e-12)
    els = [0, 7, n - 1]
    ga, gd = H.fixed_loss_grad(F, y0, dts, target, els)
    for k, j in enumerate(els):
        for which, g, rel in (("a", ga[k], 1e-5), ("dc", gd[k], 1e-4)):
            base = getattr(F, which)
            d = rel * base[j]
            p, q = base.copy(), base.copy()
            p[j] += d
            q[j] -= d
            fd = (H.fixed_loss(dataclasses.replace(F, **{which: p}), y0, dts, target)[0] -
                  H.fixed_loss(dataclasses.replace(F, **{which: q}), y0, dts, target)[0]) / (2 * d)
            assert g == pytest.approx(fd, rel=1e-6), (which, j)
