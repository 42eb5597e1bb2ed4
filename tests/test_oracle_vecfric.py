"""Pins of the oracle's rake-free (vector) friction.

(1) One square element: its in-plane self-stiffness has no strike/dip coupling (mirror
    symmetry), so with the loading along strike or along dip the traction stays parallel to
    it and the vector system is the scalar one of Eqs. 5-16 (same RK steps, 1e-10).
(2) The quasi-dynamic balance: along any state, dtau/dt + eta dV/dt (dV/dt by central
    differences of V along (dphi, dtau, dsigma)) equals the elastic stress rate H (V - V_pl r)
    of the oracle's own product; this pins the 2x2 solve and every partial derivative.
(3) A velocity-strengthening fault started off the plate direction relaxes to V = V_pl r.
"""
import dataclasses

import numpy as np
import pytest

import oracle
from synthetic import friction, meshes, rng

MU, NU, CS = 32e9, 0.25, 3464.0


def _fric(n, a, b, rake, dc=0.01):
    return friction.Friction(a=np.full(n, a), b=np.full(n, b), dc=np.full(n, dc), sigma0=np.full(n, 50e6),
                             rake=np.full(n, rake), V_init=np.full(n, 1e-9), mu=MU, nu=NU, cs=CS)


@pytest.mark.parametrize("rake", [0.0, np.pi / 2])
def test_single_square_element_reduces_to_the_scalar_law(rake):
    m = meshes.planar_vertical_rect(1, 1, 500.0)
    F = _fric(1, 0.010, 0.015, rake)
    H = oracle.HMatrix(m, oracle.OP_VEC_FULL, 1e-8, 4, 0, MU, NU, rake=F.rake)
    V = np.array([1.3e-9])
    phi, tau = oracle.steady_state(V, F.a, F.b, F.sigma0, F.f0, F.V0)
    phi = phi - 0.02                                     # away from steady state: it accelerates
    y_s = np.concatenate([phi, tau, F.sigma0])
    td, sd = H.loading(F.rake, F.Vpl)
    ys, Ds, ts, dts, rec_s = H.run(F, y_s, np.zeros(1), 0.0, 1e4, 1e-4, 40, td, sd)
    y_v = np.concatenate([phi, tau * np.cos(rake), tau * np.sin(rake), F.sigma0])
    yv, Dv, tv, dtv, rec_v = H.run_vec(F, y_v, np.zeros(2), 0.0, 1e4, 1e-4, 40)
    assert np.allclose(rec_v[:, :3], rec_s[:, :3], rtol=1e-10, atol=0)
    tau_v = np.hypot(yv[1], yv[2])
    assert np.allclose([yv[0], tau_v, yv[3]], ys, rtol=1e-10, atol=0)
    d_ang = np.arctan2(yv[2], yv[1]) - rake                # traction still along the loading
    assert abs(np.sin(d_ang)) < 1e-12 and np.cos(d_ang) > 0
    assert np.allclose(np.hypot(Dv[0], Dv[1]), Ds, rtol=1e-10)


def test_quasi_dynamic_balance_and_partials():
    m = meshes.dipping_rect(4, 3, 500.0, 35.0)          # 12 elements, planar dipping
    n = m.n_elem
    F = _fric(n, 0.010, 0.014, np.deg2rad(70.0))
    H = oracle.HMatrix(m, oracle.OP_VEC_FULL, 1e-9, 4, 0, MU, NU, rake=F.rake)
    phi, tau = oracle.steady_state(np.full(n, 2e-9), F.a, F.b, F.sigma0, F.f0, F.V0)
    ang = F.rake + 0.3 * rng.normal(3, n)               # traction off the loading direction
    y = np.concatenate([phi + 0.01 * rng.normal(4, n), tau * np.cos(ang), tau * np.sin(ang),
                        F.sigma0 * (1 + 0.01 * rng.normal(5, n))])
    dy, V = H.rhs_vec(F, y)
    # elastic stress rate of the slip-rate deficit
    x = np.concatenate([V[:n] - F.Vpl * np.cos(F.rake), V[n:] - F.Vpl * np.sin(F.rake)])
    s = H.matvec(x)
    eta = MU / (2 * CS)
    h = 1e-4
    _, Vp = H.rhs_vec(F, y + h * dy)
    _, Vm = H.rhs_vec(F, y - h * dy)
    dV = (Vp - Vm) / (2 * h)
    assert np.allclose(dy[n:3 * n] + eta * dV, s[:2 * n], rtol=1e-6, atol=1e-9 * np.abs(s[:2 * n]).max())
    assert np.allclose(dy[3 * n:], s[2 * n:], rtol=1e-12, atol=0)            # dsigma/dt (Eq. 10)
    # V is parallel to the traction
    assert np.allclose(V[:n] * y[2 * n:3 * n] - V[n:] * y[n:2 * n], 0.0, atol=1e-15 * np.abs(V).max() * tau.max())


def test_velocity_strengthening_fault_relaxes_to_plate_motion():
    m = meshes.planar_vertical_rect(4, 2, 500.0)
    n = m.n_elem
    F = _fric(n, 0.015, 0.010, np.deg2rad(30.0), dc=0.002)
    H = oracle.HMatrix(m, oracle.OP_VEC_FULL, 1e-9, 4, 0, MU, NU, rake=F.rake)
    V0 = np.full(n, 3e-9)
    phi, tau = oracle.steady_state(V0, F.a, F.b, F.sigma0, F.f0, F.V0)
    ang = F.rake + np.deg2rad(40.0)                       # started 40 degrees off the plate direction
    y = np.concatenate([phi, tau * np.cos(ang), tau * np.sin(ang), F.sigma0])
    y, D, t, dt, rec = H.run_vec(F, y, np.zeros(2 * n), 0.0, 1e5, 1e-6, 600)
    _, V = H.rhs_vec(F, y)
    Vm = np.hypot(V[:n], V[n:])
    assert np.allclose(Vm, F.Vpl, rtol=1e-3)
    assert np.allclose(np.arctan2(V[n:], V[:n]), F.rake, atol=1e-3)


def test_non_finite_trial_is_rejected():
    """A non-finite state gives an infinite error estimate (the trial is rejected, reading of
    Eqs. 14-15), also when only some of the three relative changes are NaN."""
    m = meshes.planar_vertical_rect(4, 2, 500.0)
    n = m.n_elem
    F = _fric(n, 0.010, 0.015, 0.0)
    H = oracle.HMatrix(m, oracle.OP_VEC_SHEAR, 1e-9, 4, 0, MU, NU, rake=F.rake)
    phi, tau = oracle.steady_state(np.full(n, 1e-9), F.a, F.b, F.sigma0, F.f0, F.V0)
    y = np.concatenate([phi, tau, np.zeros(n), F.sigma0])
    _, err = H.rk_attempt_vec(F, y, 1e3)
    assert np.isfinite(err)
    y[n + 3] = np.nan
    _, err = H.rk_attempt_vec(F, y, 1e3)
    assert err == np.inf


def test_zero_traction_is_the_limit_along_the_rake():
    """|tau| = 0 (V = 0, direction undefined): the right-hand side takes the loading direction
    and g/|tau| -> g', i.e. the limit of a traction that vanishes along the rake."""
    m = meshes.dipping_rect(3, 2, 500.0, 40.0)
    n = m.n_elem
    F = _fric(n, 0.010, 0.014, np.deg2rad(60.0))
    H = oracle.HMatrix(m, oracle.OP_VEC_FULL, 1e-9, 4, 0, MU, NU, rake=F.rake)
    phi, tau = oracle.steady_state(np.full(n, 2e-9), F.a, F.b, F.sigma0, F.f0, F.V0)
    y0 = np.concatenate([phi, tau * np.cos(F.rake), tau * np.sin(F.rake), F.sigma0])
    y0[n + 2] = y0[2 * n + 2] = 0.0                      # element 2: no shear traction
    dy0, V0 = H.rhs_vec(F, y0)
    assert V0[2] == 0.0 and V0[n + 2] == 0.0
    y1 = y0.copy()
    r = F.rake[2]
    y1[n + 2], y1[2 * n + 2] = 1e-3 * np.cos(r), 1e-3 * np.sin(r)    # 1 mPa along the rake
    dy1, _ = H.rhs_vec(F, y1)
    scale = np.abs(dy0).reshape(4, n).max(axis=1)
    for c in range(4):
        assert abs(dy1[c * n + 2] - dy0[c * n + 2]) <= 1e-6 * scale[c] + 1e-12, c
