"""Pins of the oracle's elastic kernel (Sec. 2.1, Eqs. 3-6) against facts fixed by
elasticity, not by the oracle: the Kelvin solution's field equation and force balance,
the Volterra surface representation, textbook 2-D dislocation limits, physical signs,
equilibrium, superposition and symmetry.  CPU only."""
import numpy as np
import pytest

import oracle
from synthetic import meshes, rng

MU, NU = 32e9, 0.25
LAM = 2 * MU * NU / (1 - 2 * NU)


def cijkl():
    d = np.eye(3)
    return (LAM * np.einsum("ij,kl->ijkl", d, d)
            + MU * (np.einsum("ik,jl->ijkl", d, d) + np.einsum("il,jk->ijkl", d, d)))


def test_gauss_legendre_exact_to_degree_15():
    x, w = oracle.gauss_legendre()
    for k in range(16):
        exact = 0.0 if k % 2 else 2.0 / (k + 1)
        assert abs(np.sum(w * x ** k) - exact) < 1e-14


def test_kelvin_dG_is_derivative_of_G():
    r = np.array([0.7, -1.3, 0.4])
    dG = oracle.kelvin_dG(r, MU, NU)
    h = 1e-3
    for q in range(3):
        e = np.zeros(3); e[q] = h
        fd = (-oracle.kelvin_G(r + 2 * e, MU, NU) + 8 * oracle.kelvin_G(r + e, MU, NU)
              - 8 * oracle.kelvin_G(r - e, MU, NU) + oracle.kelvin_G(r - 2 * e, MU, NU)) / (12 * h)
        assert np.allclose(dG[:, :, q], fd, rtol=0, atol=1e-9 * np.abs(dG).max())


def test_kelvin_satisfies_navier_equation():
    """mu lap(u) + (lam+mu) grad div u = 0 away from the point force (u = G F; second
    derivatives by 4th-order differences of the analytic first derivative)."""
    F = np.array([0.3, -0.5, 0.8])
    grad_u = lambda x: np.einsum("kpl,p->kl", oracle.kelvin_dG(x, MU, NU), F)  # d_l u_k
    x0 = np.array([1.1, 0.6, -0.9])
    h = 1e-3
    H = np.zeros((3, 3, 3))   # H[k, l, b] = d_b d_l u_k
    for b in range(3):
        e = np.zeros(3); e[b] = h
        H[:, :, b] = (-grad_u(x0 + 2 * e) + 8 * grad_u(x0 + e) - 8 * grad_u(x0 - e)
                      + grad_u(x0 - 2 * e)) / (12 * h)
    lap = np.einsum("kll->k", H)
    graddiv = np.einsum("llk->k", H)
    res = MU * lap + (LAM + MU) * graddiv
    scale = MU * np.linalg.norm(oracle.kelvin_G(x0, MU, NU) @ F) / np.dot(x0, x0)
    assert np.linalg.norm(res) < 1e-8 * scale


def test_kelvin_force_balance_on_sphere():
    """Tractions on any sphere around the point force sum to -F (equilibrium of the ball)."""
    F = np.array([0.3, -0.5, 0.8])
    c = cijkl()
    R = 2.5
    ct, wt = np.polynomial.legendre.leggauss(24)
    nphi = 48
    phis = 2 * np.pi * np.arange(nphi) / nphi
    total = np.zeros(3)
    for cth, w in zip(ct, wt):
        sth = np.sqrt(1 - cth ** 2)
        for ph in phis:
            n = np.array([sth * np.cos(ph), sth * np.sin(ph), cth])
            dG = oracle.kelvin_dG(R * n, MU, NU)
            grad = np.einsum("kpl,p->kl", dG, F)          # d_l u_k
            sig = np.einsum("ijkl,kl->ij", c, grad)
            total += w * (2 * np.pi / nphi) * R * R * sig @ n
    assert np.allclose(total, -F, atol=1e-10)


def _surface_stress(P, b, x):
    """Volterra representation u_n(x) = int b_i c_ijpq n_j dG_np/dxi_q dS (Aki & Richards
    Eq. 3.3, static) by 2-D Gauss quadrature over a triangle, then stress by 4th-order
    finite differences of u.  Independent of the loop-integral route of the oracle."""
    c = cijkl()
    P0, P1, P2 = P
    e1, e2 = P1 - P0, P2 - P0
    nn = np.cross(e1, e2)
    J = np.linalg.norm(nn)
    nrm = nn / J
    g, w = np.polynomial.legendre.leggauss(30)
    g = 0.5 * (g + 1); w = 0.5 * w
    coef = np.einsum("i,ijpq,j->pq", b, c, nrm)
    def u(xx):
        acc = np.zeros(3)
        for s, ws in zip(g, w):
            for t, wt in zip(g, w):
                xi = P0 + s * (1 - t) * e1 + s * t * e2
                dG = oracle.kelvin_dG(xx - xi, MU, NU)   # dG_np/dr_q; d/dxi_q = -d/dr_q
                acc += -ws * wt * s * J * np.einsum("pq,npq->n", coef, dG)
        return acc
    h = 1e-2 * np.linalg.norm(x - P0)
    grad = np.zeros((3, 3))
    for m in range(3):
        e = np.zeros(3); e[m] = h
        grad[:, m] = (-u(x + 2 * e) + 8 * u(x + e) - 8 * u(x - e) + u(x - 2 * e)) / (12 * h)
    eps = 0.5 * (grad + grad.T)
    return LAM * np.trace(eps) * np.eye(3) + 2 * MU * eps


@pytest.mark.parametrize("xoff", [np.array([3.0, 1.0, 2.0]), np.array([-2.5, 0.5, -1.5]),
                                  np.array([1.0, -3.0, 0.3])])
def test_loop_integral_matches_volterra_surface_integral(xoff):
    P = np.array([[0.0, 0.0, 0.0], [1.0, 0.2, 0.1], [0.3, 1.1, -0.2]])
    b = np.array([0.6, -0.3, 0.74])
    x = P.mean(0) + xoff
    s_loop = oracle.stress_polygon(P, b, MU, NU, x)[0]
    s_surf = _surface_stress(P, b, x)
    assert np.allclose(s_loop, s_surf, rtol=0, atol=2e-6 * np.abs(s_surf).max())


def _strip(L, W):
    return np.array([[-L / 2, 0, -W / 2], [L / 2, 0, -W / 2], [L / 2, 0, W / 2], [-L / 2, 0, W / 2]])


def test_long_strip_reduces_to_2d_dislocation_pairs():
    """Center of a long strip (L/W = 2000) with uniform slip: antiplane (two screw
    dislocations) -2 mu b/(pi W); in-plane (two edge dislocations) and opening
    -2 mu b/(pi (1-nu) W).  Negative = stress drop / compression (Hirth & Lothe, Segall)."""
    L, W = 2000.0, 1.0
    P = _strip(L, W)
    n = oracle.elem_frames(P[None])["normal"][0]
    sig = oracle.stress_polygon(P, [[1, 0, 0], [0, 0, 1], list(n)], MU, NU, np.zeros(3))
    screw = np.array([1, 0, 0]) @ sig[0] @ n
    edge = np.array([0, 0, 1]) @ sig[1] @ n
    opening = n @ sig[2] @ n
    assert screw == pytest.approx(-2 * MU / (np.pi * W), rel=1e-5)
    assert edge == pytest.approx(-2 * MU / (np.pi * (1 - NU) * W), rel=1e-5)
    assert opening == pytest.approx(-2 * MU / (np.pi * (1 - NU) * W), rel=1e-5)


def test_2d_screw_field_off_plane():
    """Off the plane the long strip gives the field of two opposite screw dislocations."""
    L, W = 4000.0, 1.0
    P = _strip(L, W)
    x = np.array([0.0, 0.37, 0.21])
    sig = oracle.stress_polygon(P, [[1, 0, 0]], MU, NU, x)[0]
    # screw dislocation along x at (y0, z0): sigma_xy = -k (z - z0)/r^2, sigma_xz = k (y - y0)/r^2
    def pair(y, z):
        sxy, sxz = 0.0, 0.0
        for z0, sgn in ((-W / 2, 1.0), (W / 2, -1.0)):
            r2 = y * y + (z - z0) ** 2
            sxy += sgn * (-(z - z0) / r2)
            sxz += sgn * (y / r2)
        return sxy, sxz
    sxy, sxz = pair(x[1], x[2])
    k = sig[0, 1] / sxy
    assert abs(k) == pytest.approx(MU / (2 * np.pi), rel=1e-5)
    assert sig[0, 2] == pytest.approx(k * sxz, rel=1e-5)


def test_self_stress_signs_on_nonplanar_mesh():
    m = meshes.scaled_thrust_mesh(6, 3, seed=9)
    n = m.n_elem
    idx = np.arange(n)
    E = oracle.pair_entries(m, oracle.OP_VEC_FULL, idx, idx, MU, NU)
    assert np.all(E[:, 0, 0] < 0) and np.all(E[:, 1, 1] < 0)
    P = m.verts[0]
    fr = oracle.elem_frames(P[None])
    nn = fr["normal"][0]
    s_open = oracle.stress_polygon(P, nn, MU, NU, fr["centroid"][0])[0]
    assert nn @ s_open @ nn < 0


def test_equilibrium_div_sigma_zero():
    P = np.array([[0.0, 0.0, 0.0], [1.0, 0.2, 0.1], [0.3, 1.1, -0.2]])
    b = np.array([0.2, 0.9, -0.4])
    x0 = P.mean(0) + np.array([0.4, -0.3, 0.6])
    h = 1e-3
    div = np.zeros(3)
    for j in range(3):
        e = np.zeros(3); e[j] = h
        f = lambda xx: oracle.stress_polygon(P, b, MU, NU, xx)[0][:, j]
        div += (-f(x0 + 2 * e) + 8 * f(x0 + e) - 8 * f(x0 - e) + f(x0 - 2 * e)) / (12 * h)
    scale = np.abs(oracle.stress_polygon(P, b, MU, NU, x0)[0]).max() / 0.5
    assert np.linalg.norm(div) < 1e-7 * scale


def test_rectangle_equals_two_triangles():
    R = np.array([[0.0, 0.0, 0.0], [2.0, 0.0, 0.0], [2.0, 0.3, -1.0], [0.0, 0.3, -1.0]])
    b = np.array([0.5, -0.1, 0.3])
    for x in (np.array([0.9, 0.15, -0.5]), np.array([3.0, 1.0, 1.0]), np.array([-0.7, 0.2, -0.2])):
        s_r = oracle.stress_polygon(R, b, MU, NU, x)[0]
        s_t = (oracle.stress_polygon(R[[0, 1, 2]], b, MU, NU, x)[0]
               + oracle.stress_polygon(R[[0, 2, 3]], b, MU, NU, x)[0])
        assert np.allclose(s_r, s_t, rtol=0, atol=1e-10 * np.abs(s_r).max())


def test_superposition_of_subdivided_patch():
    """A uniform-slip square equals the sum of its 3x3 sub-squares (linearity, exact)."""
    big = meshes.planar_vertical_rect(1, 1, 3.0).verts[0]
    small = meshes.planar_vertical_rect(3, 3, 1.0).verts
    b = np.array([0.7, 0.0, -0.4])
    for x in (np.array([4.0, 0.5, -1.0]), np.array([1.5, 2.0, -1.5]), np.array([-1.0, 0.0, -4.0])):
        s_big = oracle.stress_polygon(big, b, MU, NU, x)[0]
        s_sum = sum(oracle.stress_polygon(q, b, MU, NU, x)[0] for q in small)
        assert np.allclose(s_big, s_sum, rtol=0, atol=1e-10 * np.abs(s_big).max())


def test_rotation_and_translation_covariance():
    P = np.array([[0.0, 0.0, 0.0], [1.0, 0.2, 0.1], [0.3, 1.1, -0.2]])
    b = np.array([0.2, 0.9, -0.4])
    x = np.array([0.8, -0.6, 0.9])
    th = 0.7
    Rz = np.array([[np.cos(th), -np.sin(th), 0], [np.sin(th), np.cos(th), 0], [0, 0, 1]])
    Rx = np.array([[1, 0, 0], [0, np.cos(1.1), -np.sin(1.1)], [0, np.sin(1.1), np.cos(1.1)]])
    R = Rx @ Rz
    T = np.array([10.0, -4.0, 7.0])
    s0 = oracle.stress_polygon(P, b, MU, NU, x)[0]
    s1 = oracle.stress_polygon(P @ R.T + T, R @ b, MU, NU, R @ x + T)[0]
    assert np.allclose(s1, R @ s0 @ R.T, rtol=0, atol=1e-11 * np.abs(s0).max())


def test_far_field_decays_as_inverse_cube():
    P = np.array([[0.0, 0.0, 0.0], [1.0, 0.0, 0.0], [0.0, 1.0, 0.0]])
    b = np.array([1.0, 0.0, 0.0])
    d = np.array([0.3, 0.5, 0.81]); d /= np.linalg.norm(d)
    c = P.mean(0)
    s1 = oracle.stress_polygon(P, b, MU, NU, c + 1000 * d)[0]
    s2 = oracle.stress_polygon(P, b, MU, NU, c + 2000 * d)[0]
    k = np.unravel_index(np.abs(s1).argmax(), s1.shape)
    assert s2[k] / s1[k] == pytest.approx(1 / 8, rel=1e-4)


def test_planar_fault_no_normal_coupling_and_symmetry():
    m = meshes.planar_vertical_rect(6, 4, 250.0)
    n = m.n_elem
    i, j = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    E = oracle.pair_entries(m, oracle.OP_VEC_FULL, i.ravel(), j.ravel(), MU, NU).reshape(n, n, 3, 2)
    scale = np.abs(E[:, :, :2, :]).max()
    assert np.abs(E[:, :, 2, :]).max() < 1e-10 * scale          # B = 0 on a plane
    A = E[:, :, 0, 0]
    assert np.allclose(A, A.T, rtol=0, atol=1e-10 * np.abs(A).max())   # uniform grid
    assert np.all(np.diag(A) < 0)


def test_dense_rows_consistent_with_pair_entries():
    m = meshes.scaled_thrust_mesh(4, 3, seed=5)
    n = m.n_elem
    x = rng.normal(7, 2 * n)
    rows = np.array([0, 5, n - 1])
    y = oracle.dense_rows(m, oracle.OP_VEC_FULL, rows, x, MU, NU)
    for r, i in enumerate(rows):
        E = oracle.pair_entries(m, oracle.OP_VEC_FULL, np.full(n, i), np.arange(n), MU, NU)
        ref = np.einsum("jac,cj->a", E, x.reshape(2, n))
        assert np.allclose(y[r], ref, rtol=1e-13, atol=0)
