"""Pins of the oracle's half-space element solution (Sec. 2.1: the elements live in an elastic
half space with a traction-free surface).  The oracle adds to its full-space element stress
the difference between Mindlin's point-force solution and Kelvin's, carried over the element
by the Volterra representation.  What fixes it, independently of its own formulas:

- the point-force solution against the textbook surface-load limits (Boussinesq's normal load,
  Cerruti's tangential load, on the surface of the half space);
- reciprocity G_kp(x, xi) = G_pk(xi, x) of the half-space Green's function;
- Navier's equations (equilibrium) of the point-force correction and of the element
  correction field, by finite differences;
- a traction-free surface for the complete element solution (full space + correction) of a
  buried element, for both slip directions -- with equilibrium and decay this determines the
  correction uniquely, and it ties the correction's sign and scale to the full-space part;
- decay of the correction with depth, and convergence of the element quadrature."""
import numpy as np
import pytest

import oracle

MU, NU = 32e9, 0.25
LAM = 2 * MU * NU / (1 - 2 * NU)


def _rect(top=-1000.0, L=2000.0, W=1000.0, dip_deg=30.0, x0=0.0):
    d = np.radians(dip_deg)
    return np.array([[x0, 0, top], [x0 + L, 0, top], [x0 + L, W * np.cos(d), top - W * np.sin(d)],
                     [x0, W * np.cos(d), top - W * np.sin(d)]])


def _slips(P):
    fr = oracle.elem_frames(P[None])
    return np.stack([fr["strike"][0], fr["dip"][0]])


def test_boussinesq_and_cerruti_surface_displacements():
    """Unit force at the surface (source 1e-9 m deep), receiver on the surface at distance r:
    normal load (Boussinesq): u_z = (1 - nu) / (2 pi mu r) along the force, radial
    (1 - 2 nu) / (4 pi mu r) away from it for a force pointing out of the solid; tangential
    load (Cerruti): u_x = [(1 - nu) / r + nu x^2 / r^3] / (2 pi mu), u_y = nu x y / (2 pi mu r^3),
    u_z = -(1 - 2 nu) x / (4 pi mu r^2)."""
    xi = np.array([0.0, 0.0, -1e-9])
    for x in ([3.0, 4.0, 0.0], [-2.0, 0.5, 0.0], [0.0, -7.0, 0.0]):
        x = np.array(x)
        r = np.hypot(x[0], x[1])
        G = oracle.halfspace_G(x, xi, MU, NU)
        tp = 1 / (2 * np.pi * MU)
        # force along +z (out of the solid)
        assert G[2, 2] == pytest.approx((1 - NU) * tp / r, rel=1e-8)
        ur = (G[0, 2] * x[0] + G[1, 2] * x[1]) / r
        assert ur == pytest.approx((1 - 2 * NU) / (4 * np.pi * MU * r), rel=1e-8)
        assert abs(G[0, 2] * x[1] - G[1, 2] * x[0]) < 1e-12 * tp / r
        # force along +x
        assert G[0, 0] == pytest.approx(tp * ((1 - NU) / r + NU * x[0] ** 2 / r ** 3), rel=1e-8)
        assert G[1, 0] == pytest.approx(tp * NU * x[0] * x[1] / r ** 3, rel=1e-8, abs=1e-12 * tp / r)
        assert G[2, 0] == pytest.approx(-(1 - 2 * NU) * x[0] / (4 * np.pi * MU * r ** 2), rel=1e-8,
                                        abs=1e-12 * tp / r)


def test_reciprocity():
    rng = np.random.default_rng(5)
    for _ in range(20):
        x = rng.uniform(-3, 3, 3); x[2] = -rng.uniform(0.1, 3)
        xi = rng.uniform(-3, 3, 3); xi[2] = -rng.uniform(0.1, 3)
        G, Gt = oracle.halfspace_G(x, xi, MU, NU), oracle.halfspace_G(xi, x, MU, NU)
        assert np.abs(G - Gt.T).max() <= 1e-13 * np.abs(G).max()


def _navier(u, x, h):
    """mu lap u + (lam + mu) grad div u at x by central differences of u (3-vector field)."""
    e = np.eye(3)
    H = np.zeros((3, 3, 3))   # H[k, i, j] = d2 u_k / dx_i dx_j
    for i in range(3):
        for j in range(3):
            H[:, i, j] = (u(x + h * e[i] + h * e[j]) - u(x + h * e[i] - h * e[j]) - u(x - h * e[i] + h * e[j])
                          + u(x - h * e[i] - h * e[j])) / (4 * h * h)
    lap = np.array([np.trace(H[k]) for k in range(3)])
    grad_div = np.array([sum(H[k, i, k] for k in range(3)) for i in range(3)])
    return MU * lap + (LAM + MU) * grad_div, H


@pytest.mark.parametrize("p", [0, 1, 2])
def test_point_force_correction_is_elastostatic_and_clears_the_surface(p):
    xi = np.array([0.3, -0.2, -1.0])
    u = lambda x: oracle.halfspace_G(x, xi, MU, NU, with_kelvin=False)[:, p]
    for x in ([0.8, 0.4, -0.7], [-1.5, 1.0, -2.5], [2.0, 0.0, -0.2]):
        res, H = _navier(u, np.array(x), 1e-4)
        assert np.abs(res).max() < 1e-6 * MU * np.abs(H).max()
    # complete solution (Kelvin + correction): traction sigma_iz = 0 on z = 0
    full = lambda x: oracle.halfspace_G(x, xi, MU, NU)[:, p]
    for x in ([0.5, 0.7, 0.0], [-2.0, 1.0, 0.0]):
        x = np.array(x)
        h, e = 1e-4, np.eye(3)
        # one-sided (into the solid) second-order differences for d/dz; central for x, y
        grad = np.zeros((3, 3))
        for m in range(2):
            grad[:, m] = (full(x + h * e[m]) - full(x - h * e[m])) / (2 * h)
        grad[:, 2] = (-3 * full(x) + 4 * full(x - h * e[2]) - full(x - 2 * h * e[2])) / (-2 * h)
        sig = LAM * np.trace(grad) * np.eye(3) + MU * (grad + grad.T)
        assert np.abs(sig[:, 2]).max() < 1e-6 * np.abs(sig).max()


def test_buried_element_leaves_the_surface_traction_free():
    """Complete half-space stress of a buried 2 km x 1 km rectangle (top 1 km deep, dip 30
    degrees) at points of the free surface: sigma_xz = sigma_yz = sigma_zz = 0, while the
    full-space part alone has tractions of hundreds of kPa there."""
    P = _rect()
    b = _slips(P)
    for x in ([500.0, -800.0, 0.0], [1200.0, 300.0, 0.0], [3000.0, 2000.0, 0.0], [-400.0, 900.0, 0.0]):
        s_hs = oracle.stress_polygon_hs(P, b, MU, NU, x)
        s_fs = oracle.stress_polygon(P, b, MU, NU, x)
        for ib in range(2):
            assert np.abs(s_fs[ib][:, 2]).max() > 1e-2 * np.abs(s_fs[ib]).max()
            assert np.abs(s_hs[ib][:, 2]).max() < 1e-9 * np.abs(s_fs[ib]).max()


def test_buried_triangle_leaves_the_surface_traction_free():
    T = np.array([[0.0, 0.0, -500.0], [800.0, 200.0, -900.0], [100.0, 700.0, -1300.0]])
    b = _slips(T)
    for x in ([300.0, 300.0, 0.0], [-600.0, 100.0, 0.0]):
        s_hs = oracle.stress_polygon_hs(T, b, MU, NU, x)
        s_fs = oracle.stress_polygon(T, b, MU, NU, x)
        for ib in range(2):
            assert np.abs(s_hs[ib][:, 2]).max() < 1e-9 * np.abs(s_fs[ib]).max()


def test_element_correction_is_in_equilibrium():
    P = _rect()
    b = _slips(P)[1]
    e = np.eye(3)
    for x in ([1000.0, 400.0, -600.0], [2500.0, -300.0, -1500.0]):
        x = np.array(x)
        h = 2.0
        sig = lambda y: oracle.stress_polygon_hs(P, b, MU, NU, y, corr_only=True)[0]
        div = sum((sig(x + h * e[j])[:, j] - sig(x - h * e[j])[:, j]) / (2 * h) for j in range(3))
        scale = np.abs(sig(x)).max() / 1000.0     # stress over the depth scale
        assert np.abs(div).max() < 1e-5 * scale


def test_correction_decays_with_depth():
    """The correction at the element's own centre falls off as (size / depth)^3 once the
    element is deep (the image is a source 2 |z| away)."""
    ratios = []
    for top in (-20e3, -40e3, -80e3):
        P = _rect(top=top, L=1000.0, W=1000.0)
        fr = oracle.elem_frames(P[None])
        c = fr["centroid"][0]
        s_c = oracle.stress_polygon_hs(P, _slips(P), MU, NU, c, corr_only=True)
        ratios.append(np.abs(s_c).max())
    assert ratios[0] / ratios[1] == pytest.approx(8.0, rel=0.1)
    assert ratios[1] / ratios[2] == pytest.approx(8.0, rel=0.05)


def test_element_quadrature_converges():
    P = _rect(top=-300.0)
    b = _slips(P)
    x = np.array([900.0, 500.0, -500.0])
    try:
        oracle.set_halfspace_ratio(0.5)
        a = oracle.stress_polygon_hs(P, b, MU, NU, x, corr_only=True)
        oracle.set_halfspace_ratio(0.25)
        c = oracle.stress_polygon_hs(P, b, MU, NU, x, corr_only=True)
    finally:
        oracle.set_halfspace_ratio(0.5)
    assert np.abs(a - c).max() < 1e-9 * np.abs(c).max()


def test_half_space_entries_reduce_to_full_space_at_depth():
    """Operator entries of a small fault 200 km deep: the half-space entries equal the
    full-space ones to the decay of the correction (about (2 km / 400 km)^3)."""
    from synthetic import meshes
    m = meshes.planar_vertical_rect(4, 3, 500.0, origin=(0.0, 0.0, -200e3))
    recv = np.repeat(np.arange(12), 12).astype(np.int32)
    src = np.tile(np.arange(12), 12).astype(np.int32)
    Ef = oracle.pair_entries(m, oracle.OP_VEC_FULL, recv, src, MU, NU)
    Eh = oracle.pair_entries(m, oracle.OP_VEC_FULL, recv, src, MU, NU, half_space=True)
    assert np.abs(Eh - Ef).max() < 1e-6 * np.abs(Ef).max()
    assert np.abs(Eh - Ef).max() > 0


def test_half_space_h_matrix_reproduces_the_dense_operator():
    """The oracle's tree, ACA and H-matvec (Secs. 3.1-3.2, Eq. 20) on the half-space entries:
    eps -> 0 gives the dense half-space operator; eps = 1e-4 compresses (low-rank blocks) and
    stays within 10 eps of it."""
    from synthetic import meshes
    m = meshes.dipping_rect(16, 8, 250.0, 30.0, origin=(0.0, 0.0, -200.0))
    n = m.n_elem
    op = oracle.OP_VEC_FULL
    x = np.random.default_rng(7).normal(size=2 * n)
    yd = oracle.dense_matvec(m, op, x, MU, NU, half_space=True)
    for eps, tol in ((1e-12, 1e-10), (1e-4, 1e-3)):
        H = oracle.HMatrix(m, op, eps, 8, 1, MU, NU, half_space=True)
        y = H.matvec(x)
        assert np.linalg.norm(y - yd) / np.linalg.norm(yd) < tol
    assert H.n_lowrank > 0


def test_distance_based_rule_order_matches_the_full_rule():
    """The element quadrature picks its Gauss-Legendre order from the distance to the image
    (an n x n rule errs by about (diam / 2R)^(2n)); it must agree with the 8 x 8 rule on every
    pair: a shallow fault (all pairs) and 2,000 sampled pairs of the 160,000-element thrust
    fault (mostly far from their images), self pairs included."""
    from synthetic import meshes, rng
    big = meshes.scaled_thrust_mesh(400, 200, seed=3)
    u = rng.uniform(90, 4000)
    rb, sb = (u[:2000] * big.n_elem).astype(np.int32), (u[2000:] * big.n_elem).astype(np.int32)
    rb[:100] = sb[:100]
    small = meshes.dipping_rect(6, 4, 250.0, 40.0, origin=(0.0, 0.0, -50.0))
    i, j = np.meshgrid(np.arange(small.n_elem), np.arange(small.n_elem), indexing="ij")
    for m, recv, src in ((big, rb, sb), (small, i.ravel().astype(np.int32), j.ravel().astype(np.int32))):
        try:
            oracle.set_halfspace_adaptive(False)
            full = oracle.pair_entries(m, oracle.OP_VEC_FULL, recv, src, MU, NU, half_space=True)
        finally:
            oracle.set_halfspace_adaptive(True)
        adap = oracle.pair_entries(m, oracle.OP_VEC_FULL, recv, src, MU, NU, half_space=True)
        scale = np.abs(full).max(axis=(1, 2), keepdims=True)
        assert (np.abs(adap - full) / scale).max() < 1e-10
