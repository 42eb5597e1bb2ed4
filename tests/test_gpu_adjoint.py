"""The transposed product H^T and the discrete adjoint of the rate-state RK integration.

H^T is packed from the same partition and factors as H, so <H x, v> = <x, H^T v> holds to
rounding (FP64 storage: 1e-12 relative to |H x| |v|); against the oracle's dense operator
the transposed product carries the same ACA error as H (10 eps)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
import paper_2110_12165_gb300 as hbi
from synthetic import friction, meshes, rng
from gpu_util import dev, host, import_oracle, rel_l2

pytestmark = pytest.mark.gpu

MU, NU = 32e9, 0.25


def _cases():
    m1 = meshes.scaled_thrust_mesh(24, 12, seed=3)          # 576 triangles, 2 -> 3 operator
    m2 = meshes.dipping_rect(20, 10, 250.0, 40.0)           # 200 rectangles, rake shear
    return [(m1, oracle.OP_VEC_FULL, np.full(m1.n_elem, np.pi / 2)),
            (m2, oracle.OP_RAKE_SHEAR, np.full(m2.n_elem, np.pi / 2)),
            (m1, oracle.OP_RAKE_SHEAR_NORMAL, np.full(m1.n_elem, 1.0))]


@pytest.mark.parametrize("case", [0, 1, 2])
@pytest.mark.parametrize("storage,tol", [("fp64", 1e-12), ("fp32", 1e-6), ("mixed", 1e-6), ("adaptive", 1e-6)])
def test_transpose_is_the_adjoint_of_the_product(case, storage, tol):
    m, op, rake = _cases()[case]
    n = m.n_elem
    nin, nout = hbi.OP_NIN[op], hbi.OP_NOUT[op]
    h = hbi.hbi_build(m.verts, MU, NU, op, 1e-6, 16, 2, storage, rake=rake, transpose=True)
    x, v = rng.normal(31, nin * n), rng.normal(32, nout * n)
    Hx = torch.zeros(nout * n, dtype=torch.float64, device="cuda")
    Htv = torch.zeros(nin * n, dtype=torch.float64, device="cuda")
    hbi.hbi_matvec(h, dev(x), Hx)
    hbi.hbi_matvec_transpose(h, dev(v), Htv)
    lhs, rhs = float(np.dot(host(Hx), v)), float(np.dot(x, host(Htv)))
    scale = np.linalg.norm(host(Hx)) * np.linalg.norm(v)
    assert abs(lhs - rhs) <= tol * scale
    # against the oracle's dense operator: H^T v = sum_i v_i H[i, :], by linearity of the
    # dense rows in x (one product per input component and element would be too slow, so
    # compare the scalar <x, H_dense^T v> = <H_dense x, v> and the GPU H^T v on random x')
    Hd = oracle.dense_matvec(m, op, x, MU, NU, rake=rake)
    assert abs(float(np.dot(Hd, v)) - rhs) <= 10 * 1e-6 * np.linalg.norm(Hd) * np.linalg.norm(v) + tol * scale


def test_transpose_requires_the_build_flag():
    m, op, rake = _cases()[1]
    h = hbi.hbi_build(m.verts, MU, NU, op, 1e-4, 16, 1, "fp32", rake=rake)
    v = torch.zeros(m.n_elem, dtype=torch.float64, device="cuda")
    with pytest.raises(hbi.HbiError):
        hbi.hbi_matvec_transpose(h, v, v.clone())


# ------------------------------------------------------------------ adjoint of the RHS / RK
def _ode_case(op=oracle.OP_VEC_FULL):
    m = meshes.scaled_thrust_mesh(24, 12, seed=3)           # N = 576, nonplanar, normal coupling
    F = friction.thrust_friction(m, seed=3)
    h = hbi.hbi_build(m.verts, F.mu, F.nu, op, 1e-6, 16, 2, "fp64", rake=F.rake, transpose=True)
    phi, tau = oracle.steady_state(F.V_init, F.a, F.b, F.sigma0, F.f0, F.V0)
    return m, F, h, np.concatenate([phi, tau, F.sigma0])


def _fric(F, a=None, dc=None):
    return hbi.friction(dev(F.a if a is None else a), dev(F.b), dev(F.dc if dc is None else dc), dev(F.rake),
                        F.f0, F.V0, F.Vpl, F.mu, F.cs)


def _rhs(h, fr, y):
    out = torch.zeros(len(y), dtype=torch.float64, device="cuda")
    hbi.hbi_rhs(h, fr, dev(y), out)
    return host(out)


def test_rhs_vjp_matches_directional_derivatives():
    """<v, J w> by central differences of hbi_rhs equals <J^T v, w>; the same for the
    parameters a (b fixed) and d_c.  Steps are scaled per component (phi ~ 1, stresses ~
    1e7 Pa), so the O(eps^2) truncation stays below 1e-7 relative.  The state is moved away
    from steady sliding (phi by ~2e-2) so that dphi/dt, the only route of d_c, is not a
    cancellation of equal terms (else the differences would be rounding noise)."""
    m, F, h, y = _ode_case()
    n = m.n_elem
    y = y + np.concatenate([2e-2 * rng.normal(60, n), 1e4 * rng.normal(61, n), 1e4 * rng.normal(62, n)])
    v = rng.normal(63, 3 * n) * np.concatenate([np.full(n, 1e-6), np.full(n, 1.0), np.full(n, 1.0)])
    fr = _fric(F)
    yb, ga, gdc = (torch.zeros(k, dtype=torch.float64, device="cuda") for k in (3 * n, n, n))
    hbi.hbi_rhs_vjp(h, fr, dev(y), dev(v), yb, ga, gdc)
    yb, ga, gdc = host(yb), host(ga), host(gdc)
    w = np.concatenate([1e-3 * rng.normal(64, n), 1e4 * rng.normal(65, n), 1e4 * rng.normal(66, n)])
    eps = 1e-3
    fd = (_rhs(h, fr, y + eps * w) - _rhs(h, fr, y - eps * w)) / (2 * eps)
    assert abs(np.dot(v, fd) - np.dot(yb, w)) <= 1e-6 * np.linalg.norm(v) * np.linalg.norm(fd) * 10
    da = 1e-4 * F.a * rng.normal(67, n)
    fd_a = (_rhs(h, _fric(F, a=F.a + da), y) - _rhs(h, _fric(F, a=F.a - da), y)) / 2
    assert np.isclose(np.dot(v, fd_a), np.dot(ga, da), rtol=1e-6, atol=0)
    ddc = 1e-4 * F.dc * rng.normal(68, n)
    fd_dc = (_rhs(h, _fric(F, dc=F.dc + ddc), y) - _rhs(h, _fric(F, dc=F.dc - ddc), y)) / 2
    assert np.isclose(np.dot(v, fd_dc), np.dot(gdc, ddc), rtol=1e-6, atol=0)


def _loss_host(F, yN, target):
    n = len(F.a)
    phi, tau, sig = yN[:n], yN[n:2 * n], yN[2 * n:3 * n]
    a = F.a
    V = F.V0 * (np.exp((tau / sig - phi) / a) - np.exp((-tau / sig - phi) / a))
    return 0.5 * np.sum((np.log(V) - target) ** 2)


def _run_fixed(h, F, y0, dts, a=None, dc=None):
    s = dev(np.concatenate([y0, np.zeros(len(F.a))]))
    hbi.hbi_rk_fixed(h, _fric(F, a, dc), s, dts)
    return host(s)


def test_adjoint_gradient_matches_central_differences():
    m, F, h, y0 = _ode_case()
    n = m.n_elem
    # the step sizes of an adaptive run, frozen, capped at 5e5 s: the controller lets steps
    # grow to the edge of the explicit scheme's stability region, where the frozen schedule
    # would amplify the parameter changes of the differences without bound
    s = dev(np.concatenate([y0, np.zeros(n)]))
    st, done, rec = hbi.hbi_step(h, _fric(F), s, dev([0.0]), dev([1e4]), 1e-4, 12)
    assert st == 0
    dts = np.minimum(rec[:, 1], 5e5)
    phi, tau = y0[:n], y0[n:2 * n]
    V0 = F.V0 * (np.exp((tau / y0[2 * n:] - phi) / F.a) - np.exp((-tau / y0[2 * n:] - phi) / F.a))
    target = np.log(V0) + 0.1 * rng.normal(70, n)
    g_amb, g_dc = torch.zeros(n, dtype=torch.float64, device="cuda"), torch.zeros(n, dtype=torch.float64, device="cuda")
    sf = torch.zeros(4 * n, dtype=torch.float64, device="cuda")
    loss = hbi.hbi_adjoint(h, _fric(F), dev(np.concatenate([y0, np.zeros(n)])), dts, dev(target), g_amb, g_dc,
                           checkpoint_every=5, state_final=sf)
    yN = _run_fixed(h, F, y0, dts)
    assert np.array_equal(host(sf), yN)                      # the adjoint's forward run is the plain one
    assert np.isclose(loss, _loss_host(F, yN, target), rtol=1e-12)
    g_amb, g_dc = host(g_amb), host(g_dc)
    els = np.unique(rng.splitmix64(71, 8) % np.uint64(n)).astype(int)
    for i in els:
        for which, g in (("a", g_amb), ("dc", g_dc)):
            base = F.a if which == "a" else F.dc
            # steps: large enough that the loss change stands well above the rounding of the
            # loss sum (1e-14 relative), small enough for the O(d^2) truncation
            d = (1e-5 if which == "a" else 1e-3) * base[i]
            p, q = base.copy(), base.copy()
            p[i] += d
            q[i] -= d
            kw_p, kw_q = ({"a": p}, {"a": q}) if which == "a" else ({"dc": p}, {"dc": q})
            fd = (_loss_host(_with(F, **kw_p), _run_fixed(h, F, y0, dts, **kw_p), target) -
                  _loss_host(_with(F, **kw_q), _run_fixed(h, F, y0, dts, **kw_q), target)) / (2 * d)
            # rounding of the two loss sums (~ n u |L|) divided by the step
            noise = 2 * n * 1.1e-16 * loss / (2 * d)
            assert np.isclose(g[i], fd, rtol=2e-5, atol=noise), (which, i, g[i], fd, noise)


def _with(F, a=None, dc=None):
    import dataclasses
    return dataclasses.replace(F, a=F.a if a is None else a, dc=F.dc if dc is None else dc)


def test_adjoint_checkpoint_interval_does_not_change_the_result():
    m, F, h, y0 = _ode_case()
    n = m.n_elem
    dts = np.full(12, 3e5)
    target = rng.normal(72, n) - 20.0
    res = []
    for every in (1, 5, 12, 50):
        ga, gd = torch.zeros(n, dtype=torch.float64, device="cuda"), torch.zeros(n, dtype=torch.float64, device="cuda")
        L = hbi.hbi_adjoint(h, _fric(F), dev(np.concatenate([y0, np.zeros(n)])), dts, dev(target), ga, gd, every)
        res.append((L, host(ga), host(gd)))
    for L, ga, gd in res[1:]:
        assert L == res[0][0] and np.array_equal(ga, res[0][1]) and np.array_equal(gd, res[0][2])


def test_autograd_function_gives_the_adjoint_gradient():
    m, F, h, y0 = _ode_case()
    n = m.n_elem
    dts = np.full(6, 2e5)
    target = dev(rng.normal(73, n) - 20.0)
    amb = dev(F.a - F.b).requires_grad_(True)
    dc = dev(F.dc).requires_grad_(True)
    state0 = dev(np.concatenate([y0, np.zeros(n)]))
    loss = hbi.sequence_loss(h, amb, dc, dev(F.b), dev(F.rake), (F.f0, F.V0, F.Vpl, F.mu, F.cs), state0, dts,
                             target, checkpoint_every=4)
    (3.0 * loss).backward()
    ga, gd = torch.zeros(n, dtype=torch.float64, device="cuda"), torch.zeros(n, dtype=torch.float64, device="cuda")
    L = hbi.hbi_adjoint(h, _fric(F), state0, dts, target, ga, gd, 4)
    assert float(loss) == L
    assert torch.equal(amb.grad, 3.0 * ga) and torch.equal(dc.grad, 3.0 * gd)


def test_adjoint_gradient_matches_the_oracle_complex_step():
    """hbi_adjoint on the oracle's own factors (FP64 storage, H^T packed from the same factors)
    against the oracle's complex-step derivative of the same fixed-step loss, an independent
    route (the whole Cash-Karp map in complex arithmetic).  Both are exact derivatives of the
    same discrete map and differ only by rounding (the library folds the loading into the
    product input): loss to 1e-10, gradients to 1e-7 relative or 1e-9 of the largest entry."""
    m = meshes.scaled_thrust_mesh(12, 6, seed=3)             # N = 144, nonplanar, 2 -> 3
    F = friction.thrust_friction(m, seed=3)
    n = m.n_elem
    H = oracle.HMatrix(m, oracle.OP_VEC_FULL, 1e-8, 8, 1, F.mu, F.nu, rake=F.rake)
    h = import_oracle(H, "fp64", transpose=True)
    phi, tau = oracle.steady_state(F.V_init, F.a, F.b, F.sigma0, F.f0, F.V0)
    y0 = np.concatenate([phi + 0.01 * rng.normal(80, n), tau, F.sigma0])
    dts = np.full(10, 2e4)          # well inside the explicit scheme's stability region here
    target = np.log(1e-9) + 0.1 * rng.normal(81, n)
    ga = torch.zeros(n, dtype=torch.float64, device="cuda")
    gd = torch.zeros(n, dtype=torch.float64, device="cuda")
    L = hbi.hbi_adjoint(h, _fric(F), dev(np.concatenate([y0, np.zeros(n)])), dts, dev(target), ga, gd,
                        checkpoint_every=4)
    L_ref, _ = H.fixed_loss(F, y0, dts, target)
    assert L == pytest.approx(L_ref, rel=1e-10)
    ga, gd = host(ga), host(gd)
    els = sorted(set([0, n - 1] + (rng.splitmix64(82, 10) % np.uint64(n)).astype(int).tolist()))
    ga_ref, gd_ref = H.fixed_loss_grad(F, y0, dts, target, els)
    for g, ref, full in ((ga[els], ga_ref, ga), (gd[els], gd_ref, gd)):
        assert np.allclose(g, ref, rtol=1e-7, atol=1e-9 * np.abs(full).max()), np.abs(g - ref).max()
