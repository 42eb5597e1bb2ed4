"""Batched ensemble (many independent faults in one handle): each member must be computed
exactly as when it is built and stepped alone.

The ensemble operator is block diagonal over the members, each built from its own tree,
partition and ACA, and one attempt graph advances all members, each with its own step size
and accept/reject decisions.  With every member's DOF count a multiple of 4 (its product
input then starts on a 16-byte boundary, as in a single build) the member's products and
trajectory equal the single-model ones bit for bit; the single-model path is pinned to the
oracle elsewhere, and the products are also checked against the oracle's dense operator."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
import paper_2110_12165_gb300 as hbi
from synthetic import friction, meshes, rng
from gpu_util import dev, host, rel_l2

pytestmark = pytest.mark.gpu

MU, NU = 32e9, 0.25


def _members():
    # rectangular faults of uneven size and dip (N = 128, 72, 200, 32)
    return [meshes.dipping_rect(16, 8, 250.0, 30.0), meshes.dipping_rect(12, 6, 250.0, 90.0),
            meshes.dipping_rect(20, 10, 250.0, 45.0), meshes.dipping_rect(8, 4, 250.0, 60.0)]


def _rakes(ms):
    return [np.full(m.n_elem, np.pi / 2) for m in ms]


@pytest.mark.parametrize("storage", ["fp32", "mixed", "adaptive", "fp64"])
def test_ensemble_products_equal_single_models(storage):
    ms = _members()
    rk = _rakes(ms)
    eps, leaf, L = 1e-6, 8, 2
    hE, starts = hbi.hbi_build_ensemble([m.verts for m in ms], MU, NU, oracle.OP_RAKE_SHEAR, eps, leaf, L,
                                        storage, rakes=rk)
    assert hE.stats()["n_models"] == len(ms)
    x = rng.normal(5, int(starts[-1]))
    yE = torch.zeros(int(starts[-1]), dtype=torch.float64, device="cuda")
    hbi.hbi_matvec(hE, dev(x), yE)
    yE = host(yE)
    for k, m in enumerate(ms):
        a, b = int(starts[k]), int(starts[k + 1])
        h1 = hbi.hbi_build(m.verts, MU, NU, oracle.OP_RAKE_SHEAR, eps, leaf, L, storage, rake=rk[k])
        y1 = torch.zeros(b - a, dtype=torch.float64, device="cuda")
        hbi.hbi_matvec(h1, dev(x[a:b]), y1)
        assert np.array_equal(yE[a:b], host(y1)), f"member {k} differs from its single build"
        # and the member against the oracle's dense operator (GPU-built factors: <= 10 eps;
        # FP16 factors of the mixed storage: the storage tolerance)
        yd = oracle.dense_matvec(m, oracle.OP_RAKE_SHEAR, x[a:b], MU, NU, rake=rk[k])
        tol = 2e-3 if storage in ("mixed", "adaptive") else 10 * eps
        assert rel_l2(yE[a:b], yd) < tol


def test_ensemble_steps_equal_single_runs():
    ms = _members()
    rk = _rakes(ms)
    Fs = [friction.ensemble_friction(m, seed=40 + k) for k, m in enumerate(ms)]
    eps, leaf, L = 1e-6, 8, 2
    hE, starts = hbi.hbi_build_ensemble([m.verts for m in ms], MU, NU, oracle.OP_RAKE_SHEAR, eps, leaf, L, "fp32",
                                        rakes=rk)
    cat = lambda f: np.concatenate([getattr(F, f) for F in Fs])
    F0 = Fs[0]
    fr = hbi.friction(dev(cat("a")), dev(cat("b")), dev(cat("dc")), dev(cat("rake")), F0.f0, F0.V0, F0.Vpl,
                      F0.mu, F0.cs)
    states = []
    for F in Fs:
        phi, tau = oracle.steady_state(F.V_init, F.a, F.b, F.sigma0, F.f0, F.V0)
        states.append(np.concatenate([phi, tau, F.sigma0, np.zeros(len(phi))]))
    # ensemble state: each component block concatenated over the members
    comp = lambda s, c: s[c * (len(s) // 4):(c + 1) * (len(s) // 4)]
    sE = dev(np.concatenate([np.concatenate([comp(s, c) for s in states]) for c in range(4)]))
    nm = len(ms)
    dt0 = np.array([1e4 * (k + 1) for k in range(nm)])
    tE, dtE = dev(np.zeros(nm)), dev(dt0)
    n_steps = 40
    st, done, recE = hbi.hbi_step_ensemble(hE, fr, sE, tE, dtE, 1e-4, n_steps)
    assert st == 0 and list(done) == [n_steps] * nm
    sE = host(sE)
    NT = int(starts[-1])
    for k, (m, F) in enumerate(zip(ms, Fs)):
        h1 = hbi.hbi_build(m.verts, MU, NU, oracle.OP_RAKE_SHEAR, eps, leaf, L, "fp32", rake=rk[k])
        f1 = hbi.friction(dev(F.a), dev(F.b), dev(F.dc), dev(F.rake), F.f0, F.V0, F.Vpl, F.mu, F.cs)
        s1, t1, dt1 = dev(states[k]), dev([0.0]), dev([dt0[k]])
        st1, done1, rec1 = hbi.hbi_step(h1, f1, s1, t1, dt1, 1e-4, n_steps)
        assert st1 == 0 and done1 == n_steps
        a, b = int(starts[k]), int(starts[k + 1])
        got = np.concatenate([sE[c * NT + a:c * NT + b] for c in range(4)])
        assert np.array_equal(got, host(s1)), f"member {k}: state differs from its single run"
        assert host(tE)[k] == host(t1)[0] and host(dtE)[k] == host(dt1)[0]
        assert np.array_equal(recE[k], rec1)


def test_plain_step_rejects_an_ensemble_handle():
    ms = _members()[:2]
    hE, starts = hbi.hbi_build_ensemble([m.verts for m in ms], MU, NU, oracle.OP_RAKE_SHEAR, 1e-4, 8, 1, "fp32",
                                        rakes=_rakes(ms))
    n = int(starts[-1])
    F = friction.ensemble_friction(ms[0], seed=1)
    fr = hbi.friction(dev(np.full(n, F.a[0])), dev(np.full(n, F.b[0])), dev(np.full(n, F.dc[0])),
                      dev(np.full(n, np.pi / 2)), F.f0, F.V0, F.Vpl, F.mu, F.cs)
    s = dev(np.zeros(4 * n))
    st, done, _ = hbi.hbi_step(hE, fr, s, dev([0.0]), dev([1.0]), 1e-4, 1)
    assert st == -1 and done == 0


def test_ensemble_members_follow_the_oracle():
    """Each member's 40 ensemble steps against the oracle's own run of that member (its own
    tree, ACA and Cash-Karp loop on the host).  The ensemble is built with FP64 storage at
    eps_ACA = 1e-10, so its operators and the oracle's differ from the dense operator, and
    from each other, by about 1e-10.  The oracle adds the loading separately from H V, which
    near steady sliding cancels by up to 1e3 (|H V| / |H (V - V_pl)|), so the two stress rates
    differ by up to about 1e-7 relative; the error estimate, and with it the step size
    (proportional to err^-0.2), inherits that.  So the members must take the oracle's
    accept/reject decisions exactly, and times, step sizes and states agree to 1e-6."""
    ms = _members()
    rk = _rakes(ms)
    Fs = [friction.ensemble_friction(m, seed=40 + k) for k, m in enumerate(ms)]
    eps, leaf, L = 1e-10, 8, 2
    hE, starts = hbi.hbi_build_ensemble([m.verts for m in ms], MU, NU, oracle.OP_RAKE_SHEAR, eps, leaf, L, "fp64",
                                        rakes=rk)
    cat = lambda f: np.concatenate([getattr(F, f) for F in Fs])
    F0 = Fs[0]
    fr = hbi.friction(dev(cat("a")), dev(cat("b")), dev(cat("dc")), dev(cat("rake")), F0.f0, F0.V0, F0.Vpl,
                      F0.mu, F0.cs)
    y0s = []
    for F in Fs:
        phi, tau = oracle.steady_state(F.V_init, F.a, F.b, F.sigma0, F.f0, F.V0)
        y0s.append(np.concatenate([phi, tau, F.sigma0]))
    comp = lambda y, c: y[c * (len(y) // 3):(c + 1) * (len(y) // 3)]
    NT = int(starts[-1])
    sE = dev(np.concatenate([np.concatenate([comp(y, c) for y in y0s]) for c in range(3)] + [np.zeros(NT)]))
    nm = len(ms)
    dt0 = np.array([1e4 * (k + 1) for k in range(nm)])
    tE, dtE = dev(np.zeros(nm)), dev(dt0)
    n_steps = 40
    st, done, recE = hbi.hbi_step_ensemble(hE, fr, sE, tE, dtE, 1e-4, n_steps)
    assert st == 0 and list(done) == [n_steps] * nm
    sE = host(sE)
    for k, (m, F) in enumerate(zip(ms, Fs)):
        H = oracle.HMatrix(m, oracle.OP_RAKE_SHEAR, eps, leaf, L, MU, NU, rake=rk[k])
        td, sd = H.loading(F.rake, F.Vpl)
        y_ref, D_ref, t_ref, dt_ref, rec_ref = H.run(F, y0s[k], np.zeros(m.n_elem), 0.0, dt0[k], 1e-4, n_steps,
                                                     td, sd)
        a, b = int(starts[k]), int(starts[k + 1])
        assert np.array_equal(recE[k][:, 3], rec_ref[:, 3]), f"member {k}: rejections differ"
        assert np.allclose(recE[k][:, 0], rec_ref[:, 0], rtol=1e-6, atol=0), k
        assert np.allclose(recE[k][:, 1], rec_ref[:, 1], rtol=1e-6, atol=0), k
        assert np.allclose(recE[k][:, 2], rec_ref[:, 2], rtol=1e-6, atol=0), k
        got = np.concatenate([sE[c * NT + a:c * NT + b] for c in range(3)])
        assert np.allclose(got, y_ref, rtol=1e-6, atol=0), k
        assert np.allclose(sE[3 * NT + a:3 * NT + b], D_ref, rtol=1e-5, atol=1e-20), k
        assert host(tE)[k] == pytest.approx(t_ref, rel=1e-6)
