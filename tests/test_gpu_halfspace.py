"""GPU parity of the half-space operator (Sec. 2.1: elements in an elastic half space with a
traction-free surface z = 0) against the FP64 oracle, through the C ABI.

The CUDA entries add to the closed-form full-space entries Mindlin's point-force correction,
differentiated exactly with jets and integrated with Radon's seven-point rule on a
subdivision of the source (sub-triangles at most 1/4 of their vertical distance to the
receiver's image); the oracle differentiates by the complex step and finite differences and
integrates with subdivided Gauss-Legendre product rules.  The degree-5 rule at that ratio
leaves a relative error of about 3e-7 of a pair's largest entry (it falls as the sixth power
of the ratio), so entries are compared to 2e-6 of each pair's largest entry.  The H-matrix
product is compared on sampled rows to 10 eps_ACA, as the full-space build."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
import paper_2110_12165_gb300 as hbi
from synthetic import meshes, rng
from gpu_util import dev, host, rel_l2

pytestmark = pytest.mark.gpu
MU, NU = 32e9, 0.25


def _gpu_matvec(h, x):
    y = torch.zeros(h.nout * h.n, dtype=torch.float64, device="cuda")
    hbi.hbi_matvec(h, dev(x), y)
    torch.cuda.synchronize()
    return host(y)


def _dense_gpu(m, op, half_space):
    n = m.n_elem
    h = hbi.hbi_build(m.verts, MU, NU, op, 1e-8, n, 0, "fp64", half_space=half_space)
    assert h.stats()["n_lowrank"] == 0
    ni, no = oracle.OP_NIN[op], oracle.OP_NOUT[op]
    E = np.zeros((no * n, ni * n))
    for c in range(ni * n):
        e = np.zeros(ni * n); e[c] = 1.0
        E[:, c] = _gpu_matvec(h, e)
    return E.reshape(no, n, ni, n).transpose(1, 3, 0, 2)     # [i, j, c_out, c_in]


MESHES = {
    # top edge 50 m below the surface: the correction is as large as the entries themselves
    "shallow-rect-40deg": lambda: meshes.dipping_rect(6, 4, 250.0, 40.0, origin=(0.0, 0.0, -50.0)),
    "thrust-tri-top-1km": lambda: meshes.scaled_thrust_mesh(5, 3, seed=8),
}


@pytest.mark.parametrize("kind", list(MESHES))
def test_half_space_entries_equal_oracle_entries(kind):
    m = MESHES[kind]()
    n = m.n_elem
    op = oracle.OP_VEC_FULL
    E = _dense_gpu(m, op, True)
    i, j = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    ref = oracle.pair_entries(m, op, i.ravel(), j.ravel(), MU, NU, half_space=True).reshape(n, n, 3, 2)
    full = oracle.pair_entries(m, op, i.ravel(), j.ravel(), MU, NU).reshape(n, n, 3, 2)
    scale = np.abs(ref).max(axis=(2, 3), keepdims=True)
    assert (np.abs(E - ref) / scale).max() < 2e-6
    # the flag reaches the kernels: the correction is far above the tolerance
    assert (np.abs(full - ref) / scale).max() > 1e-2


def test_half_space_rake_operator_entries():
    m = MESHES["shallow-rect-40deg"]()
    n = m.n_elem
    op = oracle.OP_RAKE_SHEAR_NORMAL
    rake = rng.uniform(71, n) * np.pi
    h = hbi.hbi_build(m.verts, MU, NU, op, 1e-8, n, 0, "fp64", rake=rake, half_space=True)
    E = np.zeros((2 * n, n))
    for c in range(n):
        e = np.zeros(n); e[c] = 1.0
        E[:, c] = _gpu_matvec(h, e)
    i, j = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    ref = oracle.pair_entries(m, op, i.ravel(), j.ravel(), MU, NU, rake=rake, half_space=True).reshape(n, n, 2, 1)
    ref_full = ref.transpose(2, 0, 3, 1).reshape(2 * n, n)
    assert np.abs(E - ref_full).max() < 2e-6 * np.abs(ref_full).max()


@pytest.mark.parametrize("storage,tol", [("fp64", 1e-4), ("mixed", 2e-3)])
def test_half_space_h_matrix_product_on_sampled_rows(storage, tol):
    """GPU entries + GPU ACA + packing of the half-space operator (thrust fault, 576
    triangles, top 1 km deep) against rows of the oracle's dense half-space operator."""
    m = meshes.scaled_thrust_mesh(24, 12, seed=3)
    n = m.n_elem
    op = oracle.OP_VEC_FULL
    eps = 1e-5
    h = hbi.hbi_build(m.verts, MU, NU, op, eps, 16, 1, storage, half_space=True)
    assert h.stats()["n_lowrank"] > 0
    x = rng.normal(72, 2 * n)
    y = _gpu_matvec(h, x)
    rows = np.arange(0, n, 48)
    ref = oracle.dense_rows(m, op, rows, x, MU, NU, half_space=True)
    got = np.stack([y[c * n + rows] for c in range(3)], 1)
    assert rel_l2(got, ref) < tol, rel_l2(got, ref)
    full = oracle.dense_rows(m, op, rows, x, MU, NU)
    assert rel_l2(full, ref) > 10 * tol


def test_half_space_ensemble_members_equal_single_builds():
    """hbi_build_ensemble passes the half-space choice to every member: each member's product
    equals its single half-space build bit for bit (member DOF counts are multiples of 4, as
    in the full-space ensemble test), and a member matches the oracle's dense rows."""
    ms = [meshes.dipping_rect(16, 8, 250.0, 30.0, origin=(0.0, 0.0, -200.0)),
          meshes.dipping_rect(12, 6, 250.0, 90.0, origin=(0.0, 0.0, -100.0)),
          meshes.dipping_rect(8, 4, 250.0, 60.0, origin=(0.0, 0.0, -400.0))]
    rk = [np.full(m.n_elem, np.pi / 2) for m in ms]
    op, eps, leaf, L = oracle.OP_RAKE_SHEAR, 1e-6, 8, 1
    hE, starts = hbi.hbi_build_ensemble([m.verts for m in ms], MU, NU, op, eps, leaf, L, "fp64", rakes=rk,
                                        half_space=True)
    x = rng.normal(73, int(starts[-1]))
    yE = _gpu_matvec(hE, x)
    for k, m in enumerate(ms):
        a, b = int(starts[k]), int(starts[k + 1])
        h1 = hbi.hbi_build(m.verts, MU, NU, op, eps, leaf, L, "fp64", rake=rk[k], half_space=True)
        assert np.array_equal(yE[a:b], _gpu_matvec(h1, x[a:b])), f"member {k} differs from its single build"
    m, a, b = ms[1], int(starts[1]), int(starts[2])
    rows = np.arange(0, m.n_elem, 9)
    ref = oracle.dense_rows(m, op, rows, x[a:b], MU, NU, rake=rk[1], half_space=True)[:, 0]
    assert rel_l2(yE[a:b][rows], ref) < 10 * eps


def test_half_space_transpose_is_the_adjoint():
    """The adjoint's H^T on a half-space handle: <H x, v> = <x, H^T v> (FP64 storage) and
    <H_dense x, v> from the oracle's dense half-space operator."""
    m = meshes.dipping_rect(8, 6, 250.0, 30.0, origin=(0.0, 0.0, -200.0))
    n = m.n_elem
    op = oracle.OP_VEC_FULL
    h = hbi.hbi_build(m.verts, MU, NU, op, 1e-6, 8, 1, "fp64", transpose=True, half_space=True)
    x, v = rng.normal(74, 2 * n), rng.normal(75, 3 * n)
    Hx = _gpu_matvec(h, x)
    Htv = torch.zeros(2 * n, dtype=torch.float64, device="cuda")
    hbi.hbi_matvec_transpose(h, dev(v), Htv)
    lhs, rhs = float(np.dot(Hx, v)), float(np.dot(x, host(Htv)))
    scale = np.linalg.norm(Hx) * np.linalg.norm(v)
    assert abs(lhs - rhs) <= 1e-12 * scale
    Hd = oracle.dense_matvec(m, op, x, MU, NU, half_space=True)
    assert abs(float(np.dot(Hd, v)) - rhs) <= 1e-5 * np.linalg.norm(Hd) * np.linalg.norm(v)
