"""The multi-RHS product on the tensor cores (hbi_matvec_multi): Y = H X for k slip-rate
vectors at once, against the single-vector product on the same handle and against the
oracle's dense operator (Eqs. 5-6).

Tolerances.  The panels hold exactly the entries of the single-vector storage (FP16 with
per-column power-of-two scales; the FP32 near field of HBI_MIXED as an FP16 pair with 22
significant bits), and each input is split into FP16 hi + lo parts (22 bits) after a power-of-
two scaling per right-hand side, so the two products differ by the input split (2^-22
relative per input), the dropped lo x lo term (2^-22) and FP32 summation order: 2e-5 relative
in L2 per right-hand side covers this with margin (measured about 1e-6).  Against the dense
operator the error is the storage's own (FP16 far field: 2e-3, as for hbi_matvec)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
import paper_2110_12165_gb300 as hbi
from synthetic import meshes, rng
from gpu_util import dev, host, rel_l2

pytestmark = pytest.mark.gpu
MU, NU = 32e9, 0.25


def _single(h, X, k):
    n = h.n
    out = []
    y = torch.zeros(h.nout * n, dtype=torch.float64, device="cuda")
    for r in range(k):
        hbi.hbi_matvec(h, dev(X[r]), y)
        out.append(host(y).copy())
    return np.array(out)


def _multi(h, X, k):
    Y = torch.full((k * h.nout * h.n,), float("nan"), dtype=torch.float64, device="cuda")
    hbi.hbi_matvec_multi(h, k, dev(X.reshape(-1)), Y)
    return host(Y).reshape(k, -1)


@pytest.mark.parametrize("storage", ["mixed", "fp16"])
@pytest.mark.parametrize("k", [1, 7, 16, 33, 64])
def test_multi_matches_single_and_dense(storage, k):
    m = meshes.scaled_thrust_mesh(30, 20, seed=2)            # N = 1200, 2 -> 3 components
    n = m.n_elem
    h = hbi.hbi_build(m.verts, MU, NU, oracle.OP_VEC_FULL, 1e-5, 16, 2, storage, recompress_eps=1e-5,
                      multi_rhs=True)
    X = rng.normal(300 + k, k * 2 * n).reshape(k, 2 * n)
    Ym = _multi(h, X, k)
    Ys = _single(h, X, k)
    assert np.isfinite(Ym).all()
    for r in range(k):
        assert rel_l2(Ym[r], Ys[r]) < 2e-5, (r, rel_l2(Ym[r], Ys[r]))
    # against the oracle's dense operator on a few of the right-hand sides
    for r in sorted({0, k // 2, k - 1}):
        yd = oracle.dense_matvec(m, oracle.OP_VEC_FULL, X[r], MU, NU)
        assert rel_l2(Ym[r], yd) < 2e-3
    # the same call again gives the same bits (no atomics in the sums)
    assert np.array_equal(_multi(h, X, k), Ym)


def test_multi_scales_each_right_hand_side_on_its_own():
    """Right-hand sides 12 orders of magnitude apart (slip rates of 1e-9 m/s next to 1e3):
    each keeps its own relative accuracy (one power-of-two scale per right-hand side)."""
    m = meshes.scaled_thrust_mesh(24, 12, seed=5)
    n = m.n_elem
    h = hbi.hbi_build(m.verts, MU, NU, oracle.OP_VEC_FULL, 1e-5, 16, 1, "mixed", multi_rhs=True)
    k = 16
    X = rng.normal(41, k * 2 * n).reshape(k, 2 * n) * (10.0 ** np.linspace(-9, 3, k))[:, None]
    X[5] = 0.0                                                # an all-zero right-hand side
    Ym = _multi(h, X, k)
    Ys = _single(h, X, k)
    assert np.all(Ym[5] == 0.0)
    for r in range(k):
        if r != 5:
            assert rel_l2(Ym[r], Ys[r]) < 2e-5, r


def test_multi_spans_many_tiles_and_two_row_tiles_per_unit():
    """Leaf 64 with three outputs per element: leaf row units of up to 192 rows (two 128-row
    tiles sharing one gather list), column groups with more than 128 V^T rows, groups wider
    than 2048 columns (cut into K slices whose partial sums are reduced), many chunks; the
    single-vector product of the same handle is the reference."""
    m = meshes.scaled_thrust_mesh(100, 50, seed=3)           # N = 10,000
    n = m.n_elem
    h = hbi.hbi_build(m.verts, MU, NU, oracle.OP_VEC_FULL, 1e-4, 64, 2, "mixed", recompress_eps=1e-4,
                      multi_rhs=True)
    st = hbi.hbi_multi_stats(h)
    assert st["n_tasks_uy"] > h.stats()["n_leaves"]              # some units take two row tiles
    assert st["n_split_tiles"] > 0                                 # V^T groups cut along K, then reduced
    k = 20
    X = rng.normal(77, k * 2 * n).reshape(k, 2 * n)
    Ym = _multi(h, X, k)
    Ys = _single(h, X, k)
    for r in range(k):
        assert rel_l2(Ym[r], Ys[r]) < 2e-5, r
    rows = np.array([0, 17, n // 3, n - 1], dtype=np.int32)
    yr = oracle.dense_rows(m, oracle.OP_VEC_FULL, rows, X[3], MU, NU)
    got = np.stack([Ym[3][c * n + rows] for c in range(3)], 1)
    assert np.linalg.norm(got - yr) / np.linalg.norm(yr) < 2e-3


def test_multi_on_an_ensemble_handle():
    ms = [meshes.dipping_rect(16, 8, 250.0, 30.0), meshes.dipping_rect(12, 6, 250.0, 90.0)]
    rk = [np.full(mm.n_elem, np.pi / 2) for mm in ms]
    hE, starts = hbi.hbi_build_ensemble([mm.verts for mm in ms], MU, NU, oracle.OP_RAKE_SHEAR, 1e-6, 8, 2, "mixed",
                                        rakes=rk, multi_rhs=True)
    k = 9
    NT = int(starts[-1])
    X = rng.normal(90, k * NT).reshape(k, NT)
    Ym = _multi(hE, X, k)
    Ys = _single(hE, X, k)
    for r in range(k):
        assert rel_l2(Ym[r], Ys[r]) < 2e-5


def test_multi_rejects_bad_arguments():
    m = meshes.scaled_thrust_mesh(8, 4, seed=2)
    n = m.n_elem
    h_plain = hbi.hbi_build(m.verts, MU, NU, oracle.OP_VEC_FULL, 1e-5, 8, 1, "mixed")
    X = torch.zeros(2 * n * 64 + 2 * n, dtype=torch.float64, device="cuda")
    Y = torch.zeros(3 * n * 65, dtype=torch.float64, device="cuda")
    with pytest.raises(hbi.HbiError, match="INVALID_ARG"):
        hbi.hbi_matvec_multi(h_plain, 2, X, Y)                # built without the panels
    h = hbi.hbi_build(m.verts, MU, NU, oracle.OP_VEC_FULL, 1e-5, 8, 1, "mixed", multi_rhs=True)
    for k in (0, 65):
        with pytest.raises(hbi.HbiError, match="INVALID_ARG"):
            hbi.hbi_matvec_multi(h, k, X, Y)
    with pytest.raises(hbi.HbiError, match="INVALID_ARG"):   # the panels are FP16-based
        hbi.hbi_build(m.verts, MU, NU, oracle.OP_VEC_FULL, 1e-5, 8, 1, "fp32", multi_rhs=True)
