"""GPU parity of the HMVM and the GPU build against the FP64 oracle (through the C ABI).

Tolerances (relative L2 over the whole output):
  FP64 storage on the oracle's own factors: 1e-12 (same sums, another order).
  FP32 storage: 2e-6 (unit roundoff 6e-8 in every stored entry and in FP32 accumulation,
    amplified by the cancellation of the near-field sums).
  FP16 storage: 2e-3, BF16: 2e-2 (unit roundoffs 4.9e-4 and 3.9e-3 per stored entry; one
    power-of-two scale per column keeps every entry in the normal range).
  MIXED (FP32 dense near field, FP16 low-rank far field): 2e-3, and never worse than FP16.
  GPU-built factors vs the dense operator: 10 x eps_ACA (the ACA stopping rule bounds each
    block's relative Frobenius error by about eps; pivots may differ from the oracle's).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
import paper_2110_12165_gb300 as hbi
from synthetic import meshes, rng
from gpu_util import dev, host, import_oracle, rel_l2

pytestmark = pytest.mark.gpu
MU, NU = 32e9, 0.25

CASES = {
    # name: (mesh factory, op, eps, leaf, lattice depth)
    "planar-rect-N2048-scalar": (lambda: meshes.config1_mesh(), 0, 1e-6, 32, 0),
    "thrust-tri-N1200-full-L2": (lambda: meshes.scaled_thrust_mesh(30, 20, seed=2), 3, 1e-4, 16, 2),
    "thrust-tri-N594-rake-normal": (lambda: meshes.scaled_thrust_mesh(33, 9, seed=4), 1, 1e-5, 24, 1),
    "planar-rect-N150-vecshear-ragged": (lambda: meshes.planar_vertical_rect(15, 10, 250.0), 2, 1e-6, 7, 0),
}


@pytest.fixture(scope="module", params=list(CASES))
def case(request):
    mk, op, eps, leaf, L = CASES[request.param]
    m = mk()
    rake = rng.uniform(61, m.n_elem) * np.pi
    H = oracle.HMatrix(m, op, eps, leaf, L, MU, NU, rake=rake)
    x = rng.normal(62, H.nin * m.n_elem)
    return request.param, m, H, x, rake


def _gpu_matvec(h, x):
    xd = dev(x)
    yd = torch.zeros(h.nout * h.n, dtype=torch.float64, device="cuda")
    hbi.hbi_matvec(h, xd, yd)
    torch.cuda.synchronize()
    return host(yd)


@pytest.mark.parametrize("storage,tol", [("fp64", 1e-12), ("fp32", 2e-6), ("fp16", 2e-3), ("bf16", 2e-2),
                                         ("mixed", 2e-3), ("adaptive", 2e-3)])
def test_hmvm_on_oracle_factors(case, storage, tol):
    name, m, H, x, rake = case
    h = import_oracle(H, storage)
    y_ref = H.matvec(x)
    y = _gpu_matvec(h, x)
    assert rel_l2(y, y_ref) < tol, (name, storage, rel_l2(y, y_ref))
    st = h.stats()
    assert st["n_blocks"] == H.n_blocks and st["n_lowrank"] == H.n_lowrank


def test_mixed_storage_is_more_accurate_than_fp16(case):
    name, m, H, x, rake = case
    y_ref = H.matvec(x)
    e16 = rel_l2(_gpu_matvec(import_oracle(H, "fp16"), x), y_ref)
    emx = rel_l2(_gpu_matvec(import_oracle(H, "mixed"), x), y_ref)
    assert emx <= e16


def test_adaptive_storage_is_not_less_accurate_than_mixed(case):
    """HBI_ADAPTIVE keeps each low-rank block's leading pair in FP32 and is otherwise HBI_MIXED,
    so its rounding error is at most the mixed one (within 10 %: the remaining FP16 errors of
    the two products are the same numbers, summed in another order)."""
    name, m, H, x, rake = case
    y_ref = H.matvec(x)
    emx = rel_l2(_gpu_matvec(import_oracle(H, "mixed"), x), y_ref)
    ead = rel_l2(_gpu_matvec(import_oracle(H, "adaptive"), x), y_ref)
    assert ead <= 1.1 * emx, (name, ead, emx)


def test_hmvm_deterministic_and_linear(case):
    name, m, H, x, rake = case
    h = import_oracle(H, "fp32")
    y1 = _gpu_matvec(h, x)
    y2 = _gpu_matvec(h, x)
    assert np.array_equal(y1, y2)                 # fixed-order sums, no atomics in the data path
    y3 = _gpu_matvec(h, 2.0 * x)
    assert np.array_equal(y3, 2.0 * y1)           # exact scaling by a power of two
    yz = _gpu_matvec(h, np.zeros_like(x))
    assert not yz.any()


def test_gpu_build_matches_dense_operator():
    """GPU entries + GPU ACA + packing vs the oracle's dense operator (Eqs. 5-6)."""
    for mk, op, eps, leaf, L in ((lambda: meshes.planar_vertical_rect(32, 16, 250.0), 0, 1e-6, 16, 0),
                                 (lambda: meshes.scaled_thrust_mesh(24, 12, seed=22), 3, 1e-5, 16, 1)):
        m = mk()
        x = rng.normal(63, oracle.OP_NIN[op] * m.n_elem)
        yd = oracle.dense_matvec(m, op, x, MU, NU)
        h = hbi.hbi_build(m.verts, MU, NU, op, eps, leaf, L, "fp64")
        st = h.stats()
        assert st["n_lowrank"] > 0
        y = _gpu_matvec(h, x)
        assert rel_l2(y, yd) < 10 * eps, rel_l2(y, yd)


@pytest.mark.parametrize("kind", ["rect", "tri"])
def test_gpu_entries_equal_oracle_entries(kind):
    """All-dense build (one leaf): the closed-form entries of the CUDA kernel vs the oracle's
    quadrature of the same loop integral, entry by entry through unit vectors."""
    m = meshes.planar_vertical_rect(5, 4, 250.0) if kind == "rect" else meshes.scaled_thrust_mesh(5, 3, seed=8)
    n = m.n_elem
    op = oracle.OP_VEC_FULL
    h = hbi.hbi_build(m.verts, MU, NU, op, 1e-8, n, 0, "fp64")
    assert h.stats()["n_lowrank"] == 0
    E = np.zeros((3 * n, 2 * n))
    for c in range(2 * n):
        e = np.zeros(2 * n); e[c] = 1.0
        E[:, c] = _gpu_matvec(h, e)
    i, j = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    ref = oracle.pair_entries(m, op, i.ravel(), j.ravel(), MU, NU).reshape(n, n, 3, 2)
    ref_full = ref.transpose(2, 0, 3, 1).reshape(3 * n, 2 * n)   # rows comp-major, cols comp-major
    scale = np.abs(ref_full).max()
    assert np.abs(E - ref_full).max() < 1e-9 * scale


@pytest.mark.parametrize("storage", ["fp64", "fp16"])
def test_recompression_reduces_ranks_within_tolerance(storage):
    """SVD recompression of the ACA factors: fewer stored entries, still within 10 eps of the
    dense operator (FP16: within the storage tolerance)."""
    m = meshes.scaled_thrust_mesh(30, 20, seed=2)
    eps = 1e-5
    x = rng.normal(66, 2 * m.n_elem)
    yd = oracle.dense_matvec(m, oracle.OP_VEC_FULL, x, MU, NU)
    h0 = hbi.hbi_build(m.verts, MU, NU, oracle.OP_VEC_FULL, eps, 16, 1, storage)
    h1 = hbi.hbi_build(m.verts, MU, NU, oracle.OP_VEC_FULL, eps, 16, 1, storage, recompress_eps=eps)
    s0, s1 = h0.stats(), h1.stats()
    assert s1["entries_lowrank"] < 0.95 * s0["entries_lowrank"]
    assert s1["n_lowrank"] == s0["n_lowrank"]
    tol = 10 * eps if storage == "fp64" else 2e-3
    assert rel_l2(_gpu_matvec(h0, x), yd) < tol
    assert rel_l2(_gpu_matvec(h1, x), yd) < tol


@pytest.mark.parametrize("storage,tol", [("fp64", 1e-12), ("fp16", 2e-3), ("adaptive", 2e-3)])
def test_split_vt_group_with_tiny_tail_chunk(storage, tol):
    """Hand-built operator whose column cluster [4, N) carries two low-rank blocks (16 V^T rows)
    and is split into column chunks ending in a 2-column tail, checked against the dense
    product of the same factors (which the library takes as given)."""
    es = 8 if storage == "fp64" else 2
    cw = (192 << 10) // (16 * es)             # chunk width the packer picks for 16 rows
    M = 4 * cw + 2
    N = M + 4
    verts = meshes.planar_vertical_rect(N, 1, 10.0).verts     # geometry is not used here
    U2, V2 = rng.normal(71, 4 * 8).reshape(4, 8), rng.normal(72, M * 8).reshape(M, 8)
    U3, V3 = rng.normal(73, M * 2).reshape(M, 2), rng.normal(74, 4 * 2).reshape(4, 2)
    U4, V4 = rng.normal(75, M * 8).reshape(M, 8), rng.normal(76, M * 8).reshape(M, 8)
    D1 = rng.normal(77, 16).reshape(4, 4)
    blocks, offs, data = [], [], []
    def add(row0, m, col0, nc, lr, r, arrays):
        blocks.append([row0, m, col0, nc, lr, r]); offs.append(sum(a.size for a in data))
        data.extend(arrays)
    add(0, 4, 0, 4, 0, 0, [D1.ravel()])
    add(0, 4, 4, M, 1, 8, [U2.T.ravel(), V2.T.ravel()])          # column-major U, V
    add(4, M, 0, 4, 1, 2, [U3.T.ravel(), V3.T.ravel()])
    add(4, M, 4, M, 1, 8, [U4.T.ravel(), V4.T.ravel()])
    h = hbi.hbi_build_from_factors(verts, MU, NU, oracle.OP_RAKE_SHEAR, storage, np.arange(N),
                                   np.array(blocks), np.array(offs), np.concatenate(data),
                                   np.array([0, 4, N]))
    x = rng.normal(78, N)
    y_ref = np.zeros(N)
    y_ref[:4] = D1 @ x[:4] + U2 @ (V2.T @ x[4:])
    y_ref[4:] = U3 @ (V3.T @ x[:4]) + U4 @ (V4.T @ x[4:])
    for _ in range(2):                          # twice: stale running sums would show
        assert rel_l2(_gpu_matvec(h, x), y_ref) < tol
        assert rel_l2(_gpu_matvec(h, -3.0 * x), -3.0 * y_ref) < tol


def test_handles_with_different_panel_sizes_coexist():
    """A handle built after another one (with smaller shared-memory panels) must not
    invalidate the first handle's launches."""
    m1 = meshes.scaled_thrust_mesh(30, 20, seed=2)
    h1 = hbi.hbi_build(m1.verts, MU, NU, oracle.OP_VEC_FULL, 1e-5, 16, 2, "fp32")
    x1 = rng.normal(64, 2 * m1.n_elem)
    y1 = _gpu_matvec(h1, x1)
    m2 = meshes.planar_vertical_rect(6, 4, 250.0)
    h2 = hbi.hbi_build(m2.verts, MU, NU, oracle.OP_RAKE_SHEAR, 1e-5, 4, 0, "fp32")
    y2 = _gpu_matvec(h2, rng.normal(65, m2.n_elem))
    assert np.isfinite(y2).all()
    assert np.array_equal(_gpu_matvec(h1, x1), y1)


def test_single_element_and_deep_lattice():
    m = meshes.planar_vertical_rect(1, 1, 250.0)
    h = hbi.hbi_build(m.verts, MU, NU, 0, 1e-4, 32, 4, "fp32")
    y = _gpu_matvec(h, np.array([2.0]))
    a11 = oracle.pair_entries(m, 0, [0], [0], MU, NU)[0, 0, 0]
    assert y[0] == pytest.approx(2.0 * a11, rel=1e-6)
