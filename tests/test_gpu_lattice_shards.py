"""One rank's share of the paper's distributed lattice H-matrix (Sec. 3.2) built and multiplied
by the library (hbi_build_shard): every rank of a P_r x P_c grid in turn on the one GPU of the
run.  Each shard's partial product is zero outside its process row's lattice rows; the partial
products summed in the paper's order (a reduction along each process row, then the row sums
combined) equal the product of the whole operator; and each shard holds about its share of the
blocks.  The exchange between processes itself is exercised on CPU ranks
(tests/test_lattice_dist.py)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
import paper_2110_12165_gb300 as hbi
from oracle import lattice_dist
from synthetic import meshes, rng
from gpu_util import dev, host, rel_l2

pytestmark = pytest.mark.gpu
MU, NU = 32e9, 0.25


def _product(h, x):
    y = torch.zeros(h.nout * h.n, dtype=torch.float64, device="cuda")
    hbi.hbi_matvec(h, dev(x), y)
    return host(y)


@pytest.mark.parametrize("storage,tol", [("fp64", 1e-13), ("mixed", 1e-6)])
@pytest.mark.parametrize("pr,pc", [(2, 2), (2, 1), (1, 3), (3, 2)])
def test_shards_sum_to_the_whole_product(storage, tol, pr, pc):
    m = meshes.scaled_thrust_mesh(40, 20, seed=2)             # N = 1600, 2 -> 3 components
    n = m.n_elem
    args = (m.verts, MU, NU, oracle.OP_VEC_FULL, 1e-6, 16, 2, storage)
    h = hbi.hbi_build(*args, recompress_eps=1e-6 if storage == "mixed" else 0.0)
    x = rng.normal(61, 2 * n)
    y = _product(h, x)
    # lattice rows of each process row, in the caller's order (the rows' DOFs are permuted)
    H = oracle.HMatrix(m, oracle.OP_VEC_FULL, 1e-6, 16, 2, MU, NU)   # the same tree and lattice
    ex = H.export()
    bounds = lattice_dist.lattice_index(H, ex)
    perm = ex["perm"]
    owned_rows = [np.zeros(3 * n, dtype=bool) for _ in range(pr)]
    for I in range(len(bounds) - 1):
        for p in range(bounds[I], bounds[I + 1]):
            for c in range(3):
                owned_rows[I % pr][c * n + perm[p]] = True
    row_sums = []
    nblocks = 0
    for i in range(pr):
        acc = np.zeros(3 * n)
        for j in range(pc):
            hs = hbi.hbi_build_shard(*args, pr, pc, i * pc + j, recompress_eps=1e-6 if storage == "mixed" else 0.0)
            nblocks += hs.stats()["n_blocks"]
            yp = _product(hs, x)
            assert np.all(yp[~owned_rows[i]] == 0.0), (i, j)
            acc += yp                                             # reduction along process row i
        row_sums.append(acc)
    y_dist = np.sum(row_sums, axis=0)                             # the rows' sums combined
    assert nblocks == h.stats()["n_blocks"]                       # every block in exactly one shard
    assert rel_l2(y_dist, y) < tol


def test_shard_share_and_rejections():
    m = meshes.scaled_thrust_mesh(40, 20, seed=2)
    args = (m.verts, MU, NU, oracle.OP_VEC_FULL, 1e-5, 16, 2, "fp32")
    whole = hbi.hbi_build(*args).stats()
    shares = [hbi.hbi_build_shard(*args, 2, 2, r).stats() for r in range(4)]
    tot = sum(s["bytes_factors"] for s in shares)
    assert tot == pytest.approx(whole["bytes_factors"], rel=0.1)       # row padding per shard
    assert max(s["bytes_factors"] for s in shares) < 0.5 * whole["bytes_factors"]
    with pytest.raises(hbi.HbiError, match="INVALID_ARG"):
        hbi.hbi_build_shard(*args, 2, 2, 4)
    hs = hbi.hbi_build_shard(*args, 2, 1, 0)
    F = __import__("synthetic.friction", fromlist=["x"]).thrust_friction(m, seed=2)
    fr = hbi.friction(dev(F.a), dev(F.b), dev(F.dc), dev(F.rake), F.f0, F.V0, F.Vpl, F.mu, F.cs)
    st, done, _ = hbi.hbi_step(hs, fr, dev(np.zeros(4 * m.n_elem)), dev([0.0]), dev([1.0]), 1e-4, 1)
    assert st == -1 and done == 0
