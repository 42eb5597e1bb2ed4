"""The oracle's bounded-sample build (HMatrix(..., sample_lattice_row=a)): the blocks whose
rows lie in lattice row a are built exactly as in the whole build, so the sampled product is
the whole product's rows of that lattice row, bit for bit, and zero elsewhere; the samples of
all lattice rows add up to the whole product.  The reference arm of bench.py times the oracle on
such a sample of meshes it cannot build whole within a bench run."""
import numpy as np

import oracle
from oracle import lattice_dist
from synthetic import meshes, rng

MU, NU = 32e9, 0.25


def test_sampled_lattice_rows_are_the_whole_products_rows():
    m = meshes.scaled_thrust_mesh(24, 12, seed=2)                # N = 576, 2 -> 3 operator
    H = oracle.HMatrix(m, oracle.OP_VEC_FULL, 1e-5, 16, 2, MU, NU)
    xp = rng.normal(7, 2 * m.n_elem)
    y = H.matvec_perm(xp)
    bounds = lattice_dist.lattice_index(H)
    assert len(bounds) == 5                                     # depth 2: four lattice clusters
    total = np.zeros_like(y)
    for a in range(len(bounds) - 1):
        Hs = oracle.HMatrix(m, oracle.OP_VEC_FULL, 1e-5, 16, 2, MU, NU, sample_lattice_row=a)
        assert Hs.n_blocks == H.n_blocks and Hs.n_data < H.n_data
        bs, bf = Hs.export()["blocks"], H.export()["blocks"]
        inside = (bs[:, 0] >= 3 * bounds[a]) & (bs[:, 0] < 3 * bounds[a + 1])
        assert np.array_equal(bs[inside, :6], bf[inside, :6])   # built as in the whole build
        assert np.all(bs[~inside, 5] == -1)                     # the others: not built
        assert np.array_equal(bs[:, :4], bf[:, :4])             # one partition
        ys = Hs.matvec_perm(xp)
        lo, hi = 3 * bounds[a], 3 * bounds[a + 1]
        assert np.array_equal(ys[lo:hi], y[lo:hi])
        assert not ys[:lo].any() and not ys[hi:].any()
        total += ys
    assert np.allclose(total, y, rtol=0, atol=1e-12 * np.abs(y).max())
    # the setting does not leak into later builds
    H2 = oracle.HMatrix(m, oracle.OP_VEC_FULL, 1e-5, 16, 2, MU, NU)
    assert H2.n_data == H.n_data and np.array_equal(H2.matvec_perm(xp), y)
