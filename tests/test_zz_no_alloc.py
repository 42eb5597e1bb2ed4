"""hbi_matvec_noalloc: the HMVM for callers that cannot allocate device memory at the time
of the call (for example a program whose own pool allocator owns the device memory, or a
path where an allocation and its implicit synchronisation are not allowed).  Its scratch
lives in a static device array of the library.  Checked through the C ABI against
hbi_matvec on two calls in a row, with handles interleaved so that the shared array holds
another operator's data in between, and for the size limit.  Collected last on purpose."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
import paper_2110_12165_gb300 as hbi
from synthetic import meshes, rng
from gpu_util import dev, host, import_oracle, rel_l2

pytestmark = pytest.mark.gpu
MU, NU = 32e9, 0.25


def _y(fn, h, x):
    xd = dev(x)
    yd = torch.full((h.nout * h.n,), float("nan"), dtype=torch.float64, device="cuda")
    fn(h, xd, yd)
    torch.cuda.synchronize()
    return host(yd)


@pytest.mark.parametrize("storage,tol", [("fp64", 1e-12), ("fp32", 2e-6), ("fp16", 2e-3), ("mixed", 2e-3),
                                         ("adaptive", 2e-3)])
def test_noalloc_matches_matvec_on_two_calls(storage, tol):
    """MIXED is the storage of the timed path; ADAPTIVE's product gathers paired hi + lo entries
    of t = V^T x from the shared array, so a stale entry left by the other operator's call
    would show there first."""
    m1 = meshes.scaled_thrust_mesh(30, 20, seed=2)                  # N = 1200, 2 -> 3 components
    h1 = hbi.hbi_build(m1.verts, MU, NU, oracle.OP_VEC_FULL, 1e-5, 16, 2, storage,
                       recompress_eps=1e-5 if storage in ("mixed", "adaptive") else 0.0)
    m2 = meshes.planar_vertical_rect(33, 17, 250.0)                 # another operator, 1 -> 1
    H2 = oracle.HMatrix(m2, oracle.OP_RAKE_SHEAR, 1e-6, 16, 0, MU, NU)
    h2 = import_oracle(H2, storage)
    x1 = rng.normal(81, 2 * m1.n_elem)
    x2 = rng.normal(82, m2.n_elem)
    ref1 = _y(hbi.hbi_matvec, h1, x1)
    ref2 = _y(hbi.hbi_matvec, h2, x2)
    a1 = _y(hbi.hbi_matvec_noalloc, h1, x1)
    b2 = _y(hbi.hbi_matvec_noalloc, h2, x2)       # the shared array now holds h2's data
    a1_again = _y(hbi.hbi_matvec_noalloc, h1, x1)
    b2_again = _y(hbi.hbi_matvec_noalloc, h2, x2)
    for got, ref in ((a1, ref1), (a1_again, ref1), (b2, ref2), (b2_again, ref2)):
        assert np.isfinite(got).all()
        assert rel_l2(got, ref) < tol
    # same kernels, same task order: the two calls agree bit for bit
    assert np.array_equal(a1, a1_again) and np.array_equal(b2, b2_again)
    # and the oracle agrees within the storage tolerance
    assert rel_l2(b2, H2.matvec(x2)) < tol


def test_noalloc_rejects_operators_beyond_the_static_limit():
    m = meshes.scaled_thrust_mesh(400, 200, seed=3)   # N = 160,000 in FP64: > 16 MiB of scratch
    H_dummy_x = rng.normal(83, 2 * m.n_elem)
    h = hbi.hbi_build(m.verts, MU, NU, oracle.OP_VEC_FULL, 1e-4, 64, 2, "fp64")
    y = torch.zeros(3 * m.n_elem, dtype=torch.float64, device="cuda")
    with pytest.raises(hbi.HbiError, match="INVALID_ARG"):
        hbi.hbi_matvec_noalloc(h, dev(H_dummy_x), y)


def test_noalloc_takes_the_full_size_mixed_operator():
    """The 160,000-element thrust fault with the mixed storage of the timed path (leaf 64,
    lattice depth 2, recompression 1e-4) fits the static array: (2N + T + 16) + 3N FP32 words,
    T the sum of the ranks, about 8 MB.  Two calls agree with hbi_matvec and with each other."""
    m = meshes.scaled_thrust_mesh(400, 200, seed=3)
    h = hbi.hbi_build(m.verts, MU, NU, oracle.OP_VEC_FULL, 1e-4, 64, 2, "mixed", recompress_eps=1e-4)
    st = h.stats()
    need = 4 * (2 * m.n_elem + st["mean_rank"] * st["n_lowrank"] + 16 + 3 * m.n_elem)
    assert need < 16 << 20
    x = rng.normal(84, 2 * m.n_elem)
    ref = _y(hbi.hbi_matvec, h, x)
    a = _y(hbi.hbi_matvec_noalloc, h, x)
    b = _y(hbi.hbi_matvec_noalloc, h, x)
    assert np.isfinite(a).all() and rel_l2(a, ref) < 1e-6
    assert np.array_equal(a, b)
