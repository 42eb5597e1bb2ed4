"""The paper's distributed lattice product (Sec. 3.2) on CPU ranks (gloo): every H-matrix
block has exactly one owner under the 2D-cyclic map, each rank owns the expected share of
lattice blocks, and the product assembled from the ranks' partial products by the row
reductions and the broadcast equals the serial H-matvec.  The library itself runs one GPU
per process; this checks the parallel scheme's logic, not a GPU path."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp

import oracle
from oracle import lattice_dist
from synthetic import meshes, rng

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _case():
    m = meshes.scaled_thrust_mesh(12, 6, seed=2)             # N = 144, nonplanar
    return m, oracle.HMatrix(m, oracle.OP_VEC_FULL, 1e-6, 8, 2, 32e9, 0.25, rake=rng.uniform(3, m.n_elem))


def test_owner_map_is_a_2d_cyclic_partition():
    m, H = _case()
    ex = H.export()
    bounds = lattice_dist.lattice_index(H, ex)
    assert len(bounds) == 5                                  # depth 2: a 4 x 4 lattice
    for pr, pc in ((2, 2), (4, 1), (1, 4), (2, 1)):
        own = lattice_dist.block_owners(H, pr, pc, ex)
        assert own.min() >= 0 and own.max() < pr * pc
        # blocks of one lattice block share its owner; each rank owns 16 / (pr pc) lattice blocks
        lat_of = {}
        for b, (row0, mm, col0, nc, *_r) in enumerate(ex["blocks"]):
            I = int(np.searchsorted(bounds, row0 // H.nout, side="right") - 1)
            J = int(np.searchsorted(bounds, col0 // H.nin, side="right") - 1)
            assert lat_of.setdefault((I, J), own[b]) == own[b]
            assert own[b] == (I % pr) * pc + J % pc
        counts = np.bincount(list(lat_of.values()), minlength=pr * pc)
        assert np.all(counts == 16 // (pr * pc))


def _worker(rank, world, pr, pc, port, out, library_owners=False):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    m, H = _case()
    x = rng.normal(5, 2 * m.n_elem)
    owners = None
    if library_owners:   # the library's owner map (host only) drives the ranks' shares
        import paper_2110_12165_gb300 as hbi
        owners = hbi.hbi_lattice_owners(m.verts, oracle.OP_VEC_FULL, 8, 2, pr, pc)
    # the shares themselves: every block of this rank lies in a lattice block (I, J) with
    # I = rank // pc (mod pr) and J = rank % pc (mod pc), and its partial product touches only
    # the rows of those lattice rows (an owner map that merely tiles the blocks fails here)
    ex = H.export()
    bounds = lattice_dist.lattice_index(H, ex)
    own = lattice_dist.block_owners(H, pr, pc, ex) if owners is None else np.asarray(owners)
    mine = np.nonzero(own == rank)[0]
    row_ok = np.zeros(H.nout * H.n, dtype=bool)
    for I in range(len(bounds) - 1):
        if I % pr == rank // pc:
            row_ok[H.nout * bounds[I]:H.nout * bounds[I + 1]] = True
    for b in mine:
        row0, mm, col0, nc = (int(v) for v in ex["blocks"][b][:4])
        I = int(np.searchsorted(bounds, row0 // H.nout, side="right") - 1)
        J = int(np.searchsorted(bounds, col0 // H.nin, side="right") - 1)
        assert I % pr == rank // pc and J % pc == rank % pc, (rank, b, I, J)
        assert row_ok[row0:row0 + mm].all()
    xp = np.zeros(H.nin * H.n)
    for c in range(H.nin):
        xp[c::H.nin] = x[c * H.n + ex["perm"]]
    part = lattice_dist.partial_product(H, xp, mine, ex)
    assert np.all(part[~row_ok] == 0.0) and np.any(part[row_ok] != 0.0)
    y = lattice_dist.distributed_matvec(H, x, rank, pr, pc, dist, owners)
    out[rank] = float(np.linalg.norm(y - H.matvec(x)) / np.linalg.norm(H.matvec(x)))
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("pr,pc,library_owners", [(2, 2, False), (2, 1, False), (2, 2, True)])
def test_distributed_product_equals_serial(pr, pc, library_owners):
    ctx = mp.get_context("spawn")
    with ctx.Manager() as mgr:
        out = mgr.dict()
        mp.start_processes(_worker, args=(pr * pc, pr, pc, _free_port(), out, library_owners), nprocs=pr * pc,
                           join=True, start_method="spawn")
        errs = dict(out)
    assert len(errs) == pr * pc and max(errs.values()) < 1e-13, errs


@pytest.mark.parametrize("mk,op,leaf,L", [
    (lambda: meshes.scaled_thrust_mesh(12, 6, seed=2), 3, 8, 2),
    (lambda: meshes.planar_vertical_rect(40, 13, 250.0), 0, 32, 3),
    (lambda: meshes.planar_vertical_rect(7, 3, 250.0), 0, 4, 5),       # lattice deeper than the tree
])
def test_library_owner_map_equals_the_emulation(mk, op, leaf, L):
    """The library keeps the owner map as data (hbi_lattice_owners, host only, the partition
    of hbi_plan in its block order): it equals the owners the emulation above derives from the
    oracle's partition, for square and rectangular process grids."""
    import paper_2110_12165_gb300 as hbi
    m = mk()
    H = oracle.HMatrix(m, op, 1e-4, leaf, L, 32e9, 0.25)
    ex = H.export()
    for pr, pc in ((1, 1), (2, 2), (4, 4), (2, 3), (3, 1)):
        own = hbi.hbi_lattice_owners(m.verts, op, leaf, L, pr, pc)
        assert np.array_equal(own, lattice_dist.block_owners(H, pr, pc, ex)), (pr, pc)
        assert own.min() >= 0 and own.max() < pr * pc


def test_library_owner_map_rejects_an_empty_grid():
    import paper_2110_12165_gb300 as hbi
    m = meshes.planar_vertical_rect(4, 4, 250.0)
    with pytest.raises(hbi.HbiError, match="INVALID_ARG"):
        hbi.hbi_lattice_owners(m.verts, 0, 4, 1, 0, 2)
