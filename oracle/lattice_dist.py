"""The paper's distributed lattice H-matrix product (Sec. 3.2) on CPU ranks.

TEST INFRASTRUCTURE ONLY (like the rest of `oracle/`): it checks the owner map and the
communication pattern of the paper's parallel scheme with torch.distributed ranks on the
host.  The library runs on one GPU per process and does not distribute an operator.

Sec. 3.2 cuts the index set into a P_r x P_c lattice of clusters and hands the lattice blocks
to the ranks cyclically in both directions (rank (I mod P_r, J mod P_c) owns lattice block
(I, J)).  A rank computes Eq. 20 over the H-matrix blocks inside its lattice blocks; the
partial results of the lattice rows of one process row are summed by a reduction along that
process row, and the (disjoint) row sums are then combined over the row roots and broadcast
so that every rank holds the whole product.
"""
import numpy as np


def lattice_index(H, ex=None):
    """Element ranges [start, end) of the lattice clusters, in permuted order."""
    ex = ex or H.export()
    cl = ex["clusters"]
    lat = ex["lattice"] if len(ex["lattice"]) else np.array([0])
    starts = sorted(int(cl[k, 0]) for k in lat)
    return np.array(starts + [H.n])


def block_owners(H, pr, pc, ex=None):
    """Owning rank of every H-matrix block: the 2D-cyclic owner of its lattice block."""
    ex = ex or H.export()
    bounds = lattice_index(H, ex)
    owners = np.zeros(len(ex["blocks"]), dtype=np.int64)
    for b, (row0, m, col0, nc, *_rest) in enumerate(ex["blocks"]):
        e_row, e_col = row0 // H.nout, col0 // H.nin
        I = int(np.searchsorted(bounds, e_row, side="right") - 1)
        J = int(np.searchsorted(bounds, e_col, side="right") - 1)
        owners[b] = (I % pr) * pc + (J % pc)
    return owners


def partial_product(H, xp, blocks_mine, ex):
    """Eq. 20 over the given blocks in the permuted, component-interleaved index space."""
    data = ex["data"]
    yp = np.zeros(H.nout * H.n)
    for b in blocks_mine:
        row0, m, col0, nc, lowrank, r, off = (int(v) for v in ex["blocks"][b][:7])
        if r < 0:            # not built (a sampled build's block outside its lattice row)
            continue
        if not lowrank:
            D = data[off:off + m * nc].reshape(m, nc)
            yp[row0:row0 + m] += D @ xp[col0:col0 + nc]
        elif r > 0:
            U = data[off:off + m * r].reshape(r, m).T
            V = data[off + m * r:off + (m + nc) * r].reshape(r, nc).T
            yp[row0:row0 + m] += U @ (V.T @ xp[col0:col0 + nc])
    return yp


def distributed_matvec(H, x, rank, pr, pc, dist, owners=None):
    """y = H x on a P_r x P_c grid of ranks (world size P_r P_c, process groups of `dist`):
    2D-cyclic owners (or the given owner of every block, in the partition's block order), a
    reduction along each process row to its first rank, the row sums combined over those roots
    and broadcast.  x and y in the caller's order (component-major)."""
    import torch
    ex = H.export()
    n, perm = H.n, ex["perm"]
    xp = np.zeros(H.nin * n)
    for c in range(H.nin):
        xp[c::H.nin] = np.asarray(x)[c * n + perm]
    owners = block_owners(H, pr, pc, ex) if owners is None else np.asarray(owners)
    yp = partial_product(H, xp, np.nonzero(owners == rank)[0], ex)
    t = torch.tensor(yp, dtype=torch.float64)
    my_row = rank // pc
    for i in range(pr):   # every rank creates every group, in the same order
        g = dist.new_group(ranks=[i * pc + j for j in range(pc)])
        if i == my_row:
            dist.reduce(t, dst=i * pc, group=g)
    # the row roots hold disjoint lattice rows' sums: their sum over the roots is the product
    roots = dist.new_group(ranks=[i * pc for i in range(pr)])
    if rank % pc == 0:
        dist.all_reduce(t, group=roots)
    dist.broadcast(t, src=0)
    yp = t.numpy()
    y = np.zeros(H.nout * n)
    for c in range(H.nout):
        y[c * n + perm] = yp[c::H.nout]
    return y
