"""Helpers shared by the GPU parity tests: import an oracle H-matrix into the CUDA library
(same partition and factors) and move arrays between numpy and torch."""
import numpy as np

import oracle
import paper_2110_12165_gb300 as hbi


def leaf_starts_from_export(ex, n):
    cl = ex["clusters"]
    starts = sorted(int(c[0]) for c in cl if c[3] < 0)
    return np.array(starts + [n], dtype=np.int32)


def import_oracle(H, storage, rake=None, transpose=False):
    """hbi handle holding exactly the oracle's partition and factors (and H^T on request)."""
    ex = H.export()
    blocks = ex["blocks"]
    return hbi.hbi_build_from_factors(H.mesh.verts, H.mu, H.nu, H.op, storage, ex["perm"], blocks[:, :6],
                                      blocks[:, 6], ex["data"], leaf_starts_from_export(ex, H.n),
                                      rake=H.rake if rake is None else rake, transpose=transpose)


def dev(a):
    import torch
    return torch.tensor(np.ascontiguousarray(a, dtype=np.float64), device="cuda")


def host(t):
    return t.detach().cpu().numpy()


def rel_l2(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))
