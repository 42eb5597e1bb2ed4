"""Seeded synthetic fault meshes shaped like the paper's workloads (Section 4.1, Fig. 4).

Every generator returns a `Mesh`: element vertices in metres, shape (n_elem, nv, 3),
nv = 4 for rectangles (two sides horizontal, as the Okada-type element of Section 2.1
requires) and nv = 3 for triangles.  Vertices are ordered counter-clockwise in the
(along-strike x, down-dip s) parameter plane, which makes the right-hand normal point
into the hanging wall (upward) for the dipping faults.  `param_center` holds each
element's (x, s) parameter coordinates, used only to place friction patches.

No part of the method's arithmetic lives here: element centroids, normals, frames and
kernels are computed by the oracle and by the CUDA library independently.
"""
from dataclasses import dataclass, field

import numpy as np

from . import rng

KM = 1000.0


@dataclass
class Mesh:
    kind: str                  # "rect" or "tri"
    verts: np.ndarray          # (n_elem, nv, 3) float64, metres
    param_center: np.ndarray   # (n_elem, 2) float64, (x along strike, s down-dip), metres
    meta: dict = field(default_factory=dict)

    @property
    def n_elem(self):
        return self.verts.shape[0]

    @property
    def nv(self):
        return self.verts.shape[1]


def planar_vertical_rect(nx, nz, h, origin=(0.0, 0.0, 0.0)):
    """nx x nz squares of side h in the vertical plane y = 0 (strike along x, depth -z)."""
    ox, oy, oz = origin
    v = np.zeros((nx * nz, 4, 3))
    pc = np.zeros((nx * nz, 2))
    e = 0
    for j in range(nz):
        for i in range(nx):
            x0, x1 = i * h, (i + 1) * h
            s0, s1 = j * h, (j + 1) * h
            for k, (xx, ss) in enumerate(((x0, s0), (x1, s0), (x1, s1), (x0, s1))):
                v[e, k] = (ox + xx, oy, oz - ss)
            pc[e] = (0.5 * (x0 + x1), 0.5 * (s0 + s1))
            e += 1
    return Mesh("rect", v, pc, {"nx": nx, "nz": nz, "h": h})


def planar_vertical_tri(nx, nz, h, origin=(0.0, 0.0, 0.0)):
    """Each square of planar_vertical_rect split into two triangles (alternating diagonals)."""
    ox, oy, oz = origin
    P = lambda xx, ss: (ox + xx, oy, oz - ss)
    tris, pcs = [], []
    for j in range(nz):
        for i in range(nx):
            c = [(i * h, j * h), ((i + 1) * h, j * h), ((i + 1) * h, (j + 1) * h), (i * h, (j + 1) * h)]
            if (i + j) % 2 == 0:
                tt = ((0, 1, 2), (0, 2, 3))
            else:
                tt = ((0, 1, 3), (1, 2, 3))
            for t in tt:
                tris.append([P(*c[k]) for k in t])
                pcs.append(np.mean([c[k] for k in t], axis=0))
    return Mesh("tri", np.array(tris, dtype=np.float64), np.array(pcs), {"nx": nx, "nz": nz, "h": h})


def config1_mesh():
    """Planar vertical strike-slip fault: 64 x 32 squares of 250 m (N = 2048)."""
    m = planar_vertical_rect(64, 32, 250.0)
    m.meta.update(name="planar-strike-slip-rect-N2048", length=16 * KM, width=8 * KM)
    return m


def _thrust_surface(x, s, amp, wavelength, dip0_deg, dip1_deg, width, top_depth):
    """Map parameter coordinates (x along strike, s down-dip arc length) to 3-D points.

    The dip rises linearly with s from dip0 to dip1; the trace undulates along strike.
    """
    d0 = np.deg2rad(dip0_deg)
    k = np.deg2rad(dip1_deg - dip0_deg) / width
    if abs(k) > 0:
        Y = (np.sin(d0 + k * s) - np.sin(d0)) / k
        Z = (np.cos(d0) - np.cos(d0 + k * s)) / k
    else:
        Y = s * np.cos(d0)
        Z = s * np.sin(d0)
    X = x
    Y = Y + amp * np.sin(2.0 * np.pi * x / wavelength)
    Zc = -(top_depth + Z)
    return np.stack([X, Y, Zc], axis=-1)


def nonplanar_thrust_tri(n_strike, n_dip, seed, length=100 * KM, width=50 * KM, amp=2 * KM,
                         wavelength=40 * KM, dip0=10.0, dip1=30.0, top_depth=1 * KM, jitter=0.15):
    """Nonplanar thrust fault split into triangles with alternating diagonals.

    A quad grid of n_strike x n_dip cells over (x, s) in [0, length] x [0, width]; interior
    nodes receive a seeded in-surface jitter of +-jitter cell sizes (a stand-in for the
    side-length variability of an unstructured mesher); each quad gives two triangles.
    """
    dx, ds = length / n_strike, width / n_dip
    xi = np.arange(n_strike + 1) * dx
    si = np.arange(n_dip + 1) * ds
    X, S = np.meshgrid(xi, si, indexing="ij")
    interior = np.zeros_like(X, dtype=bool)
    interior[1:-1, 1:-1] = True
    n_int = int(interior.sum())
    ux = rng.uniform(rng.substream(seed, 11), n_int)
    us = rng.uniform(rng.substream(seed, 12), n_int)
    Xj, Sj = X.copy(), S.copy()
    Xj[interior] += jitter * dx * (2.0 * ux - 1.0)
    Sj[interior] += jitter * ds * (2.0 * us - 1.0)
    P = _thrust_surface(Xj, Sj, amp, wavelength, dip0, dip1, width, top_depth)
    i = np.arange(n_strike)[:, None]
    j = np.arange(n_dip)[None, :]
    i = np.broadcast_to(i, (n_strike, n_dip)).ravel()
    j = np.broadcast_to(j, (n_strike, n_dip)).ravel()
    c00 = np.stack([i, j], 1)
    c10 = np.stack([i + 1, j], 1)
    c11 = np.stack([i + 1, j + 1], 1)
    c01 = np.stack([i, j + 1], 1)
    even = ((i + j) % 2 == 0)
    # counter-clockwise in (x, s): (00,10,11),(00,11,01) or (00,10,01),(10,11,01)
    t1 = np.where(even[:, None, None], np.stack([c00, c10, c11], 1), np.stack([c00, c10, c01], 1))
    t2 = np.where(even[:, None, None], np.stack([c00, c11, c01], 1), np.stack([c10, c11, c01], 1))
    tri_idx = np.empty((2 * len(i), 3, 2), dtype=np.int64)
    tri_idx[0::2] = t1
    tri_idx[1::2] = t2
    verts = P[tri_idx[..., 0], tri_idx[..., 1]]
    pc = np.stack([Xj[tri_idx[..., 0], tri_idx[..., 1]].mean(1),
                   Sj[tri_idx[..., 0], tri_idx[..., 1]].mean(1)], 1)
    return Mesh("tri", np.ascontiguousarray(verts), pc,
                {"n_strike": n_strike, "n_dip": n_dip, "length": length, "width": width,
                 "seed": seed})


def config2_mesh(seed=2):
    """100 x 50 km nonplanar thrust, 141 x 71 quads -> N = 20,022 triangles (~0.7 km)."""
    m = nonplanar_thrust_tri(141, 71, seed)
    m.meta["name"] = "nonplanar-thrust-tri-N20022"
    return m


def config3_mesh(seed=3):
    """Same surface refined to 400 x 200 quads -> N = 160,000 triangles (0.25 km)."""
    m = nonplanar_thrust_tri(400, 200, seed)
    m.meta["name"] = "nonplanar-thrust-tri-N160000"
    return m


def scaled_thrust_mesh(n_strike, n_dip, seed):
    """Thrust surface at another resolution (parity and scaling cases)."""
    m = nonplanar_thrust_tri(n_strike, n_dip, seed)
    m.meta["name"] = f"nonplanar-thrust-tri-N{2 * n_strike * n_dip}"
    return m


def dipping_rect(nx, nd, h, dip_deg, origin=(0.0, 0.0, 0.0)):
    """Planar rectangular fault of nx x nd squares dipping at dip_deg (strike along x)."""
    dip = np.deg2rad(dip_deg)
    ox, oy, oz = origin
    v = np.zeros((nx * nd, 4, 3))
    pc = np.zeros((nx * nd, 2))
    e = 0
    for j in range(nd):
        for i in range(nx):
            x0, x1, s0, s1 = i * h, (i + 1) * h, j * h, (j + 1) * h
            for k, (xx, ss) in enumerate(((x0, s0), (x1, s0), (x1, s1), (x0, s1))):
                v[e, k] = (ox + xx, oy + ss * np.cos(dip), oz - ss * np.sin(dip))
            pc[e] = (0.5 * (x0 + x1), 0.5 * (s0 + s1))
            e += 1
    return Mesh("rect", v, pc, {"nx": nx, "nd": nd, "h": h, "dip": dip_deg})


def ensemble_meshes(n_models=64, seed=4, n_min=2000, n_max=40000, h=250.0):
    """Independent rectangular faults of uneven size, aspect 2:1, dip U[15,60] deg or vertical."""
    u = rng.uniform(rng.substream(seed, 21), n_models)
    ud = rng.uniform(rng.substream(seed, 22), n_models)
    uv = rng.uniform(rng.substream(seed, 23), n_models)
    out = []
    for k in range(n_models):
        n_target = n_min + u[k] * (n_max - n_min)
        # an even number of rows: N = 2 nd^2 is a multiple of 8, so every model of the
        # concatenated ensemble starts on a 16-byte boundary of the product input
        nd = max(2, 2 * int(round(np.sqrt(n_target / 2.0) / 2.0)))
        nx = 2 * nd
        dip = 90.0 if uv[k] < 0.25 else 15.0 + 45.0 * ud[k]
        out.append(dipping_rect(nx, nd, h, dip))
    return out
