"""Seeded rate-and-state parameter fields for the synthetic workloads.

Returns plain arrays (a, b, d_c, sigma0, rake, V_init) and the scalar constants; the
state (phi, tau) implied by V_init is computed by the method, not here.
"""
from dataclasses import dataclass

import numpy as np

from . import rng

KM = 1000.0


@dataclass
class Friction:
    a: np.ndarray          # direct-effect coefficient per element
    b: np.ndarray          # evolution-effect coefficient per element
    dc: np.ndarray         # characteristic slip distance per element (m)
    sigma0: np.ndarray     # initial effective normal stress (Pa, compression positive)
    rake: np.ndarray       # slip direction angle in the (strike, dip) element frame (rad)
    V_init: np.ndarray     # initial slip rate (m/s)
    f0: float = 0.6
    V0: float = 1e-6
    Vpl: float = 1e-9
    mu: float = 32e9
    nu: float = 0.25
    cs: float = 3464.0


def _perturbed_plate_rate(seed, n, Vpl, amp=1e-3):
    u = rng.uniform(rng.substream(seed, 31), n)
    return Vpl * (1.0 + amp * (2.0 * u - 1.0))


def config1_friction(mesh, seed=1):
    """VW patch 8 x 4 km at the centre (a=0.010, b=0.015); a-b=+0.004 elsewhere."""
    n = mesh.n_elem
    x, s = mesh.param_center[:, 0], mesh.param_center[:, 1]
    L, W = mesh.meta["length"], mesh.meta["width"]
    vw = (np.abs(x - L / 2) <= 4 * KM) & (np.abs(s - W / 2) <= 2 * KM)
    b = np.full(n, 0.015)
    a = np.where(vw, 0.010, 0.019)
    return Friction(a=a, b=b, dc=np.full(n, 0.005), sigma0=np.full(n, 50e6),
                    rake=np.zeros(n), V_init=_perturbed_plate_rate(seed, n, 1e-9),
                    mu=32e9, nu=0.25, cs=3460.0)


def thrust_friction(mesh, seed):
    """Randomly placed 30 x 20 km VW asperity on the thrust surface; pure thrust rake."""
    n = mesh.n_elem
    x, s = mesh.param_center[:, 0], mesh.param_center[:, 1]
    L, W = mesh.meta["length"], mesh.meta["width"]
    u = rng.uniform(rng.substream(seed, 41), 2)
    xc = 20 * KM + u[0] * (L - 40 * KM)
    sc = 12 * KM + u[1] * (W - 24 * KM)
    vw = (np.abs(x - xc) <= 15 * KM) & (np.abs(s - sc) <= 10 * KM)
    b = np.full(n, 0.015)
    a = np.where(vw, 0.010, 0.019)
    return Friction(a=a, b=b, dc=np.full(n, 0.005), sigma0=np.full(n, 50e6),
                    rake=np.full(n, np.pi / 2), V_init=_perturbed_plate_rate(seed, n, 1e-9),
                    mu=32e9, nu=0.25, cs=3460.0)


def velocity_strengthening(mesh, seed, amp=0.3):
    """All elements a-b=+0.004: the fault must relax to plate rate (a stability check)."""
    n = mesh.n_elem
    return Friction(a=np.full(n, 0.019), b=np.full(n, 0.015), dc=np.full(n, 0.005),
                    sigma0=np.full(n, 50e6), rake=np.zeros(n),
                    V_init=_perturbed_plate_rate(seed, n, 1e-9, amp=amp),
                    mu=32e9, nu=0.25, cs=3460.0)


def ensemble_friction(mesh, seed):
    """Per-model a, b-a, d_c drawn from a in [0.008,0.012], b-a in [-0.004,0.006], d_c in [2,20] mm."""
    n = mesh.n_elem
    u = rng.uniform(rng.substream(seed, 51), 3)
    a = 0.008 + 0.004 * u[0]
    bma = -0.004 + 0.010 * u[1]
    dc = 0.002 + 0.018 * u[2]
    return Friction(a=np.full(n, a), b=np.full(n, a + bma), dc=np.full(n, dc),
                    sigma0=np.full(n, 50e6), rake=np.full(n, np.pi / 2),
                    V_init=_perturbed_plate_rate(seed, n, 1e-9),
                    mu=32e9, nu=0.25, cs=3460.0)
