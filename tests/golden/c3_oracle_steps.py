"""Write c3_oracle_steps.json: the oracle's own first 200 accepted adaptive Cash-Karp steps
(Eqs. 14-16) on the 160,000-element nonplanar thrust fault of the timed workload (400 x 200
quads split into triangles, seed 3, the 2 -> 3 operator in full space, eps_ACA = 1e-4, leaf 64,
lattice depth 2, eta = 2) from steady sliding at V_init, through the late interseismic period
into the start of the first earthquake: the step records (t, dt, max V, rejected attempts) and
the state (phi, tau, sigma) after step 50 (interseismic) and after step 200 at 64 seeded sample
elements.

The oracle needs about half a minute per step at this size (and tens of minutes to build its
operator), far too slow for a test, so its run is stored and the GPU test compares against it.
This script calls only the oracle and the seeded input generators.
Usage: python tests/golden/c3_oracle_steps.py
"""
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle                                  # noqa: E402
from synthetic import friction, meshes         # noqa: E402

N_STEPS = 200
N_SAMPLE = 64
STATE_STEP = 50
EPS, LEAF, DEPTH, ETA_ADM = 1e-4, 64, 2, 2.0
EPS_RK, DT0 = 1e-4, 1e5


def sample_elements(n, k, seed=71):
    """k distinct element indices from a counter-based generator (SplitMix64 of seed + i)."""
    out, i = [], 0
    mask = (1 << 64) - 1
    while len(out) < k:
        z = (seed * 0x9E3779B97F4A7C15 + (i + 1) * 0x9E3779B97F4A7C15) & mask
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & mask
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & mask
        z ^= z >> 31
        e = int(z % n)
        if e not in out:
            out.append(e)
        i += 1
    return sorted(out)


def main():
    m = meshes.scaled_thrust_mesh(400, 200, seed=3)
    F = friction.thrust_friction(m, seed=3)
    n = m.n_elem
    t0 = time.time()
    H = oracle.HMatrix(m, oracle.OP_VEC_FULL, EPS, LEAF, DEPTH, F.mu, F.nu, rake=F.rake, eta=ETA_ADM)
    t_build = time.time() - t0
    print(f"built N = {n} in {t_build:.1f} s on {oracle.num_threads()} threads", flush=True)
    td, sd = H.loading(F.rake, F.Vpl)
    phi, tau = oracle.steady_state(F.V_init, F.a, F.b, F.sigma0, F.f0, F.V0)
    y = np.concatenate([phi, tau, F.sigma0])
    D = np.zeros(n)
    t, dt = 0.0, DT0
    recs = []
    idx = sample_elements(n, N_SAMPLE)
    mid = None
    t1 = time.time()
    for k in range(N_STEPS):            # one call per step, so that progress shows
        y, D, t, dt, rec = H.run(F, y, D, t, dt, EPS_RK, 1, td, sd)
        recs.append([float(v) for v in rec[0]])
        if k + 1 == STATE_STEP:
            mid = {"phi": [float(y[i]) for i in idx], "tau": [float(y[n + i]) for i in idx],
                   "sigma": [float(y[2 * n + i]) for i in idx], "t": float(t), "dt": float(dt)}
        if (k + 1) % 20 == 0:
            print(f"step {k + 1}: t = {t:.6e} s, {(time.time() - t1) / (k + 1):.1f} s per step", flush=True)
    t_run = time.time() - t1
    out = {"what": "oracle run of the 400 x 200 nonplanar thrust fault (N = 160,000), first 200 accepted steps",
           "mesh": {"generator": "synthetic.meshes.scaled_thrust_mesh", "n_strike": 400, "n_dip": 200, "seed": 3,
                    "n_elem": int(n)},
           "friction": {"generator": "synthetic.friction.thrust_friction", "seed": 3},
           "operator": "OP_VEC_FULL (2 slip -> 3 stress components), full space",
           "aca_eps": EPS, "leaf": LEAF, "lattice_depth": DEPTH, "eta": ETA_ADM, "eps_rk": EPS_RK, "dt0": DT0,
           "n_steps": N_STEPS, "oracle_threads": oracle.num_threads(),
           "oracle_build_s": round(t_build, 1), "oracle_s_per_step": round(t_run / N_STEPS, 3),
           "records_t_dt_vmax_rejects": recs,
           "sample_elements": idx, "state_step": STATE_STEP, "state_at_step": mid,
           "final_phi": [float(y[i]) for i in idx], "final_tau": [float(y[n + i]) for i in idx],
           "final_sigma": [float(y[2 * n + i]) for i in idx], "final_t": float(t), "final_dt": float(dt)}
    with open(os.path.join(HERE, "c3_oracle_steps.json"), "w") as f:
        json.dump(out, f, indent=0)
    print(f"done: build {t_build:.1f} s, {t_run / N_STEPS:.2f} s per step", flush=True)


if __name__ == "__main__":
    main()
