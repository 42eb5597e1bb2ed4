"""Write c2_oracle_sequence.json: the oracle's own run of the 20,022-element nonplanar thrust
fault (141 x 71 quads split into triangles, seed 2, the 2 -> 3 operator in full space,
eps_ACA = 1e-4, leaf 64, lattice depth 2, eta = 2) from steady sliding at V_init, through its
first earthquakes: the step records (t, dt, max V, rejected attempts) of every accepted
adaptive Cash-Karp step (Eqs. 14-16).

The oracle needs about two to three seconds per step at this size, too slow for a test, so
its run is stored and the GPU test compares against it.  This script calls only the oracle
and the seeded input generators.  Usage: python tests/golden/c2_oracle_sequence.py
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

N_STEPS = 240          # the first three earthquakes of this run start at steps ~140, ~167, ~220
EPS, LEAF, DEPTH, ETA_ADM = 1e-4, 64, 2, 2.0
EPS_RK, DT0 = 1e-4, 1e5


def main():
    m = meshes.config2_mesh(seed=2)
    F = friction.thrust_friction(m, seed=2)
    t0 = time.time()
    H = oracle.HMatrix(m, oracle.OP_VEC_FULL, EPS, LEAF, DEPTH, F.mu, F.nu, rake=F.rake, eta=ETA_ADM)
    t_build = time.time() - t0
    td, sd = H.loading(F.rake, F.Vpl)
    phi, tau = oracle.steady_state(F.V_init, F.a, F.b, F.sigma0, F.f0, F.V0)
    y0 = np.concatenate([phi, tau, F.sigma0])
    t1 = time.time()
    _, _, _, _, rec = H.run(F, y0, np.zeros(m.n_elem), 0.0, DT0, EPS_RK, N_STEPS, td, sd)
    t_run = time.time() - t1
    out = {"what": "oracle run of the 141 x 71 nonplanar thrust fault (N = 20,022), first earthquakes",
           "mesh": {"generator": "synthetic.meshes.config2_mesh", "seed": 2, "n_elem": int(m.n_elem)},
           "friction": {"generator": "synthetic.friction.thrust_friction", "seed": 2},
           "operator": "OP_VEC_FULL (2 slip -> 3 stress components), full space",
           "aca_eps": EPS, "leaf": LEAF, "lattice_depth": DEPTH, "eta": ETA_ADM, "eps_rk": EPS_RK, "dt0": DT0,
           "n_steps": N_STEPS, "oracle_threads": oracle.num_threads(),
           "oracle_build_s": round(t_build, 1), "oracle_s_per_step": round(t_run / N_STEPS, 3),
           "records_t_dt_vmax_rejects": [[float(v) for v in r] for r in rec]}
    with open(os.path.join(HERE, "c2_oracle_sequence.json"), "w") as f:
        json.dump(out, f, indent=0)
    print(f"N = {m.n_elem}: build {t_build:.1f} s, {t_run / N_STEPS:.3f} s per step on {oracle.num_threads()} threads")


if __name__ == "__main__":
    main()
