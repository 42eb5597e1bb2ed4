"""The bounds-checked build of the product kernels (HBI_BOUNDS_CHECK; compute-sanitizer is not
available on this pool): in a subprocess that loads that build, products through every table
layout the library makes -- the oracle's factors in FP64 and mixed storage, a GPU-built mixed
operator (ADAPTIVE storage: paired gather indices) with its transpose, an ensemble, the no-allocation product -- and a
run of adaptive steps (the products inside the captured attempt graph) count no violation, and
give bit for bit the results of the normal build (the checks change no arithmetic)."""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu
HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)

SCRIPT = r'''
import json, sys
import numpy as np, torch
sys.path.insert(0, ROOT); sys.path.insert(0, HERE)
import oracle
import paper_2110_12165_gb300 as hbi
from synthetic import friction, meshes, rng
from gpu_util import dev, host, import_oracle
out = {}
m = meshes.scaled_thrust_mesh(24, 12, seed=2)
n = m.n_elem
F = friction.thrust_friction(m, seed=2)
H = oracle.HMatrix(m, oracle.OP_VEC_FULL, 1e-5, 16, 2, F.mu, F.nu, rake=F.rake)
x = rng.normal(3, 2 * n)
y = torch.zeros(3 * n, dtype=torch.float64, device="cuda")
for stg in ("fp64", "mixed"):
    h = import_oracle(H, stg)
    hbi.hbi_matvec(h, dev(x), y)
    out["oracle_" + stg] = host(y).tolist()
hg = hbi.hbi_build(m.verts, F.mu, F.nu, oracle.OP_VEC_FULL, 1e-4, 16, 2, "adaptive", rake=F.rake, recompress_eps=1e-4,
                   transpose=True)

hbi.hbi_matvec(hg, dev(x), y); out["built"] = host(y).tolist()
w = torch.zeros(2 * n, dtype=torch.float64, device="cuda")
hbi.hbi_matvec_transpose(hg, dev(rng.normal(4, 3 * n)), w); out["transpose"] = host(w).tolist()
hbi.hbi_matvec_noalloc(hg, dev(x), y); out["noalloc"] = host(y).tolist()
ms = [meshes.dipping_rect(16, 8, 250.0, 30.0), meshes.dipping_rect(12, 6, 250.0, 90.0)]
hE, st = hbi.hbi_build_ensemble([mm.verts for mm in ms], F.mu, F.nu, oracle.OP_RAKE_SHEAR, 1e-5, 8, 2, "mixed")
ye = torch.zeros(int(st[-1]), dtype=torch.float64, device="cuda")
hbi.hbi_matvec(hE, dev(rng.normal(5, int(st[-1]))), ye); out["ensemble"] = host(ye).tolist()
phi, tau = oracle.steady_state(F.V_init, F.a, F.b, F.sigma0, F.f0, F.V0)
fr = hbi.friction(dev(F.a), dev(F.b), dev(F.dc), dev(F.rake), F.f0, F.V0, F.Vpl, F.mu, F.cs)
s = dev(np.concatenate([phi, tau, F.sigma0, np.zeros(n)]))
code, done, rec = hbi.hbi_step(hg, fr, s, dev([0.0]), dev([1e5]), 1e-4, 30)
out["steps"] = host(s).tolist(); out["records"] = rec.tolist(); out["status"] = int(code)
try:
    out["violations"] = hbi.hbi_bounds_violations()
except hbi.HbiError:
    out["violations"] = None
print(json.dumps(out))
'''


def _run(checked):
    env = dict(os.environ, HBI_BOUNDS_CHECK="1" if checked else "0")
    code = "ROOT = %r\nHERE = %r\n" % (ROOT, HERE) + SCRIPT
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env, timeout=1200)
    assert r.returncode == 0, r.stderr[-3000:]
    return json.loads(r.stdout.strip().splitlines()[-1])


def test_checked_build_counts_no_violation_and_matches_the_normal_build():
    chk = _run(True)
    ref = _run(False)
    assert ref["violations"] is None                 # the normal build has no counter
    assert chk["violations"] == 0
    assert chk["status"] == 0 and ref["status"] == 0
    for key in ("oracle_fp64", "oracle_mixed", "built", "transpose", "noalloc", "ensemble", "steps", "records"):
        assert np.array_equal(np.array(chk[key]), np.array(ref[key])), key
