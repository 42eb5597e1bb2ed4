"""hbi_step runs each Cash-Karp stage of the fixed-rake law inside the UY launch of the product
before it (stage_elem / final_unit, as the product's rows are written); hbi_rk_fixed runs the
same per-element stage arithmetic as kernels of its own.  Replaying the accepted step sizes of
an adaptive run with hbi_rk_fixed from the same state gives the same state to the last bit: a
rejected attempt leaves y unchanged, and the retry's first stage equals the one it reuses.  The
run starts with a step far too large, so that it begins with rejected attempts (the path that
skips the first product and keeps k_1)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
import paper_2110_12165_gb300 as hbi
from synthetic import friction, meshes
from gpu_util import dev, host

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("storage", ["mixed", "fp64"])
def test_adaptive_steps_equal_their_fixed_replay_bit_for_bit(storage):
    m = meshes.scaled_thrust_mesh(40, 20, seed=11)            # N = 1600, 2 -> 3 operator
    F = friction.thrust_friction(m, seed=11)
    n = m.n_elem
    h = hbi.hbi_build(m.verts, F.mu, F.nu, oracle.OP_VEC_FULL, 1e-4, 16, 2, storage, rake=F.rake,
                      recompress_eps=1e-4 if storage == "mixed" else 0.0)
    fr = hbi.friction(dev(F.a), dev(F.b), dev(F.dc), dev(F.rake), F.f0, F.V0, F.Vpl, F.mu, F.cs)
    phi, tau = oracle.steady_state(F.V_init, F.a, F.b, F.sigma0, F.f0, F.V0)
    y0 = np.concatenate([phi, tau, F.sigma0, np.zeros(n)])
    s, t, dt = dev(y0), dev([0.0]), dev([3e9])
    st, done, rec = hbi.hbi_step(h, fr, s, t, dt, 1e-4, 120)
    assert st == 0 and done == 120
    assert rec[0, 3] >= 1, "the first step should follow rejected attempts"
    s_fixed = dev(y0)
    hbi.hbi_rk_fixed(h, fr, s_fixed, rec[:, 1])
    assert torch.equal(s, s_fixed), float((s - s_fixed).abs().max())
    assert np.isclose(host(t)[0], rec[-1, 0], rtol=0, atol=0)
