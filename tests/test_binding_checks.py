"""The Python binding checks every device array before the C ABI sees it: type, float64,
contiguity, the minimum length the entry point reads or writes (from N, the operator's
component counts and the number of models), and that it lives on the GPU.  None of these
checks needs a GPU, so they run here on CPU tensors."""
import pytest

torch = pytest.importorskip("torch")

import paper_2110_12165_gb300 as hbi

N = 10


def _h(op=hbi.HBI_OP_VEC_FULL, n_models=1):
    return hbi.Handle(None, N, op, n_models)


def _z(n, dtype=torch.float64):
    return torch.zeros(n, dtype=dtype)


def _raises(match, fn, *args, **kw):
    with pytest.raises(ValueError, match=match):
        fn(*args, **kw)


def test_matvec_lengths_follow_the_component_counts():
    h = _h()                                   # 2 slip components in, 3 stress components out
    _raises("x: 19 elements, needs at least 20", hbi.hbi_matvec, h, _z(19), _z(30))
    _raises("y: 29 elements, needs at least 30", hbi.hbi_matvec, h, _z(20), _z(29))
    _raises("expected a CUDA tensor", hbi.hbi_matvec, h, _z(20), _z(30))
    _raises("x: 29 elements, needs at least 30", hbi.hbi_matvec_transpose, h, _z(29), _z(20))
    _raises("y: 19 elements, needs at least 20", hbi.hbi_matvec_transpose, h, _z(30), _z(19))
    h1 = _h(hbi.HBI_OP_RAKE_SHEAR)
    _raises("expected a CUDA tensor", hbi.hbi_matvec_noalloc, h1, _z(10), _z(10))
    _raises("x: 9 elements", hbi.hbi_matvec_async, h1, _z(9), _z(10))


def test_dtype_contiguity_and_type():
    h = _h()
    _raises("expected float64", hbi.hbi_matvec, h, _z(20, torch.float32), _z(30))
    _raises("expected a contiguous", hbi.hbi_matvec, h, _z(40)[::2], _z(30))
    _raises("expected a torch tensor", hbi.hbi_matvec, h, [0.0] * 20, _z(30))
    _raises("x: required", hbi.hbi_matvec, h, None, _z(30))


def _fr(n):
    return hbi.hbi_friction(), (_z(n), _z(n), _z(n), _z(n))


def test_rhs_state_lengths_and_friction_arrays():
    h = _h()
    _raises("friction a: 9 elements, needs at least 10", hbi.hbi_rhs, h, _fr(9), _z(30), _z(30))
    _raises("state: 29 elements, needs at least 30", hbi.hbi_rhs, h, _fr(10), _z(29), _z(30))
    _raises("V: 9 elements", hbi.hbi_rhs, h, _fr(10), _z(30), _z(30), _z(9))
    _raises("state: 39 elements, needs at least 40", hbi.hbi_rhs_vec, h, _fr(10), _z(39), _z(40))
    _raises("V: 19 elements, needs at least 20", hbi.hbi_rhs_vec, h, _fr(10), _z(40), _z(40), _z(19))
    _raises("ybar: 29 elements", hbi.hbi_rhs_vjp, h, _fr(10), _z(30), _z(30), _z(29))
    _raises("grad_dc: 9 elements", hbi.hbi_rhs_vjp, h, _fr(10), _z(30), _z(30), _z(30), None, _z(9))


def test_integrator_state_lengths():
    h = _h()
    _raises("state: 39 elements, needs at least 40", hbi.hbi_step, h, _fr(10), _z(39), _z(1), _z(1), 1e-4, 1)
    _raises("dt: 0 elements, needs at least 1", hbi.hbi_step, h, _fr(10), _z(40), _z(1), _z(0), 1e-4, 1)
    _raises("state: 39 elements", hbi.hbi_rk_fixed, h, _fr(10), _z(39), [1.0])
    _raises("target: 9 elements", hbi.hbi_adjoint, h, _fr(10), _z(40), [1.0], _z(9), _z(10), _z(10))
    _raises("grad_amb: required", hbi.hbi_adjoint, h, _fr(10), _z(40), [1.0], _z(10), None, _z(10))
    _raises("state_final: 39 elements", hbi.hbi_adjoint, h, _fr(10), _z(40), [1.0], _z(10), _z(10), _z(10),
            state_final=_z(39))


def test_ensemble_and_vector_steps_need_one_time_per_model():
    h = _h(n_models=3)
    _raises("t: 2 elements, needs at least 3", hbi.hbi_step_ensemble, h, _fr(10), _z(40), _z(2), _z(3), 1e-4, 1)
    _raises("dt: 2 elements, needs at least 3", hbi.hbi_step_ensemble, h, _fr(10), _z(40), _z(3), _z(2), 1e-4, 1)
    _raises("state: 59 elements, needs at least 60", hbi.hbi_step_vector, h, _fr(10), _z(59), _z(3), _z(3),
            1e-4, 1)
    _raises("expected a CUDA tensor", hbi.hbi_step_vector, h, _fr(10), _z(60), _z(3), _z(3), 1e-4, 1)


def test_half_space_rejects_geometry_on_or_above_the_surface():
    """hbi_build validates the half-space geometry before it touches the GPU: every vertex
    at z <= 0 and every element centre below the free surface z = 0."""
    from synthetic import meshes
    m = meshes.dipping_rect(4, 3, 250.0, 40.0, origin=(0.0, 0.0, 100.0))
    with pytest.raises(hbi.HbiError, match="every vertex needs z <= 0"):
        hbi.hbi_build(m.verts, 32e9, 0.25, hbi.HBI_OP_VEC_FULL, 1e-4, 8, 0, "fp64", half_space=True)
    v = meshes.dipping_rect(4, 3, 250.0, 90.0).verts.copy()
    v[0, :, 2] = 0.0                                   # one element lying in the surface
    with pytest.raises(hbi.HbiError, match="every element centre needs z < 0"):
        hbi.hbi_build(v, 32e9, 0.25, hbi.HBI_OP_VEC_FULL, 1e-4, 8, 0, "fp64", half_space=True)


def test_steady_state_arrays_match_V():
    _raises("tau: 4 elements, needs at least 5", hbi.hbi_steady_state, _z(5), _z(5), _z(5), _z(5), 0.6, 1e-6,
            _z(5), _z(4))
