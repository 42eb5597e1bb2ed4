"""Python binding of the hbi C ABI (include/hbi.h): argument marshalling only.

Every computation runs in the CUDA library `_build/libhbi.so` (built for sm_103a by
`build.py`).  There is no CPU fallback: if the library cannot be loaded, importing a
function raises.  Device arrays are torch CUDA tensors (float64, contiguous); the current
torch stream is passed to the library unless a stream is given.
"""
import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))

HBI_RECT, HBI_TRI = 4, 3
HBI_OP_RAKE_SHEAR, HBI_OP_RAKE_SHEAR_NORMAL, HBI_OP_VEC_SHEAR, HBI_OP_VEC_FULL = 0, 1, 2, 3
HBI_FP64, HBI_FP32, HBI_FP16, HBI_BF16, HBI_MIXED, HBI_ADAPTIVE = 0, 1, 2, 3, 4, 5
STORAGE = {"fp64": HBI_FP64, "fp32": HBI_FP32, "fp16": HBI_FP16, "bf16": HBI_BF16, "mixed": HBI_MIXED,
           "adaptive": HBI_ADAPTIVE}
OP_NIN = {0: 1, 1: 1, 2: 2, 3: 2}
OP_NOUT = {0: 1, 1: 2, 2: 2, 3: 3}

# exported symbols, in the order declared in include/hbi.h
SYMBOLS = ["hbi_build", "hbi_plan", "hbi_lattice_owners", "hbi_build_shard", "hbi_build_from_factors", "hbi_matvec", "hbi_matvec_async",
           "hbi_matvec_noalloc", "hbi_matvec_transpose", "hbi_matvec_multi", "hbi_time_multi", "hbi_multi_stats",
           "hbi_build_ensemble", "hbi_steady_state",
           "hbi_rhs", "hbi_rhs_vec", "hbi_rhs_vjp", "hbi_rk_fixed", "hbi_adjoint", "hbi_step", "hbi_step_ensemble",
           "hbi_step_vector", "hbi_time_attempts",
           "hbi_stats", "hbi_time_hmvm", "hbi_autotune", "hbi_stalled_wait_status", "hbi_inject_failure",
           "hbi_bounds_violations",
           "hbi_destroy", "hbi_status_string", "hbi_last_error"]


class hbi_mesh(C.Structure):
    _fields_ = [("n_elem", C.c_int), ("kind", C.c_int), ("h_verts", C.c_void_p), ("h_rake", C.c_void_p)]


class hbi_elastic(C.Structure):
    _fields_ = [("mu", C.c_double), ("nu", C.c_double), ("op", C.c_int), ("half_space", C.c_int)]


class hbi_build_params(C.Structure):
    _fields_ = [("aca_eps", C.c_double), ("leaf_size", C.c_int), ("lattice_depth", C.c_int),
                ("eta", C.c_double), ("storage", C.c_int), ("recompress_eps", C.c_double),
                ("with_transpose", C.c_int), ("multi_rhs", C.c_int)]


class hbi_friction(C.Structure):
    _fields_ = [("d_a", C.c_void_p), ("d_b", C.c_void_p), ("d_dc", C.c_void_p), ("d_rake", C.c_void_p),
                ("f0", C.c_double), ("V0", C.c_double), ("Vpl", C.c_double), ("mu", C.c_double),
                ("cs", C.c_double)]


class hbi_step_record(C.Structure):
    _fields_ = [("t", C.c_double), ("dt", C.c_double), ("vmax", C.c_double), ("rejects", C.c_double),
                ("mu_mean", C.c_double)]


class hbi_stats_t(C.Structure):
    _fields_ = [(k, C.c_int64) for k in ("n_elem", "n_in", "n_out", "n_clusters", "n_leaves", "n_lattice",
                                         "n_blocks", "n_lowrank", "n_dense", "max_rank")] + \
               [("mean_rank", C.c_double)] + \
               [(k, C.c_int64) for k in ("entries_lowrank", "entries_dense", "bytes_factors",
                                         "bytes_algorithmic", "n_tasks_vt", "n_tasks_uy")] + \
               [("storage", C.c_int), ("build_seconds", C.c_double), ("bytes_alg_vt", C.c_int64),
                ("bytes_alg_uy", C.c_int64), ("last_step_attempts", C.c_int64), ("last_step_kernels", C.c_int64),
                ("n_models", C.c_int64)]


class hbi_multi_stats_t(C.Structure):
    _fields_ = [(k, C.c_int64) for k in ("panel_bytes", "bytes_panels_algorithmic", "vector_bytes_per_rhs")] + \
               [("flops_per_rhs", C.c_double), ("mma_flops_per_rhs", C.c_double)] + \
               [(k, C.c_int64) for k in ("n_tasks_vt", "n_tasks_uy", "n_t", "n_split_tiles")]


class HbiError(RuntimeError):
    pass


_lib = None


def library_path():
    return os.path.join(HERE, "_build", "libhbi.so")


def lib():
    """Load libhbi.so (building it with nvcc if it is missing or stale)."""
    global _lib
    if _lib is None:
        import torch  # noqa: F401  (loads the CUDA runtime the library shares)
        from . import build as _b
        # HBI_BOUNDS_CHECK=1: the bounds-checked build of the product kernels (hbi_bounds_violations)
        path = _b.build(checked=os.environ.get("HBI_BOUNDS_CHECK", "0") == "1")
        L = C.CDLL(path)
        vp, i, d = C.c_void_p, C.c_int, C.c_double
        L.hbi_build.argtypes = [C.POINTER(hbi_mesh), C.POINTER(hbi_elastic), C.POINTER(hbi_build_params),
                                C.POINTER(vp)]
        L.hbi_plan.argtypes = [C.POINTER(hbi_mesh), C.POINTER(hbi_elastic), C.POINTER(hbi_build_params), vp, vp,
                               C.POINTER(i), vp, i, C.POINTER(i)]
        L.hbi_lattice_owners.argtypes = [C.POINTER(hbi_mesh), C.POINTER(hbi_elastic), C.POINTER(hbi_build_params),
                                         i, i, vp, i, C.POINTER(i)]
        L.hbi_build_shard.argtypes = [C.POINTER(hbi_mesh), C.POINTER(hbi_elastic), C.POINTER(hbi_build_params),
                                      i, i, i, C.POINTER(vp)]
        L.hbi_build_from_factors.argtypes = [C.POINTER(hbi_mesh), C.POINTER(hbi_elastic), i, vp, i, vp, vp, vp,
                                             i, vp, i, C.POINTER(vp)]
        L.hbi_matvec.argtypes = [vp, vp, vp, vp]
        L.hbi_matvec_async.argtypes = [vp, vp, vp, vp]
        L.hbi_matvec_noalloc.argtypes = [vp, vp, vp, vp]
        L.hbi_matvec_transpose.argtypes = [vp, vp, vp, vp]
        L.hbi_matvec_multi.argtypes = [vp, i, vp, vp, vp]
        L.hbi_time_multi.argtypes = [vp, i, i, vp, vp]
        L.hbi_multi_stats.argtypes = [vp, C.POINTER(hbi_multi_stats_t)]
        L.hbi_steady_state.argtypes = [i, vp, vp, vp, vp, d, d, vp, vp, vp]
        L.hbi_rhs.argtypes = [vp, C.POINTER(hbi_friction), vp, vp, vp, vp]
        L.hbi_rhs_vec.argtypes = [vp, C.POINTER(hbi_friction), vp, vp, vp, vp]
        L.hbi_rhs_vjp.argtypes = [vp, C.POINTER(hbi_friction), vp, vp, vp, vp, vp, vp]
        L.hbi_rk_fixed.argtypes = [vp, C.POINTER(hbi_friction), vp, vp, i, vp]
        L.hbi_adjoint.argtypes = [vp, C.POINTER(hbi_friction), vp, vp, i, i, vp, C.POINTER(d), vp, vp, vp, vp]
        L.hbi_step.argtypes = [vp, C.POINTER(hbi_friction), vp, vp, vp, d, i, vp, C.POINTER(i), vp]
        L.hbi_build_ensemble.argtypes = [i, C.POINTER(hbi_mesh), C.POINTER(hbi_elastic), C.POINTER(hbi_build_params),
                                         C.POINTER(vp)]
        L.hbi_step_ensemble.argtypes = [vp, C.POINTER(hbi_friction), vp, vp, vp, d, i, vp, vp, vp]
        L.hbi_step_vector.argtypes = [vp, C.POINTER(hbi_friction), vp, vp, vp, d, i, vp, vp, vp]
        L.hbi_stats.argtypes = [vp, C.POINTER(hbi_stats_t)]
        L.hbi_time_attempts.argtypes = [vp, C.POINTER(hbi_friction), vp, vp, vp, d, i, vp, vp]
        L.hbi_time_hmvm.argtypes = [vp, i, vp, vp]
        L.hbi_autotune.argtypes = [vp, i, vp, C.POINTER(d), vp]
        L.hbi_stalled_wait_status.argtypes = [vp]
        L.hbi_inject_failure.argtypes = [i, C.c_longlong]
        L.hbi_bounds_violations.argtypes = [C.POINTER(C.c_longlong)]
        L.hbi_destroy.argtypes = [vp]
        L.hbi_destroy.restype = None
        L.hbi_status_string.argtypes = [i]
        L.hbi_status_string.restype = C.c_char_p
        L.hbi_last_error.argtypes = []
        L.hbi_last_error.restype = C.c_char_p
        _lib = L
    return _lib


def _check(st, what):
    if st != 0:
        L = lib()
        raise HbiError(f"{what}: {L.hbi_status_string(st).decode()} ({L.hbi_last_error().decode()})")


def _ptrs(*specs):
    """Device addresses of the arrays given as (tensor, min_numel, name, optional) specs.  All
    are checked -- torch tensor, float64, contiguous, at least min_numel elements -- before
    any is required to be on the GPU, and before the library reads or writes one of them; an
    absent optional array gives None."""
    import torch
    for t, numel, what, optional in specs:
        if t is None:
            if optional:
                continue
            raise ValueError(f"{what}: required")
        if not isinstance(t, torch.Tensor):
            raise ValueError(f"{what}: expected a torch tensor, got {type(t).__name__}")
        if t.dtype != torch.float64:
            raise ValueError(f"{what}: expected float64, got {t.dtype}")
        if not t.is_contiguous():
            raise ValueError(f"{what}: expected a contiguous tensor")
        if t.numel() < numel:
            raise ValueError(f"{what}: {t.numel()} elements, needs at least {numel}")
    for t, _, what, _ in specs:
        if t is not None and not t.is_cuda:
            raise ValueError(f"{what}: expected a CUDA tensor")
    return tuple(None if t is None else t.data_ptr() for t, *_ in specs)


def _args(h, fric, *specs):
    """(hbi_friction, device addresses of specs); when the friction was built by friction(),
    its per-element arrays are checked against N with the others."""
    if isinstance(fric, tuple):
        f = fric[0]
        specs = tuple((t, h.n, f"friction {w}", False) for t, w in zip(fric[1], ("a", "b", "dc", "rake"))) + specs
        return f, _ptrs(*specs)[4:]
    return fric, _ptrs(*specs)


def _stream(stream):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return s.cuda_stream


class Handle:
    """Owner of an hbi_handle; destroyed with the object."""

    def __init__(self, ptr, n, op, n_models=1):
        self.ptr, self.n, self.op, self.n_models = ptr, n, op, n_models
        self.nin, self.nout = OP_NIN[op], OP_NOUT[op]

    def __del__(self):
        if getattr(self, "ptr", None) and _lib is not None:
            _lib.hbi_destroy(self.ptr)
            self.ptr = None

    def stats(self):
        return hbi_stats(self)


def _mesh(verts, rake):
    v = np.ascontiguousarray(verts, dtype=np.float64)
    r = None if rake is None else np.ascontiguousarray(rake, dtype=np.float64)
    m = hbi_mesh(v.shape[0], v.shape[1], v.ctypes.data, None if r is None else r.ctypes.data)
    return m, (v, r)


def hbi_build(verts, mu, nu, op, aca_eps, leaf_size, lattice_depth, storage, rake=None, eta=2.0,
              recompress_eps=0.0, transpose=False, half_space=False, multi_rhs=False):
    """Build the lattice H-matrix of the operator on the device.  half_space: the elements lie
    in the half space z < 0 with a traction-free surface z = 0 (every vertex z <= 0).
    multi_rhs: also pack the tensor-core panels of hbi_matvec_multi (fp16 or mixed storage)."""
    m, keep = _mesh(verts, rake)
    ek = hbi_elastic(mu, nu, op, int(bool(half_space)))
    bp = hbi_build_params(aca_eps, leaf_size, lattice_depth, eta, STORAGE.get(storage, storage), recompress_eps,
                          int(transpose), int(bool(multi_rhs)))
    out = C.c_void_p()
    _check(lib().hbi_build(C.byref(m), C.byref(ek), C.byref(bp), C.byref(out)), "hbi_build")
    return Handle(out.value, m.n_elem, op)


def hbi_build_shard(verts, mu, nu, op, aca_eps, leaf_size, lattice_depth, storage, p_rows, p_cols, rank, rake=None,
                    eta=2.0, recompress_eps=0.0, half_space=False):
    """The blocks of one rank of a p_rows x p_cols process grid (2D-cyclic over the lattice
    blocks, Sec. 3.2); hbi_matvec on it gives that rank's partial product."""
    m, keep = _mesh(verts, rake)
    ek = hbi_elastic(mu, nu, op, int(bool(half_space)))
    bp = hbi_build_params(aca_eps, leaf_size, lattice_depth, eta, STORAGE.get(storage, storage), recompress_eps, 0, 0)
    out = C.c_void_p()
    _check(lib().hbi_build_shard(C.byref(m), C.byref(ek), C.byref(bp), int(p_rows), int(p_cols), int(rank),
                                 C.byref(out)), "hbi_build_shard")
    return Handle(out.value, m.n_elem, op)


def hbi_build_ensemble(verts_list, mu, nu, op, aca_eps, leaf_size, lattice_depth, storage, rakes=None, eta=2.0,
                       recompress_eps=0.0, transpose=False, half_space=False, multi_rhs=False):
    """One handle for many independent models (block-diagonal operator, elements of the
    models concatenated in order).  Returns (Handle, model_starts)."""
    rakes = rakes if rakes is not None else [None] * len(verts_list)
    built = [_mesh(v, r) for v, r in zip(verts_list, rakes)]
    arr = (hbi_mesh * len(built))(*[m for m, _ in built])
    ek = hbi_elastic(mu, nu, op, int(bool(half_space)))
    bp = hbi_build_params(aca_eps, leaf_size, lattice_depth, eta, STORAGE.get(storage, storage), recompress_eps,
                          int(transpose), int(bool(multi_rhs)))
    out = C.c_void_p()
    _check(lib().hbi_build_ensemble(len(built), arr, C.byref(ek), C.byref(bp), C.byref(out)), "hbi_build_ensemble")
    starts = np.concatenate([[0], np.cumsum([m.n_elem for m, _ in built])]).astype(np.int64)
    return Handle(out.value, int(starts[-1]), op, len(built)), starts


def hbi_plan(verts, op, leaf_size, lattice_depth, rake=None, eta=2.0, mu=32e9, nu=0.25):
    """Host-only tree + partition: returns (perm, leaf_starts, blocks[n, 6])."""
    m, keep = _mesh(verts, rake)
    ek = hbi_elastic(mu, nu, op)
    bp = hbi_build_params(1e-4, leaf_size, lattice_depth, eta, HBI_FP32, 0.0)
    n = m.n_elem
    perm = np.zeros(n, dtype=np.int32)
    starts = np.zeros(n + 1, dtype=np.int32)
    nl, nb = C.c_int(0), C.c_int(0)
    L = lib()
    _check(L.hbi_plan(C.byref(m), C.byref(ek), C.byref(bp), perm.ctypes.data, starts.ctypes.data, C.byref(nl),
                      None, 0, C.byref(nb)), "hbi_plan")
    blocks = np.zeros((nb.value, 6), dtype=np.int64)
    _check(L.hbi_plan(C.byref(m), C.byref(ek), C.byref(bp), perm.ctypes.data, starts.ctypes.data, C.byref(nl),
                      blocks.ctypes.data, nb.value, C.byref(nb)), "hbi_plan")
    return perm, starts[: nl.value + 1], blocks


def hbi_lattice_owners(verts, op, leaf_size, lattice_depth, p_rows, p_cols, rake=None, eta=2.0, mu=32e9,
                       nu=0.25):
    """Host-only owner rank of every block of the hbi_plan partition on a p_rows x p_cols
    process grid (2D-cyclic over the lattice blocks, Sec. 3.2): ndarray[n_blocks] of int32."""
    m, keep = _mesh(verts, rake)
    ek = hbi_elastic(mu, nu, op)
    bp = hbi_build_params(1e-4, leaf_size, lattice_depth, eta, HBI_FP32, 0.0)
    nb = C.c_int(0)
    L = lib()
    _check(L.hbi_lattice_owners(C.byref(m), C.byref(ek), C.byref(bp), p_rows, p_cols, None, 0, C.byref(nb)),
           "hbi_lattice_owners")
    owners = np.zeros(nb.value, dtype=np.int32)
    _check(L.hbi_lattice_owners(C.byref(m), C.byref(ek), C.byref(bp), p_rows, p_cols, owners.ctypes.data, nb.value,
                                C.byref(nb)), "hbi_lattice_owners")
    return owners


def hbi_build_from_factors(verts, mu, nu, op, storage, perm, blocks, offsets, data, leaf_starts, rake=None,
                           transpose=False):
    m, keep = _mesh(verts, rake)
    ek = hbi_elastic(mu, nu, op)
    perm = np.ascontiguousarray(perm, dtype=np.int32)
    blocks = np.ascontiguousarray(blocks, dtype=np.int64)
    offsets = np.ascontiguousarray(offsets, dtype=np.int64)
    data = np.ascontiguousarray(data, dtype=np.float64)
    leaf_starts = np.ascontiguousarray(leaf_starts, dtype=np.int32)
    out = C.c_void_p()
    _check(lib().hbi_build_from_factors(C.byref(m), C.byref(ek), STORAGE.get(storage, storage), perm.ctypes.data,
                                        blocks.shape[0], blocks.ctypes.data, offsets.ctypes.data,
                                        data.ctypes.data, len(leaf_starts) - 1, leaf_starts.ctypes.data,
                                        int(bool(transpose)), C.byref(out)), "hbi_build_from_factors")
    return Handle(out.value, m.n_elem, op)


def _xy(h, x, y, transpose=False):
    nx, ny = (h.nout, h.nin) if transpose else (h.nin, h.nout)
    return _ptrs((x, nx * h.n, "x", False), (y, ny * h.n, "y", False))


def hbi_matvec(h, x, y, stream=None):
    px, py = _xy(h, x, y)
    _check(lib().hbi_matvec(h.ptr, px, py, _stream(stream)), "hbi_matvec")


def hbi_matvec_transpose(h, v, w, stream=None):
    """w = H^T v (handle built with transpose=True)."""
    pv, pw = _xy(h, v, w, transpose=True)
    _check(lib().hbi_matvec_transpose(h.ptr, pv, pw, _stream(stream)), "hbi_matvec_transpose")


def hbi_matvec_async(h, x, y, stream=None):
    px, py = _xy(h, x, y)
    _check(lib().hbi_matvec_async(h.ptr, px, py, _stream(stream)), "hbi_matvec_async")


def hbi_matvec_multi(h, k, X, Y, stream=None):
    """Y = H X for k right-hand sides on the tensor cores (handle built with multi_rhs=True):
    X is k x n_in N, Y is k x n_out N, each right-hand side laid out as hbi_matvec's x / y."""
    px, py = _ptrs((X, k * h.nin * h.n, "X", False), (Y, k * h.nout * h.n, "Y", False))
    _check(lib().hbi_matvec_multi(h.ptr, int(k), px, py, _stream(stream)), "hbi_matvec_multi")


def hbi_time_multi(h, k, n_rep, stream=None):
    """Average device ms of the multi-RHS product on the last hbi_matvec_multi input:
    dict(vt, uy, total)."""
    out = (C.c_double * 3)()
    _check(lib().hbi_time_multi(h.ptr, int(k), int(n_rep), C.cast(out, C.c_void_p), _stream(stream)),
           "hbi_time_multi")
    return dict(vt=out[0], uy=out[1], total=out[2])


def hbi_multi_stats(h):
    s = hbi_multi_stats_t()
    _check(lib().hbi_multi_stats(h.ptr, C.byref(s)), "hbi_multi_stats")
    return {k: getattr(s, k) for k, _ in s._fields_}


def hbi_matvec_noalloc(h, x, y, stream=None):
    """hbi_matvec with its scratch in the library's static device array (no allocation)."""
    px, py = _xy(h, x, y)
    _check(lib().hbi_matvec_noalloc(h.ptr, px, py, _stream(stream)), "hbi_matvec_noalloc")


def hbi_steady_state(V, a, b, sigma, f0, V0, phi, tau, stream=None):
    n = V.numel()
    p = _ptrs(*[(t, n, w, False) for t, w in ((V, "V"), (a, "a"), (b, "b"), (sigma, "sigma"), (phi, "phi"),
                                               (tau, "tau"))])
    _check(lib().hbi_steady_state(n, p[0], p[1], p[2], p[3], f0, V0, p[4], p[5], _stream(stream)),
           "hbi_steady_state")


def friction(a, b, dc, rake, f0, V0, Vpl, mu, cs):
    """hbi_friction from device tensors (kept alive by the returned tuple)."""
    p = _ptrs(*[(t, 1, w, False) for t, w in ((a, "a"), (b, "b"), (dc, "dc"), (rake, "rake"))])
    f = hbi_friction(*p, f0, V0, Vpl, mu, cs)
    return f, (a, b, dc, rake)


def hbi_rhs(h, fric, state, dydt, V=None, stream=None):
    n = h.n
    f, p = _args(h, fric, (state, 3 * n, "state", False), (dydt, 3 * n, "dydt", False), (V, n, "V", True))
    _check(lib().hbi_rhs(h.ptr, C.byref(f), *p, _stream(stream)), "hbi_rhs")


def hbi_rhs_vec(h, fric, state, dydt, V=None, stream=None):
    """Rake-free friction: state (phi, tau_s, tau_d, sigma: 4N) -> dydt (4N), V (V_s, V_d: 2N)."""
    n = h.n
    f, p = _args(h, fric, (state, 4 * n, "state", False), (dydt, 4 * n, "dydt", False), (V, 2 * n, "V", True))
    _check(lib().hbi_rhs_vec(h.ptr, C.byref(f), *p, _stream(stream)), "hbi_rhs_vec")


def hbi_rhs_vjp(h, fric, state, v, ybar, grad_a=None, grad_dc=None, stream=None):
    n = h.n
    f, p = _args(h, fric, (state, 3 * n, "state", False), (v, 3 * n, "v", False), (ybar, 3 * n, "ybar", False),
                 (grad_a, n, "grad_a", True), (grad_dc, n, "grad_dc", True))
    _check(lib().hbi_rhs_vjp(h.ptr, C.byref(f), *p, _stream(stream)), "hbi_rhs_vjp")


def hbi_rk_fixed(h, fric, state, dts, stream=None):
    """Fixed steps of the sizes dts (sequence of floats) from state (4N, updated in place)."""
    f, (ps,) = _args(h, fric, (state, 4 * h.n, "state", False))
    d = np.ascontiguousarray(dts, dtype=np.float64)
    _check(lib().hbi_rk_fixed(h.ptr, C.byref(f), ps, d.ctypes.data, len(d), _stream(stream)), "hbi_rk_fixed")


def hbi_adjoint(h, fric, state0, dts, target, grad_amb, grad_dc, checkpoint_every=50, state_final=None,
                stream=None):
    """Loss 1/2 |ln V(y_N) - target|^2 after the fixed steps dts, and its gradients with
    respect to a - b (at fixed b) and d_c (written into grad_amb, grad_dc).  Returns the loss."""
    n = h.n
    f, (p0, pt, pa, pd, pf) = _args(h, fric, (state0, 4 * n, "state0", False), (target, n, "target", False),
                                    (grad_amb, n, "grad_amb", False), (grad_dc, n, "grad_dc", False),
                                    (state_final, 4 * n, "state_final", True))
    d = np.ascontiguousarray(dts, dtype=np.float64)
    loss = C.c_double(0.0)
    _check(lib().hbi_adjoint(h.ptr, C.byref(f), p0, d.ctypes.data, len(d), checkpoint_every, pt, C.byref(loss),
                             pa, pd, pf, _stream(stream)), "hbi_adjoint")
    return loss.value


def sequence_loss(h, a_minus_b, dc, b, rake, consts, state0, dts, target, checkpoint_every=50):
    """L = 1/2 |ln V(y_N) - target|^2 of a fixed-step run as a differentiable function of the
    per-element a - b and d_c (torch tensors on the GPU); backward uses hbi_adjoint."""
    return _SequenceLoss.apply(a_minus_b, dc, h, b, rake, consts, state0, dts, target, checkpoint_every)


def _sequence_loss_cls():
    import torch

    class SequenceLoss(torch.autograd.Function):
        @staticmethod
        def forward(ctx, a_minus_b, dc, h, b, rake, consts, state0, dts, target, every):
            f0, V0, Vpl, mu, cs = consts
            a = (b + a_minus_b).contiguous()
            fr = friction(a, b.contiguous(), dc.contiguous(), rake.contiguous(), f0, V0, Vpl, mu, cs)
            g_amb, g_dc = torch.zeros_like(a), torch.zeros_like(a)
            loss = hbi_adjoint(h, fr, state0.contiguous(), dts, target.contiguous(), g_amb, g_dc, every)
            ctx.save_for_backward(g_amb, g_dc)
            return torch.tensor(loss, dtype=torch.float64, device=a.device)

        @staticmethod
        def backward(ctx, gout):
            g_amb, g_dc = ctx.saved_tensors
            return gout * g_amb, gout * g_dc, None, None, None, None, None, None, None, None

    return SequenceLoss


class _Lazy:
    def __init__(self, make):
        self.make, self.obj = make, None

    def apply(self, *args):
        if self.obj is None:
            self.obj = self.make()
        return self.obj.apply(*args)


_SequenceLoss = _Lazy(_sequence_loss_cls)


def hbi_step(h, fric, state, t, dt, eps_rk, n_steps, records=True, stream=None):
    """Returns (status, n_done, records ndarray[n_done, 5] of t, dt, vmax, rejects, mean tau/sigma)."""
    f, p = _args(h, fric, (state, 4 * h.n, "state", False), (t, 1, "t", False), (dt, 1, "dt", False))
    rec = (hbi_step_record * n_steps)() if records else None
    n_done = C.c_int(0)
    st = lib().hbi_step(h.ptr, C.byref(f), *p, eps_rk, n_steps,
                        C.cast(rec, C.c_void_p) if rec is not None else None, C.byref(n_done),
                        _stream(stream))
    out = None
    if rec is not None:
        out = np.array([(r.t, r.dt, r.vmax, r.rejects, r.mu_mean) for r in rec[: n_done.value]]).reshape(-1, 5)
    return st, n_done.value, out


def _step_models(fn, h, fric, state, n_state, t, dt, eps_rk, n_steps, records, stream):
    nm = h.n_models
    f, p = _args(h, fric, (state, n_state * h.n, "state", False), (t, nm, "t", False), (dt, nm, "dt", False))
    rec = (hbi_step_record * (nm * n_steps))() if records else None
    n_done = (C.c_int * nm)()
    st = fn(h.ptr, C.byref(f), *p, eps_rk, n_steps,
            C.cast(rec, C.c_void_p) if rec is not None else None, C.cast(n_done, C.c_void_p), _stream(stream))
    done = np.array(n_done[:], dtype=np.int64)
    out = None
    if rec is not None:
        out = [np.array([(r.t, r.dt, r.vmax, r.rejects, r.mu_mean) for r in rec[m * n_steps: m * n_steps + done[m]]])
               .reshape(-1, 5) for m in range(nm)]
    return st, done, out


def hbi_step_ensemble(h, fric, state, t, dt, eps_rk, n_steps, records=True, stream=None):
    """All models of an ensemble handle.  t, dt: device tensors of n_models doubles.
    Returns (status, n_done[n_models], records list of ndarray[n_done_m, 4] or None)."""
    return _step_models(lib().hbi_step_ensemble, h, fric, state, 4, t, dt, eps_rk, n_steps, records, stream)


def hbi_step_vector(h, fric, state, t, dt, eps_rk, n_steps, records=True, stream=None):
    """Rake-free friction: state (phi, tau_s, tau_d, sigma, D_s, D_d: 6N), t, dt one double
    per model (device).  Returns as hbi_step_ensemble."""
    return _step_models(lib().hbi_step_vector, h, fric, state, 6, t, dt, eps_rk, n_steps, records, stream)


def hbi_stats(h):
    s = hbi_stats_t()
    _check(lib().hbi_stats(h.ptr, C.byref(s)), "hbi_stats")
    return {k: getattr(s, k) for k, _ in s._fields_}


def hbi_time_hmvm(h, n_rep, stream=None):
    """Average device ms of the HMVM phases: dict(vt, uy, total)."""
    out = (C.c_double * 4)()
    _check(lib().hbi_time_hmvm(h.ptr, n_rep, C.cast(out, C.c_void_p), _stream(stream)), "hbi_time_hmvm")
    return dict(vt=out[0], uy=out[2], total=out[3])


def hbi_time_attempts(h, fric, state, t, dt, eps_rk, n_attempts, stream=None):
    """Per-kernel device times (ms per attempt) of adaptive Cash-Karp attempts from the given
    state: dict(products, stages, final, controller, commit, stop, eager_total, graph); the
    eager launches run each stage as a kernel of its own, the graph (the captured attempt of
    hbi_step) runs the stages inside the UY launches of the products."""
    n = h.n
    f, p = _args(h, fric, (state, 4 * n, "state", False), (t, 1, "t", False), (dt, 1, "dt", False))
    out = (C.c_double * 8)()
    _check(lib().hbi_time_attempts(h.ptr, C.byref(f), *p, eps_rk, int(n_attempts), C.cast(out, C.c_void_p),
                                   _stream(stream)), "hbi_time_attempts")
    keys = ("products", "stages", "final", "controller", "commit", "stop", "eager_total", "graph")
    return {k: out[i] for i, k in enumerate(keys)}


HBI_INJECT_NONE, HBI_INJECT_ALLOC, HBI_INJECT_ACA = 0, 1, 2


def hbi_inject_failure(what, count=0):
    """Host-side failure injection for error-path tests (see include/hbi.h)."""
    _check(lib().hbi_inject_failure(int(what), int(count)), "hbi_inject_failure")


def hbi_bounds_violations():
    """Table or index violations the bounds-checked build counted since the last call (it
    reads and clears the device counter); raises HbiError in the normal build."""
    v = C.c_longlong(0)
    _check(lib().hbi_bounds_violations(C.byref(v)), "hbi_bounds_violations")
    return v.value


def hbi_autotune(h, n_rep=10, stream=None):
    """Time the launch configurations of the handle's HMVM and keep the fastest.
    Returns dict(uy_rows, uy_ctas_per_sm, vt_pass_cost, ms)."""
    out = (C.c_int * 3)()
    ms = C.c_double(0.0)
    _check(lib().hbi_autotune(h.ptr, n_rep, C.cast(out, C.c_void_p), C.byref(ms), _stream(stream)), "hbi_autotune")
    return dict(uy_rows=out[0], uy_ctas_per_sm=out[1], vt_pass_cost=out[2], ms=ms.value)


def hbi_stalled_wait_status(stream=None):
    """Status of a device wait that can never complete (expected: HBI_ERR_TIMEOUT = -8)."""
    return lib().hbi_stalled_wait_status(_stream(stream))


def events(records, vth=1e-3):
    """(start time, peak max slip rate) of each event in step records (t, dt, vmax, ...): an
    event starts when the maximum slip rate exceeds vth and ends when it drops below."""
    rec = np.asarray(records)
    out, k = [], 0
    while k < len(rec):
        if rec[k, 2] > vth:
            k1 = k
            while k1 + 1 < len(rec) and rec[k1 + 1, 2] > vth:
                k1 += 1
            out.append((float(rec[k, 0]), float(rec[k:k1 + 1, 2].max())))
            k = k1 + 1
        else:
            k += 1
    return out


def checkpoint_save(path, state, t, dt, **build):
    """FP64 dump of a run (state phi, tau, sigma, D; t; dt) and the build parameters that
    rebuild the same handle (the build is deterministic), to resume bit for bit."""
    np.savez(path, state=state.detach().cpu().numpy(), t=t.detach().cpu().numpy(),
             dt=dt.detach().cpu().numpy(), **{k: np.asarray(v) for k, v in build.items()})


def checkpoint_load(path):
    """(state, t, dt, build dict) as numpy arrays, from checkpoint_save."""
    d = np.load(path)
    build = {k: d[k] for k in d.files if k not in ("state", "t", "dt")}
    return d["state"], d["t"], d["dt"], build


def status_string(st):
    return lib().hbi_status_string(st).decode()
