"""FP64 CPU oracle for the BEM / lattice-H-matrix hot path (test infrastructure only).

Only tests/, `__graft_entry__.smoke()` and the CPU-baseline leg of `bench.py` may import
this package.  The numerics live in `hbi_oracle.c` (plain C, FP64); this module compiles
it with gcc and exposes it through ctypes.  It shares no code with the CUDA library.

Parity status of each function (what pins it) is recorded in the tests under
tests/test_oracle_*.py; every oracle function has at least one pin there.
"""
import ctypes as C
import os
import subprocess

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "hbi_oracle.c")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "libhbi_oracle.so")

OP_RAKE_SHEAR, OP_RAKE_SHEAR_NORMAL, OP_VEC_SHEAR, OP_VEC_FULL = 0, 1, 2, 3
OP_NIN = {0: 1, 1: 1, 2: 2, 3: 2}
OP_NOUT = {0: 1, 1: 2, 2: 2, 3: 3}
HALF_SPACE = 16   # flag on an operator kind: the half-space form (free surface z = 0)


def build(force=False):
    """Compile the oracle shared library (gcc, -O2, OpenMP)."""
    os.makedirs(BUILD, exist_ok=True)
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= os.path.getmtime(SRC):
        return LIB
    tmp = LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-fPIC", "-shared", "-fopenmp", "-std=c11", "-o", tmp, SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, LIB)
    return LIB


_lib = None
_dp = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")
_ip = np.ctypeslib.ndpointer(dtype=np.int32, flags="C_CONTIGUOUS")
_lp = np.ctypeslib.ndpointer(dtype=np.int64, flags="C_CONTIGUOUS")


class _Fric(C.Structure):
    _fields_ = [("a", C.c_void_p), ("b", C.c_void_p), ("dc", C.c_void_p), ("rake", C.c_void_p),
                ("tau_dot", C.c_void_p), ("sig_dot", C.c_void_p),
                ("f0", C.c_double), ("V0", C.c_double), ("Vpl", C.c_double),
                ("mu", C.c_double), ("cs", C.c_double)]


def lib():
    global _lib
    if _lib is None:
        L = C.CDLL(build())
        L.ho_gauss_legendre.argtypes = [_dp, _dp]
        L.ho_elem_frames.argtypes = [C.c_int, C.c_int, _dp, _dp, _dp, _dp, _dp, _dp]
        L.ho_kelvin_G.argtypes = [_dp, C.c_double, C.c_double, _dp]
        L.ho_kelvin_dG.argtypes = [_dp, C.c_double, C.c_double, _dp]
        L.ho_stress_polygon.argtypes = [C.c_int, _dp, C.c_int, _dp, C.c_double, C.c_double, _dp, _dp]
        L.ho_stress_polygon_hs.argtypes = [C.c_int, _dp, C.c_int, _dp, C.c_double, C.c_double, _dp, C.c_int, _dp]
        L.ho_halfspace_G.argtypes = [_dp, _dp, C.c_double, C.c_double, C.c_int, _dp]
        L.ho_set_halfspace_ratio.argtypes = [C.c_double]
        L.ho_set_halfspace_ratio.restype = None
        L.ho_set_halfspace_adaptive.argtypes = [C.c_int]
        L.ho_set_halfspace_adaptive.restype = None
        L.ho_pair_entries.argtypes = [C.c_int, C.c_int, _dp, C.c_double, C.c_double, C.c_int, _dp,
                                      C.c_int, _ip, _ip, _dp]
        L.ho_dense_rows.argtypes = [C.c_int, C.c_int, _dp, C.c_double, C.c_double, C.c_int, _dp,
                                    C.c_int, _ip, _dp, _dp]
        L.ho_set_sample_lattice_row.argtypes = [C.c_int]
        L.ho_set_sample_lattice_row.restype = None
        L.ho_build.restype = C.c_void_p
        L.ho_build.argtypes = [C.c_int, C.c_int, _dp, C.c_double, C.c_double, C.c_int, _dp,
                               C.c_double, C.c_int, C.c_int, C.c_double]
        L.ho_free.argtypes = [C.c_void_p]
        L.ho_info.argtypes = [C.c_void_p, _lp]
        L.ho_export.argtypes = [C.c_void_p, _ip, _lp, _dp, _lp, _dp, _lp]
        L.ho_hmatvec.argtypes = [C.c_void_p, _dp, _dp]
        L.ho_hmatvec_perm.argtypes = [C.c_void_p, _dp, _dp]
        L.ho_steady_state.argtypes = [C.c_int, _dp, _dp, _dp, _dp, C.c_double, C.c_double, _dp, _dp]
        L.ho_loading.argtypes = [C.c_void_p, _dp, C.c_double, _dp, _dp]
        L.ho_rhs.argtypes = [C.c_void_p, C.POINTER(_Fric), _dp, _dp, _dp]
        L.ho_fixed_loss_cs.argtypes = [C.c_void_p, C.POINTER(_Fric), C.c_void_p, C.c_void_p, C.c_double, _dp, _dp,
                                       C.c_int, _dp, _dp]
        L.ho_rhs_rows.argtypes = [C.c_int, C.POINTER(_Fric), C.c_int, _dp, C.c_int, _ip, _dp, _dp]
        L.ho_rk_attempt.argtypes = [C.c_void_p, C.POINTER(_Fric), _dp, C.c_double, _dp,
                                    C.POINTER(C.c_double)]
        L.ho_run.argtypes = [C.c_void_p, C.POINTER(_Fric), _dp, _dp, C.POINTER(C.c_double),
                             C.POINTER(C.c_double), C.c_double, C.c_int, _dp]
        L.ho_aca_matrix.argtypes = [C.c_int, C.c_int, _dp, C.c_double, C.c_int, _dp, _dp]
        L.ho_rhs_vec.argtypes = [C.c_void_p, C.POINTER(_Fric), _dp, _dp, _dp]
        L.ho_rk_attempt_vec.argtypes = [C.c_void_p, C.POINTER(_Fric), _dp, C.c_double, _dp,
                                        C.POINTER(C.c_double)]
        L.ho_run_vec.argtypes = [C.c_void_p, C.POINTER(_Fric), _dp, _dp, C.POINTER(C.c_double),
                                 C.POINTER(C.c_double), C.c_double, C.c_int, _dp]
        L.ho_slip_rate.argtypes = [C.c_int, _dp, _dp, _dp, _dp, C.c_double, _dp, _dp]
        L.ho_cash_karp_tableau.argtypes = [_dp, _dp, _dp, _dp]
        L.ho_controller.argtypes = [C.c_double, C.c_double, C.c_double, C.POINTER(C.c_double)]
        L.ho_ck_linear_step.argtypes = [C.c_double, C.c_double, C.c_double, C.POINTER(C.c_double),
                                        C.POINTER(C.c_double)]
        _lib = L
    return _lib


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def num_threads():
    return lib().ho_num_threads()


def set_num_threads(k):
    """Threads of the oracle's OpenMP loops from now on; returns the previous count."""
    return lib().ho_set_num_threads(int(k))


# --------------------------------------------------------------------- geometry
def gauss_legendre():
    x, w = np.zeros(8), np.zeros(8)
    lib().ho_gauss_legendre(x, w)
    return x, w


def elem_frames(verts):
    v = _f64(verts)
    n, nv = v.shape[0], v.shape[1]
    out = [np.zeros((n, 3)) for _ in range(4)] + [np.zeros(n)]
    lib().ho_elem_frames(n, nv, v.reshape(-1), *out)
    return dict(centroid=out[0], normal=out[1], strike=out[2], dip=out[3], area=out[4])


def kelvin_G(r, mu, nu):
    G = np.zeros(9)
    lib().ho_kelvin_G(_f64(r), mu, nu, G)
    return G.reshape(3, 3)


def kelvin_dG(r, mu, nu):
    d = np.zeros(27)
    lib().ho_kelvin_dG(_f64(r), mu, nu, d)
    return d.reshape(3, 3, 3)


def stress_polygon(P, b, mu, nu, x):
    """Stress tensors (nb, 3, 3) at x from uniform slip vectors b (nb, 3) on polygon P."""
    P = _f64(P)
    b = _f64(np.atleast_2d(b))
    sig = np.zeros(9 * b.shape[0])
    rc = lib().ho_stress_polygon(P.shape[0], P.reshape(-1), b.shape[0], b.reshape(-1), mu, nu,
                                 _f64(x), sig)
    if rc != 0:
        raise ValueError("receiver lies on the element boundary")
    return sig.reshape(-1, 3, 3)


def halfspace_G(x, xi, mu, nu, with_kelvin=True):
    """Displacement G[k, p] at x from a unit force along axis p at xi in the half space
    z < 0 with a traction-free surface z = 0 (Mindlin 1936); the correction to Kelvin's
    solution alone with with_kelvin=False."""
    G = np.zeros(9)
    if lib().ho_halfspace_G(_f64(x), _f64(xi), mu, nu, int(with_kelvin), G) != 0:
        raise ValueError("points must lie in the closed half space, not both on the surface")
    return G.reshape(3, 3)


def stress_polygon_hs(P, b, mu, nu, x, corr_only=False):
    """Half-space stress tensors (nb, 3, 3) at x (z <= 0) from uniform slip vectors b (nb, 3)
    on the buried polygon P: the full-space stress plus the Mindlin correction (or the
    correction alone)."""
    P = _f64(P)
    b = _f64(np.atleast_2d(b))
    sig = np.zeros(9 * b.shape[0])
    rc = lib().ho_stress_polygon_hs(P.shape[0], P.reshape(-1), b.shape[0], b.reshape(-1), mu, nu, _f64(x),
                                    int(corr_only), sig)
    if rc != 0:
        raise ValueError("element not below the surface, or receiver on its boundary")
    return sig.reshape(-1, 3, 3)


def set_halfspace_ratio(r):
    """Subdivision rule of the half-space element quadrature (triangle diameter over its
    vertical distance to the receiver's image; default 0.5)."""
    lib().ho_set_halfspace_ratio(float(r))


def set_halfspace_adaptive(on):
    """1 (default): the Gauss-Legendre order of the half-space element quadrature follows the
    distance to the image; 0: the 8 x 8 rule everywhere."""
    lib().ho_set_halfspace_adaptive(int(bool(on)))


def _op_code(op, half_space):
    return op | (HALF_SPACE if half_space else 0)


def pair_entries(mesh, op, recv, src, mu, nu, rake=None, half_space=False):
    v = _f64(mesh.verts)
    n = v.shape[0]
    rk = _f64(rake if rake is not None else np.zeros(n))
    recv = np.ascontiguousarray(recv, dtype=np.int32)
    src = np.ascontiguousarray(src, dtype=np.int32)
    out = np.zeros(len(recv) * OP_NIN[op] * OP_NOUT[op])
    rc = lib().ho_pair_entries(n, v.shape[1], v.reshape(-1), mu, nu, _op_code(op, half_space), rk, len(recv),
                               recv, src, out)
    if rc != 0:
        raise ValueError("singular receiver")
    return out.reshape(len(recv), OP_NOUT[op], OP_NIN[op])


def dense_rows(mesh, op, rows, x, mu, nu, rake=None, half_space=False):
    """Rows of the dense operator (Eqs. 5-6) applied to x (component-major, original order).

    Returns (len(rows), n_out)."""
    v = _f64(mesh.verts)
    n = v.shape[0]
    rk = _f64(rake if rake is not None else np.zeros(n))
    rows = np.ascontiguousarray(rows, dtype=np.int32)
    y = np.zeros(len(rows) * OP_NOUT[op])
    rc = lib().ho_dense_rows(n, v.shape[1], v.reshape(-1), mu, nu, _op_code(op, half_space), rk, len(rows), rows,
                             _f64(x), y)
    if rc != 0:
        raise ValueError("singular receiver")
    return y.reshape(len(rows), OP_NOUT[op])


def rhs_rows(op, F, y, rows, s_rows):
    """dy/dt (Eqs. 8, 10, 12, 13) at the elements rows of the state y = (phi, tau, sigma) (3n),
    given their stress rates s_rows (len(rows), n_out), e.g. dense_rows of the slip-rate
    deficit (V - V_pl) r, which includes the backslip loading.  Returns (len(rows), 3)."""
    y = _f64(y)
    n = len(y) // 3
    z = np.zeros(n)
    keep = [_f64(F.a), _f64(F.b), _f64(F.dc), _f64(F.rake), z]
    f = _Fric(*[k.ctypes.data for k in keep[:4]], z.ctypes.data, z.ctypes.data, F.f0, F.V0, F.Vpl, F.mu, F.cs)
    rows = np.ascontiguousarray(rows, dtype=np.int32)
    out = np.zeros(3 * len(rows))
    if lib().ho_rhs_rows(op, C.byref(f), n, y, len(rows), rows, _f64(s_rows).reshape(-1), out) != 0:
        raise ValueError("row index out of range")
    return out.reshape(len(rows), 3)


def dense_matvec(mesh, op, x, mu, nu, rake=None, half_space=False):
    """Full dense operator applied to x; returns component-major (n_out * n)."""
    n = mesh.n_elem
    y = dense_rows(mesh, op, np.arange(n), x, mu, nu, rake, half_space)
    return np.ascontiguousarray(y.T).reshape(-1)


# ---------------------------------------------------------------- H-matrix
class HMatrix:
    """Oracle lattice H-matrix (Sec. 3.1-3.2): tree, partition, ACA factors, Eq. 20."""

    def __init__(self, mesh, op, eps, leaf, lattice_depth, mu, nu, rake=None, eta=2.0, half_space=False,
                 sample_lattice_row=None):
        """sample_lattice_row = a: build only the blocks whose rows lie in lattice cluster a (a
        bounded sample of the operator for timing: its product is the whole product's rows
        of that lattice row, zero elsewhere)."""
        self.mesh = mesh
        self._verts = _f64(mesh.verts)
        n = mesh.n_elem
        self.n, self.op = n, op
        self.nin, self.nout = OP_NIN[op], OP_NOUT[op]
        self.rake = _f64(rake if rake is not None else np.zeros(n))
        self.mu, self.nu, self.half_space = mu, nu, half_space
        self.sample_lattice_row = sample_lattice_row
        lib().ho_set_sample_lattice_row(-1 if sample_lattice_row is None else int(sample_lattice_row))
        try:
            self._h = lib().ho_build(n, self._verts.shape[1], self._verts.reshape(-1), mu, nu,
                                     _op_code(op, half_space), self.rake, eps, leaf, lattice_depth, eta)
        finally:
            lib().ho_set_sample_lattice_row(-1)
        info = np.zeros(8, dtype=np.int64)
        lib().ho_info(self._h, info)
        self.n_clusters, self.n_blocks, self.n_data, self.n_lattice = map(int, info[1:5])
        self.n_lowrank = int(info[7])

    def __del__(self):
        if getattr(self, "_h", None):
            lib().ho_free(self._h)
            self._h = None

    def export(self):
        perm = np.zeros(self.n, dtype=np.int32)
        cl = np.zeros(6 * self.n_clusters, dtype=np.int64)
        box = np.zeros(6 * self.n_clusters)
        blk = np.zeros(8 * self.n_blocks, dtype=np.int64)
        data = np.zeros(max(self.n_data, 1))
        lat = np.zeros(max(self.n_lattice, 1), dtype=np.int64)
        lib().ho_export(self._h, perm, cl, box, blk, data, lat)
        return dict(perm=perm, clusters=cl.reshape(-1, 6), boxes=box.reshape(-1, 6),
                    blocks=blk.reshape(-1, 8), data=data[: self.n_data],
                    lattice=lat[: self.n_lattice])

    def matvec(self, x):
        x = _f64(x)
        y = np.zeros(self.nout * self.n)
        lib().ho_hmatvec(self._h, x, y)
        return y

    def matvec_perm(self, xp):
        y = np.zeros(self.nout * self.n)
        lib().ho_hmatvec_perm(self._h, _f64(xp), y)
        return y

    def storage_entries(self):
        return self.n_data

    def loading(self, rake, Vpl):
        td, sd = np.zeros(self.n), np.zeros(self.n)
        lib().ho_loading(self._h, _f64(rake), Vpl, td, sd)
        return td, sd

    def _fric(self, F, tau_dot, sig_dot):
        keep = [_f64(F.a), _f64(F.b), _f64(F.dc), _f64(F.rake), _f64(tau_dot), _f64(sig_dot)]
        f = _Fric(*[k.ctypes.data for k in keep], F.f0, F.V0, F.Vpl, F.mu, F.cs)
        return f, keep

    def rhs(self, F, y, tau_dot, sig_dot):
        f, keep = self._fric(F, tau_dot, sig_dot)
        dy, V = np.zeros(3 * self.n), np.zeros(self.n)
        lib().ho_rhs(self._h, C.byref(f), _f64(y), dy, V)
        return dy, V

    def rk_attempt(self, F, y, dt, tau_dot, sig_dot):
        f, keep = self._fric(F, tau_dot, sig_dot)
        yn, err = np.zeros(3 * self.n), C.c_double()
        lib().ho_rk_attempt(self._h, C.byref(f), _f64(y), dt, yn, C.byref(err))
        return yn, err.value

    def fixed_loss(self, F, y0, dts, target, a_dir=None, dc_dir=None, step=1e-30):
        """Loss 1/2 |ln V(y_N) - target|^2 after fixed Cash-Karp steps dts from y0 (3n), with
        the loading of Eqs. 21-22, and its derivative along (a_dir, dc_dir) (b fixed) by the
        complex step: returns (L, dL)."""
        td, sd = self.loading(F.rake, F.Vpl)
        f, keep = self._fric(F, td, sd)
        ad = None if a_dir is None else _f64(a_dir)
        dd = None if dc_dir is None else _f64(dc_dir)
        out = np.zeros(2)
        dts = _f64(dts)
        lib().ho_fixed_loss_cs(self._h, C.byref(f), None if ad is None else ad.ctypes.data,
                               None if dd is None else dd.ctypes.data, step, _f64(y0), dts, len(dts),
                               _f64(target), out)
        return float(out[0]), float(out[1])

    def fixed_loss_grad(self, F, y0, dts, target, elements):
        """dL/da_j (b fixed) and dL/d(d_c)_j for the listed elements j, one complex-step run
        each (exact to rounding)."""
        ga, gd = [], []
        for j in elements:
            e = np.zeros(self.n)
            e[j] = 1.0
            ga.append(self.fixed_loss(F, y0, dts, target, a_dir=e)[1])
            gd.append(self.fixed_loss(F, y0, dts, target, dc_dir=e)[1])
        return np.array(ga), np.array(gd)

    def rhs_vec(self, F, y):
        """Rake-free friction: dy/dt of y = (phi, tau_s, tau_d, sigma) and V = (V_s, V_d); the
        plate motion is V_pl along F.rake (the loading direction)."""
        z = np.zeros(self.n)
        f, keep = self._fric(F, z, z)
        dy, V = np.zeros(4 * self.n), np.zeros(2 * self.n)
        if lib().ho_rhs_vec(self._h, C.byref(f), _f64(y), dy, V) != 0:
            raise ValueError("rake-free friction needs a 2-component operator")
        return dy, V

    def rk_attempt_vec(self, F, y, dt):
        z = np.zeros(self.n)
        f, keep = self._fric(F, z, z)
        yn, err = np.zeros(4 * self.n), C.c_double()
        lib().ho_rk_attempt_vec(self._h, C.byref(f), _f64(y), dt, yn, C.byref(err))
        return yn, err.value

    def run_vec(self, F, y, D, t, dt, eps_rk, n_steps):
        """Rake-free friction: n_steps accepted steps of y (4n) and D (2n)."""
        z = np.zeros(self.n)
        f, keep = self._fric(F, z, z)
        y = _f64(y).copy()
        D = _f64(D).copy()
        tt, dd = C.c_double(t), C.c_double(dt)
        rec = np.zeros(4 * n_steps)
        k = lib().ho_run_vec(self._h, C.byref(f), y, D, C.byref(tt), C.byref(dd), eps_rk, n_steps, rec)
        if k < 0:
            raise FloatingPointError("RK step size underflow")
        return y, D, tt.value, dd.value, rec.reshape(n_steps, 4)

    def run(self, F, y, D, t, dt, eps_rk, n_steps, tau_dot, sig_dot):
        """Advance n_steps accepted steps; returns (y, D, t, dt, records[n,4])."""
        f, keep = self._fric(F, tau_dot, sig_dot)
        y = _f64(y).copy()
        D = _f64(D).copy()
        tt, dd = C.c_double(t), C.c_double(dt)
        rec = np.zeros(4 * n_steps)
        k = lib().ho_run(self._h, C.byref(f), y, D, C.byref(tt), C.byref(dd), eps_rk, n_steps, rec)
        if k < 0:
            raise FloatingPointError("RK step size underflow")
        return y, D, tt.value, dd.value, rec.reshape(n_steps, 4)


# ------------------------------------------------------------------ ODE helpers
def steady_state(V, a, b, sig, f0, V0):
    n = len(V)
    phi, tau = np.zeros(n), np.zeros(n)
    lib().ho_steady_state(n, _f64(V), _f64(a), _f64(b), _f64(sig), f0, V0, phi, tau)
    return phi, tau


def aca_matrix(A, eps, rmax=None):
    """The oracle's ACA (Sec. 3.1.2) on an explicit matrix: returns (U, V) or None if capped."""
    A = _f64(A)
    m, nc = A.shape
    rmax = rmax or min(m, nc)
    U, V = np.zeros(m * rmax), np.zeros(nc * rmax)
    r = lib().ho_aca_matrix(m, nc, A.reshape(-1), eps, rmax, U, V)
    if r < 0:
        return None
    return U[: m * r].reshape(r, m).T, V[: nc * r].reshape(r, nc).T


def slip_rate(phi, tau, sig, a, V0):
    """V from Eq. 7 and the partials of Eqs. 13a-c: returns V, (n, 3) [dV/dtau, dV/dsig, dV/dphi]."""
    n = len(phi)
    V, P = np.zeros(n), np.zeros(3 * n)
    lib().ho_slip_rate(n, _f64(phi), _f64(tau), _f64(sig), _f64(a), V0, V, P)
    return V, P.reshape(n, 3)


def cash_karp_tableau():
    c, a, b5, b4 = np.zeros(6), np.zeros(30), np.zeros(6), np.zeros(6)
    lib().ho_cash_karp_tableau(c, a, b5, b4)
    return c, a.reshape(6, 5), b5, b4


def controller(err, eps, dt):
    out = C.c_double()
    acc = lib().ho_controller(err, eps, dt, C.byref(out))
    return bool(acc), out.value


def ck_linear_step(lam, y0, dt):
    y5, err = C.c_double(), C.c_double()
    lib().ho_ck_linear_step(lam, y0, dt, C.byref(y5), C.byref(err))
    return y5.value, err.value
