// Test infrastructure: the library's element-wise rate-and-state functions
// (hbi_ode_math.cuh, __host__ __device__) run on the host, so that the CPU tests can compare
// the CUDA path's right-hand side with the oracle's without a GPU.
//
// usage: host_rhs <in.bin> <out.bin>
//   step control (vec = 2): in int32 n, op, 2; float64 (err, eps_RK, dt)[n];
//                           out float64 (accept, dt_new)[n]
//   right-hand side (vec = 0 or 1):
//   in:  int32 n, op, vec; float64 f0, V0, Vpl, eta; float64 a[n], b[n], dc[n], rake[n];
//        float64 state[nc][n] (nc = 3: phi, tau, sigma; vec: nc = 4: phi, tau_s, tau_d, sigma);
//        float64 s[n][n_out] (the product of the slip-rate deficit, element by element)
//   out: float64 dydt[nc][n]; float64 V[n] (vec: V_s[n], V_d[n])
#include <cstdio>
#include <vector>

#include "../paper_2110_12165_gb300/csrc/hbi_ode_math.cuh"

template <typename T>
static bool rd(FILE *f, T *p, size_t n) { return fread(p, sizeof(T), n, f) == n; }

int main(int argc, char **argv) {
    if (argc != 3) return 1;
    FILE *f = fopen(argv[1], "rb");
    if (!f) return 1;
    int hdr[3];
    if (!rd(f, hdr, 3)) return 1;
    const int n = hdr[0], op = hdr[1], vec = hdr[2], nc = vec ? 4 : 3;
    if (vec == 2) {   // step control
        std::vector<double> in(3 * (size_t)n), out(2 * (size_t)n);
        if (!rd(f, in.data(), in.size())) return 1;
        fclose(f);
        for (int i = 0; i < n; ++i) {
            double dt_new;
            out[2 * i] = hbi::step_control(in[3 * i], in[3 * i + 1], in[3 * i + 2], dt_new);
            out[2 * i + 1] = dt_new;
        }
        FILE *o = fopen(argv[2], "wb");
        if (!o) return 1;
        fwrite(out.data(), sizeof(double), out.size(), o);
        fclose(o);
        return 0;
    }
    double c[4];
    if (!rd(f, c, 4)) return 1;
    const int nin = (op == HBI_OP_VEC_SHEAR || op == HBI_OP_VEC_FULL) ? 2 : 1;
    const int nout = op == HBI_OP_RAKE_SHEAR ? 1 : (op == HBI_OP_VEC_FULL ? 3 : 2);
    std::vector<double> a(n), b(n), dc(n), rake(n), y((size_t)nc * n), s((size_t)nout * n);
    if (!rd(f, a.data(), n) || !rd(f, b.data(), n) || !rd(f, dc.data(), n) || !rd(f, rake.data(), n) ||
        !rd(f, y.data(), y.size()) || !rd(f, s.data(), s.size()))
        return 1;
    fclose(f);
    std::vector<double> inv_a(n), inv_b(n), b_dc(n), cr(n), sr(n);
    for (int i = 0; i < n; ++i) {
        inv_a[i] = 1.0 / a[i]; inv_b[i] = 1.0 / b[i]; b_dc[i] = b[i] / dc[i];
        cr[i] = std::cos(rake[i]); sr[i] = std::sin(rake[i]);
    }
    hbi::OdeArgs A{};
    A.n = n; A.nin = nin; A.nout = nout;
    A.inv_a = inv_a.data(); A.inv_b = inv_b.data(); A.b_dc = b_dc.data();
    A.cr = cr.data(); A.sr = sr.data();
    A.f0 = c[0]; A.V0 = c[1]; A.Vpl = c[2]; A.eta = c[3];
    A.yp = s.data(); A.acc_double = 1;
    std::vector<double> dy((size_t)nc * n), V((size_t)(vec ? 2 : 1) * n);
    for (int i = 0; i < n; ++i) {
        if (!vec) {
            double dV, dphi, dtau, dsig;
            const double Vi = hbi::slip_rate(y[i], y[n + i], y[2 * (size_t)n + i], inv_a[i], A.V0, dV);
            hbi::rhs_elem(A, i, y[i], y[n + i], y[2 * (size_t)n + i], Vi, dV, dphi, dtau, dsig);
            dy[i] = dphi; dy[n + i] = dtau; dy[2 * (size_t)n + i] = dsig;
            V[i] = Vi;
        } else {
            const double phi = y[i], ts = y[n + i], td = y[2 * (size_t)n + i], sig = y[3 * (size_t)n + i];
            double tn, ux, uy, g1, dphi, dts, dtd, dsig;
            hbi::traction_dir(ts, td, cr[i], sr[i], tn, ux, uy);
            const double g = hbi::slip_rate(phi, tn, sig, inv_a[i], A.V0, g1);
            hbi::rhs_vec_elem(A, i, phi, ts, td, sig, g, g1, dphi, dts, dtd, dsig);
            dy[i] = dphi; dy[n + i] = dts; dy[2 * (size_t)n + i] = dtd; dy[3 * (size_t)n + i] = dsig;
            V[i] = g * ux; V[n + i] = g * uy;
        }
    }
    FILE *o = fopen(argv[2], "wb");
    if (!o) return 1;
    fwrite(dy.data(), sizeof(double), dy.size(), o);
    fwrite(V.data(), sizeof(double), V.size(), o);
    fclose(o);
    return 0;
}
