// Element-wise rate-and-state arithmetic (Eqs. 7-13, 21-22, and the rake-free form), host
// and device: the stage kernels of hbi_ode.cu use these functions on the device, and the CPU
// tests compile them for the host to check them against the oracle without a GPU.
#pragma once

#include <cuda_runtime.h>

#include <cmath>

#include "hbi_internal.h"

namespace hbi {

struct OdeArgs {
    int n, nin, nout;
    double *y, *D, *ys, *Vs, *Vold, *k;     // permuted FP64 state and stage storage
    double *dVs, *dVold;                    // dV/dtau at the stage state and at y
    const double *inv_a, *inv_b, *b_dc;     // friction: 1/a, 1/b, b/d_c
    const double *cr, *sr;                  // rake cosine/sine
    double f0, V0, Vpl, eta;                // eta = mu / (2 c_s)
    void *xt;                               // HMVM input head (accumulation type)
    const void *yp;                         // HMVM output
    int acc_double;
    int n_models, rec_cap;
    const int *model;                       // model index of each element
    StepCtl *ctl;                           // one per model
    GlobalCtl *g;
    int *mskip;                             // 2 x n_models product skip flags (first stage | others)
    hbi_step_record *rec;                   // n_models x rec_cap
    // adjoint support: with store != 0 the stage kernels keep every stage state Y_s (6 x 3N)
    // and the product outputs S_s (6 x n_out N, FP64) of the step for the reverse sweep
    int store;
    double *st_Y, *st_S;
};

// Eq. 7 solved for V: V = 2 V0 exp(-phi/a) sinh(tau/(a sigma)), written as a difference of
// two exponentials so neither factor can overflow; with it dV/dtau (Eq. 13a), which costs
// no further exponential.  FP64 divisions and exponentials are the expensive operations of
// the element-wise work, so the friction constants come as reciprocals and a stage state's
// V and dV/dtau are computed once, when the state is formed, and kept.
// tau / sigma (a friction coefficient) in fixed point 2^-40 for an exact, order-independent sum
// over the elements (|q| clamped to 2^20; a non-finite q counts as 0: its trial is rejected)
__host__ __device__ __forceinline__ long long mu_fixed(double q) {
    if (!(q == q) || !isfinite(q)) return 0;
    q = fmin(fmax(q, -1048576.0), 1048576.0);
    return (long long)llrint(q * 1099511627776.0);
}

// The two exponentials differ by the factor exp(2 q / a): once |2 q / a| > 40 the smaller one
// is below 4.3e-18 of the larger, under half an ulp of it, so the sum and the difference round
// to the larger alone and the smaller is not evaluated (the same bits, one exponential fewer;
// at frictional sliding q / a is about f0 / a, far above 20).
__host__ __device__ __forceinline__ double slip_rate(double phi, double tau, double sig, double inv_a, double V0,
                                            double &dVdtau, double &q) {
    const double inv_sig = 1.0 / sig;
    q = tau * inv_sig;   // the friction coefficient tau / sigma
    const double r = 2.0 * q * inv_a;
    double ep, em;
    if (r > 40.0) {
        ep = exp((q - phi) * inv_a);
        em = 0.0;
    } else if (r < -40.0) {
        ep = 0.0;
        em = exp((-q - phi) * inv_a);
    } else {
        ep = exp((q - phi) * inv_a);
        em = exp((-q - phi) * inv_a);
    }
    dVdtau = V0 * (ep + em) * inv_a * inv_sig;   // Eq. 13a
    return V0 * (ep - em);
}
__host__ __device__ __forceinline__ double slip_rate(double phi, double tau, double sig, double inv_a, double V0,
                                            double &dVdtau) {
    double q;
    return slip_rate(phi, tau, sig, inv_a, V0, dVdtau, q);
}

__host__ __device__ __forceinline__ void write_x(const OdeArgs &A, int i, double V) {
    const double dv = V - A.Vpl;
    if (A.nin == 1) {
        if (A.acc_double) ((double *)A.xt)[i] = dv;
        else ((float *)A.xt)[i] = (float)dv;
    } else {
        const double xs = dv * A.cr[i], xd = dv * A.sr[i];
        if (A.acc_double) { ((double *)A.xt)[2 * i] = xs; ((double *)A.xt)[2 * i + 1] = xd; }
        else { ((float *)A.xt)[2 * i] = (float)xs; ((float *)A.xt)[2 * i + 1] = (float)xd; }
    }
}

__host__ __device__ __forceinline__ double read_y(const OdeArgs &A, int64_t k) {
    return A.acc_double ? ((const double *)A.yp)[k] : (double)((const float *)A.yp)[k];
}

// shear rate (projected on the rake) and normal-stress rate from the HMVM output
__host__ __device__ __forceinline__ void stress_rates(const OdeArgs &A, int i, double &AV, double &BV) {
    const int64_t o = (int64_t)A.nout * i;
    if (A.nout == 1) { AV = read_y(A, o); BV = 0.0; return; }
    if (A.nin == 1) { AV = read_y(A, o); BV = read_y(A, o + 1); return; }   // (tau_r, sigma)
    AV = A.cr[i] * read_y(A, o) + A.sr[i] * read_y(A, o + 1);
    BV = A.nout == 3 ? read_y(A, o + 2) : 0.0;
}

// dy/dt at element i for stage state (phi, tau, sig) with slip rate V and q = tau / sig
// (Eqs. 8, 10, 12, 13)
__host__ __device__ __forceinline__ void rhs_elem_q(const OdeArgs &A, int i, double phi, double V, double dVdtau,
                                           double q, double &dphi, double &dtau, double &dsig) {
    double AV, BV;
    stress_rates(A, i, AV, BV);
    dphi = A.b_dc[i] * (A.V0 * exp((A.f0 - phi) * A.inv_b[i]) - V);   // Eq. 8
    dsig = BV;                                                          // Eq. 10 (+ loading)
    const double dVdsig = -q * dVdtau;                                  // Eq. 13b
    const double dVdphi = -V * A.inv_a[i];                              // Eq. 13c
    dtau = (AV - A.eta * (dVdsig * dsig + dVdphi * dphi)) / (1.0 + A.eta * dVdtau);   // Eq. 12
}
__host__ __device__ __forceinline__ void rhs_elem(const OdeArgs &A, int i, double phi, double tau, double sig, double V,
                                         double dVdtau, double &dphi, double &dtau, double &dsig) {
    rhs_elem_q(A, i, phi, V, dVdtau, tau / sig, dphi, dtau, dsig);
}

// Step control (Eqs. 14-15, read with the error ratio err/eps_RK carrying the exponents):
// reject unless err <= eps_RK, with dt' = max(dt/2, 0.9 dt (err/eps_RK)^-0.25) (dt/2 when err
// is NaN or infinite: a non-finite trial is rejected); otherwise accept with
// dt' = min(2 dt, 0.9 dt (err/eps_RK)^-0.2) (2 dt when err = 0).  Returns 1 on accept.
__host__ __device__ __forceinline__ int step_control(double err, double eps, double dt, double &dt_new) {
    if (!(err <= eps)) {
        const double d = 0.9 * dt * pow(err / eps, -0.25);
        dt_new = d > 0.5 * dt ? d : 0.5 * dt;   // NaN compares false: dt/2
        return 0;
    }
    dt_new = err > 0.0 ? fmin(2.0 * dt, 0.9 * dt * pow(err / eps, -0.2)) : 2.0 * dt;
    return 1;
}

// ------------------------------------------------------------- rake-free friction
// (the layouts and the 2x2 solve are described with the rake-free kernels in hbi_ode.cu)

// |tau| and its direction (the loading direction when the traction vanishes)
__host__ __device__ __forceinline__ void traction_dir(double ts, double td, double cr, double sr, double &tn, double &ux,
                                             double &uy) {
    tn = sqrt(ts * ts + td * td);
    if (tn > 0.0) {
        const double it = 1.0 / tn;
        ux = ts * it; uy = td * it;
    } else {
        ux = cr; uy = sr;
    }
}

// slip-rate deficit V - V_pl r as the product input
__host__ __device__ __forceinline__ void write_xv(const OdeArgs &A, int i, double vs, double vd) {
    const double xs = vs - A.Vpl * A.cr[i], xd = vd - A.Vpl * A.sr[i];
    if (A.acc_double) { ((double *)A.xt)[2 * i] = xs; ((double *)A.xt)[2 * i + 1] = xd; }
    else { ((float *)A.xt)[2 * i] = (float)xs; ((float *)A.xt)[2 * i + 1] = (float)xd; }
}

// the stage-state slip rate: g, (V_s, V_d) and g' into Vs / dVs
__host__ __device__ __forceinline__ void vec_state(const OdeArgs &A, int i, double phi, double ts, double td, double sig) {
    const int n = A.n;
    double tn, ux, uy, g1;
    traction_dir(ts, td, A.cr[i], A.sr[i], tn, ux, uy);
    const double g = slip_rate(phi, tn, sig, A.inv_a[i], A.V0, g1);
    A.Vs[i] = g; A.Vs[n + i] = g * ux; A.Vs[2 * n + i] = g * uy;
    A.dVs[i] = g1;
    write_xv(A, i, g * ux, g * uy);
}

// dy/dt of element i at stage state (phi, tau_s, tau_d, sigma) with slip-rate magnitude g and g'
__host__ __device__ __forceinline__ void rhs_vec_elem(const OdeArgs &A, int i, double phi, double ts, double td, double sig,
                                             double g, double g1, double &dphi, double &dts, double &dtd,
                                             double &dsig) {
    const int64_t o = (int64_t)A.nout * i;
    const double ss = read_y(A, o), sd = read_y(A, o + 1);
    dsig = A.nout == 3 ? read_y(A, o + 2) : 0.0;                       // Eq. 10
    double tn, ux, uy;
    traction_dir(ts, td, A.cr[i], A.sr[i], tn, ux, uy);
    dphi = A.b_dc[i] * (A.V0 * exp((A.f0 - phi) * A.inv_b[i]) - g);   // Eq. 8
    const double Vphi = -g * A.inv_a[i], Vsig = -(tn / sig) * g1;
    const double gt = tn > 0.0 ? g / tn : g1;
    const double c = A.eta * (Vphi * dphi + Vsig * dsig);
    const double rs = ss - c * ux, rd = sd - c * uy;
    const double par = rs * ux + rd * uy;
    const double kpar = par / (1.0 + A.eta * g1), kper = 1.0 / (1.0 + A.eta * gt);
    dts = kpar * ux + kper * (rs - par * ux);
    dtd = kpar * uy + kper * (rd - par * uy);
}

}  // namespace hbi
