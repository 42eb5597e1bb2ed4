// One Cash-Karp stage of one element, device side: the Cash & Karp (1990) embedded 4(5)
// tableau and the per-element bodies of stages 1-5 and of stage 6 (with the error norm), for
// the fixed-rake and the rake-free law, shared by the separate stage kernels (hbi_ode.cu) and
// the product's UY phase, which runs them for the elements of a leaf row unit as soon as
// their output rows are written (hbi_hmvm.cu).  Each translation unit that includes this header holds its own
// copy of the tableau in constant memory.
#pragma once

#include <climits>

#include "hbi_ode_math.cuh"

namespace hbi {

static __constant__ double c_A[6][5] = {
    {0, 0, 0, 0, 0},
    {1.0 / 5.0, 0, 0, 0, 0},
    {3.0 / 40.0, 9.0 / 40.0, 0, 0, 0},
    {3.0 / 10.0, -9.0 / 10.0, 6.0 / 5.0, 0, 0},
    {-11.0 / 54.0, 5.0 / 2.0, -70.0 / 27.0, 35.0 / 27.0, 0},
    {1631.0 / 55296.0, 175.0 / 512.0, 575.0 / 13824.0, 44275.0 / 110592.0, 253.0 / 4096.0}};
static __constant__ double c_B5[6] = {37.0 / 378.0, 0.0, 250.0 / 621.0, 125.0 / 594.0, 0.0, 512.0 / 1771.0};
static __constant__ double c_B4[6] = {2825.0 / 27648.0, 0.0, 18575.0 / 48384.0, 13525.0 / 55296.0, 277.0 / 14336.0,
                                      0.25};

// Stage s (0-based, 0..4) at element i: k_s = f(y_s) from the product output (Eqs. 8, 10,
// 12, 13a-c), then the stage s+1 state y + dt sum_l a_{s+1,l} k_l, its slip rate (Eq. 7), V,
// dV/dtau and tau/sigma kept beside it, and the next product input (V - V_pl) r into A.xt.
// After a rejected attempt y is unchanged, so stage 0 keeps k_0 = f(y) from its slot (its
// product was skipped) and only forms the stage inputs for the new step size.
__device__ __forceinline__ void stage_elem(const OdeArgs &A, int s, int i) {
    const int n = A.n;
    const StepCtl &C = A.ctl[A.model[i]];
    if (C.stop) return;
    const double dt = C.dt;
    const bool keep_k0 = s == 0 && C.reuse_k0;
    double *ks_ = A.k + (size_t)s * 3 * n;
    if (A.store) {
        if (s == 0)
            for (int c = 0; c < 3; ++c) A.st_Y[(size_t)c * n + i] = A.y[(size_t)c * n + i];
        for (int c = 0; c < A.nout; ++c)
            A.st_S[(size_t)s * A.nout * n + (size_t)A.nout * i + c] = read_y(A, (int64_t)A.nout * i + c);
    }
    if (!keep_k0) {
        double kp, kt, ks;
        rhs_elem_q(A, i, A.ys[i], A.Vs[i], A.dVs[i], A.Vs[n + i], kp, kt, ks);
        ks_[i] = kp; ks_[n + i] = kt; ks_[2 * n + i] = ks;
    }
    double acc[3] = {0.0, 0.0, 0.0};
    for (int l = 0; l <= s; ++l) {
        const double c = c_A[s + 1][l];
        const double *kl = A.k + (size_t)l * 3 * n;
        acc[0] += c * kl[i]; acc[1] += c * kl[n + i]; acc[2] += c * kl[2 * n + i];
    }
    const double p1 = A.y[i] + dt * acc[0], t1 = A.y[n + i] + dt * acc[1], s1 = A.y[2 * n + i] + dt * acc[2];
    A.ys[i] = p1; A.ys[n + i] = t1; A.ys[2 * n + i] = s1;
    if (A.store) {
        double *Y = A.st_Y + (size_t)(s + 1) * 3 * n;
        Y[i] = p1; Y[n + i] = t1; Y[2 * n + i] = s1;
    }
    double dV1, q1;
    const double V1 = slip_rate(p1, t1, s1, A.inv_a[i], A.V0, dV1, q1);
    A.Vs[i] = V1; A.dVs[i] = dV1; A.Vs[n + i] = q1;
    write_x(A, i, V1);
}

__device__ __forceinline__ unsigned long long dbits(double v) { return (unsigned long long)__double_as_longlong(v); }

// Stage 6 at element i: k_5 from the last product's rows, the solutions of order 5 and 4, the
// element error max_c |y5 - y4| / max(|y5|, 1e-30) (the largest ratio found by cross-multiplied
// comparison, all terms non-negative, and divided out once; infinite, with the model's flag,
// when not finite or when sigma5 <= 0), y5 with its slip rate as the stage state, and the
// element's contributions to the model's reductions: the error and |V5| as the ordered bit
// patterns of non-negative doubles, tau5/sigma5 in fixed point.  Returns the model index, or
// -1 for an element of a stopped model (nothing written).
__device__ __forceinline__ int final_elem(const OdeArgs &A, int i, unsigned long long &eb, unsigned long long &vb,
                                          unsigned long long &mu) {
    const int n = A.n;
    const int m = A.model[i];
    StepCtl &C = A.ctl[m];
    if (C.stop) return -1;
    const double dt = C.dt;
    if (A.store)
        for (int c = 0; c < A.nout; ++c)
            A.st_S[(size_t)5 * A.nout * n + (size_t)A.nout * i + c] = read_y(A, (int64_t)A.nout * i + c);
    double kp, kt, ks;
    rhs_elem_q(A, i, A.ys[i], A.Vs[i], A.dVs[i], A.Vs[n + i], kp, kt, ks);
    double *k5 = A.k + (size_t)5 * 3 * n;
    k5[i] = kp; k5[n + i] = kt; k5[2 * n + i] = ks;
    double y5[3], num = 0.0, den = 1.0;
    bool bad = false;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        double s5 = 0.0, s4 = 0.0;
#pragma unroll
        for (int l = 0; l < 6; ++l) {
            const double kv = A.k[(size_t)l * 3 * n + (size_t)c * n + i];
            s5 += c_B5[l] * kv;
            s4 += c_B4[l] * kv;
        }
        const double y0 = A.y[(size_t)c * n + i];
        y5[c] = y0 + dt * s5;
        const double y4 = y0 + dt * s4;
        const double d = fabs(y5[c] - y4), mg = fmax(fabs(y5[c]), 1e-30);
        bad |= !isfinite(d) || !isfinite(mg);
        if (d * den > num * mg) { num = d; den = mg; }
    }
    double e = num / den;
    if (bad || !isfinite(e)) { e = INFINITY; atomicOr(&C.flags, 2); }   // rejected
    if (!(y5[2] > 0.0)) { e = INFINITY; atomicOr(&C.flags, 1); }     // sigma <= 0: rejected
    A.ys[i] = y5[0]; A.ys[n + i] = y5[1]; A.ys[2 * n + i] = y5[2];
    double dV5, q5;
    const double V5 = slip_rate(y5[0], y5[1], y5[2], A.inv_a[i], A.V0, dV5, q5);
    A.Vs[i] = V5; A.dVs[i] = dV5; A.Vs[n + i] = q5;
    eb = dbits(e);
    vb = dbits(isfinite(V5) ? fabs(V5) : 0.0);
    mu = (unsigned long long)mu_fixed(q5);   // summed in two's complement
    return m;
}

// Rake-free friction (layouts y, ys: phi | tau_s | tau_d | sigma; Vs: g | V_s | V_d; the
// stage vectors 4N apart), stage s (0..4) at element i: k_s from the product rows, the stage
// s+1 state, its slip-rate vector and the next product input (vec_state).
__device__ __forceinline__ void stage_vec_elem(const OdeArgs &A, int s, int i) {
    const int n = A.n;
    const StepCtl &C = A.ctl[A.model[i]];
    if (C.stop) return;
    const double dt = C.dt;
    double *ks_ = A.k + (size_t)s * 4 * n;
    if (!(s == 0 && C.reuse_k0)) {
        double kp, kts, ktd, ks;
        rhs_vec_elem(A, i, A.ys[i], A.ys[n + i], A.ys[2 * n + i], A.ys[3 * n + i], A.Vs[i], A.dVs[i], kp, kts, ktd,
                     ks);
        ks_[i] = kp; ks_[n + i] = kts; ks_[2 * n + i] = ktd; ks_[3 * n + i] = ks;
    }
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
    for (int l = 0; l <= s; ++l) {
        const double c = c_A[s + 1][l];
        const double *kl = A.k + (size_t)l * 4 * n;
        for (int q = 0; q < 4; ++q) acc[q] += c * kl[(size_t)q * n + i];
    }
    double v[4];
    for (int q = 0; q < 4; ++q) {
        v[q] = A.y[(size_t)q * n + i] + dt * acc[q];
        A.ys[(size_t)q * n + i] = v[q];
    }
    vec_state(A, i, v[0], v[1], v[2], v[3]);
}

// Rake-free stage 6 at element i: the element error is its largest relative change among
// phi, the traction vector (relative to |tau5|) and sigma; otherwise as final_elem.
__device__ __forceinline__ int final_vec_elem(const OdeArgs &A, int i, unsigned long long &eb, unsigned long long &vb,
                                              unsigned long long &mu) {
    const int n = A.n;
    const int m = A.model[i];
    StepCtl &C = A.ctl[m];
    if (C.stop) return -1;
    const double dt = C.dt;
    double kp, kts, ktd, ks;
    rhs_vec_elem(A, i, A.ys[i], A.ys[n + i], A.ys[2 * n + i], A.ys[3 * n + i], A.Vs[i], A.dVs[i], kp, kts, ktd, ks);
    double *k5 = A.k + (size_t)5 * 4 * n;
    k5[i] = kp; k5[n + i] = kts; k5[2 * n + i] = ktd; k5[3 * n + i] = ks;
    double y5[4], y4[4];
    for (int c = 0; c < 4; ++c) {
        double s5 = 0.0, s4 = 0.0;
#pragma unroll
        for (int l = 0; l < 6; ++l) {
            const double kv = A.k[(size_t)l * 4 * n + (size_t)c * n + i];
            s5 += c_B5[l] * kv;
            s4 += c_B4[l] * kv;
        }
        const double y0 = A.y[(size_t)c * n + i];
        y5[c] = y0 + dt * s5;
        y4[c] = y0 + dt * s4;
    }
    const double tn5 = sqrt(y5[1] * y5[1] + y5[2] * y5[2]);
    const double dts = y5[1] - y4[1], dtd = y5[2] - y4[2];
    const double e0 = fabs(y5[0] - y4[0]) / fmax(fabs(y5[0]), 1e-30);
    const double e1 = sqrt(dts * dts + dtd * dtd) / fmax(tn5, 1e-30);
    const double e2 = fabs(y5[3] - y4[3]) / fmax(fabs(y5[3]), 1e-30);
    // fmax drops a NaN operand: test the three changes themselves
    double e = fmax(e0, fmax(e1, e2));
    if (!isfinite(e0) || !isfinite(e1) || !isfinite(e2)) { e = INFINITY; atomicOr(&C.flags, 2); }
    if (!(y5[3] > 0.0)) { e = INFINITY; atomicOr(&C.flags, 1); }
    for (int c = 0; c < 4; ++c) A.ys[(size_t)c * n + i] = y5[c];
    vec_state(A, i, y5[0], y5[1], y5[2], y5[3]);
    eb = dbits(e);
    vb = dbits(isfinite(A.Vs[i]) ? fabs(A.Vs[i]) : 0.0);
    mu = (unsigned long long)mu_fixed(tn5 / y5[3]);
    return m;
}

// final_elem (VEC: final_vec_elem) over the elements [e0, e0 + ne) of one leaf row unit by the
// first nthreads (a multiple of 32) threads of a CTA, each warp combining its lanes'
// contributions when they all belong to one model (one atomic per quantity and warp), else
// lane by lane.
template <bool VEC>
__device__ __forceinline__ void final_unit(const OdeArgs &A, int e0, int ne, int nthreads) {
    const int lane = threadIdx.x & 31;
    for (int w0 = threadIdx.x - lane; w0 < ne; w0 += nthreads) {
        unsigned long long eb = 0ull, vb = 0ull, mu = 0ull;
        int m = -1;
        if (w0 + lane < ne)
            m = VEC ? final_vec_elem(A, e0 + w0 + lane, eb, vb, mu) : final_elem(A, e0 + w0 + lane, eb, vb, mu);
        const int mlo = __reduce_min_sync(0xffffffffu, m < 0 ? INT_MAX : m), mhi = __reduce_max_sync(0xffffffffu, m);
        if (mhi < 0) continue;
        if (mlo == mhi) {
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                const unsigned long long e2 = __shfl_xor_sync(0xffffffffu, eb, o);
                const unsigned long long v2 = __shfl_xor_sync(0xffffffffu, vb, o);
                eb = e2 > eb ? e2 : eb;
                vb = v2 > vb ? v2 : vb;
                mu += __shfl_xor_sync(0xffffffffu, mu, o);
            }
            if (lane == 0) {
                StepCtl &C = A.ctl[mhi];
                atomicMax(&C.err_bits, eb);
                atomicMax(&C.vmax_bits, vb);
                atomicAdd((unsigned long long *)&C.mu_fix, mu);
            }
        } else if (m >= 0) {
            StepCtl &C = A.ctl[m];
            atomicMax(&C.err_bits, eb);
            atomicMax(&C.vmax_bits, vb);
            atomicAdd((unsigned long long *)&C.mu_fix, mu);
        }
    }
}

}  // namespace hbi
