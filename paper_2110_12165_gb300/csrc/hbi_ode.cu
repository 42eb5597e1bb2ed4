// Rate-and-state right-hand side and adaptive Runge-Kutta attempt (Eqs. 7-16, 21-22),
// element-wise in FP64 in the permuted element order of the H-matrix.
//
// One attempt = six stages.  Stage s feeds the HMVM with x = (V_s - V_pl) r (the backslip
// loading of Eqs. 21-22 folded into the product), then k_s = f(y_s) (Eqs. 8, 10, 12,
// 13a-c) is evaluated and immediately forms the next stage state
// y_{s+1} = y + dt sum_l a_{s+1,l} k_l, its slip rate (Eq. 7) and the next HMVM input: for
// inside the product's UY phase (stage_elem / stage_vec_elem, hbi_stage.cuh); the fixed-rake
// stages also run as kernels of their own (eager timing, fixed steps of the adjoint).
// The last stage also forms the 5th/4th-order solutions, the error
// err = max_i |y5_i - y4_i| / max(|y5_i|, 1e-30), reduced over the grid; the last CTA to
// finish runs the step controller (Eqs. 14-15), so accept/reject never leaves the GPU.
// Every kernel returns immediately once the control block says the requested number of
// steps is done, which lets the host replay a captured attempt graph freely.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>

#include "hbi_internal.h"
#include "hbi_ode_math.cuh"
#include "hbi_stage.cuh"

namespace hbi {

__device__ __forceinline__ bool all_stopped(const OdeArgs &A) { return *(volatile int *)&A.g->stop != 0; }

// Start of a call: stage-1 state = y, V from Eq. 7, HMVM input.
// Fixed-rake friction keeps, beside V and dV/dtau of the stage state (Vs, dVs) and of y (Vold,
// dVold), its friction coefficient q = tau / sigma (formed by slip_rate) in Vs[n + i] and
// Vold[n + i], the slots the rake-free form uses for its slip-rate components.
__global__ void prep_kernel(OdeArgs A) {
    const int n = A.n;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const double phi = A.y[i], tau = A.y[n + i], sig = A.y[2 * n + i];
        A.ys[i] = phi; A.ys[n + i] = tau; A.ys[2 * n + i] = sig;
        double dV, q;
        const double V = slip_rate(phi, tau, sig, A.inv_a[i], A.V0, dV, q);
        A.Vs[i] = V; A.dVs[i] = dV; A.Vs[n + i] = q;
        A.Vold[i] = V; A.dVold[i] = dV; A.Vold[n + i] = q;
        write_x(A, i, V);
    }
}

// Stage s (0-based, 0..4) as its own launch: stage_elem over every element.
__global__ void stage_kernel(OdeArgs A, int s) {
    if (all_stopped(A)) return;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < A.n; i += gridDim.x * blockDim.x) stage_elem(A, s, i);
}

// Stage 6 as its own launch (final_elem), with the per-model maxima of the error and of |V|
// and the friction sum.  One element per thread; a block covers a contiguous element range
// and so at most a few models, whose reductions it gathers in shared memory before one atomic
// per model.
constexpr int FINAL_SEG = 8;
__global__ void final_kernel(OdeArgs A) {
    if (all_stopped(A)) return;
    __shared__ unsigned long long s_err[FINAL_SEG], s_vm[FINAL_SEG], s_mu[FINAL_SEG];
    const int n = A.n;
    const int i0 = blockIdx.x * blockDim.x, i = i0 + threadIdx.x;
    const int m0 = A.model[min(i0, n - 1)];
    if (threadIdx.x < FINAL_SEG) { s_err[threadIdx.x] = 0ull; s_vm[threadIdx.x] = 0ull; s_mu[threadIdx.x] = 0ull; }
    __syncthreads();
    if (i < n) {
        unsigned long long eb, vb, mu;
        const int m = final_elem(A, i, eb, vb, mu);
        if (m >= 0) {
            if (m - m0 < FINAL_SEG) {
                atomicMax(&s_err[m - m0], eb);
                atomicMax(&s_vm[m - m0], vb);
                atomicAdd(&s_mu[m - m0], mu);
            } else {
                StepCtl &C = A.ctl[m];
                atomicMax(&C.err_bits, eb);
                atomicMax(&C.vmax_bits, vb);
                atomicAdd((unsigned long long *)&C.mu_fix, mu);
            }
        }
    }
    __syncthreads();
    if (threadIdx.x < FINAL_SEG && m0 + (int)threadIdx.x < A.n_models &&
        (s_err[threadIdx.x] | s_vm[threadIdx.x] | s_mu[threadIdx.x]) != 0ull) {
        StepCtl &C = A.ctl[m0 + threadIdx.x];
        atomicMax(&C.err_bits, s_err[threadIdx.x]);
        atomicMax(&C.vmax_bits, s_vm[threadIdx.x]);
        atomicAdd((unsigned long long *)&C.mu_fix, s_mu[threadIdx.x]);
    }
}

// The step controller of every active model (Eqs. 14-15, exponents read on err/eps): accept
// or reject, step records, the next dt, stop conditions, reset of the maxima.  Run by one CTA.
__device__ void control_models(const OdeArgs &A) {
    for (int m = threadIdx.x; m < A.n_models; m += blockDim.x) {
        StepCtl *C = &A.ctl[m];
        if (C->stop) continue;
        const double dt = C->dt;
        const double e = __longlong_as_double((long long)C->err_bits);
        const double vm = __longlong_as_double((long long)C->vmax_bits);
        const double eps = C->eps;
        double dt_new;
        const int accept = step_control(e, eps, dt, dt_new);
        C->accept_flag = accept;
        C->dt_used = dt;
        if (accept) {
            C->t += dt;
            if (A.rec != nullptr && C->accepted < C->target) {
                hbi_step_record r;
                r.t = C->t; r.dt = dt; r.vmax = vm; r.rejects = (double)C->rejects;
                r.mu_mean = (double)C->mu_fix * (1.0 / 1099511627776.0) / (double)max(1, C->nelem);
                A.rec[(size_t)m * A.rec_cap + C->accepted] = r;
            }
            C->accepted += 1;
            C->rejects = 0;
            if (C->accepted >= C->target) C->done_pending = 1;
        } else {
            C->rejects += 1;
        }
        C->reuse_k0 = !accept;
        C->dt = dt_new;
        if (!(dt_new > 1e-12)) {
            C->status = (C->flags & 1) ? HBI_ERR_NEG_NORMAL : ((C->flags & 2) ? HBI_ERR_NONFINITE : HBI_ERR_DT_UNDERFLOW);
            C->done_pending = 1;
        }
        C->flags = 0;
        C->err_bits = 0ull;
        C->vmax_bits = 0ull;
        C->mu_fix = 0;
    }
}
__global__ void controller_kernel(OdeArgs A) {
    if (all_stopped(A)) return;
    control_models(A);
}

// Accept: y <- y5, slip by the trapezoid of Eq. 16; either way prepare stage 1 of the next
// attempt (the HMVM input of the current state).
__global__ void commit_kernel(OdeArgs A) {
    if (all_stopped(A)) return;
    const int n = A.n;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const StepCtl &C = A.ctl[A.model[i]];
        if (C.stop) continue;
        const double dt = C.dt_used;
        if (C.accept_flag) {
            const double V5 = A.Vs[i];
            A.D[i] += 0.5 * dt * (A.Vold[i] + V5);
            A.y[i] = A.ys[i]; A.y[n + i] = A.ys[n + i]; A.y[2 * n + i] = A.ys[2 * n + i];
            A.Vold[i] = V5; A.dVold[i] = A.dVs[i]; A.Vold[n + i] = A.Vs[n + i];
        } else {
            A.ys[i] = A.y[i]; A.ys[n + i] = A.y[n + i]; A.ys[2 * n + i] = A.y[2 * n + i];
            A.Vs[i] = A.Vold[i]; A.dVs[i] = A.dVold[i]; A.Vs[n + i] = A.Vold[n + i];
        }
        write_x(A, i, A.Vold[i]);
    }
}
// Separate one-CTA kernel so that every commit CTA reads the same flags before a stop is set:
// models that reached their target (or failed) stop; the attempt graph stops when all have;
// the next attempt's first product is skipped when every active model rejected (k_0 kept).
__device__ void stop_models(const OdeArgs &A) {
    __shared__ int s_active, s_accepted;
    if (threadIdx.x == 0) { s_active = 0; s_accepted = 0; }
    __syncthreads();
    for (int m = threadIdx.x; m < A.n_models; m += blockDim.x) {
        StepCtl *C = &A.ctl[m];
        if (!C->stop && C->done_pending) C->stop = 1;
        if (!C->stop) {
            atomicOr(&s_active, 1);
            if (!C->reuse_k0) atomicOr(&s_accepted, 1);
        }
        // the next attempt's products skip this model's rows and columns once it stopped,
        // and its first product after a rejection (k_0 kept)
        A.mskip[m] = C->stop || C->reuse_k0;
        A.mskip[A.n_models + m] = C->stop;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        A.g->stop = !s_active;
        A.g->skip0 = !s_active || !s_accepted;
    }
}
__global__ void stop_kernel(OdeArgs A) { stop_models(A); }

// controller_kernel + commit_kernel + stop_kernel in one launch (fixed-rake friction).  Every
// element takes its model's decision err <= eps_RK itself (NaN rejects, as in step_control;
// the same inputs on every CTA), commits (Eq. 16) or restores, and forms the next attempt's
// first product input; the CTA that finishes last then runs the step control of every model
// (Eqs. 14-15, records, next dt) and sets the stop and skip flags, and rearms its counter.
__global__ void commit_ctl_kernel(OdeArgs A) {
    if (all_stopped(A)) return;
    __shared__ int s_last;
    const int n = A.n;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const StepCtl &C = A.ctl[A.model[i]];
        if (C.stop) continue;
        const double e = __longlong_as_double((long long)C.err_bits);
        if (e <= C.eps) {
            const double V5 = A.Vs[i];
            A.D[i] += 0.5 * C.dt * (A.Vold[i] + V5);
            A.y[i] = A.ys[i]; A.y[n + i] = A.ys[n + i]; A.y[2 * n + i] = A.ys[2 * n + i];
            A.Vold[i] = V5; A.dVold[i] = A.dVs[i]; A.Vold[n + i] = A.Vs[n + i];
        } else {
            A.ys[i] = A.y[i]; A.ys[n + i] = A.y[n + i]; A.ys[2 * n + i] = A.y[2 * n + i];
            A.Vs[i] = A.Vold[i]; A.dVs[i] = A.dVold[i]; A.Vs[n + i] = A.Vold[n + i];
        }
        write_x(A, i, A.Vold[i]);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        s_last = atomicAdd(&A.g->commit_done, 1) == (int)gridDim.x - 1;
    }
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    control_models(A);
    __syncthreads();
    stop_models(A);
    if (threadIdx.x == 0) A.g->commit_done = 0;
}

// dy/dt for a given state (hbi_rhs): first half (V and HMVM input) ...
__global__ void rhs_pre_kernel(OdeArgs A) {
    const int n = A.n;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        double dV;
        const double V = slip_rate(A.ys[i], A.ys[n + i], A.ys[2 * n + i], A.inv_a[i], A.V0, dV);
        A.Vs[i] = V; A.dVs[i] = dV;
        write_x(A, i, V);
    }
}
// ... second half, writing dy/dt and V in the caller's order
__global__ void rhs_post_kernel(OdeArgs A, const int *perm, double *dydt, double *Vout) {
    const int n = A.n;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const double phi = A.ys[i], tau = A.ys[n + i], sig = A.ys[2 * n + i];
        const double V = A.Vs[i];
        double kp, kt, ks;
        rhs_elem(A, i, phi, tau, sig, V, A.dVs[i], kp, kt, ks);
        const int e = perm[i];
        dydt[e] = kp; dydt[n + e] = kt; dydt[2 * n + e] = ks;
        if (Vout) Vout[e] = V;
    }
}

__global__ void gather_state_kernel(const double *src, const int *perm, int n, int ncomp, double *dst) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int e = perm[i];
        for (int c = 0; c < ncomp; ++c) dst[(size_t)c * n + i] = src[(size_t)c * n + e];
    }
}
__global__ void scatter_state_kernel(const double *src, const int *perm, int n, int ncomp, double *dst) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int e = perm[i];
        for (int c = 0; c < ncomp; ++c) dst[(size_t)c * n + e] = src[(size_t)c * n + i];
    }
}
__global__ void friction_kernel(const int *perm, int n, const double *a, const double *b, const double *dc,
                                const double *rake, double *inv_a, double *inv_b, double *b_dc, double *pcr,
                                double *psr) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int e = perm[i];
        inv_a[i] = 1.0 / a[e]; inv_b[i] = 1.0 / b[e]; b_dc[i] = b[e] / dc[e];
        double s, c;
        sincos(rake ? rake[e] : 0.0, &s, &c);
        pcr[i] = c; psr[i] = s;
    }
}
__global__ void steady_state_kernel(int n, const double *V, const double *a, const double *b, const double *sig,
                                    double f0, double V0, double *phi, double *tau) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const double p = f0 - b[i] * log(V[i] / V0);                                 // Eq. 8 = 0
        phi[i] = p;
        tau[i] = a[i] * sig[i] * asinh(V[i] / (2.0 * V0) * exp(p / a[i]));           // Eq. 7
    }
}

// ------------------------------------------------------------- rake-free friction
// Vector shear traction (tau_s, tau_d) with the slip rate parallel to it (an extension of the
// fixed-rake law of Eqs. 5-13): V = g t, g the Eq. 7 slip rate at |tau|, t = tau / |tau|.  The
// quasi-dynamic balance tau = tau_el - eta V gives (I + eta dV/dtau) dtau/dt = dtau_el/dt -
// eta (dV/dphi dphi/dt + dV/dsigma dsigma/dt), dV/dtau = g' t t^T + (g / |tau|)(I - t t^T):
// solved per element as a part parallel to t and a part perpendicular to it.  Layouts: y, ys
// (phi | tau_s | tau_d | sigma), Vs, Vold (g | V_s | V_d), dVs, dVold = g', D (D_s | D_d).

__global__ void prep_vec_kernel(OdeArgs A) {
    const int n = A.n;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        for (int c = 0; c < 4; ++c) A.ys[(size_t)c * n + i] = A.y[(size_t)c * n + i];
        vec_state(A, i, A.y[i], A.y[n + i], A.y[2 * n + i], A.y[3 * n + i]);
        for (int c = 0; c < 3; ++c) A.Vold[(size_t)c * n + i] = A.Vs[(size_t)c * n + i];
        A.dVold[i] = A.dVs[i];
    }
}

// dy/dt of a given state (hbi_rhs_vec): slip rates and product input from ys ...
__global__ void rhs_vec_pre_kernel(OdeArgs A) {
    const int n = A.n;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        vec_state(A, i, A.ys[i], A.ys[n + i], A.ys[2 * n + i], A.ys[3 * n + i]);
}
// ... and dy/dt (4N) and (V_s | V_d) in the caller's order
__global__ void rhs_vec_post_kernel(OdeArgs A, const int *perm, double *dydt, double *Vout) {
    const int n = A.n;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        double kp, kts, ktd, ks;
        rhs_vec_elem(A, i, A.ys[i], A.ys[n + i], A.ys[2 * n + i], A.ys[3 * n + i], A.Vs[i], A.dVs[i], kp, kts, ktd,
                     ks);
        const int e = perm[i];
        dydt[e] = kp; dydt[n + e] = kts; dydt[2 * n + e] = ktd; dydt[3 * n + e] = ks;
        if (Vout) { Vout[e] = A.Vs[n + i]; Vout[n + e] = A.Vs[2 * n + i]; }
    }
}

// accept: y <- y5, slip by the trapezoid of Eq. 16 per component; reject: back to y
__global__ void commit_vec_kernel(OdeArgs A) {
    if (all_stopped(A)) return;
    const int n = A.n;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const StepCtl &C = A.ctl[A.model[i]];
        if (C.stop) continue;
        const double dt = C.dt_used;
        if (C.accept_flag) {
            A.D[i] += 0.5 * dt * (A.Vold[n + i] + A.Vs[n + i]);
            A.D[n + i] += 0.5 * dt * (A.Vold[2 * n + i] + A.Vs[2 * n + i]);
            for (int c = 0; c < 4; ++c) A.y[(size_t)c * n + i] = A.ys[(size_t)c * n + i];
            for (int c = 0; c < 3; ++c) A.Vold[(size_t)c * n + i] = A.Vs[(size_t)c * n + i];
            A.dVold[i] = A.dVs[i];
        } else {
            for (int c = 0; c < 4; ++c) A.ys[(size_t)c * n + i] = A.y[(size_t)c * n + i];
            for (int c = 0; c < 3; ++c) A.Vs[(size_t)c * n + i] = A.Vold[(size_t)c * n + i];
            A.dVs[i] = A.dVold[i];
        }
        write_xv(A, i, A.Vold[n + i], A.Vold[2 * n + i]);
    }
}

// ------------------------------------------------------------- adjoint
// Discrete adjoint of the fixed-step Cash-Karp map y_{n+1} = y_n + dt sum_s b5_s K_s,
// K_s = f(Y_s), Y_s = y_n + dt sum_{l<s} a_{s,l} K_l, for the loss
// L = 1/2 sum_i (ln V_i(y_N) - target_i)^2.  Reverse sweep of one step, with lambda the
// adjoint of y_{n+1}:  Kbar_s = dt b5_s lambda;  for s = 5..0: Ybar_s = J_f(Y_s)^T Kbar_s,
// lambda += Ybar_s, Kbar_l += dt a_{s,l} Ybar_s (l < s).  J_f^T couples elements only through
// the product: the adjoint of the stress rates goes through H^T back to the slip rates.
// Parameters: a at fixed b (the gradient with respect to a - b) and d_c, per element.

// Adjoint of the element-wise part of f at a stage state (phi, tau, sig) with stress rates
// (AV, BV): in, the adjoints (pb, tb, sb) of (dphi/dt, dtau/dt, dsigma/dt) and VbH, the
// adjoint of V arriving through the product; out, the adjoints of the stress rates and of
// (phi, tau, sigma, a, d_c).  Same formulas as slip_rate and rhs_elem, differentiated.
__device__ __forceinline__ void rhs_vjp_elem(const OdeArgs &A, int i, double phi, double tau, double sig,
                                             double AV, double BV, double pb, double tb, double sb, double VbH,
                                             double &AVb, double &BVb, double &phib, double &taub, double &sigb,
                                             double &ab, double &dcb) {
    const double ia = A.inv_a[i], ib = A.inv_b[i], B = A.b_dc[i];
    const double isg = 1.0 / sig, q = tau * isg;
    const double Ep = exp((q - phi) * ia), Em = exp((-q - phi) * ia);
    const double V = A.V0 * (Ep - Em), Vt = A.V0 * (Ep + Em) * ia * isg;
    const double G = A.V0 * exp((A.f0 - phi) * ib);
    const double dphi = B * (G - V), dsig = BV;
    const double Vs = -q * Vt, Vp = -V * ia;
    const double N = AV - A.eta * (Vs * dsig + Vp * dphi), D = 1.0 + A.eta * Vt;
    const double dtau = N / D;
    // reverse
    const double Nb = tb / D, Db = -Nb * dtau;
    AVb = Nb;
    const double Vsb = -A.eta * dsig * Nb;
    BVb = sb - A.eta * Vs * Nb;
    const double Vpb = -A.eta * dphi * Nb;
    const double dpb = pb - A.eta * Vp * Nb;
    double Vtb = A.eta * Db;
    const double Gb = B * dpb, Bb = (G - V) * dpb;
    double Vb = -B * dpb;
    phib = -Gb * G * ib;
    const double qb = -Vt * Vsb;
    Vtb += -q * Vsb;
    Vb += -Vpb * ia;
    double iab = -Vpb * V;
    taub = qb * isg;
    sigb = -qb * q * isg;
    // Vt = V0 (Ep + Em) ia / sig
    const double ia2s2 = ia * ia * isg * isg;
    phib += Vtb * (-ia * Vt);
    taub += Vtb * V * ia2s2;
    sigb += Vtb * (-q * V * ia2s2 - Vt * isg);
    iab += Vtb * A.V0 * isg * ((Ep + Em) + ia * (q * (Ep - Em) - phi * (Ep + Em)));
    // V = V0 (Ep - Em)
    Vb += VbH;
    phib += Vb * (-ia * V);
    taub += Vb * Vt;
    sigb += Vb * (-q * Vt);
    iab += Vb * A.V0 * (q * (Ep + Em) - phi * (Ep - Em));
    ab = -iab * ia * ia;
    dcb = -Bb * B * B * ib;
}

// the stress rates (AV, BV) of element i from product outputs o (n_out per element)
__device__ __forceinline__ void stress_from(const OdeArgs &A, int i, const double *o, double &AV, double &BV) {
    if (A.nout == 1) { AV = o[0]; BV = 0.0; return; }
    if (A.nin == 1) { AV = o[0]; BV = o[1]; return; }
    AV = A.cr[i] * o[0] + A.sr[i] * o[1];
    BV = A.nout == 3 ? o[2] : 0.0;
}

// loss at y_N: per-block partial sums (summed on the host in block order), lambda_N, and
// the direct dependence of V(y_N) on a
__global__ void adj_loss_kernel(OdeArgs A, const double *__restrict__ target, double *lam, double *gA,
                                double *partial) {
    __shared__ double s_part[32];
    const int n = A.n;
    double part = 0.0;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) {
        const double phi = A.y[i], tau = A.y[n + i], sig = A.y[2 * n + i];
        const double ia = A.inv_a[i], isg = 1.0 / sig, q = tau * isg;
        const double Ep = exp((q - phi) * ia), Em = exp((-q - phi) * ia);
        const double V = A.V0 * (Ep - Em), Vt = A.V0 * (Ep + Em) * ia * isg;
        const double r = log(V) - target[i];
        part = 0.5 * r * r;
        const double Vb = r / V;
        lam[i] = Vb * (-ia * V);
        lam[n + i] = Vb * Vt;
        lam[2 * n + i] = Vb * (-q * Vt);
        gA[i] += -(Vb * A.V0 * (q * (Ep + Em) - phi * (Ep - Em))) * ia * ia;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
    if ((threadIdx.x & 31) == 0) s_part[threadIdx.x >> 5] = part;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += s_part[w];
        partial[blockIdx.x] = t;
    }
}

// start of a step's reverse sweep: Kbar_s = dt b5_s lambda
__global__ void adj_init_kernel(OdeArgs A, const double *__restrict__ lam, double *Kbar, double dt) {
    const int n3 = 3 * A.n;
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n3; j += gridDim.x * blockDim.x) {
        const double l = lam[j];
#pragma unroll
        for (int s = 0; s < 6; ++s) Kbar[(size_t)s * n3 + j] = dt * c_B5[s] * l;
    }
}

// stage s, first half: the adjoint of the stress rates, as the input of the product with H^T
__global__ void adj_pre_kernel(OdeArgs A, int s, const double *__restrict__ Kbar, void *axt) {
    const int n = A.n;
    const double *Y = A.st_Y + (size_t)s * 3 * n, *S = A.st_S + (size_t)s * A.nout * n;
    const double *K = Kbar + (size_t)s * 3 * n;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        double AV, BV, AVb, BVb, d0, d1, d2, d3, d4;
        stress_from(A, i, S + (size_t)A.nout * i, AV, BV);
        rhs_vjp_elem(A, i, Y[i], Y[n + i], Y[2 * n + i], AV, BV, K[i], K[n + i], K[2 * n + i], 0.0, AVb, BVb, d0,
                     d1, d2, d3, d4);
        double o[3];
        if (A.nout == 1) { o[0] = AVb; }
        else if (A.nin == 1) { o[0] = AVb; o[1] = BVb; }
        else { o[0] = A.cr[i] * AVb; o[1] = A.sr[i] * AVb; o[2] = BVb; }
        for (int c = 0; c < A.nout; ++c) {
            if (A.acc_double) ((double *)axt)[(size_t)A.nout * i + c] = o[c];
            else ((float *)axt)[(size_t)A.nout * i + c] = (float)o[c];
        }
    }
}

// stage s, second half: with the product H^T (adjoint stress rates) in ayp, the adjoint of
// the stage state; accumulate lambda, the earlier stages' Kbar and the parameter gradients
__global__ void adj_post_kernel(OdeArgs A, int s, const void *ayp, double *lam, double *Kbar, double *gA,
                                double *gDC, double dt) {
    const int n = A.n;
    const double *Y = A.st_Y + (size_t)s * 3 * n, *S = A.st_S + (size_t)s * A.nout * n;
    const double *K = Kbar + (size_t)s * 3 * n;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        double xb[2];
        for (int c = 0; c < A.nin; ++c)
            xb[c] = A.acc_double ? ((const double *)ayp)[(size_t)A.nin * i + c]
                                 : (double)((const float *)ayp)[(size_t)A.nin * i + c];
        const double VbH = A.nin == 1 ? xb[0] : A.cr[i] * xb[0] + A.sr[i] * xb[1];
        double AV, BV, AVb, BVb, pb, tb, sb, ab, dcb;
        stress_from(A, i, S + (size_t)A.nout * i, AV, BV);
        rhs_vjp_elem(A, i, Y[i], Y[n + i], Y[2 * n + i], AV, BV, K[i], K[n + i], K[2 * n + i], VbH, AVb, BVb, pb, tb,
                     sb, ab, dcb);
        lam[i] += pb; lam[n + i] += tb; lam[2 * n + i] += sb;
        for (int l = 0; l < s; ++l) {
            const double c = dt * c_A[s][l];
            double *Kl = Kbar + (size_t)l * 3 * n;
            Kl[i] += c * pb; Kl[n + i] += c * tb; Kl[2 * n + i] += c * sb;
        }
        gA[i] += ab;
        gDC[i] += dcb;
    }
}

// fixed-step mode: the step size of the next step, always accepted
__global__ void fixed_dt_kernel(StepCtl *C, double dt) {
    C->dt = dt; C->dt_used = dt; C->accept_flag = 1;
    C->stop = 0; C->reuse_k0 = 0;
    C->mu_fix = 0;
}

// single right-hand side: the stage-0 state and product outputs for the reverse sweep
__global__ void vjp_prep_kernel(OdeArgs A) {
    const int n = A.n;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        for (int c = 0; c < 3; ++c) A.st_Y[(size_t)c * n + i] = A.ys[(size_t)c * n + i];
        for (int c = 0; c < A.nout; ++c) A.st_S[(size_t)A.nout * i + c] = read_y(A, (int64_t)A.nout * i + c);
    }
}

// ------------------------------------------------------------- host side
namespace {
int grid_for(const hbi_handle *h) { return std::max(1, std::min((h->n + 255) / 256, 8 * std::max(1, h->num_sms))); }

// The element-wise kernels of an attempt run one element per thread in blocks of ODE_BLOCK:
// at their 54-56 registers per thread an SM holds 9 such blocks (1,152 threads) against 4 of
// 256 threads (1,024), so that one wave covers N = 160,000 elements on 152 SMs instead of
// leaving the last blocks to a second wave.
constexpr int ODE_BLOCK = 128;
int grid_ode(const hbi_handle *h) {
    return std::max(1, std::min((h->n + ODE_BLOCK - 1) / ODE_BLOCK, 16 * std::max(1, h->num_sms)));
}

OdeArgs args(hbi_handle *h) {
    OdeArgs A;
    A.n = h->n; A.nin = h->nin; A.nout = h->nout;
    A.y = h->d_y; A.D = h->d_D; A.ys = h->d_ys; A.Vs = h->d_Vs; A.Vold = h->d_Vold; A.k = h->d_k;
    A.dVs = h->d_dVs; A.dVold = h->d_dVold;
    A.inv_a = h->d_inv_a; A.inv_b = h->d_inv_b; A.b_dc = h->d_b_dc; A.cr = h->d_fcr; A.sr = h->d_fsr;
    A.f0 = h->g_f0; A.V0 = h->g_V0; A.Vpl = h->g_Vpl; A.eta = h->g_eta;
    A.xt = h->d_xt; A.yp = h->d_yp; A.acc_double = h->storage == HBI_FP64;
    A.store = 0; A.st_Y = h->d_stY; A.st_S = h->d_stS;
    A.n_models = h->n_models; A.rec_cap = h->rec_cap; A.model = h->d_model;
    A.ctl = h->d_ctl; A.g = h->d_gctl; A.rec = h->d_rec; A.mskip = h->d_mskip;
    return A;
}
}  // namespace

hbi_status ode_alloc(hbi_handle *h, int rec_cap) {
    const size_t n = (size_t)h->n;
    if (!h->d_y) {
        // sized for either friction form (rake-free: 4 state components, 3 slip-rate arrays)
        HBI_ALLOC_TRY(&h->d_y, 4 * n * sizeof(double));
        HBI_ALLOC_TRY(&h->d_D, 2 * n * sizeof(double));
        HBI_ALLOC_TRY(&h->d_ys, 4 * n * sizeof(double));
        HBI_ALLOC_TRY(&h->d_Vs, 3 * n * sizeof(double));
        HBI_ALLOC_TRY(&h->d_Vold, 3 * n * sizeof(double));
        HBI_ALLOC_TRY(&h->d_dVs, n * sizeof(double));
        HBI_ALLOC_TRY(&h->d_dVold, n * sizeof(double));
        HBI_ALLOC_TRY(&h->d_k, 24 * n * sizeof(double));
        HBI_CUDA_TRY(cudaMemset(h->d_k, 0, 24 * n * sizeof(double)));
        HBI_ALLOC_TRY(&h->d_inv_a, n * sizeof(double));
        HBI_ALLOC_TRY(&h->d_inv_b, n * sizeof(double));
        HBI_ALLOC_TRY(&h->d_b_dc, n * sizeof(double));
        HBI_ALLOC_TRY(&h->d_fcr, n * sizeof(double));
        HBI_ALLOC_TRY(&h->d_fsr, n * sizeof(double));
        const size_t nm = (size_t)h->n_models;
        HBI_ALLOC_TRY(&h->d_ctl, nm * sizeof(StepCtl));
        HBI_CUDA_TRY(cudaMemset(h->d_ctl, 0, nm * sizeof(StepCtl)));
        HBI_CUDA_TRY(cudaMallocHost(&h->h_ctl, nm * sizeof(StepCtl)));
        HBI_ALLOC_TRY(&h->d_gctl, sizeof(GlobalCtl));
        HBI_CUDA_TRY(cudaMemset(h->d_gctl, 0, sizeof(GlobalCtl)));
        HBI_CUDA_TRY(cudaMallocHost(&h->h_gctl, sizeof(GlobalCtl)));
        HBI_CUDA_TRY(cudaMallocHost(&h->h_flag, sizeof(int)));
        HBI_ALLOC_TRY(&h->d_mskip, 2 * nm * sizeof(int));
        HBI_CUDA_TRY(cudaMemset(h->d_mskip, 0, 2 * nm * sizeof(int)));
        if (!h->d_model) {
            std::vector<int> model(n, 0);
            for (int m = 0; m < h->n_models; ++m)
                for (int e = h->model_start[m]; e < h->model_start[m + 1]; ++e) model[e] = m;
            HBI_ALLOC_TRY(&h->d_model, n * sizeof(int));
            HBI_CUDA_TRY(cudaMemcpy(h->d_model, model.data(), n * sizeof(int), cudaMemcpyHostToDevice));
        }
    }
    if (rec_cap > h->rec_cap) {
        if (h->d_rec) cudaFree(h->d_rec);
        rec_cap = std::max(rec_cap, std::max(4096, 2 * h->rec_cap));   // grow rarely: re-capture
        HBI_ALLOC_TRY(&h->d_rec, (size_t)h->n_models * rec_cap * sizeof(hbi_step_record));
        h->rec_cap = rec_cap;
        drop_graphs(h);
    }
    return HBI_OK;
}

void drop_graphs(hbi_handle *h) {
    if (h->graph_exec) { cudaGraphExecDestroy(h->graph_exec); h->graph_exec = nullptr; }
    if (h->graph_exec_vec) { cudaGraphExecDestroy(h->graph_exec_vec); h->graph_exec_vec = nullptr; }
}

hbi_status ode_set_friction(hbi_handle *h, const hbi_friction *f, cudaStream_t s) {
    friction_kernel<<<grid_for(h), 256, 0, s>>>(h->d_perm, h->n, f->d_a, f->d_b, f->d_dc, f->d_rake, h->d_inv_a,
                                                h->d_inv_b, h->d_b_dc, h->d_fcr, h->d_fsr);
    HBI_CUDA_TRY(cudaGetLastError());
    const double eta = f->mu / (2.0 * f->cs);
    if (h->g_f0 != f->f0 || h->g_V0 != f->V0 || h->g_Vpl != f->Vpl || h->g_eta != eta) drop_graphs(h);
    h->g_f0 = f->f0; h->g_V0 = f->V0; h->g_Vpl = f->Vpl; h->g_eta = eta;
    return HBI_OK;
}

// state component counts: fixed rake (phi, tau, sigma | D), rake-free (phi, tau_s, tau_d, sigma | D_s, D_d)
hbi_status ode_state_in(hbi_handle *h, const double *d_state, int with_slip, cudaStream_t s, int vec) {
    const int ny = vec ? 4 : 3, nd = vec ? 2 : 1;
    gather_state_kernel<<<grid_for(h), 256, 0, s>>>(d_state, h->d_perm, h->n, ny, h->d_y);
    if (with_slip)
        gather_state_kernel<<<grid_for(h), 256, 0, s>>>(d_state + ny * (size_t)h->n, h->d_perm, h->n, nd, h->d_D);
    HBI_CUDA_TRY(cudaGetLastError());
    return HBI_OK;
}

hbi_status ode_state_out(hbi_handle *h, double *d_state, cudaStream_t s, int vec) {
    const int ny = vec ? 4 : 3, nd = vec ? 2 : 1;
    scatter_state_kernel<<<grid_for(h), 256, 0, s>>>(h->d_y, h->d_perm, h->n, ny, d_state);
    scatter_state_kernel<<<grid_for(h), 256, 0, s>>>(h->d_D, h->d_perm, h->n, nd, d_state + ny * (size_t)h->n);
    HBI_CUDA_TRY(cudaGetLastError());
    return HBI_OK;
}

hbi_status ode_rhs(hbi_handle *h, double *d_dydt, double *d_V, cudaStream_t s) {
    OdeArgs A = args(h);
    HBI_CUDA_TRY(cudaMemcpyAsync(h->d_ys, h->d_y, 3 * (size_t)h->n * sizeof(double), cudaMemcpyDeviceToDevice, s));
    rhs_pre_kernel<<<grid_for(h), 256, 0, s>>>(A);
    HBI_CUDA_TRY(cudaGetLastError());
    hbi_status st = hmvm_launch(h, s, nullptr);
    if (st) return st;
    rhs_post_kernel<<<grid_for(h), 256, 0, s>>>(A, h->d_perm, d_dydt, d_V);
    HBI_CUDA_TRY(cudaGetLastError());
    return HBI_OK;
}

hbi_status ode_rhs_vec(hbi_handle *h, double *d_dydt, double *d_V, cudaStream_t s) {
    OdeArgs A = args(h);
    HBI_CUDA_TRY(cudaMemcpyAsync(h->d_ys, h->d_y, 4 * (size_t)h->n * sizeof(double), cudaMemcpyDeviceToDevice, s));
    rhs_vec_pre_kernel<<<grid_for(h), 256, 0, s>>>(A);
    HBI_CUDA_TRY(cudaGetLastError());
    hbi_status st = hmvm_launch(h, s, nullptr);
    if (st) return st;
    rhs_vec_post_kernel<<<grid_for(h), 256, 0, s>>>(A, h->d_perm, d_dydt, d_V);
    HBI_CUDA_TRY(cudaGetLastError());
    return HBI_OK;
}

hbi_status ode_prep(hbi_handle *h, cudaStream_t s, int vec) {
    if (vec) prep_vec_kernel<<<grid_for(h), 256, 0, s>>>(args(h));
    else prep_kernel<<<grid_for(h), 256, 0, s>>>(args(h));
    HBI_CUDA_TRY(cudaGetLastError());
    return HBI_OK;
}

// One attempt: 6 x (HMVM + stage), controller, commit.  A rejected attempt leaves y
// unchanged, so the next attempt skips its first HMVM and reuses k_0.
// Stage s (0..5, the last with the error maxima) runs inside the UY phase of product s, unit by
// unit as the unit's rows are written; the products alternate between the input buffers d_xt
// (even products: prep and commit write it) and d_xt2, so that stage s can write product
// s+1's input while other CTAs still gather product s's.
hbi_status ode_attempt(hbi_handle *h, cudaStream_t s, int vec) {
    OdeArgs A = args(h);
    const int *stop = &h->d_gctl->stop;
    const int g = grid_ode(h);
    if (!vec) {
        void *xb[2] = {h->d_xt, h->d_xt2};
        for (int st = 0; st < 6; ++st) {
            OdeArgs F = A;
            F.xt = xb[(st + 1) & 1];
            hbi_status r = hmvm_launch(h, s, st == 0 ? &h->d_gctl->skip0 : stop,
                                       st == 0 ? h->d_mskip : h->d_mskip + h->n_models, false, xb[st & 1], &F, st);
            if (r) return r;
        }
        commit_ctl_kernel<<<g, ODE_BLOCK, 0, s>>>(A);   // controller, commit and stop flags in one launch
        HBI_CUDA_TRY(cudaGetLastError());
        return HBI_OK;
    }
    // rake-free friction: the same, with its stage functions; then controller, commit, stop
    void *xb[2] = {h->d_xt, h->d_xt2};
    for (int st = 0; st < 6; ++st) {
        OdeArgs F = A;
        F.xt = xb[(st + 1) & 1];
        hbi_status r = hmvm_launch(h, s, st == 0 ? &h->d_gctl->skip0 : stop,
                                   st == 0 ? h->d_mskip : h->d_mskip + h->n_models, false, xb[st & 1], &F, st, 2);
        if (r) return r;
    }
    controller_kernel<<<1, 256, 0, s>>>(A);
    commit_vec_kernel<<<g, ODE_BLOCK, 0, s>>>(A);
    stop_kernel<<<1, 256, 0, s>>>(A);
    HBI_CUDA_TRY(cudaGetLastError());
    return HBI_OK;
}

// The fixed-rake attempt launched eagerly with the stages as kernels of their own (every
// product on d_xt) and an event recorded before the first launch and after every kernel
// (per-kernel device times): interval k is of kind cat[k] (0 product, 1 stage, 2 final,
// 4 controller + commit + stop flags).  ev must hold 32 events.
hbi_status ode_attempt_profiled(hbi_handle *h, cudaStream_t s, cudaEvent_t *ev, int *cat, int &nev) {
    OdeArgs A = args(h);
    const int *stop = &h->d_gctl->stop;
    const int g = grid_ode(h);
    nev = 0;
    HBI_CUDA_TRY(cudaEventRecord(ev[nev++], s));
    auto mark = [&](int kind) -> hbi_status {
        cat[nev - 1] = kind;
        HBI_CUDA_TRY(cudaEventRecord(ev[nev++], s));
        return HBI_OK;
    };
    hbi_status r;
    for (int st = 0; st < 6; ++st) {
        if ((r = hmvm_launch(h, s, st == 0 ? &h->d_gctl->skip0 : stop, st == 0 ? h->d_mskip : h->d_mskip + h->n_models,
                             false)) ||
            (r = mark(0)))
            return r;
        if (st < 5) stage_kernel<<<g, ODE_BLOCK, 0, s>>>(A, st);
        else final_kernel<<<(h->n + ODE_BLOCK - 1) / ODE_BLOCK, ODE_BLOCK, 0, s>>>(A);
        if ((r = mark(st < 5 ? 1 : 2))) return r;
    }
    commit_ctl_kernel<<<g, ODE_BLOCK, 0, s>>>(A);   // controller, commit and stop flags in one launch
    if ((r = mark(4))) return r;
    HBI_CUDA_TRY(cudaGetLastError());
    return HBI_OK;
}

hbi_status steady_state_launch(int n, const double *V, const double *a, const double *b, const double *sig,
                               double f0, double V0, double *phi, double *tau, cudaStream_t s) {
    const int grid = std::max(1, std::min((n + 255) / 256, 1024));
    steady_state_kernel<<<grid, 256, 0, s>>>(n, V, a, b, sig, f0, V0, phi, tau);
    HBI_CUDA_TRY(cudaGetLastError());
    return HBI_OK;
}


// ------------------------------------------------------------- adjoint drivers
namespace {
hbi_status adj_alloc(hbi_handle *h, int n_ckpt, int n_seg) {
    const size_t n = (size_t)h->n, n3 = 3 * n;
    if (!h->d_stY) {
        HBI_ALLOC_TRY(&h->d_stY, 6 * n3 * sizeof(double));
        HBI_ALLOC_TRY(&h->d_stS, 6 * (size_t)h->nout * n * sizeof(double));
        HBI_ALLOC_TRY(&h->d_Kbar, 6 * n3 * sizeof(double));
        HBI_ALLOC_TRY(&h->d_lam, n3 * sizeof(double));
        HBI_ALLOC_TRY(&h->d_gA, n * sizeof(double));
        HBI_ALLOC_TRY(&h->d_gDC, n * sizeof(double));
        HBI_ALLOC_TRY(&h->d_aux, (n + (n + 255) / 256 + 1) * sizeof(double));
    }
    if ((int64_t)n_ckpt * (int64_t)n3 > h->n_ckpt) {
        if (h->d_ckpt) cudaFree(h->d_ckpt);
        HBI_ALLOC_TRY(&h->d_ckpt, (size_t)n_ckpt * n3 * sizeof(double));
        h->n_ckpt = (int64_t)n_ckpt * (int64_t)n3;
    }
    // the stage data (6 stage states, 6 product outputs) of every step of one segment
    const int64_t per_step = 6 * (int64_t)n3 + 6 * (int64_t)h->nout * (int64_t)n;
    if ((int64_t)n_seg * per_step > h->n_segY) {
        if (h->d_segY) cudaFree(h->d_segY);
        HBI_ALLOC_TRY(&h->d_segY, (size_t)n_seg * per_step * sizeof(double));
        h->n_segY = (int64_t)n_seg * per_step;
    }
    return HBI_OK;
}

// control blocks for fixed steps: one model, nothing stopped, nothing skipped
hbi_status fixed_reset(hbi_handle *h, cudaStream_t s) {
    HBI_CUDA_TRY(cudaMemsetAsync(h->d_ctl, 0, (size_t)h->n_models * sizeof(StepCtl), s));
    HBI_CUDA_TRY(cudaMemsetAsync(h->d_gctl, 0, sizeof(GlobalCtl), s));
    return HBI_OK;
}

// one Cash-Karp step of size dt from the prepared state (ys = y, V, x), always accepted
hbi_status fixed_step(hbi_handle *h, const OdeArgs &A, double dt, cudaStream_t s) {
    const int g = grid_for(h);
    fixed_dt_kernel<<<1, 1, 0, s>>>(h->d_ctl, dt);
    for (int st = 0; st < 6; ++st) {
        hbi_status r = hmvm_launch(h, s, &h->d_gctl->stop);
        if (r) return r;
        if (st < 5) stage_kernel<<<g, 256, 0, s>>>(A, st);
        else final_kernel<<<(h->n + 255) / 256, 256, 0, s>>>(A);
    }
    commit_kernel<<<g, 256, 0, s>>>(A);
    HBI_CUDA_TRY(cudaGetLastError());
    return HBI_OK;
}

// reverse sweep of one step whose stage data are stored (st_Y, st_S); lambda in d_lam
hbi_status reverse_step(hbi_handle *h, const OdeArgs &A, double dt, cudaStream_t s) {
    const int g = grid_for(h);
    adj_init_kernel<<<g, 256, 0, s>>>(A, h->d_lam, h->d_Kbar, dt);
    for (int st = 5; st >= 0; --st) {
        adj_pre_kernel<<<g, 256, 0, s>>>(A, st, h->d_Kbar, h->adj->d_xt);
        hbi_status r = hmvm_launch(h->adj, s, nullptr);
        if (r) return r;
        adj_post_kernel<<<g, 256, 0, s>>>(A, st, h->adj->d_yp, h->d_lam, h->d_Kbar, h->d_gA, h->d_gDC, dt);
    }
    HBI_CUDA_TRY(cudaGetLastError());
    return HBI_OK;
}
}  // namespace

hbi_status ode_adj_alloc(hbi_handle *h, int n_ckpt, int n_seg) { return adj_alloc(h, n_ckpt, n_seg); }

hbi_status ode_gather(hbi_handle *h, const double *src, int ncomp, double *dst, cudaStream_t s) {
    gather_state_kernel<<<grid_for(h), 256, 0, s>>>(src, h->d_perm, h->n, ncomp, dst);
    HBI_CUDA_TRY(cudaGetLastError());
    return HBI_OK;
}

hbi_status ode_scatter(hbi_handle *h, const double *src, int ncomp, double *dst, cudaStream_t s) {
    scatter_state_kernel<<<grid_for(h), 256, 0, s>>>(src, h->d_perm, h->n, ncomp, dst);
    HBI_CUDA_TRY(cudaGetLastError());
    return HBI_OK;
}

hbi_status ode_rk_fixed(hbi_handle *h, const double *h_dts, int n_steps, cudaStream_t s) {
    hbi_status st = fixed_reset(h, s);
    if (st || (st = ode_prep(h, s))) return st;
    const OdeArgs A = args(h);
    for (int k = 0; k < n_steps; ++k)
        if ((st = fixed_step(h, A, h_dts[k], s))) return st;
    return HBI_OK;
}

hbi_status ode_adjoint(hbi_handle *h, const double *h_dts, int n_steps, int every, const double *d_target,
                       double *h_loss, double *d_state_final, cudaStream_t s) {
    const size_t n = (size_t)h->n, n3 = 3 * n, bytes3 = n3 * sizeof(double);
    const int nseg = (n_steps + every - 1) / every;
    hbi_status st = adj_alloc(h, nseg, every);
    if (st || (st = fixed_reset(h, s))) return st;
    HBI_CUDA_TRY(cudaMemsetAsync(h->d_gA, 0, n * sizeof(double), s));
    HBI_CUDA_TRY(cudaMemsetAsync(h->d_gDC, 0, n * sizeof(double), s));
    const OdeArgs A = args(h);
    OdeArgs As = A;
    As.store = 1;
    // forward, keeping the state at the start of every segment
    if ((st = ode_prep(h, s))) return st;
    for (int k = 0; k < nseg; ++k) {
        HBI_CUDA_TRY(cudaMemcpyAsync(h->d_ckpt + (size_t)k * n3, h->d_y, bytes3, cudaMemcpyDeviceToDevice, s));
        for (int j = k * every; j < std::min(n_steps, (k + 1) * every); ++j)
            if ((st = fixed_step(h, A, h_dts[j], s))) return st;
    }
    if (d_state_final && (st = ode_state_out(h, d_state_final, s))) return st;
    // loss and lambda_N
    const int nb = (int)((n + 255) / 256);
    adj_loss_kernel<<<nb, 256, 0, s>>>(A, d_target, h->d_lam, h->d_gA, h->d_aux + n);
    HBI_CUDA_TRY(cudaGetLastError());
    std::vector<double> part(nb);
    HBI_CUDA_TRY(cudaMemcpyAsync(part.data(), h->d_aux + n, nb * sizeof(double), cudaMemcpyDeviceToHost, s));
    HBI_CUDA_TRY(cudaStreamSynchronize(s));
    double loss = 0.0;
    for (double p : part) loss += p;
    if (h_loss) *h_loss = loss;
    // reverse, segment by segment: recompute the segment from its checkpoint keeping every
    // step's stage data, then sweep back over its steps (last first)
    const size_t per_step = 6 * n3 + 6 * (size_t)h->nout * n;
    auto with_store = [&](int i) {
        OdeArgs Ai = As;
        Ai.st_Y = h->d_segY + (size_t)i * per_step;
        Ai.st_S = Ai.st_Y + 6 * n3;
        return Ai;
    };
    for (int k = nseg - 1; k >= 0; --k) {
        const int j0 = k * every, j1 = std::min(n_steps, (k + 1) * every);
        HBI_CUDA_TRY(cudaMemcpyAsync(h->d_y, h->d_ckpt + (size_t)k * n3, bytes3, cudaMemcpyDeviceToDevice, s));
        if ((st = ode_prep(h, s))) return st;
        for (int j = j0; j < j1; ++j)
            if ((st = fixed_step(h, with_store(j - j0), h_dts[j], s))) return st;
        for (int j = j1 - 1; j >= j0; --j)
            if ((st = reverse_step(h, with_store(j - j0), h_dts[j], s))) return st;
    }
    return HBI_OK;
}

hbi_status ode_rhs_vjp(hbi_handle *h, const double *d_v, double *d_ybar, double *d_grad_a, double *d_grad_dc,
                       cudaStream_t s) {
    const size_t n = (size_t)h->n, n3 = 3 * n;
    hbi_status st = adj_alloc(h, 1, 1);
    if (st) return st;
    const OdeArgs A = args(h);
    const int g = grid_for(h);
    HBI_CUDA_TRY(cudaMemcpyAsync(h->d_ys, h->d_y, n3 * sizeof(double), cudaMemcpyDeviceToDevice, s));
    rhs_pre_kernel<<<g, 256, 0, s>>>(A);
    if ((st = hmvm_launch(h, s, nullptr))) return st;
    vjp_prep_kernel<<<g, 256, 0, s>>>(A);
    gather_state_kernel<<<g, 256, 0, s>>>(d_v, h->d_perm, h->n, 3, h->d_Kbar);
    HBI_CUDA_TRY(cudaMemsetAsync(h->d_lam, 0, n3 * sizeof(double), s));
    HBI_CUDA_TRY(cudaMemsetAsync(h->d_gA, 0, n * sizeof(double), s));
    HBI_CUDA_TRY(cudaMemsetAsync(h->d_gDC, 0, n * sizeof(double), s));
    adj_pre_kernel<<<g, 256, 0, s>>>(A, 0, h->d_Kbar, h->adj->d_xt);
    if ((st = hmvm_launch(h->adj, s, nullptr))) return st;
    adj_post_kernel<<<g, 256, 0, s>>>(A, 0, h->adj->d_yp, h->d_lam, h->d_Kbar, h->d_gA, h->d_gDC, 0.0);
    scatter_state_kernel<<<g, 256, 0, s>>>(h->d_lam, h->d_perm, h->n, 3, d_ybar);
    if (d_grad_a) scatter_state_kernel<<<g, 256, 0, s>>>(h->d_gA, h->d_perm, h->n, 1, d_grad_a);
    if (d_grad_dc) scatter_state_kernel<<<g, 256, 0, s>>>(h->d_gDC, h->d_perm, h->n, 1, d_grad_dc);
    HBI_CUDA_TRY(cudaGetLastError());
    return HBI_OK;
}

}  // namespace hbi
