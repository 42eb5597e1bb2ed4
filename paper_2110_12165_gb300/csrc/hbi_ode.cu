// Rate-and-state right-hand side and adaptive Runge-Kutta attempt (Eqs. 7-16, 21-22),
// element-wise in FP64 in the permuted element order of the H-matrix.
//
// One attempt = six stages.  Stage s feeds the HMVM with x = (V_s - V_pl) r (the backslip
// loading of Eqs. 21-22 folded into the product), then a fused kernel evaluates
// k_s = f(y_s) (Eqs. 8, 10, 12, 13a-c) and immediately forms the next stage state
// y_{s+1} = y + dt sum_l a_{s+1,l} k_l, its slip rate (Eq. 7) and the next HMVM input.
// The last stage also forms the 5th/4th-order solutions, the error
// err = max_i |y5_i - y4_i| / max(|y5_i|, 1e-30), reduced over the grid; the last CTA to
// finish runs the step controller (Eqs. 14-15), so accept/reject never leaves the GPU.
// Every kernel returns immediately once the control block says the requested number of
// steps is done, which lets the host replay a captured attempt graph freely.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>

#include "hbi_internal.h"

namespace hbi {

// Cash & Karp (1990) embedded 4(5) tableau
__constant__ double c_A[6][5] = {
    {0, 0, 0, 0, 0},
    {1.0 / 5.0, 0, 0, 0, 0},
    {3.0 / 40.0, 9.0 / 40.0, 0, 0, 0},
    {3.0 / 10.0, -9.0 / 10.0, 6.0 / 5.0, 0, 0},
    {-11.0 / 54.0, 5.0 / 2.0, -70.0 / 27.0, 35.0 / 27.0, 0},
    {1631.0 / 55296.0, 175.0 / 512.0, 575.0 / 13824.0, 44275.0 / 110592.0, 253.0 / 4096.0}};
__constant__ double c_B5[6] = {37.0 / 378.0, 0.0, 250.0 / 621.0, 125.0 / 594.0, 0.0, 512.0 / 1771.0};
__constant__ double c_B4[6] = {2825.0 / 27648.0, 0.0, 18575.0 / 48384.0, 13525.0 / 55296.0, 277.0 / 14336.0, 0.25};

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
};

// Eq. 7 solved for V: V = 2 V0 exp(-phi/a) sinh(tau/(a sigma)), written as a difference of
// two exponentials so neither factor can overflow; with it dV/dtau (Eq. 13a), which costs
// no further exponential.  FP64 divisions and exponentials are the expensive operations of
// the element-wise work, so the friction constants come as reciprocals and a stage state's
// V and dV/dtau are computed once, when the state is formed, and kept.
__device__ __forceinline__ double slip_rate(double phi, double tau, double sig, double inv_a, double V0,
                                            double &dVdtau) {
    const double inv_sig = 1.0 / sig;
    const double q = tau * inv_sig;
    const double ep = exp((q - phi) * inv_a), em = exp((-q - phi) * inv_a);
    dVdtau = V0 * (ep + em) * inv_a * inv_sig;   // Eq. 13a
    return V0 * (ep - em);
}

__device__ __forceinline__ void write_x(const OdeArgs &A, int i, double V) {
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

__device__ __forceinline__ double read_y(const OdeArgs &A, int64_t k) {
    return A.acc_double ? ((const double *)A.yp)[k] : (double)((const float *)A.yp)[k];
}

// shear rate (projected on the rake) and normal-stress rate from the HMVM output
__device__ __forceinline__ void stress_rates(const OdeArgs &A, int i, double &AV, double &BV) {
    const int64_t o = (int64_t)A.nout * i;
    if (A.nout == 1) { AV = read_y(A, o); BV = 0.0; return; }
    if (A.nin == 1) { AV = read_y(A, o); BV = read_y(A, o + 1); return; }   // (tau_r, sigma)
    AV = A.cr[i] * read_y(A, o) + A.sr[i] * read_y(A, o + 1);
    BV = A.nout == 3 ? read_y(A, o + 2) : 0.0;
}

// dy/dt at element i for stage state (phi, tau, sig) with slip rate V (Eqs. 8, 10, 12, 13)
__device__ __forceinline__ void rhs_elem(const OdeArgs &A, int i, double phi, double tau, double sig, double V,
                                         double dVdtau, double &dphi, double &dtau, double &dsig) {
    double AV, BV;
    stress_rates(A, i, AV, BV);
    dphi = A.b_dc[i] * (A.V0 * exp((A.f0 - phi) * A.inv_b[i]) - V);   // Eq. 8
    dsig = BV;                                                          // Eq. 10 (+ loading)
    const double dVdsig = -(tau / sig) * dVdtau;                        // Eq. 13b
    const double dVdphi = -V * A.inv_a[i];                              // Eq. 13c
    dtau = (AV - A.eta * (dVdsig * dsig + dVdphi * dphi)) / (1.0 + A.eta * dVdtau);   // Eq. 12
}

__device__ __forceinline__ bool all_stopped(const OdeArgs &A) { return *(volatile int *)&A.g->stop != 0; }

// Start of a call: stage-1 state = y, V from Eq. 7, HMVM input.
__global__ void prep_kernel(OdeArgs A) {
    const int n = A.n;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const double phi = A.y[i], tau = A.y[n + i], sig = A.y[2 * n + i];
        A.ys[i] = phi; A.ys[n + i] = tau; A.ys[2 * n + i] = sig;
        double dV;
        const double V = slip_rate(phi, tau, sig, A.inv_a[i], A.V0, dV);
        A.Vs[i] = V; A.dVs[i] = dV;
        A.Vold[i] = V; A.dVold[i] = dV;
        write_x(A, i, V);
    }
}

// Stage s (0-based, 0..4): k_s from the HMVM output, then stage s+1 state and input.  After
// a rejected attempt y is unchanged, so stage 0 keeps k_0 = f(y) from its slot (its HMVM
// was skipped) and only the stage inputs for the new step size are formed.
__global__ void stage_kernel(OdeArgs A, int s) {
    if (all_stopped(A)) return;
    const int n = A.n;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const StepCtl &C = A.ctl[A.model[i]];
        if (C.stop) continue;
        const double dt = C.dt;
        const bool keep_k0 = s == 0 && C.reuse_k0;
        double *ks_ = A.k + (size_t)s * 3 * n;
        if (!keep_k0) {
            const double phi = A.ys[i], tau = A.ys[n + i], sig = A.ys[2 * n + i];
            double kp, kt, ks;
            rhs_elem(A, i, phi, tau, sig, A.Vs[i], A.dVs[i], kp, kt, ks);
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
        double dV1;
        const double V1 = slip_rate(p1, t1, s1, A.inv_a[i], A.V0, dV1);
        A.Vs[i] = V1; A.dVs[i] = dV1;
        write_x(A, i, V1);
    }
}

__device__ __forceinline__ unsigned long long dbits(double v) { return (unsigned long long)__double_as_longlong(v); }

// Stage 6, solutions of order 5 and 4, the element errors and their maxima per model.
// One element per thread; a block covers a contiguous element range and so at most a few
// models, whose maxima it gathers in shared memory before one atomic per model.
constexpr int FINAL_SEG = 8;
__global__ void final_kernel(OdeArgs A) {
    if (all_stopped(A)) return;
    __shared__ unsigned long long s_err[FINAL_SEG], s_vm[FINAL_SEG];
    const int n = A.n;
    const int i0 = blockIdx.x * blockDim.x, i = i0 + threadIdx.x;
    const int m0 = A.model[min(i0, n - 1)];
    if (threadIdx.x < FINAL_SEG) { s_err[threadIdx.x] = 0ull; s_vm[threadIdx.x] = 0ull; }
    __syncthreads();
    if (i < n) {
        const int m = A.model[i];
        StepCtl &C = A.ctl[m];
        if (!C.stop) {
            const double dt = C.dt;
            const double phi = A.ys[i], tau = A.ys[n + i], sig = A.ys[2 * n + i];
            double kp, kt, ks;
            rhs_elem(A, i, phi, tau, sig, A.Vs[i], A.dVs[i], kp, kt, ks);
            double *k5 = A.k + (size_t)5 * 3 * n;
            k5[i] = kp; k5[n + i] = kt; k5[2 * n + i] = ks;
            double y5[3], e = 0.0;
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
                double ec = fabs(y5[c] - y4) / fmax(fabs(y5[c]), 1e-30);
                if (!isfinite(ec)) { ec = INFINITY; atomicOr(&C.flags, 2); }   // rejected
                e = fmax(e, ec);
            }
            if (!(y5[2] > 0.0)) { e = INFINITY; atomicOr(&C.flags, 1); }     // sigma <= 0: rejected
            A.ys[i] = y5[0]; A.ys[n + i] = y5[1]; A.ys[2 * n + i] = y5[2];
            double dV5;
            const double V5 = slip_rate(y5[0], y5[1], y5[2], A.inv_a[i], A.V0, dV5);
            A.Vs[i] = V5; A.dVs[i] = dV5;
            const double vm = isfinite(V5) ? fabs(V5) : 0.0;
            // maxima through the ordered bit patterns of non-negative doubles
            if (m - m0 < FINAL_SEG) {
                atomicMax(&s_err[m - m0], dbits(e));
                atomicMax(&s_vm[m - m0], dbits(vm));
            } else {
                atomicMax(&C.err_bits, dbits(e));
                atomicMax(&C.vmax_bits, dbits(vm));
            }
        }
    }
    __syncthreads();
    if (threadIdx.x < FINAL_SEG && m0 + (int)threadIdx.x < A.n_models &&
        (s_err[threadIdx.x] | s_vm[threadIdx.x]) != 0ull) {
        StepCtl &C = A.ctl[m0 + threadIdx.x];
        atomicMax(&C.err_bits, s_err[threadIdx.x]);
        atomicMax(&C.vmax_bits, s_vm[threadIdx.x]);
    }
}

// The step controller of every active model (Eqs. 14-15, exponents read on err/eps): accept
// or reject, step records, the next dt, stop conditions, reset of the maxima.
__global__ void controller_kernel(OdeArgs A) {
    if (all_stopped(A)) return;
    for (int m = threadIdx.x; m < A.n_models; m += blockDim.x) {
        StepCtl *C = &A.ctl[m];
        if (C->stop) continue;
        const double dt = C->dt;
        const double e = __longlong_as_double((long long)C->err_bits);
        const double vm = __longlong_as_double((long long)C->vmax_bits);
        const double eps = C->eps;
        double dt_new;
        int accept;
        if (e > eps) {
            dt_new = fmax(0.5 * dt, 0.9 * dt * pow(e / eps, -0.25));
            accept = 0;
        } else {
            dt_new = e > 0.0 ? fmin(2.0 * dt, 0.9 * dt * pow(e / eps, -0.2)) : 2.0 * dt;
            accept = 1;
        }
        C->accept_flag = accept;
        C->dt_used = dt;
        if (accept) {
            C->t += dt;
            if (A.rec != nullptr && C->accepted < C->target) {
                hbi_step_record r;
                r.t = C->t; r.dt = dt; r.vmax = vm; r.rejects = (double)C->rejects;
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
    }
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
            A.Vold[i] = V5; A.dVold[i] = A.dVs[i];
        } else {
            A.ys[i] = A.y[i]; A.ys[n + i] = A.y[n + i]; A.ys[2 * n + i] = A.y[2 * n + i];
            A.Vs[i] = A.Vold[i]; A.dVs[i] = A.dVold[i];
        }
        write_x(A, i, A.Vold[i]);
    }
}
// Separate one-CTA kernel so that every commit CTA reads the same flags before a stop is set:
// models that reached their target (or failed) stop; the attempt graph stops when all have;
// the next attempt's first product is skipped when every active model rejected (k_0 kept).
__global__ void stop_kernel(OdeArgs A) {
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

// ------------------------------------------------------------- host side
namespace {
int grid_for(const hbi_handle *h) { return std::max(1, std::min((h->n + 255) / 256, 8 * std::max(1, h->num_sms))); }

OdeArgs args(hbi_handle *h) {
    OdeArgs A;
    A.n = h->n; A.nin = h->nin; A.nout = h->nout;
    A.y = h->d_y; A.D = h->d_D; A.ys = h->d_ys; A.Vs = h->d_Vs; A.Vold = h->d_Vold; A.k = h->d_k;
    A.dVs = h->d_dVs; A.dVold = h->d_dVold;
    A.inv_a = h->d_inv_a; A.inv_b = h->d_inv_b; A.b_dc = h->d_b_dc; A.cr = h->d_fcr; A.sr = h->d_fsr;
    A.f0 = h->g_f0; A.V0 = h->g_V0; A.Vpl = h->g_Vpl; A.eta = h->g_eta;
    A.xt = h->d_xt; A.yp = h->d_yp; A.acc_double = h->storage == HBI_FP64;
    A.n_models = h->n_models; A.rec_cap = h->rec_cap; A.model = h->d_model;
    A.ctl = h->d_ctl; A.g = h->d_gctl; A.rec = h->d_rec; A.mskip = h->d_mskip;
    return A;
}
}  // namespace

hbi_status ode_alloc(hbi_handle *h, int rec_cap) {
    const size_t n = (size_t)h->n;
    if (!h->d_y) {
        HBI_CUDA_TRY(cudaMalloc(&h->d_y, 3 * n * sizeof(double)));
        HBI_CUDA_TRY(cudaMalloc(&h->d_D, n * sizeof(double)));
        HBI_CUDA_TRY(cudaMalloc(&h->d_ys, 3 * n * sizeof(double)));
        HBI_CUDA_TRY(cudaMalloc(&h->d_Vs, n * sizeof(double)));
        HBI_CUDA_TRY(cudaMalloc(&h->d_Vold, n * sizeof(double)));
        HBI_CUDA_TRY(cudaMalloc(&h->d_dVs, n * sizeof(double)));
        HBI_CUDA_TRY(cudaMalloc(&h->d_dVold, n * sizeof(double)));
        HBI_CUDA_TRY(cudaMalloc(&h->d_k, 18 * n * sizeof(double)));
        HBI_CUDA_TRY(cudaMemset(h->d_k, 0, 18 * n * sizeof(double)));
        HBI_CUDA_TRY(cudaMalloc(&h->d_inv_a, n * sizeof(double)));
        HBI_CUDA_TRY(cudaMalloc(&h->d_inv_b, n * sizeof(double)));
        HBI_CUDA_TRY(cudaMalloc(&h->d_b_dc, n * sizeof(double)));
        HBI_CUDA_TRY(cudaMalloc(&h->d_fcr, n * sizeof(double)));
        HBI_CUDA_TRY(cudaMalloc(&h->d_fsr, n * sizeof(double)));
        const size_t nm = (size_t)h->n_models;
        HBI_CUDA_TRY(cudaMalloc(&h->d_ctl, nm * sizeof(StepCtl)));
        HBI_CUDA_TRY(cudaMemset(h->d_ctl, 0, nm * sizeof(StepCtl)));
        HBI_CUDA_TRY(cudaMallocHost(&h->h_ctl, nm * sizeof(StepCtl)));
        HBI_CUDA_TRY(cudaMalloc(&h->d_gctl, sizeof(GlobalCtl)));
        HBI_CUDA_TRY(cudaMemset(h->d_gctl, 0, sizeof(GlobalCtl)));
        HBI_CUDA_TRY(cudaMallocHost(&h->h_gctl, sizeof(GlobalCtl)));
        HBI_CUDA_TRY(cudaMalloc(&h->d_mskip, 2 * nm * sizeof(int)));
        HBI_CUDA_TRY(cudaMemset(h->d_mskip, 0, 2 * nm * sizeof(int)));
        if (!h->d_model) {
            std::vector<int> model(n, 0);
            for (int m = 0; m < h->n_models; ++m)
                for (int e = h->model_start[m]; e < h->model_start[m + 1]; ++e) model[e] = m;
            HBI_CUDA_TRY(cudaMalloc(&h->d_model, n * sizeof(int)));
            HBI_CUDA_TRY(cudaMemcpy(h->d_model, model.data(), n * sizeof(int), cudaMemcpyHostToDevice));
        }
    }
    if (rec_cap > h->rec_cap) {
        if (h->d_rec) cudaFree(h->d_rec);
        rec_cap = std::max(rec_cap, std::max(4096, 2 * h->rec_cap));   // grow rarely: re-capture
        HBI_CUDA_TRY(cudaMalloc(&h->d_rec, (size_t)h->n_models * rec_cap * sizeof(hbi_step_record)));
        h->rec_cap = rec_cap;
        if (h->graph_exec) { cudaGraphExecDestroy(h->graph_exec); h->graph_exec = nullptr; }
    }
    return HBI_OK;
}

hbi_status ode_set_friction(hbi_handle *h, const hbi_friction *f, cudaStream_t s) {
    friction_kernel<<<grid_for(h), 256, 0, s>>>(h->d_perm, h->n, f->d_a, f->d_b, f->d_dc, f->d_rake, h->d_inv_a,
                                                h->d_inv_b, h->d_b_dc, h->d_fcr, h->d_fsr);
    HBI_CUDA_TRY(cudaGetLastError());
    const double eta = f->mu / (2.0 * f->cs);
    if (h->graph_exec && (h->g_f0 != f->f0 || h->g_V0 != f->V0 || h->g_Vpl != f->Vpl || h->g_eta != eta)) {
        cudaGraphExecDestroy(h->graph_exec);
        h->graph_exec = nullptr;
    }
    h->g_f0 = f->f0; h->g_V0 = f->V0; h->g_Vpl = f->Vpl; h->g_eta = eta;
    return HBI_OK;
}

hbi_status ode_state_in(hbi_handle *h, const double *d_state, int with_slip, cudaStream_t s) {
    gather_state_kernel<<<grid_for(h), 256, 0, s>>>(d_state, h->d_perm, h->n, 3, h->d_y);
    if (with_slip)
        gather_state_kernel<<<grid_for(h), 256, 0, s>>>(d_state + 3 * (size_t)h->n, h->d_perm, h->n, 1, h->d_D);
    HBI_CUDA_TRY(cudaGetLastError());
    return HBI_OK;
}

hbi_status ode_state_out(hbi_handle *h, double *d_state, cudaStream_t s) {
    scatter_state_kernel<<<grid_for(h), 256, 0, s>>>(h->d_y, h->d_perm, h->n, 3, d_state);
    scatter_state_kernel<<<grid_for(h), 256, 0, s>>>(h->d_D, h->d_perm, h->n, 1, d_state + 3 * (size_t)h->n);
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

hbi_status ode_prep(hbi_handle *h, cudaStream_t s) {
    prep_kernel<<<grid_for(h), 256, 0, s>>>(args(h));
    HBI_CUDA_TRY(cudaGetLastError());
    return HBI_OK;
}

// One attempt: 6 x (HMVM + stage kernel), controller, commit.  A rejected attempt leaves y
// unchanged, so the next attempt skips its first HMVM and reuses k_0.
hbi_status ode_attempt(hbi_handle *h, cudaStream_t s) {
    OdeArgs A = args(h);
    const int *stop = &h->d_gctl->stop;
    const int g = grid_for(h);
    for (int st = 0; st < 6; ++st) {
        // the first product is skipped once every active model rejected (k_0 kept) or stopped
        hbi_status r = hmvm_launch(h, s, st == 0 ? &h->d_gctl->skip0 : stop,
                                   st == 0 ? h->d_mskip : h->d_mskip + h->n_models);
        if (r) return r;
        if (st < 5) stage_kernel<<<g, 256, 0, s>>>(A, st);
        else final_kernel<<<(h->n + 255) / 256, 256, 0, s>>>(A);
    }
    controller_kernel<<<1, 256, 0, s>>>(A);
    commit_kernel<<<g, 256, 0, s>>>(A);
    stop_kernel<<<1, 256, 0, s>>>(A);
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

}  // namespace hbi
