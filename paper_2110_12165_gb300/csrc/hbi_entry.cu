// Device-side entry generation and ACA (the build of the H-matrix, Sec. 3.1.2).
//
// The entries themselves (full space in closed form, the half-space correction) are in
// hbi_entry_math.cuh; this file holds the kernels that fill dense blocks and run ACA on
// them, and their host driver.
#include <cuda_runtime.h>

#include <cmath>

#include "hbi_entry_math.cuh"
#include "hbi_internal.h"

namespace hbi {

// ---------------------------------------------------------------- dense fill
struct DenseJob {
    int tau_start, tau_size, sig_start, sig_size;
    double *dst;          // row-major (nout*tau_size) x (nin*sig_size)
};

template <bool HALF>
__global__ void dense_fill_kernel(EntryGeo g, const DenseJob *jobs, int *bad) {
    const DenseJob jb = jobs[blockIdx.x];
    const int np = jb.tau_size * jb.sig_size;
    const int nc = g.nin * jb.sig_size;
    for (int p = threadIdx.x; p < np; p += blockDim.x) {
        const int ii = p / jb.sig_size, jj = p - ii * jb.sig_size;
        double E[3][2];
        if (!pair_op<HALF>(g, jb.tau_start + ii, jb.sig_start + jj, E)) atomicOr(bad, 1);
        for (int a = 0; a < g.nout; ++a)
            for (int c = 0; c < g.nin; ++c)
                jb.dst[(size_t)(ii * g.nout + a) * nc + jj * g.nin + c] = E[a][c];
    }
}

// ---------------------------------------------------------------------- ACA
struct AcaJob {
    int tau_start, tau_size, sig_start, sig_size;
    int m, nc, rmax, rcap;
    double *U, *V;        // m x rmax and nc x rmax, column-major
    unsigned char *flags; // m + nc bytes (used rows, used columns)
};
struct AcaOut { int rank, status; };  // status: 0 converged, 1 rank budget exhausted, 2 capped, 3 singular

constexpr int ACA_THREADS = 256;
constexpr int ACA_WARPS = ACA_THREADS / 32;

// block-wide argmax of (value, index) with ties to the smaller index; -1 if all excluded
__device__ void block_argmax(double v, int idx, double *sv, int *si, double &best, int &bidx) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        double ov = __shfl_down_sync(0xffffffffu, v, o);
        int oi = __shfl_down_sync(0xffffffffu, idx, o);
        if (oi >= 0 && (idx < 0 || ov > v || (ov == v && oi < idx))) { v = ov; idx = oi; }
    }
    if (lane == 0) { sv[w] = v; si[w] = idx; }
    __syncthreads();
    if (threadIdx.x == 0) {
        double bv = sv[0];
        int bi = si[0];
        for (int k = 1; k < ACA_WARPS; ++k)
            if (si[k] >= 0 && (bi < 0 || sv[k] > bv || (sv[k] == bv && si[k] < bi))) { bv = sv[k]; bi = si[k]; }
        sv[0] = bv; si[0] = bi;
    }
    __syncthreads();
    best = sv[0];
    bidx = si[0];
    __syncthreads();
}

__device__ double block_sum(double v, double *sv) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if (lane == 0) sv[w] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int k = 0; k < ACA_WARPS; ++k) s += sv[k];
        sv[0] = s;
    }
    __syncthreads();
    double r = sv[0];
    __syncthreads();
    return r;
}

// Adaptive cross approximation with partial pivoting (Sec. 3.1.2; Bebendorf 2000), one
// CTA per block: start at row 0; pivot column = argmax of the residual row over unused
// columns; next row = argmax |u_k| over unused rows (ties to the smaller index); a zero
// residual row moves on to the first unused row; stop once |u_k||v_k| <= eps ||S_k||_F
// (Frobenius norm of the approximant updated recursively).  Reaching the rank cap
// floor(m n / (m + n)) marks the block for dense storage.
template <bool HALF>
__global__ void __launch_bounds__(ACA_THREADS) aca_kernel(EntryGeo g, const AcaJob *jobs, AcaOut *outs,
                                                          double eps) {
    __shared__ double sv[ACA_WARPS];
    __shared__ int si[ACA_WARPS];
    __shared__ double s_cross[ACA_WARPS];
    const AcaJob jb = jobs[blockIdx.x];
    const int m = jb.m, nc = jb.nc;
    unsigned char *urow = jb.flags, *ucol = jb.flags + m;
    for (int k = threadIdx.x; k < m + nc; k += blockDim.x) jb.flags[k] = 0;
    __syncthreads();
    int k = 0, i = 0, status = 0;
    double normS2 = 0.0;
    bool singular = false;
    for (int guard = 0; guard < m + nc + 2; ++guard) {
        if (k >= jb.rcap) { status = 2; break; }
        if (k >= jb.rmax) { status = 1; break; }
        // residual row i -> V[:, k]
        double *vk = jb.V + (size_t)k * nc;
        {
            const int ie = jb.tau_start + i / g.nout, co = i % g.nout;
            for (int jj = threadIdx.x; jj < jb.sig_size; jj += blockDim.x) {
                double E[3][2];
                if (!pair_op<HALF>(g, ie, jb.sig_start + jj, E)) singular = true;
                for (int c = 0; c < g.nin; ++c) {
                    const int J = jj * g.nin + c;
                    double val = E[co][c];
                    for (int l = 0; l < k; ++l) val -= jb.U[(size_t)l * m + i] * jb.V[(size_t)l * nc + J];
                    vk[J] = val;
                }
            }
        }
        __syncthreads();
        if (threadIdx.x == 0) urow[i] = 1;
        double best;
        int j;
        {
            double v = -1.0;
            int idx = -1;
            for (int J = threadIdx.x; J < nc; J += blockDim.x) {
                if (ucol[J]) continue;
                double a = fabs(vk[J]);
                if (idx < 0 || a > v) { v = a; idx = J; }
            }
            block_argmax(v, idx, sv, si, best, j);
        }
        if (j < 0 || !(best > 0.0)) {
            // zero residual row: move to the first unused row
            int nxt = -1;
            {
                int idx = -1;
                for (int I = threadIdx.x; I < m; I += blockDim.x)
                    if (!urow[I]) { idx = I; break; }
                double dummy;
                block_argmax(idx >= 0 ? -(double)idx : -1e300, idx, sv, si, dummy, nxt);
            }
            if (nxt < 0) break;
            i = nxt;
            continue;
        }
        const double piv = vk[j];
        for (int J = threadIdx.x; J < nc; J += blockDim.x) vk[J] /= piv;
        // residual column j -> U[:, k]
        double *uk = jb.U + (size_t)k * m;
        {
            const int je = jb.sig_start + j / g.nin, ci = j % g.nin;
            for (int ii = threadIdx.x; ii < jb.tau_size; ii += blockDim.x) {
                double E[3][2];
                if (!pair_op<HALF>(g, jb.tau_start + ii, je, E)) singular = true;
                for (int a = 0; a < g.nout; ++a) {
                    const int I = ii * g.nout + a;
                    double val = E[a][ci];
                    for (int l = 0; l < k; ++l) val -= jb.V[(size_t)l * nc + j] * jb.U[(size_t)l * m + I];
                    uk[I] = val;
                }
            }
        }
        __syncthreads();
        if (threadIdx.x == 0) ucol[j] = 1;
        // norms: ||u||^2, ||v||^2 and sum_l (u_l . u)(v_l . v)
        double pu = 0.0, pv = 0.0;
        for (int I = threadIdx.x; I < m; I += blockDim.x) pu += uk[I] * uk[I];
        for (int J = threadIdx.x; J < nc; J += blockDim.x) pv += vk[J] * vk[J];
        const double uu = block_sum(pu, sv), vv = block_sum(pv, sv);
        {
            const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
            double cw = 0.0;
            for (int l = w; l < k; l += ACA_WARPS) {
                double a = 0.0, b = 0.0;
                const double *ul = jb.U + (size_t)l * m, *vl = jb.V + (size_t)l * nc;
                for (int I = lane; I < m; I += 32) a += ul[I] * uk[I];
                for (int J = lane; J < nc; J += 32) b += vl[J] * vk[J];
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) {
                    a += __shfl_xor_sync(0xffffffffu, a, o);
                    b += __shfl_xor_sync(0xffffffffu, b, o);
                }
                cw += a * b;
            }
            if (lane == 0) s_cross[w] = cw;
            __syncthreads();
            double cross = 0.0;
            for (int q = 0; q < ACA_WARPS; ++q) cross += s_cross[q];
            __syncthreads();
            normS2 += 2.0 * cross + uu * vv;
        }
        ++k;
        if (sqrt(uu * vv) <= eps * sqrt(normS2 > 0.0 ? normS2 : 0.0)) break;
        // next row: argmax |u_k| over unused rows
        int nxt;
        {
            double v = -1.0;
            int idx = -1;
            for (int I = threadIdx.x; I < m; I += blockDim.x) {
                if (urow[I]) continue;
                double a = fabs(uk[I]);
                if (idx < 0 || a > v) { v = a; idx = I; }
            }
            block_argmax(v, idx, sv, si, best, nxt);
        }
        if (nxt < 0) break;
        i = nxt;
    }
    // reduce the singular flag
    __shared__ int s_sing;
    if (threadIdx.x == 0) s_sing = 0;
    __syncthreads();
    if (singular) atomicOr(&s_sing, 1);
    __syncthreads();
    if (threadIdx.x == 0) {
        outs[blockIdx.x].rank = k;
        outs[blockIdx.x].status = s_sing ? 3 : status;
    }
}

// ------------------------------------------------------------- host driver
namespace {
template <typename T>
hbi_status dev_alloc(T **p, size_t count, std::vector<void *> &owned) {
    void *q = nullptr;
    if (count == 0) count = 1;
    hbi_status st = dev_malloc(&q, count * sizeof(T));
    if (st) return st;
    owned.push_back(q);
    *p = (T *)q;
    return HBI_OK;
}
}  // namespace

hbi_status device_build_factors(hbi_handle *h, const Tree &T, std::vector<Block> &blocks, double eps,
                                std::vector<void *> &owned) {
    EntryGeo g{h->d_geom, h->d_verts, h->d_rake, h->nv, h->op, h->nin, h->nout, h->mu, h->nu};
    int *d_bad = nullptr;
    hbi_status st = dev_alloc(&d_bad, 1, owned);
    if (st) return st;
    HBI_CUDA_TRY(cudaMemset(d_bad, 0, sizeof(int)));

    // ---- low-rank candidates: ACA with growing rank budgets
    std::vector<int> pending;
    for (int b = 0; b < (int)blocks.size(); ++b)
        if (blocks[b].lowrank) pending.push_back(b);
    const int budgets[] = {48, 256, 2048};
    for (int pass = 0; pass < 3 && !pending.empty(); ++pass) {
        // batches bounded by a workspace budget
        size_t free_b = 0, total_b = 0;
        HBI_CUDA_TRY(cudaMemGetInfo(&free_b, &total_b));
        const size_t cap_bytes = std::max<size_t>((size_t)(0.45 * (double)free_b), (size_t)1 << 28);
        std::vector<int> next;
        size_t pos = 0;
        while (pos < pending.size()) {
            std::vector<AcaJob> jobs;
            std::vector<int> ids;
            size_t bytes = 0;
            while (pos < pending.size()) {
                const Block &B = blocks[pending[pos]];
                const int rcap = (int)((B.m * B.nc) / (B.m + B.nc));
                const int rmax = std::max(1, std::min(rcap, budgets[pass]));
                size_t need = (size_t)(B.m + B.nc) * rmax * sizeof(double) + (size_t)(B.m + B.nc) + 64;
                if (!jobs.empty() && bytes + need > cap_bytes) break;
                const Cluster &A = T.cl[B.tau], &S = T.cl[B.sig];
                jobs.push_back(AcaJob{A.start, A.size, S.start, S.size, (int)B.m, (int)B.nc, rmax, rcap,
                                      nullptr, nullptr, nullptr});
                ids.push_back(pending[pos]);
                bytes += need;
                ++pos;
            }
            // one allocation for the batch's factors (kept until packing), one for flags
            size_t nd = 0, nf = 0;
            for (auto &J : jobs) { nd += (size_t)(J.m + J.nc) * J.rmax; nf += (size_t)(J.m + J.nc); }
            double *d_fac = nullptr;
            unsigned char *d_flags = nullptr;
            DevScratch tmp;   // flags, job and result tables of this batch
            if ((st = dev_alloc(&d_fac, nd, owned)) || (st = tmp.alloc(&d_flags, nf ? nf : 1))) return st;
            size_t od = 0, of = 0;
            for (auto &J : jobs) {
                J.U = d_fac + od;
                J.V = d_fac + od + (size_t)J.m * J.rmax;
                J.flags = d_flags + of;
                od += (size_t)(J.m + J.nc) * J.rmax;
                of += (size_t)(J.m + J.nc);
            }
            AcaJob *d_jobs = nullptr;
            AcaOut *d_outs = nullptr;
            if ((st = tmp.alloc(&d_jobs, jobs.size() * sizeof(AcaJob))) ||
                (st = tmp.alloc(&d_outs, jobs.size() * sizeof(AcaOut))))
                return st;
            HBI_CUDA_TRY(cudaMemcpy(d_jobs, jobs.data(), jobs.size() * sizeof(AcaJob), cudaMemcpyHostToDevice));
            if (h->half_space)
                aca_kernel<true><<<(unsigned)jobs.size(), ACA_THREADS>>>(g, d_jobs, d_outs, eps);
            else
                aca_kernel<false><<<(unsigned)jobs.size(), ACA_THREADS>>>(g, d_jobs, d_outs, eps);
            HBI_CUDA_TRY(cudaGetLastError());
            std::vector<AcaOut> outs(jobs.size());
            HBI_CUDA_TRY(cudaMemcpy(outs.data(), d_outs, outs.size() * sizeof(AcaOut), cudaMemcpyDeviceToHost));
            for (size_t q = 0; q < jobs.size(); ++q) {
                Block &B = blocks[ids[q]];
                if (outs[q].status == 3) {
                    set_error("receiver on an element edge (singular stress)");
                    return HBI_ERR_SINGULAR;
                }
                if (inject_aca_failure()) {   // a block's ACA reported as not converged
                    set_error("ACA did not converge within rank 2048 (injected)");
                    return HBI_ERR_ACA_FAIL;
                }
                if (outs[q].status == 0) {
                    B.rank = outs[q].rank;
                    B.d_src = jobs[q].U;       // U column-major, leading dimension m
                    B.d_src2 = jobs[q].V;      // V column-major, leading dimension nc
                } else if (outs[q].status == 2) {
                    B.lowrank = 0;             // rank cap: dense storage
                } else {
                    if (pass == 2) {
                        set_error("ACA did not converge within rank 2048");
                        return HBI_ERR_ACA_FAIL;
                    }
                    next.push_back(ids[q]);
                }
            }
        }
        pending.swap(next);
    }

    // ---- dense blocks (near field and rank-capped)
    std::vector<DenseJob> djobs;
    size_t nd = 0;
    for (auto &B : blocks)
        if (!B.lowrank) nd += (size_t)B.m * B.nc;
    double *d_dense = nullptr;
    if ((st = dev_alloc(&d_dense, nd, owned))) return st;
    size_t od = 0;
    for (auto &B : blocks) {
        if (B.lowrank) continue;
        const Cluster &A = T.cl[B.tau], &S = T.cl[B.sig];
        djobs.push_back(DenseJob{A.start, A.size, S.start, S.size, d_dense + od});
        B.d_src = d_dense + od;
        B.d_src2 = nullptr;
        B.rank = 0;
        od += (size_t)B.m * B.nc;
    }
    if (!djobs.empty()) {
        DenseJob *d_dj = nullptr;
        DevScratch tmp;
        if ((st = tmp.upload(&d_dj, djobs))) return st;
        if (h->half_space)
            dense_fill_kernel<true><<<(unsigned)djobs.size(), 256>>>(g, d_dj, d_bad);
        else
            dense_fill_kernel<false><<<(unsigned)djobs.size(), 256>>>(g, d_dj, d_bad);
        HBI_CUDA_TRY(cudaGetLastError());
        HBI_CUDA_TRY(cudaDeviceSynchronize());
    }
    int bad = 0;
    HBI_CUDA_TRY(cudaMemcpy(&bad, d_bad, sizeof(int), cudaMemcpyDeviceToHost));
    if (bad) {
        set_error("receiver on an element edge (singular stress)");
        return HBI_ERR_SINGULAR;
    }
    return HBI_OK;
}

}  // namespace hbi
