// Rank recompression of ACA factors (an optional build step after Sec. 3.1.2's ACA).
//
// ACA stops at a rank that meets Eq. 19 but is not the smallest such rank.  For a block
// A ~ U V^T (U: m x r, V: n x r) this step finds the best rank-r' approximation of U V^T
// itself: with U = Q_U R_U and V = Q_V R_V, U V^T = Q_U (R_U R_V^T) Q_V^T, so the singular
// values of U V^T are those of the r x r core C = R_U R_V^T.  Keeping the leading r' of them
// such that the discarded tail has Frobenius norm <= tol ||U V^T||_F gives
//     U' = U R_U^{-1} W_r' Sigma_r',   V' = V R_V^{-1} Z_r'   (C = W Sigma Z^T).
// R_U, R_V come from the Cholesky factors of the column-scaled Gram matrices (Cholesky-QR;
// the scaling keeps them well conditioned for ACA factors), the core's SVD from one-sided
// Jacobi (Hestenes) sweeps in a round-robin order.  All in FP64, one CTA per block; blocks
// whose Gram matrix is numerically singular are left as they are.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>

#include "hbi_internal.h"

namespace hbi {

constexpr int RC_THREADS = 256;
constexpr int RC_RMAX = 48;          // blocks of higher rank are left as they are
constexpr int RC_TILE = 32;          // rows per tile of the Gram and update passes
constexpr int RC_PAIRS = (RC_RMAX * (RC_RMAX + 1) / 2 + RC_THREADS - 1) / RC_THREADS;

struct RecompJob {
    double *U, *V;       // column-major, leading dimensions m and n, rank r (updated in place)
    int m, n, r;
};

// G = X^T X for X (len x r, column-major); tile = RC_TILE x r scratch in shared memory.
__device__ void gram(const double *X, int len, int r, double *G, double *tile) {
    const int npair = r * (r + 1) / 2;
    int pa[RC_PAIRS], pb[RC_PAIRS];
    double acc[RC_PAIRS];
#pragma unroll
    for (int q = 0; q < RC_PAIRS; ++q) {
        const int p = threadIdx.x + q * blockDim.x;
        int a = 0, rem = p;
        while (a < r && rem >= r - a) { rem -= r - a; ++a; }   // pair p -> (a, a + rem), a <= b
        pa[q] = p < npair ? a : -1;
        pb[q] = a + rem;
        acc[q] = 0.0;
    }
    for (int row0 = 0; row0 < len; row0 += RC_TILE) {
        const int rows = min(RC_TILE, len - row0);
        for (int e = threadIdx.x; e < RC_TILE * r; e += blockDim.x) {
            const int k = e / RC_TILE, i = e - k * RC_TILE;
            tile[i * r + k] = i < rows ? X[(size_t)k * len + row0 + i] : 0.0;
        }
        __syncthreads();
#pragma unroll
        for (int q = 0; q < RC_PAIRS; ++q) {
            if (pa[q] < 0) continue;
            double s = 0.0;
            for (int i = 0; i < RC_TILE; ++i) s += tile[i * r + pa[q]] * tile[i * r + pb[q]];
            acc[q] += s;
        }
        __syncthreads();
    }
#pragma unroll
    for (int q = 0; q < RC_PAIRS; ++q) {
        if (pa[q] < 0) continue;
        G[pa[q] * r + pb[q]] = acc[q];
        G[pb[q] * r + pa[q]] = acc[q];
    }
    __syncthreads();
}

// In place: G (symmetric r x r, row-major) -> upper-triangular R with G = R^T R, computed on
// the column-scaled Gram matrix and returned unscaled (R = R_scaled D).  False if singular.
__device__ bool chol_scaled(double *G, int r, double *d, int *s_ok) {
    for (int k = threadIdx.x; k < r; k += blockDim.x) d[k] = sqrt(fmax(G[k * r + k], 0.0));
    __syncthreads();
    for (int e = threadIdx.x; e < r * r; e += blockDim.x) {
        const int a = e / r, b = e - a * r;
        const double den = d[a] * d[b];
        G[e] = den > 0.0 ? G[e] / den : (a == b ? 1.0 : 0.0);
    }
    if (threadIdx.x == 0) *s_ok = 1;
    __syncthreads();
    for (int k = 0; k < r; ++k) {
        if (threadIdx.x == 0) {
            const double p = G[k * r + k];
            if (!(p > 1e-13)) *s_ok = 0;
            G[k * r + k] = sqrt(fmax(p, 1e-300));
        }
        __syncthreads();
        const double pk = G[k * r + k];
        for (int j = k + 1 + threadIdx.x; j < r; j += blockDim.x) G[k * r + j] /= pk;
        __syncthreads();
        const int rem = r - k - 1;   // trailing update of the upper triangle, k < i <= j
        for (int e = threadIdx.x; e < rem * rem; e += blockDim.x) {
            const int i = k + 1 + e / rem, j = k + 1 + e % rem;
            if (j >= i) G[i * r + j] -= G[k * r + i] * G[k * r + j];
        }
        __syncthreads();
    }
    for (int e = threadIdx.x; e < r * r; e += blockDim.x) {
        const int a = e / r, b = e - a * r;
        G[e] = b < a ? 0.0 : G[e] * d[b];
    }
    __syncthreads();
    return *s_ok != 0;
}

// shared memory (doubles): RU, RV, C, Z, TU, TV (r*r each), tile (RC_TILE*r), sv (r)
__global__ void __launch_bounds__(RC_THREADS) recompress_kernel(const RecompJob *jobs, int *new_rank, double tol) {
    extern __shared__ __align__(16) double sm[];
    __shared__ int s_ok, s_keep;
    __shared__ int s_order[RC_RMAX];
    __shared__ double s_d[RC_RMAX];
    const RecompJob J = jobs[blockIdx.x];
    const int r = J.r, rr = r * r;
    double *RU = sm, *RV = RU + rr, *C = RV + rr, *Z = C + rr, *TU = Z + rr, *TV = TU + rr;
    double *tile = TV + rr, *sv = tile + RC_TILE * r;
    if (threadIdx.x == 0) new_rank[blockIdx.x] = r;
    if (r < 2 || r > RC_RMAX) return;
    gram(J.U, J.m, r, RU, tile);
    if (!chol_scaled(RU, r, s_d, &s_ok)) return;
    gram(J.V, J.n, r, RV, tile);
    if (!chol_scaled(RV, r, s_d, &s_ok)) return;
    // core C = R_U R_V^T (column-major: C[i + j r]), Z = I
    for (int e = threadIdx.x; e < rr; e += blockDim.x) {
        const int i = e % r, j = e / r;
        double s = 0.0;
        for (int k = max(i, j); k < r; ++k) s += RU[i * r + k] * RV[j * r + k];
        C[e] = s;
        Z[e] = (i == j) ? 1.0 : 0.0;
    }
    __syncthreads();
    // one-sided Jacobi on the columns of C; disjoint pairs of one round-robin round per step
    const int np = (r + 1) & ~1;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int sweep = 0; sweep < 30; ++sweep) {
        if (threadIdx.x == 0) s_ok = 0;   // "a rotation happened in this sweep"
        __syncthreads();
        for (int round = 0; round < np - 1; ++round) {
            for (int k = warp; k < np / 2; k += nw) {
                int p = k == 0 ? 0 : (k - 1 + round) % (np - 1) + 1;
                const int kk = np - 1 - k;
                int q = kk == 0 ? 0 : (kk - 1 + round) % (np - 1) + 1;
                if (p > q) { const int t = p; p = q; q = t; }
                if (q >= r) continue;
                double a = 0.0, b = 0.0, c = 0.0;
                for (int i = lane; i < r; i += 32) {
                    const double x = C[i + p * r], y = C[i + q * r];
                    a += x * x; b += y * y; c += x * y;
                }
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) {
                    a += __shfl_xor_sync(0xffffffffu, a, o);
                    b += __shfl_xor_sync(0xffffffffu, b, o);
                    c += __shfl_xor_sync(0xffffffffu, c, o);
                }
                if (c == 0.0 || fabs(c) <= 1e-15 * sqrt(a * b)) continue;
                const double zeta = (b - a) / (2.0 * c);
                const double t = (zeta >= 0.0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
                const double cs = 1.0 / sqrt(1.0 + t * t), sn = cs * t;
                for (int i = lane; i < r; i += 32) {
                    const double x = C[i + p * r], y = C[i + q * r];
                    C[i + p * r] = cs * x - sn * y;
                    C[i + q * r] = sn * x + cs * y;
                    const double u = Z[i + p * r], v = Z[i + q * r];
                    Z[i + p * r] = cs * u - sn * v;
                    Z[i + q * r] = sn * u + cs * v;
                }
                if (lane == 0) s_ok = 1;
            }
            __syncthreads();
        }
        const int rotated = s_ok;
        __syncthreads();
        if (!rotated) break;
    }
    // singular values = column norms of C; order; smallest rank within the tolerance
    for (int k = threadIdx.x; k < r; k += blockDim.x) {
        double s = 0.0;
        for (int i = 0; i < r; ++i) s += C[i + k * r] * C[i + k * r];
        sv[k] = sqrt(s);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int k = 0; k < r; ++k) s_order[k] = k;
        for (int a = 1; a < r; ++a) {   // insertion sort, descending
            const int v = s_order[a];
            int b = a - 1;
            while (b >= 0 && sv[s_order[b]] < sv[v]) { s_order[b + 1] = s_order[b]; --b; }
            s_order[b + 1] = v;
        }
        double tot = 0.0;
        for (int k = 0; k < r; ++k) tot += sv[k] * sv[k];
        double tail = 0.0;
        int keep = r;
        while (keep > 1) {
            const double sk = sv[s_order[keep - 1]];
            if (tail + sk * sk > tol * tol * tot) break;
            tail += sk * sk;
            --keep;
        }
        s_keep = keep;
    }
    __syncthreads();
    const int rk = s_keep;
    if (rk >= r) return;   // nothing to gain
    // TU = R_U^{-1} C[:, order[:rk]], TV = R_V^{-1} Z[:, order[:rk]] (back substitution)
    for (int k = threadIdx.x; k < 2 * rk; k += blockDim.x) {
        const bool isU = k < rk;
        const int kk = isU ? k : k - rk;
        const double *R = isU ? RU : RV, *rhs = (isU ? C : Z) + s_order[kk] * r;
        double *out = (isU ? TU : TV) + kk * r;
        for (int i = r - 1; i >= 0; --i) {
            double s = rhs[i];
            for (int j = i + 1; j < r; ++j) s -= R[i * r + j] * out[j];
            out[i] = s / R[i * r + i];
        }
    }
    __syncthreads();
    // in place U <- U TU and V <- V TV, a tile of rows at a time (read fully before writing)
    for (int pass = 0; pass < 2; ++pass) {
        double *X = pass == 0 ? J.U : J.V;
        const int len = pass == 0 ? J.m : J.n;
        const double *Tm = pass == 0 ? TU : TV;
        for (int row0 = 0; row0 < len; row0 += RC_TILE) {
            const int rows = min(RC_TILE, len - row0);
            for (int e = threadIdx.x; e < RC_TILE * r; e += blockDim.x) {
                const int k = e / RC_TILE, i = e - k * RC_TILE;
                tile[i * r + k] = i < rows ? X[(size_t)k * len + row0 + i] : 0.0;
            }
            __syncthreads();
            for (int e = threadIdx.x; e < RC_TILE * rk; e += blockDim.x) {
                const int k = e / RC_TILE, i = e - k * RC_TILE;
                if (i < rows) {
                    double s = 0.0;
                    for (int j = 0; j < r; ++j) s += tile[i * r + j] * Tm[j + k * r];
                    X[(size_t)k * len + row0 + i] = s;
                }
            }
            __syncthreads();
        }
    }
    if (threadIdx.x == 0) new_rank[blockIdx.x] = rk;
}

// Recompress every low-rank block of rank 2..RC_RMAX; updates ranks in place (the first
// r' columns of the same U and V storage hold the new factors).
hbi_status recompress_lowrank(std::vector<Block> &blocks, double tol) {
    std::vector<RecompJob> jobs;
    std::vector<int> ids;
    int rmax = 0;
    for (size_t b = 0; b < blocks.size(); ++b) {
        Block &B = blocks[b];
        if (!B.lowrank || B.rank < 2 || B.rank > RC_RMAX) continue;
        jobs.push_back(RecompJob{const_cast<double *>(B.d_src), const_cast<double *>(B.d_src2), (int)B.m, (int)B.nc,
                                 B.rank});
        ids.push_back((int)b);
        rmax = std::max(rmax, B.rank);
    }
    if (jobs.empty()) return HBI_OK;
    const size_t smem = ((size_t)6 * rmax * rmax + (size_t)RC_TILE * rmax + rmax) * sizeof(double);
    HBI_CUDA_TRY(cudaFuncSetAttribute(recompress_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    RecompJob *d_jobs = nullptr;
    int *d_rank = nullptr;
    DevScratch tmp;
    hbi_status st;
    if ((st = tmp.upload(&d_jobs, jobs)) || (st = tmp.alloc(&d_rank, jobs.size() * sizeof(int)))) return st;
    recompress_kernel<<<(unsigned)jobs.size(), RC_THREADS, smem>>>(d_jobs, d_rank, tol);
    HBI_CUDA_TRY(cudaGetLastError());
    std::vector<int> nr(jobs.size());
    HBI_CUDA_TRY(cudaMemcpy(nr.data(), d_rank, nr.size() * sizeof(int), cudaMemcpyDeviceToHost));
    for (size_t q = 0; q < jobs.size(); ++q) {
        Block &B = blocks[ids[q]];
        if (nr[q] < B.rank) B.rank = nr[q];
    }
    return HBI_OK;
}

}  // namespace hbi
