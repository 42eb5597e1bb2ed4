// H-matrix x vector product (Sec. 3.1.3, Eq. 20) as two persistent GEMV phases.
//
// Eq. 20 splits every low-rank block into t_b = V_b^T x_sigma followed by y_tau += U_b t_b.
// Phase VT computes all t_b; phase UY computes every output row once.  Both phases run the
// same kernel over "tasks": a row-major panel of stored factor values with one output per
// panel row, fed by an input vector that the CTA gathers into shared memory.
//   VT tasks  : all low-rank blocks sharing a column cluster sigma stacked (rows = their
//               V columns), optionally split into column chunks (partial sums reduced in a
//               fixed order afterwards).  Input = the contiguous x_sigma slice.
//   UY tasks  : one per leaf row cluster: the concatenation over every block covering those
//               rows of its U slice (low-rank) or its dense rows.  Input = the matching
//               t_b and x_sigma values.  Each output row is written exactly once, so the
//               result needs no atomics and is bitwise reproducible.
// A UY row has two segments, the dense near-field columns and the low-rank U columns, so the
// two kinds of block can be stored in different precisions: FP64, FP32, FP16 or BF16 for
// both, or FP32 near field + FP16 far field (HBI_MIXED).  FP16/BF16 values carry one
// power-of-two scale per factor column: U and V column scales fold into the VT output,
// dense column scales into the UY gather, so the inner loops are plain dot products with
// FP32 (FP64) accumulation.
// Tasks are claimed from an atomic counter in decreasing size order (LPT), which keeps
// the persistent grid (a multiple of the SM count) busy until the end.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <map>
#include <mutex>
#include <numeric>
#include <type_traits>

#include "hbi_internal.h"

namespace hbi {

constexpr int GEMV_THREADS = 256;
constexpr int GEMV_RPW = 4;                 // rows per warp pass
constexpr int64_t VT_TARGET_BYTES = 192 << 10;  // column-chunk size target of a VT task

// -------------------------------------------------------- vector decoding
__device__ __forceinline__ uint4 ld_stream(const void *p) {
    uint4 r;
    asm volatile("ld.global.nc.L1::no_allocate.v4.u32 {%0,%1,%2,%3}, [%4];"
                 : "=r"(r.x), "=r"(r.y), "=r"(r.z), "=r"(r.w)
                 : "l"(p));
    return r;
}

template <typename T> struct Vec;
template <> struct Vec<double> {
    static constexpr int N = 2;
    using A = double;
    __device__ static void fma(const uint4 &r, const double *z, double &acc) {
        double2 v = *reinterpret_cast<const double2 *>(&r);
        acc = ::fma(v.x, z[0], acc);
        acc = ::fma(v.y, z[1], acc);
    }
};
template <> struct Vec<float> {
    static constexpr int N = 4;
    using A = float;
    __device__ static void fma(const uint4 &r, const float *z, float &acc) {
        acc = fmaf(__uint_as_float(r.x), z[0], acc);
        acc = fmaf(__uint_as_float(r.y), z[1], acc);
        acc = fmaf(__uint_as_float(r.z), z[2], acc);
        acc = fmaf(__uint_as_float(r.w), z[3], acc);
    }
};
template <> struct Vec<__half> {
    static constexpr int N = 8;
    using A = float;
    __device__ static void fma(const uint4 &r, const float *z, float &acc) {
        const unsigned w[4] = {r.x, r.y, r.z, r.w};
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            __half2 h = *reinterpret_cast<const __half2 *>(&w[q]);
            float2 f = __half22float2(h);
            acc = fmaf(f.x, z[2 * q], acc);
            acc = fmaf(f.y, z[2 * q + 1], acc);
        }
    }
};
template <> struct Vec<__nv_bfloat16> {
    static constexpr int N = 8;
    using A = float;
    __device__ static void fma(const uint4 &r, const float *z, float &acc) {
        const unsigned w[4] = {r.x, r.y, r.z, r.w};
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            // bf16 -> fp32 is a 16-bit left shift of the bit pattern
            float lo = __uint_as_float(w[q] << 16), hi = __uint_as_float(w[q] & 0xffff0000u);
            acc = fmaf(lo, z[2 * q], acc);
            acc = fmaf(hi, z[2 * q + 1], acc);
        }
    }
};

template <typename A> __device__ __forceinline__ A warp_sum(A v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// ------------------------------------------------------------- GEMV kernel
template <typename A> struct GemvBufs {
    A *xt;          // [x | t]
    A *part;        // partial sums of chunked VT groups
    A *y;           // HMVM output
    int *counter;   // work counter of this phase (zero before the launch)
    int *red_cnt;   // arrival counters of chunked VT groups (zero before the product)
};

// acc[q] += row q of a row-major segment (stride cpad) . z for q < nr <= GEMV_RPW; the row
// is split over `lpr` lanes (sub-lane sl), each taking 16-byte vectors lpr apart.
template <typename T>
__device__ __forceinline__ void segment_dot(const T *__restrict__ rowp, int cpad, int nr, const typename Vec<T>::A *z,
                                            int sl, int lpr, typename Vec<T>::A (&acc)[GEMV_RPW]) {
    using A = typename Vec<T>::A;
    constexpr int VEC = Vec<T>::N;
    const int step = lpr * VEC;
    if (nr == GEMV_RPW) {
#pragma unroll 2
        for (int c = sl * VEC; c < cpad; c += step) {
            uint4 raw[GEMV_RPW];
#pragma unroll
            for (int q = 0; q < GEMV_RPW; ++q) raw[q] = ld_stream(rowp + (size_t)q * cpad + c);
            A zv[VEC];
#pragma unroll
            for (int e = 0; e < VEC; ++e) zv[e] = z[c + e];
#pragma unroll
            for (int q = 0; q < GEMV_RPW; ++q) Vec<T>::fma(raw[q], zv, acc[q]);
        }
    } else if (nr > 0) {
        for (int c = sl * VEC; c < cpad; c += step) {
            A zv[VEC];
#pragma unroll
            for (int e = 0; e < VEC; ++e) zv[e] = z[c + e];
            for (int q = 0; q < nr; ++q) {
                uint4 raw = ld_stream(rowp + (size_t)q * cpad + c);
                Vec<T>::fma(raw, zv, acc[q]);
            }
        }
    }
}

// TD = dense-segment element type, TL = low-rank-segment element type (same accumulator).
template <typename TD, typename TL>
__global__ void __launch_bounds__(GEMV_THREADS, 5) gemv_tasks_kernel(
    const GemvTask *__restrict__ tasks, int ntasks, const TD *__restrict__ data_d, const TL *__restrict__ data_l,
    const int *__restrict__ gidx, const float *__restrict__ gscale, const float *__restrict__ rowscale,
    const ReduceGroup *__restrict__ red, GemvBufs<typename Vec<TL>::A> B, const int *stop) {
    using A = typename Vec<TL>::A;
    static_assert(std::is_same<typename Vec<TD>::A, A>::value, "segments must share the accumulator");
    constexpr int GU = 4;   // gather: independent index -> value chains per thread
    extern __shared__ __align__(16) unsigned char smem_raw[];
    A *z = reinterpret_cast<A *>(smem_raw);
    __shared__ int s_task, s_last;
    if (stop != nullptr && *(volatile const int *)stop) return;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    A *xt = B.xt;
    for (;;) {
        if (threadIdx.x == 0) s_task = atomicAdd(B.counter, 1);
        __syncthreads();
        const int ti = s_task;
        if (ti >= ntasks) break;
        const GemvTask tk = tasks[ti];
        const int ctot = tk.cpad_d + tk.cpad;
        // ---- input gather into shared memory: [dense segment | low-rank segment]
        const A *zin = z;
        if (tk.gather_off < 0) {
            const A *src = xt + tk.src_off;
            for (int c = threadIdx.x; c < ctot; c += blockDim.x) z[c] = c < tk.ncols ? src[c] : A(0);
            __syncthreads();
        } else {
            const int *gi = gidx + tk.gather_off;
            const float *gs = gscale != nullptr ? gscale + tk.gather_off : nullptr;
            for (int c0 = threadIdx.x; c0 < ctot; c0 += GU * blockDim.x) {
                int idx[GU];
#pragma unroll
                for (int u = 0; u < GU; ++u) {
                    const int c = c0 + u * blockDim.x;
                    idx[u] = c < ctot ? gi[c] : -1;
                }
                A v[GU];
#pragma unroll
                for (int u = 0; u < GU; ++u) v[u] = idx[u] >= 0 ? xt[idx[u]] : A(0);
                if (gs != nullptr) {
#pragma unroll
                    for (int u = 0; u < GU; ++u) {
                        const int c = c0 + u * blockDim.x;
                        if (c < ctot) v[u] *= (A)gs[c];
                    }
                }
#pragma unroll
                for (int u = 0; u < GU; ++u) {
                    const int c = c0 + u * blockDim.x;
                    if (c < ctot) z[c] = v[u];
                }
            }
            __syncthreads();
        }
        // ---- rows: groups of GEMV_RPW rows, each group served by `lpr` lanes of a warp (a
        //      power of two sized to the row length, so short rows do not leave lanes idle)
        A *out = tk.out_kind == 2 ? B.y : (tk.out_kind == 1 ? B.part : xt);
        const int nvec = tk.cpad_d / Vec<TD>::N + tk.cpad / Vec<TL>::N;
        int lpr = 32;   // >= GEMV_RPW: each lane of a group writes one of its rows
        while (lpr > GEMV_RPW && 2 * nvec <= lpr) lpr >>= 1;
        const int gpw = 32 / lpr, g = lane / lpr, sl = lane - g * lpr;
        for (int base = warp * gpw * GEMV_RPW; base < tk.rows; base += nwarps * gpw * GEMV_RPW) {
            const int r0 = base + g * GEMV_RPW;
            A acc[GEMV_RPW];
#pragma unroll
            for (int q = 0; q < GEMV_RPW; ++q) acc[q] = A(0);
            const int nr = max(0, min(GEMV_RPW, tk.rows - r0));
            if (tk.cpad_d > 0)
                segment_dot<TD>(data_d + tk.data_off_d + (size_t)r0 * tk.cpad_d, tk.cpad_d, nr, zin, sl, lpr, acc);
            if (tk.cpad > 0)
                segment_dot<TL>(data_l + tk.data_off + (size_t)r0 * tk.cpad, tk.cpad, nr, zin + tk.cpad_d, sl, lpr,
                                acc);
#pragma unroll
            for (int q = 0; q < GEMV_RPW; ++q)
                for (int o = lpr >> 1; o > 0; o >>= 1) acc[q] += __shfl_xor_sync(0xffffffffu, acc[q], o);
            if (sl < nr) {
                A v = acc[0];
#pragma unroll
                for (int q = 1; q < GEMV_RPW; ++q)
                    if (sl == q) v = acc[q];
                if (tk.scale_off >= 0) v *= (A)rowscale[tk.scale_off + r0 + sl];
                out[tk.out_off + r0 + sl] = v;
            }
        }
        // ---- a chunked VT group: the last chunk to finish sums the partials in fixed order
        if (tk.red >= 0) {
            __threadfence();
            __syncthreads();
            if (threadIdx.x == 0) s_last = (atomicAdd(&B.red_cnt[tk.red], 1) == red[tk.red].nchunks - 1);
            __syncthreads();
            if (s_last) {
                __threadfence();
                const ReduceGroup g = red[tk.red];
                for (int r = threadIdx.x; r < g.rows; r += blockDim.x) {
                    A sum = A(0);
                    for (int c = 0; c < g.nchunks; ++c) sum += __ldcg(&B.part[g.p_off + (int64_t)c * g.rows + r]);
                    xt[g.t_off + r] = sum;
                }
            }
        }
        __syncthreads();
    }
}

template <typename A>
__global__ void permute_in_kernel(const double *__restrict__ x, const int *__restrict__ perm, int n, int nin,
                                  A *__restrict__ xt) {
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < n; p += gridDim.x * blockDim.x) {
        const int e = perm[p];
        for (int c = 0; c < nin; ++c) xt[(size_t)nin * p + c] = (A)x[(size_t)c * n + e];
    }
}
template <typename A>
__global__ void permute_out_kernel(const A *__restrict__ yp, const int *__restrict__ perm, int n, int nout,
                                   double *__restrict__ y) {
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < n; p += gridDim.x * blockDim.x) {
        const int e = perm[p];
        for (int c = 0; c < nout; ++c) y[(size_t)c * n + e] = (double)yp[(size_t)nout * p + c];
    }
}

// ----------------------------------------------------------- packing kernels
struct ColRef {          // one factor column to scale
    const double *p;
    int64_t len, stride;
};
__global__ void colscale_kernel(const ColRef *__restrict__ cols, int64_t ncols, float *__restrict__ scale) {
    const int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (w >= ncols) return;
    const ColRef c = cols[w];
    double m = 0.0;
    for (int64_t i = lane; i < c.len; i += 32) m = fmax(m, fabs(c.p[i * c.stride]));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    if (lane == 0) {
        // power of two so that max / scale lies in (2^13, 2^14]; exact to apply and undo
        float s = 1.0f;
        if (m > 0.0 && isfinite(m)) s = (float)exp2(ceil(log2(m)) - 14.0);
        scale[w] = s;
    }
}

template <typename T> __device__ __forceinline__ T to_storage(double v);
template <> __device__ __forceinline__ double to_storage<double>(double v) { return v; }
template <> __device__ __forceinline__ float to_storage<float>(double v) { return (float)v; }
template <> __device__ __forceinline__ __half to_storage<__half>(double v) { return __double2half(v); }
template <> __device__ __forceinline__ __nv_bfloat16 to_storage<__nv_bfloat16>(double v) {
    return __double2bfloat16(v);
}


struct VtRow {           // one VT panel row: a V column of one low-rank block
    const double *v;     // V(:, k), contiguous
    float inv_scale;
};
// one CTA per VT task
template <typename T>
__global__ void pack_vt_kernel(const GemvTask *__restrict__ tasks, const int64_t *__restrict__ chunk_col0,
                               const int64_t *__restrict__ row_base, const VtRow *__restrict__ rows,
                               T *__restrict__ data) {
    const GemvTask tk = tasks[blockIdx.x];
    const int64_t c0 = chunk_col0[blockIdx.x], rb = row_base[blockIdx.x];
    const int64_t tot = (int64_t)tk.rows * tk.cpad;
    for (int64_t e = threadIdx.x; e < tot; e += blockDim.x) {
        const int r = (int)(e / tk.cpad), c = (int)(e - (int64_t)r * tk.cpad);
        double v = 0.0;
        if (c < tk.ncols) {
            const VtRow R = rows[rb + r];
            v = R.v[c0 + c] * (double)R.inv_scale;
        }
        data[tk.data_off + e] = to_storage<T>(v);
    }
}

struct UyTerm {          // one block's contribution to a leaf row unit
    const double *src;   // U (column-major, ld = m) or dense (row-major, ld = nc)
    const float *colscale;  // per-column scale of this block (U or dense), or null
    int64_t ld, roff;    // leading dimension, first block row of the unit
    int width, coloff, dense;   // coloff: column offset inside its segment
    int pad_;
};
// one CTA per UY task (leaf row unit): dense terms into the dense segment, U slices into
// the low-rank segment
template <typename TD, typename TL>
__global__ void pack_uy_kernel(const GemvTask *__restrict__ tasks, const int *__restrict__ term_begin,
                               const UyTerm *__restrict__ terms, TD *__restrict__ data_d, TL *__restrict__ data_l) {
    const GemvTask tk = tasks[blockIdx.x];
    for (int q = term_begin[blockIdx.x]; q < term_begin[blockIdx.x + 1]; ++q) {
        const UyTerm t = terms[q];
        const int64_t tot = (int64_t)tk.rows * t.width;
        for (int64_t e = threadIdx.x; e < tot; e += blockDim.x) {
            const int i = (int)(e / t.width), c = (int)(e - (int64_t)i * t.width);
            double v = t.dense ? t.src[(t.roff + i) * t.ld + c] : t.src[(int64_t)c * t.ld + t.roff + i];
            if (t.colscale) v /= (double)t.colscale[c];
            if (t.dense)
                data_d[tk.data_off_d + (int64_t)i * tk.cpad_d + t.coloff + c] = to_storage<TD>(v);
            else
                data_l[tk.data_off + (int64_t)i * tk.cpad + t.coloff + c] = to_storage<TL>(v);
        }
    }
}

// ------------------------------------------------------------- host driver
namespace {
// element sizes of the dense and low-rank streams of a storage mode
size_t esize_dense(int storage) {
    switch (storage) {
        case HBI_FP64: return 8;
        case HBI_FP32: case HBI_MIXED: return 4;
        default: return 2;
    }
}
size_t esize_lowrank(int storage) {
    switch (storage) {
        case HBI_FP64: return 8;
        case HBI_FP32: return 4;
        default: return 2;
    }
}
int64_t round_up(int64_t v, int64_t m) { return (v + m - 1) / m * m; }

struct GemvCfg {
    hbi_handle *h;
    int smem1, smem2, smax;
    template <typename TD, typename TL> hbi_status operator()() {
        const void *fn = (const void *)gemv_tasks_kernel<TD, TL>;
        // The limit is a property of the kernel, shared by every handle: only ever raise
        // it, so that building a handle with smaller panels cannot invalidate another's.
        cudaFuncAttributes fa;
        HBI_CUDA_TRY(cudaFuncGetAttributes(&fa, fn));
        if (smax > fa.maxDynamicSharedSizeBytes)
            HBI_CUDA_TRY(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smax));
        int b1 = 0, b2 = 0;
        HBI_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b1, fn, GEMV_THREADS, smem1));
        HBI_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b2, fn, GEMV_THREADS, smem2));
        h->grid1 = std::max(1, std::min(h->num_sms * std::max(1, b1), std::max(1, h->n_tasks1)));
        h->grid2 = std::max(1, std::min(h->num_sms * std::max(1, b2), std::max(1, h->n_tasks2)));
        return HBI_OK;
    }
};

struct PackLaunch {
    hbi_handle *h;
    const GemvTask *t1, *t2;
    int n1, n2;
    const int64_t *c0, *rb;
    const VtRow *rows;
    const int *tb;
    const UyTerm *terms;
    template <typename TD, typename TL> hbi_status operator()() {
        if (n1) pack_vt_kernel<TL><<<n1, 256>>>(t1, c0, rb, rows, (TL *)h->d_data1);
        HBI_CUDA_TRY(cudaGetLastError());
        if (n2) pack_uy_kernel<TD, TL><<<n2, 256>>>(t2, tb, terms, (TD *)h->d_data3, (TL *)h->d_data2);
        HBI_CUDA_TRY(cudaGetLastError());
        return HBI_OK;
    }
};

// Calls f.template operator()<TD, TL>() with the element types of a storage mode.
template <typename F> hbi_status dispatch_storage(int storage, F &&f) {
    switch (storage) {
        case HBI_FP64: return f.template operator()<double, double>();
        case HBI_FP32: return f.template operator()<float, float>();
        case HBI_FP16: return f.template operator()<__half, __half>();
        case HBI_BF16: return f.template operator()<__nv_bfloat16, __nv_bfloat16>();
        default: return f.template operator()<float, __half>();
    }
}

hbi_status gemv_config(hbi_handle *h, int smem1, int smem2) {
    const int smax = std::max(smem1, smem2);
    if (smax > 220 * 1024) {
        set_error("a leaf row unit needs more than 220 KB of gathered input");
        return HBI_ERR_INVALID_ARG;
    }
    int dev = 0;
    HBI_CUDA_TRY(cudaGetDevice(&dev));
    HBI_CUDA_TRY(cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, dev));
    GemvCfg cfg{h, smem1, smem2, smax};
    hbi_status st = dispatch_storage(h->storage, cfg);
    if (st) return st;
    h->smem1 = smem1;
    h->smem2 = smem2;
    return HBI_OK;
}

template <typename X>
hbi_status upload(X **dst, const std::vector<X> &v) {
    HBI_CUDA_TRY(cudaMalloc((void **)dst, std::max<size_t>(1, v.size()) * sizeof(X)));
    if (!v.empty()) HBI_CUDA_TRY(cudaMemcpy(*dst, v.data(), v.size() * sizeof(X), cudaMemcpyHostToDevice));
    return HBI_OK;
}
}  // namespace

hbi_status pack_operator(hbi_handle *h, const Tree *, std::vector<Block> &blocks,
                         const std::vector<int> &leaf_starts) {
    const int n = h->n, nin = h->nin, nout = h->nout;
    const size_t esd = esize_dense(h->storage), esl = esize_lowrank(h->storage);
    h->elem_bytes = esl;
    h->elem_bytes_d = esd;
    const int VECD = (int)(16 / esd), VECL = (int)(16 / esl);
    const bool scaled_d = esd == 2, scaled_l = esl == 2;
    const size_t acc_bytes = h->storage == HBI_FP64 ? 8 : 4;

    // ---- statistics
    h->n_blocks = (int64_t)blocks.size();
    h->n_lowrank = h->n_dense = h->max_rank = h->entries_lr = h->entries_dense = 0;
    double rsum = 0;
    for (auto &B : blocks) {
        if (B.lowrank) {
            ++h->n_lowrank;
            h->max_rank = std::max<int64_t>(h->max_rank, B.rank);
            rsum += B.rank;
            h->entries_lr += (B.m + B.nc) * B.rank;
        } else {
            ++h->n_dense;
            h->entries_dense += B.m * B.nc;
        }
    }
    h->mean_rank = h->n_lowrank ? rsum / (double)h->n_lowrank : 0.0;

    // ---- per-column scales of the 2-byte streams: U, V columns and dense columns
    std::vector<ColRef> cols;
    std::vector<int64_t> soffU(blocks.size(), -1), soffV(blocks.size(), -1), soffD(blocks.size(), -1);
    for (size_t b = 0; b < blocks.size(); ++b) {
        const Block &B = blocks[b];
        if (B.lowrank && scaled_l) {
            soffU[b] = (int64_t)cols.size();
            for (int k = 0; k < B.rank; ++k) cols.push_back(ColRef{B.d_src + (size_t)k * B.m, B.m, 1});
            soffV[b] = (int64_t)cols.size();
            for (int k = 0; k < B.rank; ++k) cols.push_back(ColRef{B.d_src2 + (size_t)k * B.nc, B.nc, 1});
        } else if (!B.lowrank && scaled_d) {
            soffD[b] = (int64_t)cols.size();
            for (int64_t j = 0; j < B.nc; ++j) cols.push_back(ColRef{B.d_src + j, B.m, B.nc});
        }
    }
    ColRef *d_cols = nullptr;
    float *d_colscale = nullptr;
    std::vector<float> colscale;
    if (!cols.empty()) {
        hbi_status st = upload(&d_cols, cols);
        if (st) return st;
        HBI_CUDA_TRY(cudaMalloc(&d_colscale, cols.size() * sizeof(float)));
        const int64_t threads = (int64_t)cols.size() * 32;
        colscale_kernel<<<(unsigned)((threads + 255) / 256), 256>>>(d_cols, (int64_t)cols.size(), d_colscale);
        HBI_CUDA_TRY(cudaGetLastError());
        colscale.resize(cols.size());
        HBI_CUDA_TRY(cudaMemcpy(colscale.data(), d_colscale, cols.size() * sizeof(float), cudaMemcpyDeviceToHost));
    }

    // ---- VT phase: low-rank blocks grouped by column range
    std::map<std::pair<int64_t, int64_t>, std::vector<int>> groups;
    for (size_t b = 0; b < blocks.size(); ++b)
        if (blocks[b].lowrank && blocks[b].rank > 0) groups[{blocks[b].col0, blocks[b].nc}].push_back((int)b);
    std::vector<int64_t> toff(blocks.size(), -1);
    std::vector<GemvTask> t1;
    std::vector<int64_t> chunk_col0, row_base;
    std::vector<VtRow> vrows;
    std::vector<ReduceGroup> red;
    std::vector<float> rowscale;
    int64_t tcount = 0, pcount = 0, d1 = 0;
    const int64_t ntot_in = (int64_t)nin * n;
    for (auto &kv : groups) {
        const int64_t col0 = kv.first.first, nc = kv.first.second;
        int rows = 0;
        const int64_t tbase = tcount;
        for (int b : kv.second) {
            toff[b] = tcount + rows;
            for (int k = 0; k < blocks[b].rank; ++k) {
                const float sv = scaled_l ? colscale[soffV[b] + k] : 1.0f;
                const float su = scaled_l ? colscale[soffU[b] + k] : 1.0f;
                vrows.push_back(VtRow{blocks[b].d_src2 + (size_t)k * blocks[b].nc, 1.0f / sv});
                rowscale.push_back(sv * su);
            }
            rows += blocks[b].rank;
        }
        int64_t cw = VT_TARGET_BYTES / ((int64_t)rows * (int64_t)esl);
        cw = std::max<int64_t>(256, cw / 64 * 64);
        const int64_t nchunks = (nc + cw - 1) / cw;
        if (nchunks <= 1) cw = nc;
        for (int64_t c = 0; c < nchunks; ++c) {
            const int64_t cols_c = std::min(cw, nc - c * cw);
            GemvTask T{};
            T.data_off = d1;
            T.data_off_d = 0;
            T.rows = rows;
            T.ncols = (int)cols_c;
            T.cpad = (int)round_up(cols_c, VECL);
            T.cpad_d = 0;
            T.src_off = col0 + c * cw;
            T.gather_off = -1;
            T.scale_off = scaled_l ? tbase : -1;
            T.red = -1;
            if (nchunks == 1) { T.out_kind = 0; T.out_off = ntot_in + tbase; }
            else { T.out_kind = 1; T.out_off = pcount + c * rows; T.red = (int)red.size(); }
            d1 += (int64_t)rows * T.cpad;
            t1.push_back(T);
            chunk_col0.push_back(c * cw);
            row_base.push_back(tbase);
        }
        if (nchunks > 1) {
            red.push_back(ReduceGroup{ntot_in + tbase, pcount, rows, (int)nchunks});
            pcount += nchunks * rows;
        }
        tcount += rows;
    }
    h->n_t = tcount;
    h->n_part = pcount;

    // ---- UY phase: one task per leaf row unit, [dense segment | low-rank segment]
    const int nleaves = (int)leaf_starts.size() - 1;
    std::vector<std::vector<int>> unit_terms(nleaves);
    {
        std::vector<int> leaf_of(n);
        for (int u = 0; u < nleaves; ++u)
            for (int e = leaf_starts[u]; e < leaf_starts[u + 1]; ++e) leaf_of[e] = u;
        for (size_t b = 0; b < blocks.size(); ++b) {
            const Block &B = blocks[b];
            if (B.lowrank && B.rank == 0) continue;
            const int e0 = (int)(B.row0 / nout), e1 = (int)((B.row0 + B.m) / nout);
            for (int u = leaf_of[e0]; u < nleaves && leaf_starts[u] < e1; ++u) unit_terms[u].push_back((int)b);
        }
    }
    std::vector<GemvTask> t2;
    std::vector<int> term_begin;
    std::vector<UyTerm> terms;
    std::vector<int> gidx;
    std::vector<float> gsc;
    int64_t d2 = 0, d3 = 0;
    for (int u = 0; u < nleaves; ++u) {
        const int64_t r0 = (int64_t)nout * leaf_starts[u], R = (int64_t)nout * (leaf_starts[u + 1] - leaf_starts[u]);
        term_begin.push_back((int)terms.size());
        const int64_t goff = (int64_t)gidx.size();
        int64_t Cd = 0, Cl = 0;
        // dense terms first (their gather entries lead), then the low-rank terms
        for (int pass = 0; pass < 2; ++pass) {
            for (int b : unit_terms[u]) {
                const Block &B = blocks[b];
                if ((pass == 0) == (bool)B.lowrank) continue;
                UyTerm t{};
                t.roff = r0 - B.row0;
                if (!B.lowrank) {
                    t.src = B.d_src; t.ld = B.nc; t.width = (int)B.nc; t.dense = 1; t.coloff = (int)Cd;
                    t.colscale = scaled_d ? d_colscale + soffD[b] : nullptr;
                    for (int64_t j = 0; j < B.nc; ++j) {
                        gidx.push_back((int)(B.col0 + j));
                        gsc.push_back(scaled_d ? colscale[soffD[b] + j] : 1.0f);
                    }
                    Cd += t.width;
                } else {
                    t.src = B.d_src; t.ld = B.m; t.width = B.rank; t.dense = 0; t.coloff = (int)Cl;
                    t.colscale = scaled_l ? d_colscale + soffU[b] : nullptr;
                    for (int k = 0; k < B.rank; ++k) { gidx.push_back((int)(ntot_in + toff[b] + k)); gsc.push_back(1.0f); }
                    Cl += t.width;
                }
                terms.push_back(t);
            }
            if (pass == 0) {   // pad the dense segment
                const int64_t cpd = round_up(Cd, VECD);
                for (int64_t c = Cd; c < cpd; ++c) { gidx.push_back(-1); gsc.push_back(0.0f); }
            }
        }
        const int64_t cpd = round_up(Cd, VECD), cpl = round_up(Cl, VECL);
        for (int64_t c = Cl; c < cpl; ++c) { gidx.push_back(-1); gsc.push_back(0.0f); }
        GemvTask T{};
        T.data_off = d2;
        T.data_off_d = d3;
        T.rows = (int)R;
        T.cpad = (int)cpl;
        T.cpad_d = (int)cpd;
        T.ncols = (int)(Cd + Cl);
        T.src_off = 0;
        T.gather_off = goff;
        T.scale_off = -1;
        T.out_kind = 2;
        T.out_off = r0;
        T.red = -1;
        d2 += R * cpl;
        d3 += R * cpd;
        t2.push_back(T);
    }
    term_begin.push_back((int)terms.size());
    if ((int64_t)gidx.size() > (int64_t)INT32_MAX || ntot_in + tcount > (int64_t)INT32_MAX) {
        set_error("operator too large for 32-bit gather indices");
        return HBI_ERR_INVALID_ARG;
    }

    // ---- device allocations and packing
    h->n_data1 = d1;
    h->n_data2 = d2;
    h->n_data3 = d3;
    HBI_CUDA_TRY(cudaMalloc(&h->d_data1, std::max<int64_t>(1, d1) * esl));
    HBI_CUDA_TRY(cudaMalloc(&h->d_data2, std::max<int64_t>(1, d2) * esl));
    HBI_CUDA_TRY(cudaMalloc(&h->d_data3, std::max<int64_t>(1, d3) * esd));
    HBI_CUDA_TRY(cudaMemset(h->d_data2, 0, std::max<int64_t>(1, d2) * esl));
    HBI_CUDA_TRY(cudaMemset(h->d_data3, 0, std::max<int64_t>(1, d3) * esd));
    hbi_status st;
    GemvTask *d_t1 = nullptr, *d_t2 = nullptr;
    int64_t *d_c0 = nullptr, *d_rb = nullptr;
    VtRow *d_rows = nullptr;
    int *d_tb = nullptr;
    UyTerm *d_terms = nullptr;
    if ((st = upload(&d_t1, t1)) || (st = upload(&d_t2, t2)) || (st = upload(&d_c0, chunk_col0)) ||
        (st = upload(&d_rb, row_base)) || (st = upload(&d_rows, vrows)) || (st = upload(&d_tb, term_begin)) ||
        (st = upload(&d_terms, terms)))
        return st;
    PackLaunch pk{h, d_t1, d_t2, (int)t1.size(), (int)t2.size(), d_c0, d_rb, d_rows, d_tb, d_terms};
    if ((st = dispatch_storage(h->storage, pk))) return st;
    HBI_CUDA_TRY(cudaDeviceSynchronize());
    cudaFree(d_t1); cudaFree(d_t2); cudaFree(d_c0); cudaFree(d_rb); cudaFree(d_rows); cudaFree(d_tb);
    cudaFree(d_terms); cudaFree(d_cols); cudaFree(d_colscale);

    // ---- tasks sorted by decreasing size for the dynamic scheduler (LPT)
    auto work = [&](const GemvTask &a) { return (int64_t)a.rows * ((int64_t)a.cpad * esl + (int64_t)a.cpad_d * esd); };
    auto bigger = [&](const GemvTask &a, const GemvTask &b) {
        const int64_t ca = work(a), cb = work(b);
        return ca > cb || (ca == cb && (a.data_off < b.data_off || (a.data_off == b.data_off && a.data_off_d < b.data_off_d)));
    };
    std::stable_sort(t1.begin(), t1.end(), bigger);
    std::stable_sort(t2.begin(), t2.end(), bigger);
    int smem1 = 16, smem2 = 16;
    for (auto &T : t1) smem1 = std::max<int>(smem1, (int)((T.cpad + T.cpad_d) * acc_bytes));
    for (auto &T : t2) smem2 = std::max<int>(smem2, (int)((T.cpad + T.cpad_d) * acc_bytes));
    h->n_tasks1 = (int)t1.size();
    h->n_tasks2 = (int)t2.size();
    h->n_red = (int)red.size();
    h->n_gather = (int64_t)gidx.size();
    h->n_rowscale = (int64_t)rowscale.size();
    if ((st = upload(&h->d_tasks1, t1)) || (st = upload(&h->d_tasks2, t2)) || (st = upload(&h->d_red, red)) ||
        (st = upload(&h->d_gidx, gidx)))
        return st;
    if (scaled_d && (st = upload(&h->d_gscale, gsc))) return st;
    if (scaled_l && (st = upload(&h->d_rowscale, rowscale))) return st;
    // + 16 zero guard elements: contiguous VT inputs are read up to their padded width
    HBI_CUDA_TRY(cudaMalloc(&h->d_xt, (ntot_in + tcount + 16) * acc_bytes));
    HBI_CUDA_TRY(cudaMemset(h->d_xt, 0, (ntot_in + tcount + 16) * acc_bytes));
    HBI_CUDA_TRY(cudaMalloc(&h->d_part, std::max<int64_t>(1, pcount) * acc_bytes));
    HBI_CUDA_TRY(cudaMalloc(&h->d_yp, (size_t)nout * n * acc_bytes));
    HBI_CUDA_TRY(cudaMalloc(&h->d_counters, (2 + (size_t)h->n_red) * sizeof(int)));
    HBI_CUDA_TRY(cudaMemset(h->d_counters, 0, (2 + (size_t)h->n_red) * sizeof(int)));

    // ---- bytes per HMVM: packed streams (with padding) and algorithmic (stored entries,
    //      scales, x read, y written, t written and read)
    h->bytes_factors = (d1 + d2) * (int64_t)esl + d3 * (int64_t)esd + (int64_t)gidx.size() * (scaled_d ? 8 : 4) +
                       (int64_t)rowscale.size() * 4;
    int64_t v_entries = 0, u_entries = 0, d_entries = 0, v_scales = 0, uy_scales = 0;
    for (auto &B : blocks) {
        if (B.lowrank) {
            v_entries += B.nc * B.rank;
            u_entries += B.m * B.rank;
            if (scaled_l) { v_scales += 4 * (int64_t)B.rank; uy_scales += 4 * (int64_t)B.rank; }
        } else {
            d_entries += B.m * B.nc;
            if (scaled_d) uy_scales += 4 * B.nc;
        }
    }
    h->bytes_alg_vt = v_entries * (int64_t)esl + v_scales + (ntot_in + tcount) * (int64_t)acc_bytes;
    h->bytes_alg_uy = u_entries * (int64_t)esl + d_entries * (int64_t)esd + uy_scales +
                      (ntot_in + tcount + (int64_t)nout * n) * (int64_t)acc_bytes;
    h->bytes_algorithmic = (v_entries + u_entries) * (int64_t)esl + d_entries * (int64_t)esd + v_scales + uy_scales +
                           (int64_t)(nin + nout) * n * (int64_t)acc_bytes + 2 * tcount * (int64_t)acc_bytes;
    return gemv_config(h, smem1, smem2);
}

// ----------------------------------------------------------------- launch
namespace {
// One product with explicit buffers.  phase: -1 = whole product, 0 = VT (with the counter
// reset; chunked groups are summed by their last chunk), 2 = UY; 1 launches nothing (kept
// so the phase timing keeps its layout).  `counters` holds 2 + n_red ints.
template <typename TD, typename TL>
hbi_status hmvm_run(hbi_handle *h, int phase, typename Vec<TL>::A *xt, typename Vec<TL>::A *part,
                    typename Vec<TL>::A *yp, int *counters, cudaStream_t s, const int *d_stop) {
    using A = typename Vec<TL>::A;
    if (phase <= 0) {
        HBI_CUDA_TRY(cudaMemsetAsync(counters, 0, (2 + (size_t)h->n_red) * sizeof(int), s));
        if (h->n_tasks1)
            gemv_tasks_kernel<TD, TL><<<h->grid1, GEMV_THREADS, h->smem1, s>>>(
                h->d_tasks1, h->n_tasks1, (const TD *)h->d_data3, (const TL *)h->d_data1, h->d_gidx, h->d_gscale,
                h->d_rowscale, h->d_red, GemvBufs<A>{xt, part, yp, counters, counters + 2}, d_stop);
    }
    if (phase < 0 || phase == 2)
        gemv_tasks_kernel<TD, TL><<<h->grid2, GEMV_THREADS, h->smem2, s>>>(
            h->d_tasks2, h->n_tasks2, (const TD *)h->d_data3, (const TL *)h->d_data2, h->d_gidx, h->d_gscale,
            h->d_rowscale, h->d_red, GemvBufs<A>{xt, part, yp, counters + 1, counters + 2}, d_stop);
    HBI_CUDA_TRY(cudaGetLastError());
    return HBI_OK;
}
struct PhaseRun {
    hbi_handle *h;
    int phase;
    cudaStream_t s;
    const int *stop;
    template <typename TD, typename TL> hbi_status operator()() {
        using A = typename Vec<TL>::A;
        return hmvm_run<TD, TL>(h, phase, (A *)h->d_xt, (A *)h->d_part, (A *)h->d_yp, h->d_counters, s, stop);
    }
};
}  // namespace

hbi_status hmvm_phase(hbi_handle *h, int phase, cudaStream_t s, const int *d_stop) {
    return dispatch_storage(h->storage, PhaseRun{h, phase, s, d_stop});
}

hbi_status hmvm_launch(hbi_handle *h, cudaStream_t s, const int *d_stop) { return hmvm_phase(h, -1, s, d_stop); }

hbi_status permute_x_in(hbi_handle *h, const double *d_x, cudaStream_t s) {
    const int grid = std::max(1, std::min((h->n + 255) / 256, 4 * std::max(1, h->num_sms)));
    if (h->storage == HBI_FP64)
        permute_in_kernel<double><<<grid, 256, 0, s>>>(d_x, h->d_perm, h->n, h->nin, (double *)h->d_xt);
    else
        permute_in_kernel<float><<<grid, 256, 0, s>>>(d_x, h->d_perm, h->n, h->nin, (float *)h->d_xt);
    HBI_CUDA_TRY(cudaGetLastError());
    return HBI_OK;
}

hbi_status permute_y_out(hbi_handle *h, double *d_y, cudaStream_t s) {
    const int grid = std::max(1, std::min((h->n + 255) / 256, 4 * std::max(1, h->num_sms)));
    if (h->storage == HBI_FP64)
        permute_out_kernel<double><<<grid, 256, 0, s>>>((const double *)h->d_yp, h->d_perm, h->n, h->nout, d_y);
    else
        permute_out_kernel<float><<<grid, 256, 0, s>>>((const float *)h->d_yp, h->d_perm, h->n, h->nout, d_y);
    HBI_CUDA_TRY(cudaGetLastError());
    return HBI_OK;
}

}  // namespace hbi

// ----------------------------------------------------------------------------
// HMVM for callers that cannot allocate: every per-call buffer (work counters, permuted
// input with the intermediate t = V^T x, partial sums, permuted output) lives in one static
// device array instead of the handle's buffers or fresh allocations.
namespace hbi {
namespace {
static __device__ __align__(256) unsigned char g_noalloc_scratch[HBI_NOALLOC_SCRATCH_BYTES];

constexpr int kMaxDevices = 256;
std::mutex g_noalloc_mu;
void *g_noalloc_addr[kMaxDevices] = {};

// Device address of the static array on the current device, looked up once per device.
hbi_status noalloc_scratch(void **out) {
    int dev = 0;
    HBI_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) {
        set_error("device index out of range for the static scratch table");
        return HBI_ERR_INVALID_ARG;
    }
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (g_noalloc_addr[dev] == nullptr) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || p == nullptr) {
            set_error(std::string("cudaGetSymbolAddress(scratch): ") + cudaGetErrorString(e));
            return HBI_ERR_CUDA;
        }
        g_noalloc_addr[dev] = p;
    }
    *out = g_noalloc_addr[dev];
    return HBI_OK;
}

size_t align256(size_t v) { return (v + 255) / 256 * 256; }

struct NoallocRun {
    hbi_handle *h;
    unsigned char *base;
    const double *x;
    double *y;
    cudaStream_t s;
    template <typename TD, typename TL> hbi_status operator()() {
        using A = typename Vec<TL>::A;
        size_t off = 0;
        int *counters = reinterpret_cast<int *>(base + off);
        off += align256((2 + (size_t)h->n_red) * sizeof(int));
        A *xt = reinterpret_cast<A *>(base + off);
        const size_t nxt = (size_t)h->nin * h->n + (size_t)h->n_t;
        off += align256((nxt + 16) * sizeof(A));
        A *part = reinterpret_cast<A *>(base + off);
        off += align256((size_t)std::max<int64_t>(1, h->n_part) * sizeof(A));
        A *yp = reinterpret_cast<A *>(base + off);
        const int grid = std::max(1, std::min((h->n + 255) / 256, 4 * std::max(1, h->num_sms)));
        HBI_CUDA_TRY(cudaMemsetAsync(xt + nxt, 0, 16 * sizeof(A), s));   // guard elements
        permute_in_kernel<A><<<grid, 256, 0, s>>>(x, h->d_perm, h->n, h->nin, xt);
        hbi_status st = hmvm_run<TD, TL>(h, -1, xt, part, yp, counters, s, nullptr);   // clears the counters
        if (st) return st;
        permute_out_kernel<A><<<grid, 256, 0, s>>>(yp, h->d_perm, h->n, h->nout, y);
        HBI_CUDA_TRY(cudaGetLastError());
        return HBI_OK;
    }
};
}  // namespace
}  // namespace hbi

extern "C" hbi_status hbi_matvec_noalloc(hbi_handle *h, const double *d_x, double *d_y, hbi_stream stream) {
    using namespace hbi;
    if (!h || !d_x || !d_y) {
        set_error("handle, x and y are required");
        return HBI_ERR_INVALID_ARG;
    }
    const size_t acc = h->storage == HBI_FP64 ? 8 : 4;
    const size_t need = align256((2 + (size_t)h->n_red) * sizeof(int)) +
                        align256(((size_t)h->nin * h->n + (size_t)h->n_t + 16) * acc) +
                        align256((size_t)std::max<int64_t>(1, h->n_part) * acc) + align256((size_t)h->nout * h->n * acc);
    if (need > HBI_NOALLOC_SCRATCH_BYTES) {
        set_error("operator needs " + std::to_string(need) + " bytes of scratch, more than the static " +
                  std::to_string((size_t)HBI_NOALLOC_SCRATCH_BYTES) + " bytes of hbi_matvec_noalloc");
        return HBI_ERR_INVALID_ARG;
    }
    void *base = nullptr;
    hbi_status st = noalloc_scratch(&base);
    if (st) return st;
    cudaStream_t s = (cudaStream_t)stream;
    unsigned char *b = static_cast<unsigned char *>(base);
    st = dispatch_storage(h->storage, NoallocRun{h, b, d_x, d_y, s});
    if (st) return st;
    HBI_CUDA_TRY(cudaStreamSynchronize(s));
    return HBI_OK;
}
