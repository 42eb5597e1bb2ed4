// H-matrix x vector product (Sec. 3.1.3, Eq. 20) as two persistent GEMV phases.
//
// Eq. 20 splits every low-rank block into t_b = V_b^T x_sigma followed by y_tau += U_b t_b.
// Phase VT computes all t_b; phase UY computes every output row once.  Both reduce
// row-major panels of stored factor values, one output per panel row:
//   VT items  : all low-rank blocks sharing a column cluster sigma stacked (rows = their
//               V columns), cut into row blocks and, for wide groups, column chunks whose
//               sums stay in registers of one CTA.  Input = the contiguous x_sigma slice,
//               staged with the panel through shared memory by TMA bulk copies.
//   UY tasks  : one per leaf row cluster: the concatenation over every block covering those
//               rows of its U slice (low-rank) or its dense rows.  Input = the matching
//               t_b and x_sigma values, gathered into shared memory.  Each output row is
//               written exactly once, so the result needs no atomics and is bitwise
//               reproducible.
// A UY row has two segments, the dense near-field columns and the low-rank U columns, so the
// two kinds of block can be stored in different precisions: FP64, FP32, FP16 or BF16 for
// both, FP32 near field + FP16 far field (HBI_MIXED), or HBI_MIXED with the leading pair
// (U(:,0), V(:,0)) of every low-rank block at FP32 accuracy (HBI_ADAPTIVE: V(:,0) is split
// into two FP16 VT rows, hi and lo, whose t entries the UY gather adds for an FP32 U(:,0)
// column of the near-field segment).  FP16/BF16 values carry one power-of-two scale per
// factor column: U and V column scales fold into the VT output, dense column scales into the
// UY gather, so the inner loops are plain dot products with FP32 (FP64) accumulation.
// UY tasks are claimed from an atomic counter in decreasing size order (LPT), which keeps
// the persistent grid (a multiple of the SM count) busy until the end; VT items follow a
// static LPT schedule made on the host.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <map>
#include <mutex>
#include <numeric>
#include <queue>
#include <type_traits>

#include "hbi_internal.h"
#include "hbi_stage.cuh"
#include "hbi_tables.h"

namespace hbi {

constexpr int GEMV_THREADS = 256;           // UY phase
constexpr int GEMV_RPW = 4;                 // rows per lane group and pass (VT chunks)
// UY rows per lane group and pass: 4 (registers sized for 5 CTAs per SM) or 8 (4 CTAs),
// chosen per handle (default 4; hbi_autotune times both)
template <int R> struct UyShape { static constexpr int blocks = R >= 8 ? 4 : 5; };
constexpr int VT_PASS_COST = 8;              // default per-pass cost of the VT shape choice
constexpr int64_t VT_PANEL_BYTES = 40 << 10; // VT item panel: one shared-memory stage
constexpr int64_t VT_X_BYTES = 8 << 10;      // VT item x slice
constexpr int64_t VT_STAGE_BYTES = VT_PANEL_BYTES + VT_X_BYTES;
constexpr int VT_STAGES = 2;                 // stages per CTA
constexpr int VT_CTAS_PER_SM = 2;
constexpr int VT_CW = 8;                     // consumer warps of the VT kernel
constexpr int VT_THREADS = 32 * (VT_CW + 1); // + one producer warp
constexpr int VT_MC_ROWS = VT_CW * GEMV_RPW; // rows of a row block split into column chunks
constexpr int VT_MAX_SUB = 8;                // items per stage batch (<= 32, one producer lane each)

// -------------------------------------------------------- vector decoding
__device__ __forceinline__ uint4 ld_stream(const void *p) {
    uint4 r;
    asm volatile("ld.global.nc.L1::no_allocate.v4.u32 {%0,%1,%2,%3}, [%4];"
                 : "=r"(r.x), "=r"(r.y), "=r"(r.z), "=r"(r.w)
                 : "l"(p));
    return r;
}

// Bounds-checked build (HBI_BOUNDS_CHECK): both product kernels check every table entry and
// gather index against the limits of the handle being multiplied (copied to g_lim before each
// launch) and count a violation in g_violations instead of making the access; never a trap.
#ifdef HBI_BOUNDS_CHECK
struct DevLimits {
    int64_t n_data1, n_data2, n_data3, n_x, n_xt, n_y, n_gather;
    int es_vt, smem_uy;
};
__device__ DevLimits g_lim;
__device__ unsigned long long g_violations;
__device__ __forceinline__ bool bc_violated(bool ok) {
    if (!ok) atomicAdd(&g_violations, 1ull);
    return !ok;
}
#define HBI_BC(cond) bc_violated(cond)
#else
#define HBI_BC(cond) false
#endif

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

// ------------------------------------------------------------- UY kernel
// z[c .. c + VEC) into registers with 16-byte shared-memory loads (z is 16-byte aligned).
__device__ __forceinline__ void load_z(const float *z, float (&zv)[4]) {
    const float4 a = *reinterpret_cast<const float4 *>(z);
    zv[0] = a.x; zv[1] = a.y; zv[2] = a.z; zv[3] = a.w;
}
__device__ __forceinline__ void load_z(const float *z, float (&zv)[8]) {
    const float4 a = *reinterpret_cast<const float4 *>(z), b = *reinterpret_cast<const float4 *>(z + 4);
    zv[0] = a.x; zv[1] = a.y; zv[2] = a.z; zv[3] = a.w;
    zv[4] = b.x; zv[5] = b.y; zv[6] = b.z; zv[7] = b.w;
}
__device__ __forceinline__ void load_z(const double *z, double (&zv)[2]) {
    const double2 a = *reinterpret_cast<const double2 *>(z);
    zv[0] = a.x; zv[1] = a.y;
}

// Sum R per-lane row partials over a group of lpr lanes (R <= lpr, both powers of two) by
// recursive halving: at each level a lane keeps half of its rows and adds the partner's
// copy of them, so R rows cost R - 1 + log2(lpr / R) shuffles instead of R log2(lpr).
// Returns the total of row `row`, held by the lanes with sl % (lpr / R) == 0.  The
// summation tree is fixed, so the result is reproducible.
template <int R, typename A>
__device__ __forceinline__ A reduce_scatter(A (&v)[R], int sl, int lpr, int &row) {
    row = 0;
    int h = lpr >> 1;
#pragma unroll
    for (int n = R; n > 1; n >>= 1) {
        const bool hi = (sl & h) != 0;
#pragma unroll
        for (int j = 0; j < n / 2; ++j) {
            const A keep = hi ? v[n / 2 + j] : v[j];
            const A send = hi ? v[j] : v[n / 2 + j];
            v[j] = keep + __shfl_xor_sync(0xffffffffu, send, h);
        }
        row = row * 2 + (hi ? 1 : 0);
        h >>= 1;
    }
    A sum = v[0];
    for (; h > 0; h >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, h);
    return sum;
}

// acc[q] += row q of a row-major segment (stride cpad) . z for q < nr <= R; the row is
// split over `lpr` lanes (sub-lane sl), each taking 16-byte vectors lpr apart.
template <int R, typename T>
__device__ __forceinline__ void segment_dot(const T *__restrict__ rowp, int cpad, int nr, const typename Vec<T>::A *z,
                                            int sl, int lpr, typename Vec<T>::A (&acc)[R]) {
    using A = typename Vec<T>::A;
    constexpr int VEC = Vec<T>::N;
    const int step = lpr * VEC;
    if (nr == R) {
#pragma unroll(R >= 8 ? 1 : 2)
        for (int c = sl * VEC; c < cpad; c += step) {
            uint4 raw[R];
#pragma unroll
            for (int q = 0; q < R; ++q) raw[q] = ld_stream(rowp + (size_t)q * cpad + c);
            A zv[VEC];
            load_z(z + c, zv);
#pragma unroll
            for (int q = 0; q < R; ++q) Vec<T>::fma(raw[q], zv, acc[q]);
        }
    } else if (nr > 0) {
        for (int c = sl * VEC; c < cpad; c += step) {
            A zv[VEC];
            load_z(z + c, zv);
            for (int q = 0; q < nr; ++q) {
                uint4 raw = ld_stream(rowp + (size_t)q * cpad + c);
                Vec<T>::fma(raw, zv, acc[q]);
            }
        }
    }
}

// One leaf row unit per task, claimed from a work counter in decreasing size order.  The
// CTA gathers the unit's input ([x_sigma of its dense blocks | t_b of its low-rank blocks],
// dense columns pre-multiplied by their scales) into shared memory, then every row is one
// dot product over [dense segment | low-rank segment], written once to y.
// TD = dense-segment element type, TL = low-rank-segment element type (same accumulator).
// FUSE: once a unit's rows are written (and visible to the CTA after its barrier), the CTA
// runs Cash-Karp stage `stage` for the unit's elements, whose product rows these are
// (stage_elem or stage_vec_elem for stages 0-4, final_unit with the error maxima for stage 5): once the next
// unit's input is gathered, its first FUSE_WARPS warps run the stage while the other warps
// stream the next unit's rows, whose row blocks the warps claim from a shared-memory counter
// so that the stage warps join them when done; the CTA runs the stage of its last unit with
// every thread after its last claim.  The stage's FP64
// arithmetic so overlaps the streaming instead of taking a launch of its own.  The next
// product's input goes to ode.xt, a buffer other than xt; y is read back through ode.yp (so
// y is not declared __restrict__).
// FUSE selects the law: 0 none, 1 fixed rake (stage_elem, final_elem), 2 rake-free
// (stage_vec_elem, final_vec_elem).
constexpr int FUSE_WARPS = 2;
template <int FUSE>
__device__ __forceinline__ void fused_stage(const OdeArgs &A, int stage, int e0, int ne, int nthreads) {
    if (stage < 5) {
        for (int e = threadIdx.x; e < ne; e += nthreads) {
            if (FUSE == 2) stage_vec_elem(A, stage, e0 + e);
            else stage_elem(A, stage, e0 + e);
        }
    } else {
        final_unit<FUSE == 2>(A, e0, ne, nthreads);
    }
}

template <typename TD, typename TL, int UY_RPW, int FUSE>
__global__ void __launch_bounds__(GEMV_THREADS, UyShape<UY_RPW>::blocks) uy_gemv_kernel(
    const GemvTask *__restrict__ tasks, int ntasks, const TD *__restrict__ data_d, const TL *__restrict__ data_l,
    const int *__restrict__ gidx, const float *__restrict__ gscale, const typename Vec<TL>::A *__restrict__ xt,
    typename Vec<TL>::A *y, int *counter, const int *stop, const int *__restrict__ mskip, const OdeArgs ode,
    int stage) {
    using A = typename Vec<TL>::A;
    static_assert(std::is_same<typename Vec<TD>::A, A>::value, "segments must share the accumulator");
    constexpr int GU = 4;   // gather: independent index -> value chains per thread
    extern __shared__ __align__(16) unsigned char smem_raw[];
    A *z = reinterpret_cast<A *>(smem_raw);
    __shared__ int s_task;
    if (stop != nullptr && *(volatile const int *)stop) {
        // a skipped product (every active model rejected: k_0 kept) still forms the stage
        // inputs of the new step size; once every model stopped there is nothing to do
        if (FUSE && stage < 5 && !*(volatile const int *)&ode.g->stop)
            for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < ode.n; i += gridDim.x * blockDim.x) {
                if (FUSE == 2) stage_vec_elem(ode, stage, i);
                else stage_elem(ode, stage, i);
            }
        return;
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    int prev_e0 = 0, prev_ne = 0;   // FUSE: the unit whose rows this CTA wrote last
    __shared__ int s_rowctr;        // FUSE: the unit's next row block (claimed by warps)
    for (;;) {
        if (threadIdx.x == 0) {
            s_task = atomicAdd(counter, 1);
            if (FUSE) s_rowctr = 0;
        }
        __syncthreads();
        const int ti = s_task;
        if (ti >= ntasks) {
            if (FUSE && prev_ne > 0) fused_stage<FUSE>(ode, stage, prev_e0, prev_ne, blockDim.x);
            // every CTA has made its last claim once all have counted themselves out here:
            // the last one rearms the work counter (counter[0]) and this count (counter[2])
            if (threadIdx.x == 0) {
                __threadfence();
                if (atomicAdd(counter + 2, 1) == (int)gridDim.x - 1) {
                    atomicExch(counter, 0);
                    atomicExch(counter + 2, 0);
                }
            }
            break;
        }
        const GemvTask tk = tasks[ti];
#ifdef HBI_BOUNDS_CHECK
        const bool task_bad =
            threadIdx.x == 0 &&
            HBI_BC(tk.rows >= 1 && tk.cpad >= 0 && tk.cpad_d >= 0 && tk.data_off >= 0 &&
                   tk.data_off + (int64_t)tk.rows * tk.cpad <= g_lim.n_data2 && tk.data_off_d >= 0 &&
                   tk.data_off_d + (int64_t)tk.rows * tk.cpad_d <= g_lim.n_data3 && tk.out_off >= 0 &&
                   tk.out_off + tk.rows <= g_lim.n_y && tk.gather_off >= 0 &&
                   tk.gather_off + tk.cpad + tk.cpad_d <= g_lim.n_gather &&
                   (int64_t)(tk.cpad + tk.cpad_d) * (int64_t)sizeof(A) <= g_lim.smem_uy);
        if (__syncthreads_or(task_bad)) {
            if (FUSE && prev_ne > 0) fused_stage<FUSE>(ode, stage, prev_e0, prev_ne, blockDim.x);
            prev_ne = 0;
            __syncthreads();
            continue;
        }
#endif
        const bool rows_on = mskip == nullptr || !mskip[tk.model];   // rows of a finished model: nothing to do
        if (rows_on) {
            const int ctot = tk.cpad_d + tk.cpad;
            // ---- input gather into shared memory: [dense segment | low-rank segment]
            {
                const int *gi = gidx + tk.gather_off;
                const float *gs = gscale != nullptr ? gscale + tk.gather_off : nullptr;
                const int gn = blockDim.x;   // gathering threads
                for (int c0 = threadIdx.x; c0 < ctot; c0 += GU * gn) {
                    int idx[GU];
#pragma unroll
                    for (int u = 0; u < GU; ++u) {
                        const int c = c0 + u * gn;
                        idx[u] = c < ctot ? gi[c] : -1;
#ifdef HBI_BOUNDS_CHECK
                        if (HBI_BC(idx[u] == -1 || (idx[u] >= 0 && idx[u] < g_lim.n_xt) ||
                                   (idx[u] <= -2 && -1 - (int64_t)idx[u] < g_lim.n_xt)))
                            idx[u] = -1;
#endif
                    }
                    A v[GU];
#pragma unroll
                    for (int u = 0; u < GU; ++u)   // -1: padding; <= -2: the pair at -2 - idx
                        v[u] = idx[u] >= 0 ? xt[idx[u]] : (idx[u] <= -2 ? xt[-2 - idx[u]] + xt[-1 - idx[u]] : A(0));
                    if (gs != nullptr) {
#pragma unroll
                        for (int u = 0; u < GU; ++u) {
                            const int c = c0 + u * gn;
                            if (c < ctot) v[u] *= (A)gs[c];
                        }
                    }
#pragma unroll
                    for (int u = 0; u < GU; ++u) {
                        const int c = c0 + u * gn;
                        if (c < ctot) z[c] = v[u];
                    }
                }
            }
        }
        __syncthreads();
        // FUSE: the previous unit's stage on the first FUSE_WARPS warps, which then join this
        // unit's rows, claimed a warp's row block at a time, so the stage hides behind the rows
        if (FUSE && prev_ne > 0 && warp < FUSE_WARPS) fused_stage<FUSE>(ode, stage, prev_e0, prev_ne, 32 * FUSE_WARPS);
        prev_ne = 0;
        if (rows_on) {
            // ---- rows: lanes split into groups of lpr (>= UY_RPW) per UY_RPW-row block, so
            //      that short rows still keep every lane busy
            const int nvec = tk.cpad_d / Vec<TD>::N + tk.cpad / Vec<TL>::N;
            int lpr = 32;
            while (lpr > UY_RPW && 2 * nvec <= lpr) lpr >>= 1;
            const int gpw = 32 / lpr, g = lane / lpr, sl = lane - g * lpr;
            const int wstep = gpw * UY_RPW;   // rows of one warp's block
            auto claim_rows = [&]() {
                int b = 0;
                if (lane == 0) b = atomicAdd(&s_rowctr, wstep);
                return __shfl_sync(0xffffffffu, b, 0);
            };
            for (int base = FUSE ? claim_rows() : warp * wstep; base < tk.rows;
                 base = FUSE ? claim_rows() : base + nwarps * wstep) {
                const int r0 = base + g * UY_RPW;
                const int nr = max(0, min(UY_RPW, tk.rows - r0));
                A acc[UY_RPW];
#pragma unroll
                for (int q = 0; q < UY_RPW; ++q) acc[q] = A(0);
                if (tk.cpad_d > 0)
                    segment_dot<UY_RPW, TD>(data_d + tk.data_off_d + (size_t)r0 * tk.cpad_d, tk.cpad_d, nr, z, sl, lpr,
                                            acc);
                if (tk.cpad > 0)
                    segment_dot<UY_RPW, TL>(data_l + tk.data_off + (size_t)r0 * tk.cpad, tk.cpad, nr, z + tk.cpad_d, sl,
                                            lpr, acc);
                int row;
                const A v = reduce_scatter<UY_RPW>(acc, sl, lpr, row);
                if ((sl & (lpr / UY_RPW - 1)) == 0 && row < nr) y[tk.out_off + r0 + row] = v;
            }
        }
        __syncthreads();
        if (FUSE) {   // the unit's elements (a skipped model's too: the stage decides)
            prev_e0 = (int)(tk.out_off / ode.nout);
            prev_ne = tk.rows / ode.nout;
        }
    }
}

// ------------------------------------------------ VT phase: TMA-fed, warp-specialised
// VT_CTAS_PER_SM CTAs per SM each walk a list of items made on the host (largest units
// first, balanced over the CTAs).  An item is a row block x column chunk of the stacked V^T
// panel of one column group: its panel (row-major, <= VT_PANEL_BYTES) and the matching x
// slice, which starts on a 16-byte boundary (the panel is packed with the same column
// shift, so z loads are aligned; `lo`/`hi` bound the group's columns inside it).  A
// producer warp moves both with cp.async.bulk (the TMA engine) into a ring of VT_STAGES
// shared-memory stages, completing on the stage's `full` mbarrier; VT_CW consumer warps
// reduce the rows and release the stage on its `empty` mbarrier.  A row block split into
// column chunks keeps per-lane running sums in registers across its chunks (consecutive
// items of one CTA), so t is deterministic and needs no partial sums or atomics.  Every
// wait is bounded by VT_WAIT_NS of wall time; a CTA that gives up raises the error flag and
// returns only after its bulk copies in flight have landed.
__device__ __forceinline__ unsigned smem_u32(const void *p) { return (unsigned)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mbar_init(uint64_t *bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_fence_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, unsigned bytes, uint64_t *bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(dst)),
                 "l"(src), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, unsigned parity) {
    unsigned ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
constexpr unsigned long long VT_WAIT_NS = 1000000000ull;   // 1 s
// One thread waits for the phase of the given parity; false once *fail is set or after VT_WAIT_NS.
__device__ __forceinline__ bool thread_wait(uint64_t *bar, unsigned parity, volatile int *fail) {
    if (mbar_try_wait(bar, parity)) return true;   // already complete: no timer read
    const unsigned long long t0 = global_ns();
    for (unsigned it = 0;; ++it) {
        if (mbar_try_wait(bar, parity)) return true;
        if ((it & 63u) == 63u && (*fail || global_ns() - t0 > VT_WAIT_NS)) {
            *fail = 1;
            return false;
        }
    }
}
// The same for a whole warp, with a warp-uniform outcome.
__device__ __forceinline__ bool warp_wait(uint64_t *bar, unsigned parity, volatile int *fail) {
    if (__all_sync(0xffffffffu, mbar_try_wait(bar, parity))) return true;   // already complete: no timer read
    const unsigned long long t0 = global_ns();
    for (unsigned it = 0;; ++it) {
        if (__all_sync(0xffffffffu, mbar_try_wait(bar, parity))) return true;
        if ((it & 63u) == 63u && __any_sync(0xffffffffu, *fail != 0 || global_ns() - t0 > VT_WAIT_NS)) {
            *fail = 1;
            return false;
        }
    }
}

// The rows of one whole-width VT item handled by one consumer warp: groups of lpr lanes take
// R rows per pass; the group's lanes stride the 16-byte column vectors.
template <int R, typename TL>
__device__ __forceinline__ void vt_item_rows(const VtItem &it, const TL *panel, const typename Vec<TL>::A *z,
                                             const float *__restrict__ rowscale, typename Vec<TL>::A *xt, int warp,
                                             int lane, int lpr) {
    using A = typename Vec<TL>::A;
    constexpr int VEC = Vec<TL>::N;
    const int gpw = 32 / lpr, g = lane / lpr, sl = lane - g * lpr;
    for (int base = warp * gpw * R; base < it.rows; base += VT_CW * gpw * R) {
        const int r0 = base + g * R;
        const int nr = max(0, min(R, it.rows - r0));
        // the row this lane stores after the reduction (reduce_scatter's assignment from the
        // sub-lane bits) and its scale, loaded before the column loop so that the load's
        // latency is hidden behind it
        int prow = 0;
        {
            int hh = lpr >> 1;
#pragma unroll
            for (int n = R; n > 1; n >>= 1) {
                prow = prow * 2 + ((sl & hh) ? 1 : 0);
                hh >>= 1;
            }
        }
        const bool will_store = (sl & (lpr / R - 1)) == 0 && prow < nr;
        const float rs_pre = (will_store && it.scale_off >= 0) ? rowscale[it.scale_off + r0 + prow] : 1.0f;
        A acc[R];
#pragma unroll
        for (int q = 0; q < R; ++q) acc[q] = A(0);
        for (int c = sl * VEC; c < it.cpad; c += lpr * VEC) {
            A zv[VEC];
            load_z(z + c, zv);
            if (c < it.lo || c + VEC > it.hi) {   // only a row's first or last vector
#pragma unroll
                for (int e = 0; e < VEC; ++e)
                    if (c + e < it.lo || c + e >= it.hi) zv[e] = A(0);
            }
#pragma unroll
            for (int q = 0; q < R; ++q)
                if (q < nr) {
                    const uint4 raw = *reinterpret_cast<const uint4 *>(panel + (size_t)(r0 + q) * it.cpad + c);
                    Vec<TL>::fma(raw, zv, acc[q]);
                }
        }
        int row;
        A v = reduce_scatter<R>(acc, sl, lpr, row);
        if (will_store) {
            const int r = r0 + row;
            if (it.scale_off >= 0) v *= (A)rs_pre;
            xt[it.out_off + r] = v;
        }
    }
}

// One column chunk of a split row block (<= VT_MC_ROWS rows): warp w owns rows
// [GEMV_RPW w, GEMV_RPW (w + 1)) in every chunk and its lanes add the chunk into per-lane
// running sums kept in registers across the chunks; the last chunk reduces them over the
// warp.  Fixed lane-to-column mapping and chunk order keep the result reproducible.
template <typename TL>
__device__ __forceinline__ void vt_chunk_rows(const VtItem &it, const TL *panel, const typename Vec<TL>::A *z,
                                              typename Vec<TL>::A (&acc)[GEMV_RPW], const float *__restrict__ rowscale,
                                              typename Vec<TL>::A *xt, int warp, int lane) {
    using A = typename Vec<TL>::A;
    constexpr int VEC = Vec<TL>::N;
    const int r0 = warp * GEMV_RPW;
    const int nr = max(0, min(GEMV_RPW, it.rows - r0));
    // the last chunk's storing lanes load their row scale before the column loop
    float rs_pre = 1.0f;
    int prow = 0;
    if (it.flags & 2) {
        int hh = 16;
#pragma unroll
        for (int n = GEMV_RPW; n > 1; n >>= 1) {
            prow = prow * 2 + ((lane & hh) ? 1 : 0);
            hh >>= 1;
        }
        if ((lane & (32 / GEMV_RPW - 1)) == 0 && prow < nr && it.scale_off >= 0)
            rs_pre = rowscale[it.scale_off + r0 + prow];
    }
    if (it.flags & 1) {
#pragma unroll
        for (int q = 0; q < GEMV_RPW; ++q) acc[q] = A(0);
    }
    if (nr > 0) {
        for (int c = lane * VEC; c < it.cpad; c += 32 * VEC) {
            A zv[VEC];
            load_z(z + c, zv);
            if (c < it.lo || c + VEC > it.hi) {   // only a row's first or last vector
#pragma unroll
                for (int e = 0; e < VEC; ++e)
                    if (c + e < it.lo || c + e >= it.hi) zv[e] = A(0);
            }
#pragma unroll
            for (int q = 0; q < GEMV_RPW; ++q)
                if (q < nr) {
                    const uint4 raw = *reinterpret_cast<const uint4 *>(panel + (size_t)(r0 + q) * it.cpad + c);
                    Vec<TL>::fma(raw, zv, acc[q]);
                }
        }
    }
    if ((it.flags & 2) && nr > 0) {
        int row;
        A v = reduce_scatter<GEMV_RPW>(acc, lane, 32, row);
        if ((lane & (32 / GEMV_RPW - 1)) == 0 && row < nr) {
            const int r = r0 + row;
            if (it.scale_off >= 0) v *= (A)rs_pre;
            xt[it.out_off + r] = v;
        }
    }
}

// One VT item by a consumer warp: a column chunk of a split row block, or a whole item whose
// rows per pass (8 or 4) and lanes per row group are the cheapest by a count of row-vector
// steps per warp plus a per-pass reduction cost.  TP is the item's panel element type.
template <typename TP>
__device__ __forceinline__ void vt_item(const VtItem &it, const TP *panel, const typename Vec<TP>::A *z,
                                        typename Vec<TP>::A (&macc)[GEMV_RPW], const float *__restrict__ rowscale,
                                        typename Vec<TP>::A *xt, int warp, int lane, int pass_cost) {
    constexpr int VEC = Vec<TP>::N;
    if ((it.flags & 3) != 3) {
        vt_chunk_rows<TP>(it, panel, z, macc, rowscale, xt, warp, lane);
        return;
    }
    const int nvec = it.cpad / VEC;
    int best = 1 << 30, bR = 4, blpr = 32;
#pragma unroll
    for (int R = 8; R >= 4; R >>= 1)
        for (int l = 32; l >= R; l >>= 1) {
            const int gpw = 32 / l, iters = (nvec + l - 1) / l;
            const int passes = (it.rows + R * gpw - 1) / (R * gpw);
            const int cost = (passes + VT_CW - 1) / VT_CW * (iters * R + pass_cost);
            if (cost < best) { best = cost; bR = R; blpr = l; }
        }
    if (bR == 8)
        vt_item_rows<8, TP>(it, panel, z, rowscale, xt, warp, lane, blpr);
    else
        vt_item_rows<4, TP>(it, panel, z, rowscale, xt, warp, lane, blpr);
}

template <typename TL>
__global__ void __launch_bounds__(VT_THREADS, VT_CTAS_PER_SM) vt_stream_kernel(
    const VtBatch *__restrict__ batches, const VtItem *__restrict__ items, const int *__restrict__ cta_begin,
    const TL *__restrict__ data, const float *__restrict__ rowscale, typename Vec<TL>::A *xt, const int *stop,
    int *err, int pass_cost, const int *__restrict__ mskip) {
    using A = typename Vec<TL>::A;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t full[VT_STAGES], empty[VT_STAGES];
    __shared__ VtItem desc[VT_STAGES][VT_MAX_SUB];
    __shared__ int nsub[VT_STAGES];
    __shared__ int s_fail;
    if (stop != nullptr && *(volatile const int *)stop) return;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int beg = cta_begin[blockIdx.x], n = cta_begin[blockIdx.x + 1] - beg;
    volatile int *fail = &s_fail;
    if (tid == 0) {
        for (int s = 0; s < VT_STAGES; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], VT_CW);
        }
        mbar_fence_init();
        s_fail = 0;
    }
    __syncthreads();
    auto stage_panel = [&](int s) { return smem_raw + (size_t)s * VT_STAGE_BYTES; };
    auto stage_x = [&](int s) { return reinterpret_cast<A *>(smem_raw + (size_t)s * VT_STAGE_BYTES + VT_PANEL_BYTES); };
    if (warp == VT_CW) {
        // ---- producer warp: batch i into stage i % VT_STAGES once its previous use is
        // released; lane k handles the descriptor and x slice of the batch's item k
        int i = 0;
#ifndef HBI_BOUNDS_CHECK
        // descriptors ahead of their use: the batch records two batches ahead, the items of
        // the next batch one ahead (the bounds-checked build reads each only once it is checked)
        VtBatch b_cur{}, b_next{};
        VtItem it_cur{};
        if (n > 0) b_cur = batches[beg];
        if (n > 1) b_next = batches[beg + 1];
        if (n > 0 && lane < b_cur.nitems) it_cur = items[b_cur.item0 + lane];
#endif
        for (; i < n; ++i) {
            const int s = i % VT_STAGES;
#ifndef HBI_BOUNDS_CHECK
            const VtBatch b = b_cur;
            VtItem it = it_cur;
            {
                VtItem it_n{};
                VtBatch b_nn{};
                if (i + 1 < n && lane < b_next.nitems) it_n = items[b_next.item0 + lane];
                if (i + 2 < n) b_nn = batches[beg + i + 2];
                b_cur = b_next;
                b_next = b_nn;
                it_cur = it_n;
            }
#else
            const VtBatch b = batches[beg + i];
            VtItem it{};
#endif
#ifdef HBI_BOUNDS_CHECK
            const bool batch_bad =
                lane == 0 && HBI_BC(b.nitems >= 1 && b.nitems <= VT_MAX_SUB && b.pbytes >= 0 && b.pbytes <= VT_PANEL_BYTES &&
                                    b.xbytes >= 0 && b.xbytes <= VT_X_BYTES && b.data_off >= 0 &&
                                    b.data_off * g_lim.es_vt + b.pbytes <= g_lim.n_data1 * g_lim.es_vt);
            const bool bad_b = __any_sync(0xffffffffu, batch_bad);
            if (!bad_b && lane < b.nitems) it = items[b.item0 + lane];
            const bool item_bad =
                !bad_b && lane < b.nitems &&
                HBI_BC(it.x_off >= 0 && it.x_off + it.cpad <= g_lim.n_xt + 16 && it.out_off >= g_lim.n_x &&
                       it.out_off + it.rows <= g_lim.n_xt && it.zoff >= 0 &&
                       (int64_t)it.zoff * (int64_t)sizeof(A) + (int64_t)it.cpad * (int64_t)sizeof(A) <= VT_X_BYTES);
            // a batch with a bad entry moves no bytes and is skipped
            const bool skip_all = bad_b || __any_sync(0xffffffffu, item_bad) ||
                                  (mskip != nullptr && __all_sync(0xffffffffu, lane >= b.nitems || mskip[it.model] != 0));
#else
            // a batch whose items all belong to skipped models moves no bytes
            const bool skip_all =
                mskip != nullptr && __all_sync(0xffffffffu, lane >= b.nitems || mskip[it.model] != 0);
#endif
            if (i >= VT_STAGES && !warp_wait(&empty[s], (unsigned)(i / VT_STAGES - 1) & 1u, fail)) break;
            if (skip_all) {
                if (lane == 0) {
                    nsub[s] = 0;
                    mbar_arrive(&full[s]);   // completes the phase without a transfer
                }
                __syncwarp();
                continue;
            }
            if (lane < b.nitems) desc[s][lane] = it;
            if (lane == 0) nsub[s] = b.nitems;
            __syncwarp();
            if (lane == 0) {
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                mbar_expect_tx(&full[s], (unsigned)(b.pbytes + b.xbytes));
            }
            __syncwarp();
            if (lane == 0) bulk_g2s(stage_panel(s), data + b.data_off, (unsigned)b.pbytes, &full[s]);
            if (lane < b.nitems)
                bulk_g2s(stage_x(s) + it.zoff, xt + it.x_off, (unsigned)(it.cpad * (int)sizeof(A)), &full[s]);
        }
        // the copies of the last issued batches must land before the CTA may exit
        if (lane == 0) {
            volatile int never = 0;
            for (int j = max(0, i - VT_STAGES); j < i; ++j)
                if (!thread_wait(&full[j % VT_STAGES], (unsigned)(j / VT_STAGES) & 1u, &never)) *fail = 1;
        }
        __syncwarp();
    } else {
        // ---- consumers
        A macc[GEMV_RPW];   // per-lane running sums of the current split row block
#pragma unroll
        for (int q = 0; q < GEMV_RPW; ++q) macc[q] = A(0);
        for (int i = 0; i < n; ++i) {
            const int s = i % VT_STAGES;
            if (!warp_wait(&full[s], (unsigned)(i / VT_STAGES) & 1u, fail)) break;
            const int ns = nsub[s];
            for (int k = 0; k < ns; ++k) {
                const VtItem it = desc[s][k];
                if (mskip != nullptr && mskip[it.model]) continue;   // columns of a skipped model
                const TL *panel = reinterpret_cast<const TL *>(stage_panel(s)) + it.poff;
                const A *z = stage_x(s) + it.zoff;
                vt_item<TL>(it, panel, z, macc, rowscale, xt, warp, lane, pass_cost);
            }
            __syncwarp();
            if (lane == 0) mbar_arrive(&empty[s]);
        }
    }
    __syncthreads();
    if (tid == 0 && s_fail) atomicExch(err, 1);
}

// A wait that can never complete (an mbarrier phase that expects one arrival nobody makes),
// through the same bounded helper as the V^T kernel: it gives up after VT_WAIT_NS and the
// kernel reports it through *err, as a stalled V^T stage would.  No copy is in flight.
__global__ void stalled_wait_kernel(int *err) {
    __shared__ __align__(8) uint64_t bar;
    __shared__ int fail;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        mbar_fence_init();
        fail = 0;
    }
    __syncwarp();
    const bool done = warp_wait(&bar, 0u, &fail);
    if (threadIdx.x == 0) *err = done ? 0 : 1;
}

hbi_status stalled_wait_status(cudaStream_t s) {
    int *d_err = nullptr, err = 0;
    HBI_ALLOC_TRY(&d_err, sizeof(int));
    stalled_wait_kernel<<<1, 32, 0, s>>>(d_err);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e == cudaSuccess) e = cudaMemcpy(&err, d_err, sizeof(int), cudaMemcpyDeviceToHost);
    cudaFree(d_err);
    if (e != cudaSuccess) { set_error(std::string("stalled wait check: ") + cudaGetErrorString(e)); return HBI_ERR_CUDA; }
    if (err) { set_error("a device wait timed out"); return HBI_ERR_TIMEOUT; }
    return HBI_OK;
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

// Power-of-two scales of the given FP64 columns (max |entry| / scale in (2^13, 2^14]).
hbi_status column_scales(const std::vector<ColRef> &cols, std::vector<float> &out) {
    out.assign(cols.size(), 1.0f);
    if (cols.empty()) return HBI_OK;
    ColRef *d_cols = nullptr;
    float *d_s = nullptr;
    DevScratch tmp;
    hbi_status st;
    if ((st = tmp.upload(&d_cols, cols)) || (st = tmp.alloc(&d_s, cols.size() * sizeof(float)))) return st;
    const int64_t threads = (int64_t)cols.size() * 32;
    colscale_kernel<<<(unsigned)((threads + 255) / 256), 256>>>(d_cols, (int64_t)cols.size(), d_s);
    HBI_CUDA_TRY(cudaGetLastError());
    HBI_CUDA_TRY(cudaMemcpy(out.data(), d_s, cols.size() * sizeof(float), cudaMemcpyDeviceToHost));
    return HBI_OK;
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
    float hi_inv_scale;  // > 0: the row holds v - hi(v), the part of v its FP16 hi row (scale
                         // 1 / hi_inv_scale) does not represent
};
// one CTA per VT item: panel column j holds group column chunk_col0 + j - lo for
// lo <= j < hi and zero elsewhere
template <typename T>
__global__ void pack_vt_kernel(const VtItem *__restrict__ items, const int64_t *__restrict__ chunk_col0,
                               const int64_t *__restrict__ row_base, const VtRow *__restrict__ rows,
                               T *__restrict__ data) {
    const VtItem it = items[blockIdx.x];
    const int64_t c0 = chunk_col0[blockIdx.x], rb = row_base[blockIdx.x];
    const int64_t tot = (int64_t)it.rows * it.cpad;
    for (int64_t e = threadIdx.x; e < tot; e += blockDim.x) {
        const int r = (int)(e / it.cpad), j = (int)(e - (int64_t)r * it.cpad);
        double v = 0.0;
        if (j >= it.lo && j < it.hi) {
            const VtRow R = rows[rb + r];
            v = R.v[c0 + j - it.lo];
            if (R.hi_inv_scale > 0.0f) {   // residual of the hi row, in the same element type
                const double hs = (double)R.hi_inv_scale;
                v -= (double)to_storage<T>(v * hs) / hs;
            }
            v *= (double)R.inv_scale;
        }
        data[it.data_off + e] = to_storage<T>(v);
    }
}

struct UyTerm {          // one block's contribution to a leaf row unit
    const double *src;   // U (column-major, ld = m), dense (row-major, ld = nc) or, for a
                         // transposed dense block, its original (column-major here, ld = m)
    const float *colscale;  // per-column scale of this block (U or dense), or null
    int64_t ld, roff;    // leading dimension, first block row of the unit
    int width, coloff, dense;   // coloff: column offset inside its segment
    int trans;           // dense block read transposed
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
            double v = t.dense ? (t.trans ? t.src[(int64_t)c * t.ld + t.roff + i] : t.src[(t.roff + i) * t.ld + c])
                               : t.src[(int64_t)c * t.ld + t.roff + i];
            if (t.colscale) v /= (double)t.colscale[c];
            if (t.dense)
                data_d[tk.data_off_d + (int64_t)i * tk.cpad_d + t.coloff + c] = to_storage<TD>(v);
            else
                data_l[tk.data_off + (int64_t)i * tk.cpad + t.coloff + c] = to_storage<TL>(v);
        }
    }
}

// UY grid for `per_sm` CTAs per SM (capped by the occupancy of the chosen row variant)
void set_uy_grid(hbi_handle *h, int per_sm) {
    const int occ = h->uy_occ[h->uy_rpw == 8 ? 1 : 0];
    h->uy_ctas_per_sm = std::max(1, std::min(per_sm, occ));
    h->grid2 = std::max(1, std::min(h->num_sms * h->uy_ctas_per_sm, std::max(1, h->n_tasks2)));
}

// ------------------------------------------------------------- host driver
namespace {
// element sizes of the dense and low-rank streams of a storage mode
size_t esize_dense(int storage) {
    switch (storage) {
        case HBI_FP64: return 8;
        case HBI_FP32: case HBI_MIXED: case HBI_ADAPTIVE: return 4;
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
        // The limit is a property of the kernel, shared by every handle: only ever raise
        // it, so that building a handle with smaller panels cannot invalidate another's.
        cudaFuncAttributes fa;
        // rows per pass 4 / 8, each plain and with a Cash-Karp stage of either law inside
        // (same grid: the smallest of the occupancies)
        const void *fns[2][3] = {{(const void *)uy_gemv_kernel<TD, TL, 4, 0>, (const void *)uy_gemv_kernel<TD, TL, 4, 1>,
                                  (const void *)uy_gemv_kernel<TD, TL, 4, 2>},
                                 {(const void *)uy_gemv_kernel<TD, TL, 8, 0>, (const void *)uy_gemv_kernel<TD, TL, 8, 1>,
                                  (const void *)uy_gemv_kernel<TD, TL, 8, 2>}};
        for (int v = 0; v < 2; ++v) {
            int occ = 1 << 30;
            for (int f = 0; f < 3; ++f) {
                HBI_CUDA_TRY(cudaFuncGetAttributes(&fa, fns[v][f]));
                if (smem2 > fa.maxDynamicSharedSizeBytes)
                    HBI_CUDA_TRY(cudaFuncSetAttribute(fns[v][f], cudaFuncAttributeMaxDynamicSharedMemorySize, smem2));
                int b = 0;
                HBI_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, fns[v][f], GEMV_THREADS, smem2));
                occ = std::min(occ, b);
            }
            h->uy_occ[v] = std::max(1, occ);
        }
        const void *fvt = (const void *)vt_stream_kernel<TL>;
        HBI_CUDA_TRY(cudaFuncGetAttributes(&fa, fvt));
        if (smem1 > fa.maxDynamicSharedSizeBytes)
            HBI_CUDA_TRY(cudaFuncSetAttribute(fvt, cudaFuncAttributeMaxDynamicSharedMemorySize, smem1));
        int b1 = 0;
        HBI_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b1, fvt, VT_THREADS, smem1));
        if (b1 < 1) {
            set_error("VT stage ring does not fit one SM");
            return HBI_ERR_INVALID_ARG;
        }
        h->uy_rpw = 4;
        h->vt_pass_cost = VT_PASS_COST;
        set_uy_grid(h, h->uy_occ[0]);
        return HBI_OK;
    }
};

struct PackLaunch {
    hbi_handle *h;
    const VtItem *t1;
    const GemvTask *t2;
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
    if (smem2 > 220 * 1024) {
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
    HBI_ALLOC_TRY((void **)dst, std::max<size_t>(1, v.size()) * sizeof(X));
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
    // model of an element (ensemble handles: contiguous element ranges)
    auto model_of = [&](int64_t e) {
        return (int)(std::upper_bound(h->model_start.begin(), h->model_start.end(), (int)e) - h->model_start.begin()) - 1;
    };

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
            for (int64_t j = 0; j < B.nc; ++j)
                cols.push_back(B.dense_trans ? ColRef{B.d_src + j * B.m, B.m, 1} : ColRef{B.d_src + j, B.m, B.nc});
        }
    }
    ColRef *d_cols = nullptr;
    float *d_colscale = nullptr;
    std::vector<float> colscale;
    DevScratch tmp;   // build tables, freed on every return path
    if (!cols.empty()) {
        hbi_status st = tmp.upload(&d_cols, cols);
        if (st) return st;
        if ((st = tmp.alloc(&d_colscale, cols.size() * sizeof(float)))) return st;
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
    std::vector<VtItem> t1;
    std::vector<int64_t> chunk_col0, row_base;
    std::vector<size_t> unit_first;   // first item of each row block (unit of the schedule)
    std::vector<VtRow> vrows;
    std::vector<float> rowscale;
    int64_t tcount = 0, d1 = 0;
    const int64_t ntot_in = (int64_t)nin * n;
    const int64_t ZA = 16 / (int64_t)acc_bytes;                // accumulator words per 16 bytes
    const int64_t zcap = VT_X_BYTES / (int64_t)acc_bytes;      // columns of an x slice
    // HBI_ADAPTIVE: V(:, 0) of a low-rank block as two FP16 rows, hi and lo (t entries
    // toff[b] and toff[b] + 1), then its other ranks; plain storage: rank k at toff[b] + k
    const bool dom32 = h->storage == HBI_ADAPTIVE;
    const int k0 = dom32 ? 1 : 0;
    // Items of one sub-panel of a group (`rows` panel rows from t position tb, element size
    // es): the x slice starts on the 16-byte boundary at or below col0 (shift lo).  A group
    // whose full width fits an x slice and at least min(rows, VT_MC_ROWS) rows of it fit a
    // panel is cut into row blocks only; otherwise row blocks of <= VT_MC_ROWS rows are cut
    // into column chunks.  d1 counts stream elements of the low-rank type (an FP32 panel
    // takes es / esl of them per entry).
    auto cut = [&](int64_t col0, int64_t nc, int64_t rows, int64_t tb, int64_t es, bool scaled) {
        const int64_t vec = 16 / es;
        const int64_t lo = col0 % ZA, x0 = col0 - lo;
        const int64_t cpad_full = round_up(lo + nc, vec);
        const int64_t fit = VT_PANEL_BYTES / (cpad_full * es);
        int64_t rb, cw, nch;
        if (cpad_full <= zcap && fit >= std::min<int64_t>(rows, VT_MC_ROWS)) {
            const int64_t nrb0 = (rows + fit - 1) / fit;
            rb = (rows + nrb0 - 1) / nrb0;
            cw = nc;
            nch = 1;
        } else {
            const int64_t nrb0 = (rows + VT_MC_ROWS - 1) / VT_MC_ROWS;
            rb = (rows + nrb0 - 1) / nrb0;
            // a chunk spans whole warp sweeps of 32 16-byte vectors: cw + lo rounds up to
            // k sweeps, and cw is a multiple of ZA so that every chunk keeps the shift lo
            const int64_t cw_max = std::min<int64_t>(zcap, VT_PANEL_BYTES / (rb * es));
            const int64_t sweep = 32 * vec;
            cw = std::max<int64_t>(1, cw_max / sweep) * sweep - vec;
            nch = (nc + cw - 1) / cw;
        }
        const int64_t nrb = (rows + rb - 1) / rb;
        for (int64_t q = 0; q < nrb; ++q) {
            const int64_t rows_q = std::min<int64_t>(rb, rows - q * rb);
            unit_first.push_back(t1.size());
            for (int64_t c = 0; c < nch; ++c) {
                const int64_t cols_c = std::min(cw, nc - c * cw);
                VtItem T{};
                T.data_off = d1;
                T.x_off = x0 + c * cw;
                T.out_off = ntot_in + tb + q * rb;
                T.scale_off = scaled ? tb + q * rb : -1;
                T.rows = (int)rows_q;
                T.lo = (int)lo;
                T.hi = (int)(lo + cols_c);
                T.cpad = (int)round_up(lo + cols_c, vec);
                T.flags = (c == 0 ? 1 : 0) | (c == nch - 1 ? 2 : 0);
                T.model = model_of(col0 / nin);
                d1 += rows_q * T.cpad * (es / (int64_t)esl);
                t1.push_back(T);
                chunk_col0.push_back(c * cw);
                row_base.push_back(tb + q * rb);
            }
        }
    };
    for (auto &kv : groups) {
        const int64_t col0 = kv.first.first, nc = kv.first.second;
        const int64_t tbase = tcount;
        int64_t rows = 0;
        for (int b : kv.second) {
            const Block &B = blocks[b];
            toff[b] = tbase + rows;
            if (dom32) {
                // hi and lo rows of V(:, 0): the lo row's scale sits 2^11 below the hi row's
                // (the residual is at most half an FP16 unit of the column's largest entry);
                // U(:, 0) stays FP32 in UY, so these t entries carry the V scales alone
                const float sv = colscale[soffV[b]];
                vrows.push_back(VtRow{B.d_src2, 1.0f / sv, 0.0f});
                rowscale.push_back(sv);
                vrows.push_back(VtRow{B.d_src2, 2048.0f / sv, 1.0f / sv});
                rowscale.push_back(sv / 2048.0f);
                rows += 2;
            }
            for (int k = k0; k < B.rank; ++k) {
                const float sv = scaled_l ? colscale[soffV[b] + k] : 1.0f;
                const float su = scaled_l ? colscale[soffU[b] + k] : 1.0f;
                vrows.push_back(VtRow{B.d_src2 + (size_t)k * B.nc, 1.0f / sv, 0.0f});
                rowscale.push_back(sv * su);
            }
            rows += B.rank - k0;
        }
        cut(col0, nc, rows, tbase, (int64_t)esl, scaled_l);
        tcount += rows;
    }
    unit_first.push_back(t1.size());
    h->n_t = tcount;

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
        // dense terms first (their gather entries lead), then the low-rank terms; with
        // HBI_ADAPTIVE a low-rank block's leading U column joins the dense (FP32) segment and
        // gathers the sum of its hi and lo t entries (index -2 - t)
        for (int pass = 0; pass < 2; ++pass) {
            for (int b : unit_terms[u]) {
                const Block &B = blocks[b];
                if (pass == 0 && dom32 && B.lowrank) {
                    UyTerm t{};
                    t.roff = r0 - B.row0;
                    t.src = B.d_src; t.ld = B.m; t.width = 1; t.dense = 1; t.trans = 1;   // column-major U(:, 0)
                    t.coloff = (int)Cd;
                    t.colscale = nullptr;
                    gidx.push_back((int)(-2 - (ntot_in + toff[b])));
                    gsc.push_back(1.0f);
                    Cd += 1;
                    terms.push_back(t);
                    continue;
                }
                if ((pass == 0) == (bool)B.lowrank) continue;
                if (B.lowrank && B.rank - k0 == 0) continue;
                UyTerm t{};
                t.roff = r0 - B.row0;
                if (!B.lowrank) {
                    t.src = B.d_src; t.ld = B.dense_trans ? B.m : B.nc; t.width = (int)B.nc; t.dense = 1;
                    t.coloff = (int)Cd; t.trans = B.dense_trans;
                    t.colscale = scaled_d ? d_colscale + soffD[b] : nullptr;
                    for (int64_t j = 0; j < B.nc; ++j) {
                        gidx.push_back((int)(B.col0 + j));
                        gsc.push_back(scaled_d ? colscale[soffD[b] + j] : 1.0f);
                    }
                    Cd += t.width;
                } else {
                    t.src = B.d_src + (size_t)k0 * B.m; t.ld = B.m; t.width = B.rank - k0; t.dense = 0;
                    t.coloff = (int)Cl;
                    t.colscale = scaled_l ? d_colscale + soffU[b] + k0 : nullptr;
                    for (int k = k0; k < B.rank; ++k) {
                        gidx.push_back((int)(ntot_in + toff[b] + 2 * k0 + k - k0));
                        gsc.push_back(1.0f);
                    }
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
        T.out_off = r0;
        T.gather_off = goff;
        T.rows = (int)R;
        T.cpad = (int)cpl;
        T.cpad_d = (int)cpd;
        T.model = model_of(leaf_starts[u]);
        d2 += R * cpl;
        d3 += R * cpd;
        t2.push_back(T);
    }
    term_begin.push_back((int)terms.size());
    if ((int64_t)gidx.size() > (int64_t)INT32_MAX || ntot_in + tcount > (int64_t)INT32_MAX) {
        set_error("operator too large for 32-bit gather indices");
        return HBI_ERR_INVALID_ARG;
    }

    hbi_status st;
    // ---- VT schedule: row-block units, largest first, each to the least loaded of
    // VT_CTAS_PER_SM x num_sms CTA lists (static LPT); a unit's chunks stay consecutive.
    // Panels are then laid out in list order, so consecutive items of a CTA are contiguous
    // and are grouped into stage batches (one bulk copy of their panels).
    int dev = 0;
    HBI_CUDA_TRY(cudaGetDevice(&dev));
    HBI_CUDA_TRY(cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, dev));
    const int G = std::max(1, h->num_sms) * VT_CTAS_PER_SM;
    std::vector<VtItem> items;
    std::vector<VtBatch> batches;
    std::vector<int64_t> ic0, irb;
    std::vector<int> vt_begin(G + 1, 0);
    auto es_of = [&](const VtItem &) { return (int64_t)esl; };
    auto len_of = [&](const VtItem &it) { return (int64_t)it.rows * it.cpad; };
    d1 = 0;
    {
        const size_t nunits = unit_first.size() - 1;
        std::vector<int64_t> uw(nunits, 0);
        for (size_t u = 0; u < nunits; ++u)
            for (size_t i = unit_first[u]; i < unit_first[u + 1]; ++i)
                uw[u] += (int64_t)t1[i].rows * t1[i].cpad * es_of(t1[i]) + (int64_t)t1[i].cpad * (int64_t)acc_bytes +
                         1024;   // + a per-item overhead in bytes of streaming time
        std::vector<size_t> uorder(nunits);
        std::iota(uorder.begin(), uorder.end(), (size_t)0);
        std::stable_sort(uorder.begin(), uorder.end(), [&](size_t a, size_t b) { return uw[a] > uw[b]; });
        std::vector<std::vector<size_t>> lists(G);
        using Load = std::pair<int64_t, int>;
        std::priority_queue<Load, std::vector<Load>, std::greater<Load>> pq;
        for (int g = 0; g < G; ++g) pq.push({0, g});
        for (size_t u : uorder) {
            const Load l = pq.top();
            pq.pop();
            lists[l.second].push_back(u);
            pq.push({l.first + uw[u], l.second});
        }
        for (int g = 0; g < G; ++g) {
            vt_begin[g] = (int)batches.size();
            VtBatch cur{};
            cur.nitems = 0;
            for (size_t u : lists[g]) {
                for (size_t i = unit_first[u]; i < unit_first[u + 1]; ++i) {
                    VtItem it = t1[i];
                    const int pb = (int)((int64_t)it.rows * it.cpad * es_of(it));
                    const int xb = (int)((int64_t)it.cpad * (int64_t)acc_bytes);
                    if (cur.nitems > 0 && (cur.nitems == VT_MAX_SUB || cur.pbytes + pb > VT_PANEL_BYTES ||
                                           cur.xbytes + xb > VT_X_BYTES)) {
                        batches.push_back(cur);
                        cur = VtBatch{};
                        cur.nitems = 0;
                    }
                    if (cur.nitems == 0) {
                        cur.data_off = d1;
                        cur.pbytes = cur.xbytes = 0;
                        cur.item0 = (int)items.size();
                    }
                    it.data_off = d1;
                    it.poff = (int)(cur.pbytes / (int)esl);
                    it.zoff = (int)(cur.xbytes / (int)acc_bytes);
                    cur.pbytes += pb;
                    cur.xbytes += xb;
                    ++cur.nitems;
                    d1 += len_of(it);
                    items.push_back(it);
                    ic0.push_back(chunk_col0[i]);
                    irb.push_back(row_base[i]);
                }
            }
            if (cur.nitems > 0) batches.push_back(cur);
        }
        vt_begin[G] = (int)batches.size();
    }
    if ((int64_t)items.size() > (int64_t)INT32_MAX / 2) {
        set_error("too many V^T items");
        return HBI_ERR_INVALID_ARG;
    }
    // ---- device allocations and packing
    h->n_data1 = d1;
    h->n_data2 = d2;
    h->n_data3 = d3;
    HBI_ALLOC_TRY(&h->d_data1, std::max<int64_t>(1, d1) * esl);
    HBI_ALLOC_TRY(&h->d_data2, std::max<int64_t>(1, d2) * esl);
    HBI_ALLOC_TRY(&h->d_data3, std::max<int64_t>(1, d3) * esd);
    HBI_CUDA_TRY(cudaMemset(h->d_data2, 0, std::max<int64_t>(1, d2) * esl));
    HBI_CUDA_TRY(cudaMemset(h->d_data3, 0, std::max<int64_t>(1, d3) * esd));
    VtItem *d_t1 = nullptr;
    GemvTask *d_t2 = nullptr;
    int64_t *d_c0 = nullptr, *d_rb = nullptr;
    VtRow *d_rows = nullptr;
    int *d_tb = nullptr;
    UyTerm *d_terms = nullptr;
    if ((st = tmp.upload(&d_t1, items)) || (st = tmp.upload(&d_t2, t2)) || (st = tmp.upload(&d_c0, ic0)) ||
        (st = tmp.upload(&d_rb, irb)) || (st = tmp.upload(&d_rows, vrows)) || (st = tmp.upload(&d_tb, term_begin)) ||
        (st = tmp.upload(&d_terms, terms)))
        return st;
    PackLaunch pk{h, d_t1, d_t2, (int)items.size(), (int)t2.size(), d_c0, d_rb, d_rows, d_tb, d_terms};
    if ((st = dispatch_storage(h->storage, pk))) return st;
    HBI_CUDA_TRY(cudaDeviceSynchronize());

    // ---- UY tasks sorted by decreasing size for the dynamic scheduler (LPT)
    auto work = [&](const GemvTask &a) { return (int64_t)a.rows * ((int64_t)a.cpad * esl + (int64_t)a.cpad_d * esd); };
    auto bigger = [&](const GemvTask &a, const GemvTask &b) {
        const int64_t ca = work(a), cb = work(b);
        return ca > cb || (ca == cb && (a.data_off < b.data_off || (a.data_off == b.data_off && a.data_off_d < b.data_off_d)));
    };
    std::stable_sort(t2.begin(), t2.end(), bigger);
    h->grid1 = G;
    int smem1 = (int)(VT_STAGES * VT_STAGE_BYTES), smem2 = 16;
    for (auto &T : t2) smem2 = std::max<int>(smem2, (int)((T.cpad + T.cpad_d) * acc_bytes));
    // every access of the two product kernels stays inside its buffers (the bounds-checked
    // build checks the same limits on the device)
    {
        TableLimits L;
        L.n_data1 = d1; L.n_data2 = d2; L.n_data3 = d3;
        L.n_x = ntot_in; L.n_xt = ntot_in + tcount; L.n_y = (int64_t)nout * n; L.n_gather = (int64_t)gidx.size();
        L.es_vt = (int)esl; L.es_u = (int)esl; L.es_d = (int)esd; L.acc_bytes = (int)acc_bytes;
        L.smem_uy = smem2;
        L.vt_panel_bytes = (int)VT_PANEL_BYTES; L.vt_x_bytes = (int)VT_X_BYTES; L.vt_max_sub = VT_MAX_SUB;
        L.vt_split_rows = VT_MC_ROWS;
        std::string first;
        if (check_vt_tables(batches, items, L, &first) + check_uy_tables(t2, gidx, L, &first) > 0) {
            set_error("internal error: an HMVM work table exceeds its buffers (" + first + ")");
            return HBI_ERR_INVALID_ARG;
        }
        h->lim = L;
    }
#ifdef HBI_BOUNDS_CHECK
    {
        const DevLimits dl{h->lim.n_data1, h->lim.n_data2, h->lim.n_data3, h->lim.n_x, h->lim.n_xt, h->lim.n_y,
                           h->lim.n_gather, h->lim.es_vt, h->lim.smem_uy};
        HBI_ALLOC_TRY(&h->d_lim, sizeof dl);
        HBI_CUDA_TRY(cudaMemcpy(h->d_lim, &dl, sizeof dl, cudaMemcpyHostToDevice));
    }
#endif
    h->n_tasks1 = (int)items.size();
    h->n_tasks2 = (int)t2.size();
    h->n_gather = (int64_t)gidx.size();
    h->n_rowscale = (int64_t)rowscale.size();
    if ((st = upload(&h->d_items1, items)) || (st = upload(&h->d_batches1, batches)) ||
        (st = upload(&h->d_vt_begin, vt_begin)) || (st = upload(&h->d_tasks2, t2)) || (st = upload(&h->d_gidx, gidx)))
        return st;
    if (scaled_d && (st = upload(&h->d_gscale, gsc))) return st;
    if (scaled_l && (st = upload(&h->d_rowscale, rowscale))) return st;
    // + 16 zero guard elements: VT x slices are read up to their padded width
    HBI_ALLOC_TRY(&h->d_xt, (ntot_in + tcount + 16) * acc_bytes);
    HBI_CUDA_TRY(cudaMemset(h->d_xt, 0, (ntot_in + tcount + 16) * acc_bytes));
    HBI_ALLOC_TRY(&h->d_xt2, (ntot_in + tcount + 16) * acc_bytes);
    HBI_CUDA_TRY(cudaMemset(h->d_xt2, 0, (ntot_in + tcount + 16) * acc_bytes));
    HBI_ALLOC_TRY(&h->d_yp, (size_t)nout * n * acc_bytes);
    HBI_ALLOC_TRY(&h->d_counters, 4 * sizeof(int));
    HBI_CUDA_TRY(cudaMemset(h->d_counters, 0, 4 * sizeof(int)));

    // ---- bytes per HMVM: packed streams (with padding) and algorithmic (stored entries,
    //      scales, x read, y written, t written and read)
    h->bytes_factors = (d1 + d2) * (int64_t)esl + d3 * (int64_t)esd + (int64_t)gidx.size() * (scaled_d ? 8 : 4) +
                       (int64_t)rowscale.size() * 4;
    int64_t v_entries = 0, u_entries = 0, d_entries = 0, v_scales = 0, uy_scales = 0;
    int64_t u32 = 0;   // HBI_ADAPTIVE: U(:, 0) in FP32; V(:, 0) as two FP16 rows
    for (auto &B : blocks) {
        if (B.lowrank) {
            const int64_t vr = B.rank > 0 ? B.rank + k0 : 0, ur = B.rank > 0 ? B.rank - k0 : 0;
            if (B.rank > 0 && dom32) u32 += B.m;
            v_entries += B.nc * vr;
            u_entries += B.m * ur;
            if (scaled_l) { v_scales += 4 * vr; uy_scales += 4 * ur; }
        } else {
            d_entries += B.m * B.nc;
            if (scaled_d) uy_scales += 4 * B.nc;
        }
    }
    h->bytes_alg_vt = v_entries * (int64_t)esl + v_scales + (ntot_in + tcount) * (int64_t)acc_bytes;
    h->bytes_alg_uy = u_entries * (int64_t)esl + 4 * u32 + d_entries * (int64_t)esd + uy_scales +
                      (ntot_in + tcount + (int64_t)nout * n) * (int64_t)acc_bytes;
    h->bytes_algorithmic = (v_entries + u_entries) * (int64_t)esl + 4 * u32 + d_entries * (int64_t)esd +
                           v_scales + uy_scales + (int64_t)(nin + nout) * n * (int64_t)acc_bytes +
                           2 * tcount * (int64_t)acc_bytes;
    return gemv_config(h, smem1, smem2);
}

hbi_status pack_operators(hbi_handle *h, std::vector<Block> &blocks, const std::vector<int> &leaf_starts,
                          int with_transpose, int multi_rhs) {
    // H^T has the blocks (sigma, tau): a low-rank block's factors swap (U' = V, V' = U), a
    // dense block is read transposed; rows of H^T are the n_in components of each element
    std::vector<Block> bt;
    if (with_transpose) {
        bt.reserve(blocks.size());
        for (const Block &B : blocks) {
            Block T = B;
            T.tau = B.sig; T.sig = B.tau;
            T.row0 = B.col0; T.m = B.nc;
            T.col0 = B.row0; T.nc = B.m;
            if (B.lowrank) { T.d_src = B.d_src2; T.d_src2 = B.d_src; }
            else T.dense_trans = 1;
            bt.push_back(T);
        }
    }
    hbi_status st = pack_operator(h, nullptr, blocks, leaf_starts);
    if (!st && multi_rhs) st = pack_multi(h, blocks, leaf_starts);
    if (st || !with_transpose) return st;
    hbi_handle *a = new hbi_handle();
    h->adj = a;
    a->n = h->n; a->nv = h->nv; a->op = h->op;
    a->nin = h->nout; a->nout = h->nin;
    a->mu = h->mu; a->nu = h->nu; a->storage = h->storage;
    a->perm = h->perm;
    a->n_models = h->n_models; a->model_start = h->model_start;
    HBI_ALLOC_TRY(&a->d_perm, (size_t)h->n * sizeof(int));
    HBI_CUDA_TRY(cudaMemcpy(a->d_perm, h->d_perm, (size_t)h->n * sizeof(int), cudaMemcpyDeviceToDevice));
    return pack_operator(a, nullptr, bt, leaf_starts);
}

// ----------------------------------------------------------------- launch
namespace {
// One product with explicit buffers.  phase: -1 = whole product, 0 = VT, 2 = UY (with the
// reset of its work counter unless reset = false, so that it can also be launched alone and
// repeatedly); 1 launches nothing (kept so the phase timing keeps its layout).  counters[0] is
// the UY work counter, counters[1] an error flag that a VT CTA sets when one of its bounded
// waits gives up (cleared only when it is reported), counters[2] the UY CTAs that finished
// (the last one sets counters[0] and counters[2] back to zero).
template <typename TD, typename TL>
hbi_status hmvm_run(hbi_handle *h, int phase, typename Vec<TL>::A *xt, typename Vec<TL>::A *yp, int *counters,
                    cudaStream_t s, const int *d_stop, const int *d_mskip = nullptr, bool reset = true,
                    const OdeArgs *fuse = nullptr, int stage = 0, int law = 1) {
#ifdef HBI_BOUNDS_CHECK
    // from device memory: a copy captured into the attempt graph stays valid at every replay
    HBI_CUDA_TRY(cudaMemcpyToSymbolAsync(g_lim, h->d_lim, sizeof(DevLimits), 0, cudaMemcpyDeviceToDevice, s));
#endif
    if (phase <= 0) {
        if (h->n_tasks1)
            vt_stream_kernel<TL><<<h->grid1, VT_THREADS, h->smem1, s>>>(
                h->d_batches1, h->d_items1, h->d_vt_begin, (const TL *)h->d_data1, h->d_rowscale, xt, d_stop,
                counters + 1, h->vt_pass_cost, d_mskip);
    }
    if (phase < 0 || phase == 2) {
        if (reset) HBI_CUDA_TRY(cudaMemsetAsync(counters, 0, sizeof(int), s));
        const OdeArgs none{};
        const OdeArgs &oa = fuse != nullptr ? *fuse : none;
#define HBI_UY_LAUNCH(R, F)                                                                                        \
    uy_gemv_kernel<TD, TL, R, F><<<h->grid2, GEMV_THREADS, h->smem2, s>>>(                                         \
        h->d_tasks2, h->n_tasks2, (const TD *)h->d_data3, (const TL *)h->d_data2, h->d_gidx, h->d_gscale, xt, yp,    \
        counters, d_stop, d_mskip, oa, stage)
        const int f = fuse == nullptr ? 0 : (law == 2 ? 2 : 1);
        if (h->uy_rpw == 8) {
            if (f == 2) HBI_UY_LAUNCH(8, 2);
            else if (f == 1) HBI_UY_LAUNCH(8, 1);
            else HBI_UY_LAUNCH(8, 0);
        } else {
            if (f == 2) HBI_UY_LAUNCH(4, 2);
            else if (f == 1) HBI_UY_LAUNCH(4, 1);
            else HBI_UY_LAUNCH(4, 0);
        }
#undef HBI_UY_LAUNCH
    }
    HBI_CUDA_TRY(cudaGetLastError());
    return HBI_OK;
}
struct PhaseRun {
    hbi_handle *h;
    int phase;
    cudaStream_t s;
    const int *stop, *mskip;
    bool reset;
    void *xt = nullptr;
    const OdeArgs *fuse = nullptr;
    int stage = 0;
    int law = 1;
    template <typename TD, typename TL> hbi_status operator()() {
        using A = typename Vec<TL>::A;
        return hmvm_run<TD, TL>(h, phase, (A *)(xt != nullptr ? xt : h->d_xt), (A *)h->d_yp, h->d_counters, s, stop,
                                mskip, reset, fuse, stage, law);
    }
};
}  // namespace

hbi_status hmvm_phase(hbi_handle *h, int phase, cudaStream_t s, const int *d_stop) {
    return dispatch_storage(h->storage, PhaseRun{h, phase, s, d_stop, nullptr, true});
}

hbi_status hmvm_launch(hbi_handle *h, cudaStream_t s, const int *d_stop, const int *d_mskip, bool reset_counter,
                       void *xt, const OdeArgs *fuse, int stage, int law) {
    return dispatch_storage(h->storage, PhaseRun{h, -1, s, d_stop, d_mskip, reset_counter, xt, fuse, stage, law});
}

// After the stream is synchronised: HBI_ERR_TIMEOUT if a bounded device wait gave up.
hbi_status hmvm_check(hbi_handle *h) {
    int err = 0;
    HBI_CUDA_TRY(cudaMemcpy(&err, h->d_counters + 1, sizeof(int), cudaMemcpyDeviceToHost));
    if (err) {
        HBI_CUDA_TRY(cudaMemset(h->d_counters + 1, 0, sizeof(int)));
        set_error("an HMVM stage wait timed out");
        return HBI_ERR_TIMEOUT;
    }
    return HBI_OK;
}

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
// HMVM for callers that cannot allocate: every per-call buffer (work counter and error
// flag, permuted input with the intermediate t = V^T x, permuted output) lives in one static
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
        off += align256(3 * sizeof(int));
        A *xt = reinterpret_cast<A *>(base + off);
        const size_t nxt = (size_t)h->nin * h->n + (size_t)h->n_t;
        off += align256((nxt + 16) * sizeof(A));
        A *yp = reinterpret_cast<A *>(base + off);
        const int grid = std::max(1, std::min((h->n + 255) / 256, 4 * std::max(1, h->num_sms)));
        HBI_CUDA_TRY(cudaMemsetAsync(xt + nxt, 0, 16 * sizeof(A), s));   // guard elements
        HBI_CUDA_TRY(cudaMemsetAsync(counters + 1, 0, 2 * sizeof(int), s));   // error flag, UY finish count
        permute_in_kernel<A><<<grid, 256, 0, s>>>(x, h->d_perm, h->n, h->nin, xt);
        hbi_status st = hmvm_run<TD, TL>(h, -1, xt, yp, counters, s, nullptr);   // clears the work counter
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
    const size_t need = align256(3 * sizeof(int)) + align256(((size_t)h->nin * h->n + (size_t)h->n_t + 16) * acc) +
                        align256((size_t)h->nout * h->n * acc);
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
    int err = 0;   // error flag after the counters at the start of the scratch array
    HBI_CUDA_TRY(cudaMemcpy(&err, reinterpret_cast<int *>(b) + 1, sizeof(int), cudaMemcpyDeviceToHost));
    if (err) {
        set_error("an HMVM stage wait timed out");
        return HBI_ERR_TIMEOUT;
    }
    return HBI_OK;
}

extern "C" hbi_status hbi_bounds_violations(long long *out) {
    using namespace hbi;
    if (!out) { set_error("out is required"); return HBI_ERR_INVALID_ARG; }
#ifdef HBI_BOUNDS_CHECK
    unsigned long long v = 0, zero = 0;
    HBI_CUDA_TRY(cudaDeviceSynchronize());
    HBI_CUDA_TRY(cudaMemcpyFromSymbol(&v, g_violations, sizeof v));
    HBI_CUDA_TRY(cudaMemcpyToSymbol(g_violations, &zero, sizeof zero));
    *out = (long long)v;
    return HBI_OK;
#else
    *out = -1;
    set_error("this library was built without bounds checks (build with HBI_BOUNDS_CHECK)");
    return HBI_ERR_INVALID_ARG;
#endif
}
