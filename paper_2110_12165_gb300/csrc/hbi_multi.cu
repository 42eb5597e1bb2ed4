// Multi-right-hand-side HMVM on the fifth-generation tensor cores: Y = H X for k slip-rate
// vectors at once (Eq. 20 applied to k inputs).
//
// With one right-hand side the product performs one FMA per stored entry and is bound by
// HBM; with k of them every stored entry feeds k FMAs, so from k of about 16 up the product
// needs more arithmetic than the CUDA cores give at full bandwidth, and it becomes a dense
// contraction that belongs on the tensor cores.  Both phases of Eq. 20 are batched GEMMs:
//   V^T phase: for each column group (low-rank blocks sharing a column cluster), the stacked
//              V^T rows (ranks x group columns) times the group's slice of X;
//   UY phase:  for each leaf row unit, its row panel [dense near-field | U of the low-rank
//              blocks] times the gathered [X | T] rows.
// A = the stored panel (FP16, per-column power-of-two scales as in the 2-byte storage; the
// FP32 near field of HBI_MIXED as an FP16 pair hi + 2^-11 lo), packed at build time in the
// canonical no-swizzle K-major tcgen05 layout (8 x 8 core matrices of 128 contiguous bytes),
// in chunks of MR_CW columns, so that one cp.async.bulk lands a chunk in shared memory ready
// for the MMA.  B = the inputs, FP32 in HBM, scaled per right-hand side to FP16 range and
// split into hi + 2^-11 lo FP16 parts (22 significant bits) in the canonical MN-major layout.
// The MMA (kind::f16, M = 128 panel rows, N = k padded to 16, K = 16) accumulates in FP32 in
// tensor memory: D1 = A_hi B_hi and D2 = A_hi B_lo + A_lo B_hi; y = (D1 + 2^-11 D2) / s.
//
// Persistent CTAs, warp-specialised: a producer warp streams the A pieces into a ring of MR_SA
// shared-memory stages (bulk copies on mbarriers), four warps convert one B chunk each into
// a ring of MR_SB stages, four warps run the epilogue (tcgen05.ld, one TMEM lane per panel
// row) from one of two accumulators while the next task's MMAs fill the other, and one warp
// allocates tensor memory and issues the MMAs, releasing each stage with tcgen05.commit.
// Every wait is bounded; a CTA that gives up raises the error flag, lets its copies and MMAs
// in flight finish and frees its tensor memory.
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <map>
#include <vector>

#include "hbi_internal.h"

namespace hbi {

#ifndef HBI_MR_CW
#define HBI_MR_CW 64
#endif

#ifndef HBI_MR_SB
#define HBI_MR_SB 4
#endif
constexpr int MR_CW = HBI_MR_CW;                   // K columns per chunk
// A ring stages (one panel piece of 16 KB each): three for 32 right-hand sides, so that two CTAs
// share an SM (measured 1.9x faster than one CTA with four), four otherwise
__host__ __device__ constexpr int mr_stages_a(int kp) { return kp == 32 ? 3 : 4; }
constexpr int MR_SB = HBI_MR_SB;                   // B ring stages
constexpr int MR_GW = 4;                           // converter warps (and epilogue warps: TMEM lanes 0..127)
constexpr int MR_SS = MR_SB;                       // staging stages (one per B stage)
// Converter warp w takes the chunks g = w (mod MR_GW); a stage must come back to the same warp
// (MR_SB, MR_SS multiples of MR_GW), so that no warp waits on a stage whose previous phase
// another warp has not yet consumed (a parity wait cannot tell two phases apart).
static_assert(MR_SB % MR_GW == 0 && MR_SS % MR_GW == 0, "B and staging stages: multiples of the converter warps");
static_assert(mr_stages_a(16) >= 2 && mr_stages_a(32) >= 2 && mr_stages_a(64) >= 2,
              "a dense chunk with a lo part holds two A stages");
constexpr int MR_THREADS = 32 * (2 * MR_GW + 3);   // converter, epilogue, A producer, MMA and B producer warps
constexpr int MR_ROWS = 128;                       // MMA M: panel rows of a task
constexpr int MR_A_STAGE = MR_ROWS * MR_CW * 2;    // bytes: one part (hi or lo) of a 128-row chunk
constexpr int MR_KP_MAX = 64;                      // right-hand sides per call (padded to 16)
constexpr int MR_KSLICE = 2048;                    // V^T: widest K of one task (wider groups are cut)
constexpr unsigned long long MR_WAIT_NS = 1000000000ull;   // 1 s

// One task: rows [0, rows) of one panel (a 128-row slice of a column group's V^T rows or of
// a leaf row unit).  Its K columns are kd dense columns (hi and, if lo, lo parts) followed by
// kl factor columns (U or V^T), each segment a multiple of 16 and cut into chunks of MR_CW.
struct MrTask {
    int64_t a_off;     // byte offset of the first chunk in the panel stream
    int64_t g_off;     // UY: offset of the unit's gather list; V^T: first X row of the group
    int64_t out_off;   // first output row (V^T: row of T inside xt; UY: row of yp)
    int64_t s_off;     // V^T: rowscale index of row 0; UY: -1
    int rows;          // 1..128
    int kd, kl;        // dense and factor columns (multiples of 16)
    int kreal;         // V^T: the group's columns (the padding gathers zeros)
    int lo;            // the dense chunks carry a lo part
    int partial;       // V^T: a K slice of a wide column group; its rows are partial sums
    int nd_real;       // dense columns before the padding of the dense segment (V^T: 0)
    int nl_real;       // factor columns before the padding of the factor segment (V^T: kreal)
};

// A V^T row tile of a wide column group, cut into nsl K slices: slice q wrote its partial rows
// (already scaled) at xt rows p_row + q MR_ROWS; their sum in slice order is t.
struct MrSplit {
    int64_t t_row, p_row;
    int rows, nsl;
};

// One run of the B gather: len consecutive xt rows from row src land in the chunk's staging
// buffer at columns [dst, dst + len) (one bulk copy of len x KP FP32 words).
struct MrRun {
    int64_t src;
    int len, dst;
};

}  // namespace hbi

// Everything the handle keeps for the multi-RHS product.
struct hbi::MultiRhs {
    unsigned char *d_panels = nullptr;
    int64_t panel_bytes = 0;
    MrTask *d_vt = nullptr, *d_uy = nullptr;
    int n_vt = 0, n_uy = 0;
    MrSplit *d_split = nullptr;   // V^T row tiles cut along K (reduced after the V^T phase)
    int n_split = 0;
    int64_t n_prow = 0;           // partial rows after T in xt
    // B gather runs of every chunk, per phase: host copies in task order (first run of each
    // task's chunk c at h_crun[p][c_first[task] + c]), and on the device in the order in which
    // the CTAs of a grid of `layout_grid` take the chunks (d_crun[p][d_cta[p][b] + g] is the
    // first run of chunk g of CTA b)
    std::vector<MrRun> h_runs[2];
    std::vector<int64_t> h_crun[2], h_cfirst[2];
    MrRun *d_runs[2] = {nullptr, nullptr};
    int64_t *d_crun[2] = {nullptr, nullptr}, *d_cta[2] = {nullptr, nullptr};
    int layout_grid = 0;
    float *d_cscale = nullptr;    // per X row: the scale of its dense columns (largest over the blocks)
    int *d_iperm = nullptr;       // original element -> permuted position
    float *d_rowscale = nullptr;  // V^T output row scales (sv su)
    int64_t n_t = 0;              // rows of T
    int64_t nx = 0;               // rows of X (n_in N)
    int lo = 0;
    int grid = 0;
    // per-call buffers, sized for kp_cap right-hand sides
    int kp_cap = 0;
    float *d_xt = nullptr, *d_yp = nullptr;
    unsigned *d_vmax = nullptr;   // per right-hand side: [0, 64) max |x|, [64, 128) max |t|,
                                  // [128, 192) max |x| x its row's dense column scale
    int *d_err = nullptr;
    int64_t bytes_panels_alg = 0;     // stored entries (hi + lo for the FP32 near field) + scales
    int64_t vec_bytes_per_rhs = 0;    // x read, t written and read, y written (FP32)
    double flops_per_rhs = 0;         // 2 x (dense + U + V entries)
    double mma_flops_per_rhs = 0;     // as issued (padding, hi / lo passes)
};

namespace hbi {
namespace {

// ------------------------------------------------------------------ PTX helpers
__device__ __forceinline__ unsigned mr_smem(const void *p) { return (unsigned)__cvta_generic_to_shared(p); }
__device__ __forceinline__ unsigned long long mr_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
__device__ __forceinline__ void mr_bar_init(uint64_t *b, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(mr_smem(b)), "r"(count) : "memory");
}
__device__ __forceinline__ void mr_arrive(uint64_t *b) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(mr_smem(b)) : "memory");
}
__device__ __forceinline__ void mr_expect_tx(uint64_t *b, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(mr_smem(b)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mr_try(uint64_t *b, unsigned parity) {
    unsigned ok;
    asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
                 : "=r"(ok)
                 : "r"(mr_smem(b)), "r"(parity)
                 : "memory");
    return ok != 0;
}
// One thread waits for the phase of the given parity; false once *fail is set or after MR_WAIT_NS.
__device__ __forceinline__ bool mr_wait(uint64_t *b, unsigned parity, volatile int *fail) {
    if (mr_try(b, parity)) return true;   // already complete: no timer read
    const unsigned long long t0 = mr_ns();
    for (unsigned it = 0;; ++it) {
        if (mr_try(b, parity)) return true;
        if ((it & 63u) == 63u && (*fail || mr_ns() - t0 > MR_WAIT_NS)) {
            *fail = 1;
            return false;
        }
    }
}
// The same for a whole warp, with a warp-uniform outcome.
__device__ __forceinline__ bool mr_warp_wait(uint64_t *b, unsigned parity, volatile int *fail) {
    if (__all_sync(0xffffffffu, mr_try(b, parity))) return true;   // already complete: no timer read
    const unsigned long long t0 = mr_ns();
    for (unsigned it = 0;; ++it) {
        if (__all_sync(0xffffffffu, mr_try(b, parity))) return true;
        if ((it & 63u) == 63u && __any_sync(0xffffffffu, *fail != 0 || mr_ns() - t0 > MR_WAIT_NS)) {
            *fail = 1;
            return false;
        }
    }
}
__device__ __forceinline__ void mr_bulk(void *dst, const void *src, unsigned bytes, uint64_t *b) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     mr_smem(dst)),
                 "l"(src), "r"(bytes), "r"(mr_smem(b))
                 : "memory");
}
// Shared-memory matrix descriptor, no swizzle: start address, LBO = byte stride between core
// matrices along K, SBO = byte stride between 8-row (M or N) groups; version 1 (bits 46-47).
__device__ __forceinline__ uint64_t mr_desc(unsigned saddr, unsigned lbo, unsigned sbo) {
    return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | ((uint64_t)1 << 46);
}
__device__ __forceinline__ void mr_mma(unsigned d_tmem, uint64_t a, uint64_t b, unsigned idesc, unsigned acc) {
    asm volatile("{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                 " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
                 "l"(a), "l"(b), "r"(idesc), "r"(acc)
                 : "memory");
}
__device__ __forceinline__ void mr_commit(uint64_t *b) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mr_smem(b))
                 : "memory");
}
__device__ __forceinline__ void mr_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void mr_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void mr_ld16(unsigned taddr, float *v) {
    unsigned r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
          "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
#pragma unroll
    for (int q = 0; q < 16; ++q) v[q] = __uint_as_float(r[q]);
}
__device__ __forceinline__ void mr_ld_wait() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// Chunk c of a task: dense or factor, its first column in the task's K, width, bytes of one
// part, parts (a dense chunk with a lo part holds its hi part, then its lo part) and offset.
struct MrChunk {
    int dense, col0, w, parts;
    unsigned bytes;   // of one part
    int64_t off;
};
__device__ __forceinline__ int mr_nchunks(const MrTask &t) { return (t.kd + MR_CW - 1) / MR_CW + (t.kl + MR_CW - 1) / MR_CW; }
__device__ __forceinline__ MrChunk mr_chunk(const MrTask &t, int c) {
    const int rg = (t.rows + 7) / 8, parts = 1 + t.lo;
    const int nchd = (t.kd + MR_CW - 1) / MR_CW;
    MrChunk k;
    if (c < nchd) {
        k.dense = 1;
        k.col0 = c * MR_CW;
        k.w = min(MR_CW, t.kd - k.col0);
        k.off = t.a_off + (int64_t)c * rg * MR_CW * 16 * parts;
        k.parts = parts;
    } else {
        const int cu = c - nchd;
        k.dense = 0;
        k.col0 = t.kd + cu * MR_CW;
        k.w = min(MR_CW, t.kl - cu * MR_CW);
        k.off = t.a_off + (int64_t)rg * t.kd * 16 * parts + (int64_t)cu * rg * MR_CW * 16;
        k.parts = 1;
    }
    k.bytes = (unsigned)(rg * k.w * 16);
    return k;
}

// Power of two s with max |v| s in (2^13, 2^14] (1 for 0): keeps the scaled B operand, whose
// largest entry is m s, inside FP16 range with the most significant bits.
__device__ __forceinline__ float mr_scale_for(float m) {
    if (!(m > 0.0f) || !isfinite(m)) return 1.0f;
    int e;
    const float f = frexpf(m, &e);   // m = f 2^e, f in [0.5, 1)
    const int c = f == 0.5f ? e - 1 : e;   // ceil(log2 m)
    return ldexpf(1.0f, 14 - c);
}

// ------------------------------------------------------------------ the product kernel
// vt = 1: V^T phase (B = X rows g_off + col, outputs T rows scaled by rowscale, max |t| per
// right-hand side into vmax[64 + r]); vt = 0: UY phase (B = gathered xt rows, outputs yp).
// Warp 10 copies each chunk's B rows (FP32, runs of consecutive xt rows, one bulk copy per run)
// into staging stage g (mod MR_SS) of the CTA's chunk sequence; converter warp g (mod 4) scales
// and splits them into FP16 hi / lo B stage g (mod MR_SB); warps 4-7 run the epilogue from one
// of two tensor-memory accumulators while the MMAs of the next task fill the other; warp 8
// streams the A pieces; warp 9 allocates tensor memory and issues the MMAs.
template <int KP>
__global__ void __launch_bounds__(MR_THREADS, 1)
    mr_kernel(const MrTask *__restrict__ tasks, int ntasks, int vt, const unsigned char *__restrict__ panels,
              const MrRun *__restrict__ runs, int64_t n_runs, const int64_t *__restrict__ crun,
              const int64_t *__restrict__ cta, const float *__restrict__ rowscale, float *xt, float *out, unsigned *vmax,
              int *err) {
    constexpr int MR_SA = mr_stages_a(KP);     // A ring stages
    constexpr int BSTAGE = MR_CW * KP * 2;    // bytes of one FP16 B part (hi or lo)
    constexpr int SSTAGE = MR_CW * KP * 4;    // bytes of one FP32 staging stage
    constexpr unsigned TCOLS = 4 * KP <= 64 ? 64 : (4 * KP <= 128 ? 128 : 256);   // 2 accumulators x (D1 | D2)
    extern __shared__ __align__(1024) unsigned char mr_sm[];
    unsigned char *sA = mr_sm;                                        // MR_SA x MR_A_STAGE
    unsigned char *sB = sA + MR_SA * MR_A_STAGE;                      // MR_SB x (hi | lo)
    unsigned char *sS = sB + MR_SB * 2 * BSTAGE;                      // MR_SS x staging
    __shared__ uint64_t a_full[MR_SA], a_empty[MR_SA], b_full[MR_SB], b_empty[MR_SB], s_full[MR_SS], s_empty[MR_SS];
    __shared__ uint64_t acc_full[2], acc_empty[2], fin;
    __shared__ unsigned s_taddr;
    __shared__ __align__(16) float s_scale[KP];
    __shared__ float s_inv[KP];
    __shared__ unsigned s_tmax[KP];
    __shared__ volatile int s_fail;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    constexpr int W_EPI = MR_GW, W_PROD = 2 * MR_GW, W_MMA = 2 * MR_GW + 1, W_BPROD = 2 * MR_GW + 2;

    if (threadIdx.x == 0) {
        s_fail = 0;
        for (int s = 0; s < MR_SA; ++s) { mr_bar_init(&a_full[s], 1); mr_bar_init(&a_empty[s], 1); }
        for (int s = 0; s < MR_SB; ++s) { mr_bar_init(&b_full[s], 32); mr_bar_init(&b_empty[s], 1); }
        for (int s = 0; s < MR_SS; ++s) { mr_bar_init(&s_full[s], 1); mr_bar_init(&s_empty[s], 32); }
        for (int s = 0; s < 2; ++s) { mr_bar_init(&acc_full[s], 1); mr_bar_init(&acc_empty[s], 32 * MR_GW); }
        mr_bar_init(&fin, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (threadIdx.x < KP) {
        const int r = threadIdx.x;
        const float xm = __uint_as_float(vmax[r]);
        const float m = vt ? xm : fmaxf(__uint_as_float(vmax[128 + r]), __uint_as_float(vmax[64 + r]));
        const float s = mr_scale_for(m);
        s_scale[r] = s;
        s_inv[r] = 1.0f / s;
        s_tmax[r] = 0u;
    }
    if (warp == W_MMA) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(mr_smem(&s_taddr)),
                     "r"(TCOLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    mr_fence_before();
    __syncthreads();
    mr_fence_after();
    const unsigned taddr = s_taddr;
    volatile int *fail = &s_fail;

    if (warp == W_PROD) {
        // ---------------------------------------------------------------- A producer (one lane)
        if (lane == 0) {
            unsigned g = 0;
            bool ok = true;
            MrTask tn;
            if (blockIdx.x < ntasks) tn = tasks[blockIdx.x];
            for (int ti = blockIdx.x; ti < ntasks && ok && !*fail; ti += gridDim.x) {
                const MrTask t = tn;
                if (ti + (int)gridDim.x < ntasks) tn = tasks[ti + gridDim.x];   // the next task, in flight
                const int nch = mr_nchunks(t);
                for (int c = 0; c < nch && ok; ++c) {
                    const MrChunk k = mr_chunk(t, c);
                    for (int p = 0; p < k.parts; ++p) {
                        const int s = g % MR_SA;
                        if (g >= (unsigned)MR_SA && !mr_wait(&a_empty[s], ((g / MR_SA) - 1) & 1, fail)) { ok = false; break; }
                        mr_expect_tx(&a_full[s], k.bytes);
                        mr_bulk(sA + (size_t)s * MR_A_STAGE, panels + k.off + (int64_t)p * k.bytes, k.bytes, &a_full[s]);
                        ++g;
                    }
                }
            }
            if (*fail) {   // let the copies in flight land before the CTA exits
                for (int s = 0; s < MR_SA; ++s) {
                    const unsigned uses = g / MR_SA + (s < (int)(g % MR_SA) ? 1u : 0u);
                    if (uses == 0) continue;
                    const unsigned long long t0 = mr_ns();
                    while (!mr_try(&a_full[s], (uses - 1) & 1) && mr_ns() - t0 < MR_WAIT_NS) {
                    }
                }
            }
        }
    } else if (warp == W_BPROD) {
        // ---------------------------------------------------------------- B producer (whole warp)
        // This CTA's chunks g = 0 .. nchk - 1 take the runs [crun[c0 + g], crun[c0 + g + 1]).  The
        // lanes hold 32 chunk boundaries and three windows of 32 runs (a 64-column chunk has at
        // most 64 runs, so it lies inside the three), with the next boundaries and the third
        // window loaded ahead of use; each lane issues the bulk copies of the runs it holds.
        const int64_t c0 = cta[blockIdx.x];
        const int nchk = (int)(cta[blockIdx.x + 1] - c0 - 1);
        auto bload = [&](int j) -> int64_t { return j <= nchk ? crun[c0 + j] : 0; };
        auto rload = [&](int64_t i) -> MrRun { MrRun r{0, 0, 0}; if (i >= 0 && i < n_runs) r = runs[i]; return r; };
        int64_t bnd = bload(lane), bnd_next = bload(31 + lane);
        int cb = 0;
        int64_t rb = __shfl_sync(0xffffffffu, bnd, 0);
        MrRun w0 = rload(rb + lane), w1 = rload(rb + 32 + lane), w2 = rload(rb + 64 + lane);
        bool ok = true;
        int issued = 0;
        for (int g = 0; g < nchk && ok; ++g) {
            if (g - cb >= 31) {
                cb += 31;
                bnd = bnd_next;
                bnd_next = bload(cb + 31 + lane);
            }
            const int64_t r0 = __shfl_sync(0xffffffffu, bnd, g - cb), r1 = __shfl_sync(0xffffffffu, bnd, g - cb + 1);
            while (r0 >= rb + 32) {
                rb += 32;
                w0 = w1;
                w1 = w2;
                w2 = rload(rb + 64 + lane);
            }
            const int64_t i0 = rb + lane, i1 = i0 + 32, i2 = i0 + 64;
            const bool h0 = i0 >= r0 && i0 < r1, h1 = i1 >= r0 && i1 < r1, h2 = i2 >= r0 && i2 < r1;
            unsigned bytes = ((h0 ? w0.len : 0) + (h1 ? w1.len : 0) + (h2 ? w2.len : 0)) * (unsigned)KP * 4u;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) bytes += __shfl_xor_sync(0xffffffffu, bytes, o);
            const int s = g % MR_SS;
            if (g >= MR_SS && !mr_warp_wait(&s_empty[s], ((g / MR_SS) - 1) & 1, fail)) { ok = false; break; }
            if (lane == 0) mr_expect_tx(&s_full[s], bytes);   // 0 bytes: the phase completes on the arrival
            __syncwarp();
            unsigned char *stg = sS + (size_t)s * SSTAGE;
            if (h0) mr_bulk(stg + (size_t)w0.dst * KP * 4, xt + w0.src * KP, (unsigned)w0.len * KP * 4u, &s_full[s]);
            if (h1) mr_bulk(stg + (size_t)w1.dst * KP * 4, xt + w1.src * KP, (unsigned)w1.len * KP * 4u, &s_full[s]);
            if (h2) mr_bulk(stg + (size_t)w2.dst * KP * 4, xt + w2.src * KP, (unsigned)w2.len * KP * 4u, &s_full[s]);
            ++issued;
        }
        if (*fail && lane == 0) {   // let the copies in flight land before the CTA exits
            const unsigned g = (unsigned)issued;
            for (int s = 0; s < MR_SS; ++s) {
                const unsigned uses = g / MR_SS + (s < (int)(g % MR_SS) ? 1u : 0u);
                if (uses == 0) continue;
                const unsigned long long t0 = mr_ns();
                while (!mr_try(&s_full[s], (uses - 1) & 1) && mr_ns() - t0 < MR_WAIT_NS) {
                }
            }
        }
    } else if (warp == W_MMA) {
        // ---------------------------------------------------------------- MMA issuer
        if (lane == 0) {
            // D F32 (bits 4-5 = 1), A and B F16, A K-major, B MN-major (bit 16), M = 128; N = 2 KP
            // for A_hi [B_hi | B_lo] into the adjacent accumulators D1 | D2, N = KP for A_lo B_hi
            const unsigned idesc2 = (1u << 4) | (1u << 16) | ((unsigned)((2 * KP) >> 3) << 17) |
                                    ((unsigned)(MR_ROWS >> 4) << 24);
            const unsigned idesc1 = (1u << 4) | (1u << 16) | ((unsigned)(KP >> 3) << 17) | ((unsigned)(MR_ROWS >> 4) << 24);
            unsigned ga = 0, gb = 0, nt = 0;
            bool ok = true;
            MrTask tn;
            if (blockIdx.x < ntasks) tn = tasks[blockIdx.x];
            for (int ti = blockIdx.x; ti < ntasks && ok && !*fail; ti += gridDim.x) {
                const MrTask t = tn;
                if (ti + (int)gridDim.x < ntasks) tn = tasks[ti + gridDim.x];
                const unsigned ab = nt & 1;
                if (nt >= 2 && !mr_wait(&acc_empty[ab], ((nt >> 1) - 1) & 1, fail)) break;
                mr_fence_after();
                const unsigned d1 = taddr + ab * 2 * KP, d2 = d1 + KP;
                const int nch = mr_nchunks(t);
                unsigned acc1 = 0;
                for (int c = 0; c < nch; ++c) {
                    const MrChunk k = mr_chunk(t, c);
                    const int sa = ga % MR_SA, sa2 = (ga + 1) % MR_SA, sb = gb % MR_SB;
                    if (!mr_wait(&a_full[sa], (ga / MR_SA) & 1, fail) ||
                        (k.parts == 2 && !mr_wait(&a_full[sa2], ((ga + 1) / MR_SA) & 1, fail)) ||
                        !mr_wait(&b_full[sb], (gb / MR_SB) & 1, fail)) {
                        ok = false;
                        break;
                    }
                    mr_fence_after();
                    const unsigned a0 = mr_smem(sA + (size_t)sa * MR_A_STAGE);
                    const unsigned a1 = mr_smem(sA + (size_t)sa2 * MR_A_STAGE);
                    const unsigned bst = mr_smem(sB + (size_t)sb * 2 * BSTAGE);
                    const unsigned sbo_a = (unsigned)k.w * 16u;
                    // descriptors of the chunk's first K step: the B operand's K groups are 2 KP x 16
                    // bytes apart, its N groups 128; a K step of 16 columns moves A by two core
                    // matrices (256 bytes) and B by two K groups (64 KP bytes), i.e. the start-address
                    // field (address / 16, low bits) by 16 and 4 KP.  The N = KP descriptor reads the
                    // hi half (the first RQ N groups) of the same operand.
                    uint64_t ah = mr_desc(a0, 128u, sbo_a), al = mr_desc(a1, 128u, sbo_a);
                    uint64_t bd = mr_desc(bst, (unsigned)KP * 32u, 128u);
                    const int nk = k.w / 16;
                    for (int kk = 0; kk < nk; ++kk) {
                        mr_mma(d1, ah, bd, idesc2, acc1);
                        acc1 = 1;
                        if (k.parts == 2) mr_mma(d2, al, bd, idesc1, 1u);
                        ah += 16u;
                        al += 16u;
                        bd += 4u * KP;
                    }
                    mr_commit(&a_empty[sa]);
                    if (k.parts == 2) mr_commit(&a_empty[sa2]);
                    mr_commit(&b_empty[sb]);
                    ga += k.parts;
                    ++gb;
                }
                if (!ok) break;
                mr_commit(&acc_full[ab]);
                ++nt;
            }
            // every MMA issued so far has completed once this phase does
            mr_commit(&fin);
            const unsigned long long t0 = mr_ns();
            while (!mr_try(&fin, 0) && mr_ns() - t0 < MR_WAIT_NS) {
            }
        }
    } else if (warp < MR_GW) {
        // ---------------------------------------------------------------- converters (warp w: chunks w mod 4)
        unsigned gc = 0;   // chunk index in this CTA's sequence
        bool ok = true;
        MrTask tn;
        if (blockIdx.x < ntasks) tn = tasks[blockIdx.x];
        for (int ti = blockIdx.x; ti < ntasks && ok; ti += gridDim.x) {
            const MrTask t = tn;
            if (ti + (int)gridDim.x < ntasks) tn = tasks[ti + gridDim.x];
            const int nch = mr_nchunks(t);
            for (int c = 0; c < nch; ++c, ++gc) {
                if ((int)(gc % MR_GW) != warp) continue;
                const MrChunk k = mr_chunk(t, c);
                const int sb = gc % MR_SB, ss = gc % MR_SS;
                if (gc >= MR_SB && !mr_warp_wait(&b_empty[sb], ((gc / MR_SB) - 1) & 1, fail)) { ok = false; break; }
                if (!mr_warp_wait(&s_full[ss], (gc / MR_SS) & 1, fail)) { ok = false; break; }
                __syncwarp();
                const float *stg = reinterpret_cast<const float *>(sS + (size_t)ss * SSTAGE);
                unsigned char *bst = sB + (size_t)sb * 2 * BSTAGE;
                // Vector (kc, rq): K row kc = 8 kg + kr, right-hand sides 8 rq .. 8 rq + 7, one
                // 16-byte row of core matrix (kg, rq).  A 16-byte shared-memory access is served
                // eight lanes at a time; those eight lanes take the eight K rows kr = p of one kg
                // (their stores hit eight different 16-byte bank groups of a core-matrix row
                // set) with right-hand-side blocks rq = base + off(p) and the two float4 halves
                // of their staging row read in the order h(p), 1 - h(p): the staging word
                // kc KP + 8 rq + 4 h lies in bank group (kc KP / 4 + 2 rq + h) mod 8, and off,
                // h are chosen so that these eight groups differ as well.
                constexpr int RQ = KP / 8;
                constexpr bool KP_MOD32 = (KP / 4) % 8 == 0;   // KP = 32, 64: kc KP / 4 = 0 mod 8
                const int p = lane & 7;
                const int h = KP_MOD32 ? (p & 1) : ((p >> 1) & 1);
                const int roff = KP_MOD32 ? (p >> 1) : (p >> 2);
                const int npairs = (k.w / 8) * RQ;
                for (int u = lane >> 3; u < npairs; u += 4) {
                    const int kg = u / RQ, base = u - kg * RQ;
                    const int rq = base + roff < RQ ? base + roff : base + roff - RQ;
                    const int kr = p;
                    const int kc = 8 * kg + kr, col = k.col0 + kc;
                    // padding at the end of the dense and of the factor segment: zeros (not copied)
                    const bool pad = col < t.kd ? col >= t.nd_real : col - t.kd >= t.nl_real;
                    __align__(16) __half hi[8], lo[8];
                    if (!pad) {
                        const float *src = stg + kc * KP + 8 * rq, *scl = s_scale + 8 * rq;
                        const float4 xa = *reinterpret_cast<const float4 *>(src + 4 * h);
                        const float4 xb = *reinterpret_cast<const float4 *>(src + 4 - 4 * h);
                        const float4 sa = *reinterpret_cast<const float4 *>(scl + 4 * h);
                        const float4 sb = *reinterpret_cast<const float4 *>(scl + 4 - 4 * h);
                        const float4 x0 = h ? xb : xa, x1 = h ? xa : xb;
                        const float4 s0 = h ? sb : sa, s1 = h ? sa : sb;
                        const float xs[8] = {x0.x, x0.y, x0.z, x0.w, x1.x, x1.y, x1.z, x1.w};
                        const float ss[8] = {s0.x, s0.y, s0.z, s0.w, s1.x, s1.y, s1.z, s1.w};
#pragma unroll
                        for (int q = 0; q < 8; ++q) {
                            const float b = xs[q] * ss[q];
                            hi[q] = __float2half_rn(b);
                            lo[q] = __float2half_rn((b - __half2float(hi[q])) * 2048.0f);
                        }
                    } else {
#pragma unroll
                        for (int q = 0; q < 8; ++q) hi[q] = lo[q] = __float2half_rn(0.0f);
                    }
                    // one B operand of N = 2 KP: K group kg holds the hi core matrices (N groups
                    // 0 .. RQ - 1) and then the lo ones (RQ .. 2 RQ - 1), 128 bytes each
                    const int off = (kg * 2 * RQ + rq) * 128 + kr * 16;
                    *reinterpret_cast<uint4 *>(bst + off) = *reinterpret_cast<const uint4 *>(hi);
                    *reinterpret_cast<uint4 *>(bst + off + RQ * 128) = *reinterpret_cast<const uint4 *>(lo);
                }
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                mr_arrive(&s_empty[ss]);
                mr_arrive(&b_full[sb]);
                __syncwarp();
            }
        }
    } else {
        // ---------------------------------------------------------------- epilogue (warps 4-7)
        const int row = threadIdx.x - 32 * W_EPI;          // 0..127 = TMEM lane = panel row
        const unsigned lane_base = (unsigned)(32 * (warp & 3)) << 16;
        unsigned nt = 0;
        MrTask tn;
        if (blockIdx.x < ntasks) tn = tasks[blockIdx.x];
        for (int ti = blockIdx.x; ti < ntasks; ti += gridDim.x, ++nt) {
            const MrTask t = tn;
            if (ti + (int)gridDim.x < ntasks) tn = tasks[ti + gridDim.x];
            const unsigned ab = nt & 1;
            const float rs0 = (vt && row < t.rows && rowscale) ? rowscale[t.s_off + row] : 1.0f;
            if (!mr_warp_wait(&acc_full[ab], (nt >> 1) & 1, fail)) break;
            mr_fence_after();
            const bool live = row < t.rows;
            const float rs = rs0;
            float *orow = out + (t.out_off + row) * KP;
            const unsigned base = taddr + lane_base + ab * 2 * KP;
#pragma unroll 1
            for (int c0 = 0; c0 < KP; c0 += 16) {
                float a[16], b[16];
                mr_ld16(base + c0, a);
                mr_ld16(base + KP + c0, b);
                mr_ld_wait();
                float y[16];
#pragma unroll
                for (int q = 0; q < 16; ++q) y[q] = (a[q] + b[q] * (1.0f / 2048.0f)) * s_inv[c0 + q] * rs;
                if (live) {
#pragma unroll
                    for (int q = 0; q < 16; q += 4)
                        *reinterpret_cast<float4 *>(orow + c0 + q) = make_float4(y[q], y[q + 1], y[q + 2], y[q + 3]);
                }
                if (vt && !t.partial) {
                    // max |t| per right-hand side over the warp's rows: non-negative floats order
                    // as their bit patterns, so one integer warp reduction per column
#pragma unroll
                    for (int q = 0; q < 16; ++q) {
                        float m = live ? fabsf(y[q]) : 0.0f;
                        if (!(m == m)) m = 0.0f;
                        const unsigned mb = __reduce_max_sync(0xffffffffu, __float_as_uint(m));
                        if (lane == 0 && mb) atomicMax(&s_tmax[c0 + q], mb);
                    }
                }
            }
            mr_fence_before();
            mr_arrive(&acc_empty[ab]);
        }
    }
    if (threadIdx.x == 0 && s_fail) atomicExch(err, 1);
    mr_fence_before();
    __syncthreads();
    mr_fence_after();
    if (vt && threadIdx.x < KP && s_tmax[threadIdx.x]) atomicMax(vmax + 64 + threadIdx.x, s_tmax[threadIdx.x]);
    if (warp == W_MMA)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(TCOLS) : "memory");
}

constexpr int MR_TILE = 32;   // rows of the shared-memory transpose tiles of the input and output kernels

// The k inputs (caller's order, component-major, FP64) into [X | X with the dense column
// scales] in the permuted row order, KP FP32 words per row (right-hand sides k .. KP - 1 zero),
// and the largest magnitudes per right-hand side into vmax[r] (X) and vmax[128 + r] (scaled X).
// A tile of 32 consecutive elements of the caller's order, all their components, goes through
// shared memory: read with consecutive threads on consecutive elements of one component and
// right-hand side (coalesced), written as whole rows of KP words at the elements' permuted
// positions (iperm).  The block size is a multiple of KP, so a thread writes one right-hand side
// throughout and keeps its maxima in registers (one shared and one global atomic per
// right-hand side and block).
__global__ void mr_in_kernel(const double *__restrict__ X, const int *__restrict__ iperm, int n, int nin, int k, int KP,
                             const float *__restrict__ cscale, float *__restrict__ xt, unsigned *__restrict__ vmax) {
    __shared__ float tile[MR_TILE * 2][MR_KP_MAX + 1];
    __shared__ unsigned s_m[2][MR_KP_MAX];
    const int tid = threadIdx.x, nt = blockDim.x;
    const int64_t nx = (int64_t)nin * n;
    const int trows = MR_TILE * nin;
    for (int q = tid; q < 2 * MR_KP_MAX; q += nt) s_m[q / MR_KP_MAX][q % MR_KP_MAX] = 0u;
    __syncthreads();
    float m = 0.0f, mc = 0.0f;
    const int64_t ntile = ((int64_t)n + MR_TILE - 1) / MR_TILE;
    for (int64_t t = blockIdx.x; t < ntile; t += gridDim.x) {
        const int64_t j0 = t * MR_TILE;
        __syncthreads();   // the previous tile is written out
        for (int q = tid; q < trows * KP; q += nt) {
            const int jl = q % MR_TILE, cr = q / MR_TILE, c = cr % nin, r = cr / nin;
            const int64_t j = j0 + jl;
            tile[jl * nin + c][r] = (r < k && j < n) ? (float)X[(int64_t)r * nx + (int64_t)c * n + j] : 0.0f;
        }
        __syncthreads();
        for (int q = tid; q < trows * KP; q += nt) {
            const int tr = q / KP, r = q - tr * KP, jl = tr / nin, c = tr - jl * nin;
            const int64_t j = j0 + jl;
            if (j >= n) break;
            const int64_t row = (int64_t)iperm[j] * nin + c;
            const float v = tile[tr][r], vc = v * cscale[row];
            xt[row * KP + r] = v;             // X, the V^T phase's input
            xt[nx * KP + row * KP + r] = vc;  // X with the row's dense column scale, the near field's input
            const float a = fabsf(v), ac = fabsf(vc);
            if (isfinite(a)) m = fmaxf(m, a);
            if (isfinite(ac)) mc = fmaxf(mc, ac);
        }
    }
    if (m > 0.0f) atomicMax(&s_m[0][tid % KP], __float_as_uint(m));
    if (mc > 0.0f) atomicMax(&s_m[1][tid % KP], __float_as_uint(mc));
    __syncthreads();
    for (int r = tid; r < KP; r += nt) {
        if (s_m[0][r]) atomicMax(vmax + r, s_m[0][r]);
        if (s_m[1][r]) atomicMax(vmax + 128 + r, s_m[1][r]);
    }
}

// t of the V^T row tiles cut along K: the sum of their slices' partial rows, in slice order
// (deterministic), and its largest magnitude per right-hand side into vmax[64 + r].
__global__ void mr_reduce_kernel(const MrSplit *__restrict__ sp, int KP, float *xt, unsigned *vmax) {
    __shared__ unsigned s_m[MR_KP_MAX];
    const MrSplit S = sp[blockIdx.x];
    if (threadIdx.x < KP) s_m[threadIdx.x] = 0u;
    __syncthreads();
    for (int e = threadIdx.x; e < S.rows * KP; e += blockDim.x) {
        const int r = e / KP, j = e - r * KP;
        float v = 0.0f;
        for (int q = 0; q < S.nsl; ++q) v += xt[(S.p_row + (int64_t)q * MR_ROWS + r) * KP + j];
        xt[(S.t_row + r) * KP + j] = v;
        const float a = fabsf(v);
        if (a > 0.0f && isfinite(a)) atomicMax(&s_m[j], __float_as_uint(a));
    }
    __syncthreads();
    if (threadIdx.x < KP && s_m[threadIdx.x]) atomicMax(vmax + 64 + threadIdx.x, s_m[threadIdx.x]);
}

// The permuted outputs (KP FP32 words per row) into the caller's order, component-major, FP64:
// a tile of 32 consecutive elements of the caller's order, all their components, read as whole
// rows at the elements' permuted positions and written with consecutive threads on consecutive
// elements of one component and right-hand side (coalesced).
__global__ void mr_out_kernel(const float *__restrict__ yp, const int *__restrict__ iperm, int n, int nout, int k, int KP,
                              double *__restrict__ Y) {
    __shared__ float tile[MR_TILE * 3][MR_KP_MAX + 1];
    const int tid = threadIdx.x, nt = blockDim.x;
    const int64_t ny = (int64_t)nout * n;
    const int trows = MR_TILE * nout;
    const int64_t ntile = ((int64_t)n + MR_TILE - 1) / MR_TILE;
    for (int64_t t = blockIdx.x; t < ntile; t += gridDim.x) {
        const int64_t j0 = t * MR_TILE;
        __syncthreads();   // the previous tile is written out
        for (int q = tid; q < trows * KP; q += nt) {
            const int tr = q / KP, r = q - tr * KP, jl = tr / nout, c = tr - jl * nout;
            const int64_t j = j0 + jl;
            tile[tr][r] = j < n ? yp[((int64_t)iperm[j] * nout + c) * KP + r] : 0.0f;
        }
        __syncthreads();
        for (int q = tid; q < trows * k; q += nt) {
            const int jl = q % MR_TILE, cr = q / MR_TILE, c = cr % nout, r = cr / nout;
            const int64_t j = j0 + jl;
            if (j < n) Y[(int64_t)r * ny + (int64_t)c * n + j] = (double)tile[jl * nout + c][r];
        }
    }
}

// ------------------------------------------------------------------ packing
// Panel sources.  V^T task row: V(:, k) of one low-rank block (contiguous over the group's
// columns) times inv_scale.  UY term: like the main path's UyTerm.
struct MrRowSrc {
    const double *v;
    float inv_scale;
};
struct MrTerm {
    const double *src;   // U (column-major, ld = m) or dense (row-major, ld = nc)
    int64_t ld, roff;    // leading dimension, block row of the task's row 0
    int width, coloff;   // columns, first column inside its segment
    int dense;
    const float *inv_scales; // per-column 1 / scale (device), or null
};
struct MrPackTask {
    MrTask t;
    int src0, nsrc;      // V^T: rows [src0, src0 + rows); UY: terms [src0, src0 + nsrc)
};

__device__ __forceinline__ int64_t mr_elem_off(const MrTask &t, int i, int kc, int part) {
    // byte offset of panel entry (row i, task column kc) of part 0 (hi / factor) or 1 (lo)
    const int rg = (t.rows + 7) / 8, parts = 1 + t.lo;
    int64_t base;
    int w, k;
    if (kc < t.kd) {
        const int c = kc / MR_CW;
        k = kc - c * MR_CW;
        w = min(MR_CW, t.kd - c * MR_CW);
        base = t.a_off + (int64_t)c * rg * MR_CW * 16 * parts + (int64_t)part * rg * w * 16;
    } else {
        const int cu = (kc - t.kd) / MR_CW;
        k = kc - t.kd - cu * MR_CW;
        w = min(MR_CW, t.kl - cu * MR_CW);
        base = t.a_off + (int64_t)rg * t.kd * 16 * parts + (int64_t)cu * rg * MR_CW * 16;
    }
    return base + ((int64_t)(i >> 3) * (w >> 3) + (k >> 3)) * 128 + (i & 7) * 16 + (k & 7) * 2;
}

__device__ __forceinline__ void mr_put(unsigned char *panels, const MrTask &t, int i, int kc, double v, bool split) {
    const __half hi = __double2half(v);
    *reinterpret_cast<__half *>(panels + mr_elem_off(t, i, kc, 0)) = hi;
    if (split) {
        const __half lo = __double2half((v - (double)__half2float(hi)) * 2048.0);
        *reinterpret_cast<__half *>(panels + mr_elem_off(t, i, kc, 1)) = lo;
    }
}

// one CTA per task; the panel bytes were zeroed (row and column padding stays zero)
__global__ void mr_pack_kernel(const MrPackTask *__restrict__ pt, int vt, const MrRowSrc *__restrict__ rows,
                               const MrTerm *__restrict__ terms, unsigned char *__restrict__ panels) {
    const MrPackTask P = pt[blockIdx.x];
    const MrTask &t = P.t;
    if (vt) {
        const int64_t tot = (int64_t)t.rows * t.kreal;
        for (int64_t e = threadIdx.x; e < tot; e += blockDim.x) {
            const int i = (int)(e / t.kreal), kc = (int)(e % t.kreal);
            const MrRowSrc R = rows[P.src0 + i];
            mr_put(panels, t, i, t.kd + kc, R.v[kc] * (double)R.inv_scale, false);
        }
    } else {
        for (int q = P.src0; q < P.src0 + P.nsrc; ++q) {
            const MrTerm T = terms[q];
            const int64_t tot = (int64_t)t.rows * T.width;
            for (int64_t e = threadIdx.x; e < tot; e += blockDim.x) {
                const int i = (int)(e / T.width), c = (int)(e % T.width);
                double v = T.dense ? T.src[(T.roff + i) * T.ld + c] : T.src[(int64_t)c * T.ld + T.roff + i];
                if (T.inv_scales) v *= (double)T.inv_scales[c];
                mr_put(panels, t, i, (T.dense ? 0 : t.kd) + T.coloff + c, v, T.dense && t.lo);
            }
        }
    }
}

int64_t mr_round(int64_t v, int64_t m) { return (v + m - 1) / m * m; }

template <typename X>
hbi_status mr_upload(X **dst, const std::vector<X> &v) {
    HBI_ALLOC_TRY((void **)dst, std::max<size_t>(1, v.size()) * sizeof(X));
    if (!v.empty()) HBI_CUDA_TRY(cudaMemcpy(*dst, v.data(), v.size() * sizeof(X), cudaMemcpyHostToDevice));
    return HBI_OK;
}

int64_t mr_task_bytes(const MrTask &t) {
    const int64_t rg = (t.rows + 7) / 8;
    return rg * 16 * ((int64_t)t.kd * (1 + t.lo) + t.kl);
}

template <int KP> const void *mr_fn() { return (const void *)mr_kernel<KP>; }
const void *mr_fn_for(int kp) {
    switch (kp) {
        case 16: return mr_fn<16>();
        case 32: return mr_fn<32>();
        case 48: return mr_fn<48>();
        default: return mr_fn<64>();
    }
}
int mr_smem_bytes(int kp) { return mr_stages_a(kp) * MR_A_STAGE + MR_SB * 2 * MR_CW * kp * 2 + MR_SS * MR_CW * kp * 4; }

}  // namespace

void multi_free(hbi_handle *h) {
    MultiRhs *m = h->mr;
    if (!m) return;
    void *ptrs[] = {m->d_panels, m->d_vt, m->d_uy, m->d_split, m->d_runs[0], m->d_runs[1], m->d_crun[0], m->d_crun[1],
                    m->d_cta[0], m->d_cta[1], m->d_cscale, m->d_iperm, m->d_rowscale, m->d_xt, m->d_yp, m->d_vmax,
                    m->d_err};
    for (void *p : ptrs)
        if (p) cudaFree(p);
    delete m;
    h->mr = nullptr;
}

// Pack the tensor-core panels of H from the FP64 blocks (build time).
hbi_status pack_multi(hbi_handle *h, std::vector<Block> &blocks, const std::vector<int> &leaf_starts) {
    if (h->storage != HBI_FP16 && h->storage != HBI_MIXED) {
        set_error("the multi-RHS product needs HBI_FP16 or HBI_MIXED storage");
        return HBI_ERR_INVALID_ARG;
    }
    const int n = h->n, nin = h->nin, nout = h->nout;
    const int lo = h->storage == HBI_MIXED ? 1 : 0;
    MultiRhs *M = new MultiRhs();
    h->mr = M;
    M->lo = lo;
    M->nx = (int64_t)nin * n;

    // ---- per-column scales: U, V columns of low-rank blocks and dense columns
    std::vector<ColRef> cols;
    std::vector<int64_t> soffU(blocks.size(), -1), soffV(blocks.size(), -1), soffD(blocks.size(), -1);
    for (size_t b = 0; b < blocks.size(); ++b) {
        const Block &B = blocks[b];
        if (B.lowrank) {
            if (B.rank == 0) continue;
            soffU[b] = (int64_t)cols.size();
            for (int k = 0; k < B.rank; ++k) cols.push_back(ColRef{B.d_src + (size_t)k * B.m, B.m, 1});
            soffV[b] = (int64_t)cols.size();
            for (int k = 0; k < B.rank; ++k) cols.push_back(ColRef{B.d_src2 + (size_t)k * B.nc, B.nc, 1});
        } else {
            soffD[b] = (int64_t)cols.size();
            for (int64_t j = 0; j < B.nc; ++j) cols.push_back(ColRef{B.d_src + j, B.m, B.nc});
        }
    }
    std::vector<float> cs;
    hbi_status st = column_scales(cols, cs);
    if (st) return st;
    std::vector<float> inv_cs(cs.size());
    for (size_t i = 0; i < cs.size(); ++i) inv_cs[i] = 1.0f / cs[i];
    float *d_inv_cs = nullptr;
    DevScratch tmp;   // build tables, freed on every return path
    if ((st = tmp.upload(&d_inv_cs, inv_cs))) return st;
    // The dense columns of one X row (one slip component of one element) get one scale, the
    // largest over the near-field blocks that hold the column: the input gather then needs no
    // per-column scale (mr_in_kernel writes the scaled X beside X), and the near-field entries
    // of a column, within a few decades of their maximum, stay far from FP16's subnormal range.
    std::vector<float> cglob(M->nx, 0.0f);
    for (size_t b = 0; b < blocks.size(); ++b)
        if (!blocks[b].lowrank)
            for (int64_t j = 0; j < blocks[b].nc; ++j)
                cglob[blocks[b].col0 + j] = std::max(cglob[blocks[b].col0 + j], cs[soffD[b] + j]);
    std::vector<float> inv_cglob(M->nx);
    for (int64_t j = 0; j < M->nx; ++j) {
        if (!(cglob[j] > 0.0f)) cglob[j] = 1.0f;
        inv_cglob[j] = 1.0f / cglob[j];
    }
    float *d_inv_cglob = nullptr;
    if ((st = tmp.upload(&d_inv_cglob, inv_cglob)) || (st = mr_upload(&M->d_cscale, cglob))) return st;
    {
        std::vector<int> iperm(n);
        for (int p = 0; p < n; ++p) iperm[h->perm[p]] = p;
        if ((st = mr_upload(&M->d_iperm, iperm))) return st;
    }

    // ---- V^T phase: column groups, 128-row tasks
    std::map<std::pair<int64_t, int64_t>, std::vector<int>> groups;
    for (size_t b = 0; b < blocks.size(); ++b)
        if (blocks[b].lowrank && blocks[b].rank > 0) groups[{blocks[b].col0, blocks[b].nc}].push_back((int)b);
    std::vector<int64_t> toff(blocks.size(), -1);
    std::vector<MrPackTask> pvt, puy;
    std::vector<MrRowSrc> vrows;
    std::vector<MrSplit> splits;
    int64_t prow = 0;
    std::vector<float> rowscale;
    int64_t aoff = 0, tcount = 0;
    int64_t alg = 0;
    double flops = 0, mma = 0;
    for (auto &kv : groups) {
        const int64_t col0 = kv.first.first, nc = kv.first.second;
        const int64_t tbase = tcount;
        std::vector<MrRowSrc> rs;
        for (int b : kv.second) {
            const Block &B = blocks[b];
            toff[b] = tbase + (int64_t)rs.size();
            for (int k = 0; k < B.rank; ++k) {
                const float sv = cs[soffV[b] + k], su = cs[soffU[b] + k];
                rs.push_back(MrRowSrc{B.d_src2 + (size_t)k * B.nc, 1.0f / sv});
                rowscale.push_back(sv * su);
            }
            alg += 2 * B.nc * B.rank + 4 * B.rank;
            flops += 2.0 * (double)B.nc * B.rank;
        }
        const int64_t R = (int64_t)rs.size();
        const int nsl = (int)((nc + MR_KSLICE - 1) / MR_KSLICE);
        for (int64_t q = 0; q < R; q += MR_ROWS) {
            const int rows = (int)std::min<int64_t>(MR_ROWS, R - q);
            if (nsl > 1) splits.push_back(MrSplit{2 * M->nx + tbase + q, prow, rows, nsl});
            for (int sl = 0; sl < nsl; ++sl) {
                const int64_t c0 = (int64_t)sl * MR_KSLICE, w = std::min<int64_t>(MR_KSLICE, nc - c0);
                MrPackTask P{};
                P.t.a_off = aoff;
                P.t.g_off = col0 + c0;
                P.t.out_off = nsl > 1 ? prow + (int64_t)sl * MR_ROWS : 2 * M->nx + tbase + q;   // partial rows: fixed below
                P.t.s_off = tbase + q;
                P.t.rows = rows;
                P.t.kd = 0;
                P.t.kl = (int)mr_round(w, 16);
                P.t.kreal = (int)w;
                P.t.lo = 0;
                P.t.partial = nsl > 1;
                P.t.nd_real = 0;
                P.t.nl_real = (int)w;
                P.src0 = (int)vrows.size();
                P.nsrc = rows;
                for (int i = 0; i < rows; ++i) vrows.push_back(MrRowSrc{rs[q + i].v + c0, rs[q + i].inv_scale});
                aoff += mr_round(mr_task_bytes(P.t), 256);
                mma += 2.0 * 2.0 * MR_ROWS * P.t.kl;
                pvt.push_back(P);
            }
            if (nsl > 1) prow += (int64_t)nsl * MR_ROWS;
        }
        tcount += R;
    }
    M->n_t = tcount;
    M->n_prow = prow;
    // partial rows live after T in xt
    for (auto &P : pvt)
        if (P.t.partial) P.t.out_off += 2 * M->nx + tcount;
    for (auto &S : splits) S.p_row += 2 * M->nx + tcount;

    // ---- UY phase: leaf row units, 128-row tasks, [dense | U] columns
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
    std::vector<MrTerm> terms;
    std::vector<int> gidx;
    for (int u = 0; u < nleaves; ++u) {
        const int64_t r0 = (int64_t)nout * leaf_starts[u], R = (int64_t)nout * (leaf_starts[u + 1] - leaf_starts[u]);
        const int64_t goff = (int64_t)gidx.size();
        std::vector<MrTerm> ut;
        int64_t Cd = 0, Cl = 0;
        for (int pass = 0; pass < 2; ++pass) {
            for (int b : unit_terms[u]) {
                const Block &B = blocks[b];
                if ((pass == 0) == (bool)B.lowrank) continue;
                MrTerm T{};
                T.roff = r0 - B.row0;
                if (!B.lowrank) {
                    T.src = B.d_src; T.ld = B.nc; T.width = (int)B.nc; T.dense = 1; T.coloff = (int)Cd;
                    T.inv_scales = d_inv_cglob + B.col0;
                    for (int64_t j = 0; j < B.nc; ++j) gidx.push_back((int)(M->nx + B.col0 + j));   // scaled X
                    Cd += B.nc;
                    alg += R * B.nc * (lo ? 4 : 2) + 4 * B.nc;
                    flops += 2.0 * (double)R * B.nc;
                } else {
                    T.src = B.d_src; T.ld = B.m; T.width = B.rank; T.dense = 0; T.coloff = (int)Cl;
                    T.inv_scales = d_inv_cs + soffU[b];
                    for (int k = 0; k < B.rank; ++k) gidx.push_back((int)(2 * M->nx + toff[b] + k));   // T
                    Cl += B.rank;
                    alg += 2 * R * B.rank;
                    flops += 2.0 * (double)R * B.rank;
                }
                ut.push_back(T);
            }
            if (pass == 0)
                for (int64_t c = Cd; c < mr_round(Cd, 16); ++c) gidx.push_back(-1);
        }
        for (int64_t c = Cl; c < mr_round(Cl, 16); ++c) gidx.push_back(-1);
        const int64_t kd = mr_round(Cd, 16), kl = mr_round(Cl, 16);
        for (int64_t q = 0; q < R; q += MR_ROWS) {
            MrPackTask P{};
            P.t.a_off = aoff;
            P.t.g_off = goff;
            P.t.out_off = r0 + q;
            P.t.s_off = -1;
            P.t.rows = (int)std::min<int64_t>(MR_ROWS, R - q);
            P.t.kd = (int)kd;
            P.t.kl = (int)kl;
            P.t.kreal = (int)(kd + kl);
            P.t.lo = lo;
            P.t.nd_real = (int)Cd;
            P.t.nl_real = (int)Cl;
            P.src0 = (int)terms.size();
            P.nsrc = (int)ut.size();
            for (const MrTerm &T0 : ut) {
                MrTerm T = T0;
                T.roff += q;
                terms.push_back(T);
            }
            aoff += mr_round(mr_task_bytes(P.t), 256);
            mma += 2.0 * MR_ROWS * (double)(3 * kd * lo + 2 * kd * (1 - lo) + 2 * kl);
            puy.push_back(P);
        }
    }
    if ((int64_t)gidx.size() > (int64_t)INT32_MAX || 2 * M->nx + tcount > (int64_t)INT32_MAX) {
        set_error("operator too large for the multi-RHS gather indices");
        return HBI_ERR_INVALID_ARG;
    }
    // every task's chunks lie inside the panel stream and fit one A stage; its rows fit the MMA
    for (const auto *L : {&pvt, &puy})
        for (const MrPackTask &P : *L) {
            const MrTask &t = P.t;
            const bool ok = t.rows >= 1 && t.rows <= MR_ROWS && t.kd % 16 == 0 && t.kl % 16 == 0 && t.kd + t.kl > 0 &&
                            t.a_off % 256 == 0 && t.a_off + mr_task_bytes(t) <= aoff &&
                            (int64_t)((t.rows + 7) / 8) * MR_CW * 16 <= MR_A_STAGE;
            if (!ok) {
                set_error("internal error: a multi-RHS task exceeds its buffers");
                return HBI_ERR_INVALID_ARG;
            }
        }

    // ---- device data and packing
    M->panel_bytes = aoff;
    HBI_ALLOC_TRY(&M->d_panels, std::max<int64_t>(256, aoff));
    HBI_CUDA_TRY(cudaMemset(M->d_panels, 0, std::max<int64_t>(256, aoff)));
    MrPackTask *d_pvt = nullptr, *d_puy = nullptr;
    MrRowSrc *d_rows = nullptr;
    MrTerm *d_terms = nullptr;
    if ((st = tmp.upload(&d_pvt, pvt)) || (st = tmp.upload(&d_puy, puy)) || (st = tmp.upload(&d_rows, vrows)) ||
        (st = tmp.upload(&d_terms, terms)))
        return st;
    if (!pvt.empty()) mr_pack_kernel<<<(unsigned)pvt.size(), 256>>>(d_pvt, 1, d_rows, d_terms, M->d_panels);
    HBI_CUDA_TRY(cudaGetLastError());
    if (!puy.empty()) mr_pack_kernel<<<(unsigned)puy.size(), 256>>>(d_puy, 0, d_rows, d_terms, M->d_panels);
    HBI_CUDA_TRY(cudaGetLastError());
    HBI_CUDA_TRY(cudaDeviceSynchronize());

    // gather runs: per chunk, the maximal ranges of consecutive xt rows landing on consecutive
    // chunk columns (padding columns are left out and read as zeros)
    auto add_runs = [&](const MrTask &t, int phase) {
        std::vector<MrRun> &runs = M->h_runs[phase];
        std::vector<int64_t> &crun = M->h_crun[phase];
        M->h_cfirst[phase].push_back((int64_t)crun.size());
        const int nchd = (t.kd + MR_CW - 1) / MR_CW, nch = nchd + (t.kl + MR_CW - 1) / MR_CW;
        for (int c = 0; c < nch; ++c) {
            crun.push_back((int64_t)runs.size());
            const int col0 = c < nchd ? c * MR_CW : t.kd + (c - nchd) * MR_CW;
            const int w = c < nchd ? std::min(MR_CW, t.kd - col0) : std::min(MR_CW, t.kd + t.kl - col0);
            const size_t first = runs.size();
            for (int kc = 0; kc < w; ++kc) {
                const int col = col0 + kc;
                int64_t j;
                if (phase == 0) j = col < t.kreal ? t.g_off + col : -1;   // V^T: X rows of the group
                else j = gidx[t.g_off + col];
                if (j < 0) continue;
                if (runs.size() > first && runs.back().src + runs.back().len == j && runs.back().dst + runs.back().len == kc)
                    ++runs.back().len;
                else
                    runs.push_back(MrRun{j, 1, kc});
            }
        }
        crun.push_back((int64_t)runs.size());
    };
    std::vector<MrTask> tv, tu;
    for (auto &P : pvt) tv.push_back(P.t);
    for (auto &P : puy) tu.push_back(P.t);
    // V^T tasks largest first (they are independent); UY tasks in tree order, so that the
    // units running at the same time share far-field t entries in L2
    std::stable_sort(tv.begin(), tv.end(), [](const MrTask &a, const MrTask &b) { return mr_task_bytes(a) > mr_task_bytes(b); });
    for (const MrTask &t : tv) add_runs(t, 0);
    for (const MrTask &t : tu) add_runs(t, 1);
    M->n_vt = (int)tv.size();
    M->n_uy = (int)tu.size();
    M->n_split = (int)splits.size();
    if ((st = mr_upload(&M->d_vt, tv)) || (st = mr_upload(&M->d_uy, tu)) || (st = mr_upload(&M->d_split, splits)) ||
        (st = mr_upload(&M->d_rowscale, rowscale)))
        return st;
    M->bytes_panels_alg = alg;
    M->vec_bytes_per_rhs = 4 * (M->nx + 2 * tcount + (int64_t)nout * n);
    M->flops_per_rhs = flops;
    M->mma_flops_per_rhs = mma;
    return HBI_OK;
}

namespace {
// The B gather runs of phase p in the order the CTAs of a grid of g take their chunks: CTA b
// takes tasks b, b + g, ...; its chunk boundaries are d_crun[d_cta[b] ...], one more than its
// chunks, and index the reordered runs.
hbi_status mr_layout(MultiRhs *M, int p, int ntasks, int g) {
    const std::vector<int64_t> &cf = M->h_cfirst[p], &hc = M->h_crun[p];
    const std::vector<MrRun> &hr = M->h_runs[p];
    std::vector<MrRun> runs;
    std::vector<int64_t> crun, cta;
    runs.reserve(hr.size());
    crun.reserve(hc.size() + g);
    for (int b = 0; b < g; ++b) {
        cta.push_back((int64_t)crun.size());
        for (int ti = b; ti < ntasks; ti += g) {
            const int64_t f = cf[ti], e = ti + 1 < ntasks ? cf[ti + 1] : (int64_t)hc.size();
            for (int64_t c = f; c + 1 < e; ++c) {
                crun.push_back((int64_t)runs.size());
                runs.insert(runs.end(), hr.begin() + hc[c], hr.begin() + hc[c + 1]);
            }
        }
        crun.push_back((int64_t)runs.size());
    }
    cta.push_back((int64_t)crun.size());
    if (M->d_runs[p]) cudaFree(M->d_runs[p]);
    if (M->d_crun[p]) cudaFree(M->d_crun[p]);
    if (M->d_cta[p]) cudaFree(M->d_cta[p]);
    M->d_runs[p] = nullptr; M->d_crun[p] = M->d_cta[p] = nullptr;
    hbi_status st;
    if ((st = mr_upload(&M->d_runs[p], runs)) || (st = mr_upload(&M->d_crun[p], crun)) ||
        (st = mr_upload(&M->d_cta[p], cta)))
        return st;
    return HBI_OK;
}

hbi_status mr_prepare(hbi_handle *h, int kp) {
    MultiRhs *M = h->mr;
    if (M->kp_cap < kp) {
        if (M->d_xt) cudaFree(M->d_xt);
        if (M->d_yp) cudaFree(M->d_yp);
        M->d_xt = M->d_yp = nullptr;
        M->kp_cap = 0;
        // xt rows: X, X scaled per row for the near field, T, partial rows of cut V^T tiles
        HBI_ALLOC_TRY(&M->d_xt, (size_t)(2 * M->nx + M->n_t + M->n_prow) * kp * sizeof(float));
        HBI_ALLOC_TRY(&M->d_yp, (size_t)h->nout * h->n * kp * sizeof(float));
        M->kp_cap = kp;
    }
    if (!M->d_vmax) {
        HBI_ALLOC_TRY(&M->d_vmax, 192 * sizeof(unsigned));
        HBI_ALLOC_TRY(&M->d_err, sizeof(int));
        HBI_CUDA_TRY(cudaMemset(M->d_err, 0, sizeof(int)));
    }
    const void *fn = mr_fn_for(kp);
    const int smem = mr_smem_bytes(kp);
    HBI_CUDA_TRY(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    HBI_CUDA_TRY(cudaFuncSetAttribute(fn, cudaFuncAttributePreferredSharedMemoryCarveout, 100));
    // CTAs per SM from shared memory, registers and tensor memory (each CTA holds 4 kp columns,
    // two accumulators, rounded up to a power of two, of the SM's 512)
    int dev = 0, sms = 0, smem_sm = 0, resv = 0, regs_sm = 0;
    HBI_CUDA_TRY(cudaGetDevice(&dev));
    HBI_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    HBI_CUDA_TRY(cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev));
    HBI_CUDA_TRY(cudaDeviceGetAttribute(&resv, cudaDevAttrReservedSharedMemoryPerBlock, dev));
    HBI_CUDA_TRY(cudaDeviceGetAttribute(&regs_sm, cudaDevAttrMaxRegistersPerMultiprocessor, dev));
    cudaFuncAttributes fa;
    HBI_CUDA_TRY(cudaFuncGetAttributes(&fa, fn));
    const int by_smem = smem_sm / (smem + (int)fa.sharedSizeBytes + resv);
    const int regs_warp = (fa.numRegs * 32 + 255) / 256 * 256;
    const int by_regs = regs_sm / (regs_warp * (MR_THREADS / 32));
    const int tcols = 4 * kp <= 64 ? 64 : (4 * kp <= 128 ? 128 : 256);
    const int per_sm = std::max(1, std::min(std::min(by_smem, by_regs), 512 / tcols));
    M->grid = sms * per_sm;
    if (M->layout_grid != M->grid) {
        hbi_status st;
        if ((st = mr_layout(M, 0, M->n_vt, std::max(1, std::min(M->grid, M->n_vt)))) ||
            (st = mr_layout(M, 1, M->n_uy, std::max(1, std::min(M->grid, M->n_uy)))))
            return st;
        M->layout_grid = M->grid;
    }
    return HBI_OK;
}

template <int KP>
hbi_status mr_launch_phase(hbi_handle *h, int phase, cudaStream_t s) {
    MultiRhs *M = h->mr;
    const int smem = mr_smem_bytes(KP);
    if (phase == 0 && M->n_vt)
        mr_kernel<KP><<<std::min(M->grid, M->n_vt), MR_THREADS, smem, s>>>(
            M->d_vt, M->n_vt, 1, M->d_panels, M->d_runs[0], (int64_t)M->h_runs[0].size(), M->d_crun[0], M->d_cta[0],
            M->d_rowscale, M->d_xt, M->d_xt, M->d_vmax, M->d_err);
    if (phase == 0 && M->n_split)
        mr_reduce_kernel<<<M->n_split, 256, 0, s>>>(M->d_split, KP, M->d_xt, M->d_vmax);
    if (phase == 1 && M->n_uy)
        mr_kernel<KP><<<std::min(M->grid, M->n_uy), MR_THREADS, smem, s>>>(
            M->d_uy, M->n_uy, 0, M->d_panels, M->d_runs[1], (int64_t)M->h_runs[1].size(), M->d_crun[1], M->d_cta[1],
            M->d_rowscale, M->d_xt, M->d_yp, M->d_vmax, M->d_err);
    HBI_CUDA_TRY(cudaGetLastError());
    return HBI_OK;
}
hbi_status mr_phase(hbi_handle *h, int kp, int phase, cudaStream_t s) {
    switch (kp) {
        case 16: return mr_launch_phase<16>(h, phase, s);
        case 32: return mr_launch_phase<32>(h, phase, s);
        case 48: return mr_launch_phase<48>(h, phase, s);
        default: return mr_launch_phase<64>(h, phase, s);
    }
}

// the whole product on `s`, no synchronisation
hbi_status mr_enqueue(hbi_handle *h, int k, int kp, const double *d_X, double *d_Y, cudaStream_t s) {
    MultiRhs *M = h->mr;
    HBI_CUDA_TRY(cudaMemsetAsync(M->d_vmax, 0, 192 * sizeof(unsigned), s));
    const int gmax = 8 * std::max(1, h->num_sms);
    const int g = (int)std::max<int64_t>(1, std::min<int64_t>(((int64_t)h->n + MR_TILE - 1) / MR_TILE, gmax));
    // a block size that is a multiple of kp (every thread writes one right-hand side)
    if (d_X) mr_in_kernel<<<g, kp * (256 / kp), 0, s>>>(d_X, M->d_iperm, h->n, h->nin, k, kp, M->d_cscale, M->d_xt, M->d_vmax);
    HBI_CUDA_TRY(cudaGetLastError());
    hbi_status st = mr_phase(h, kp, 0, s);
    if (st) return st;
    if ((st = mr_phase(h, kp, 1, s))) return st;
    if (d_Y) {
        const int64_t ny = (int64_t)h->nout * h->n;
        const int g2 = (int)std::max<int64_t>(1, std::min<int64_t>(((int64_t)h->n + MR_TILE - 1) / MR_TILE, gmax));
        mr_out_kernel<<<g2, 256, 0, s>>>(M->d_yp, M->d_iperm, h->n, h->nout, k, kp, d_Y);
        HBI_CUDA_TRY(cudaGetLastError());
    }
    return HBI_OK;
}

hbi_status mr_check(hbi_handle *h) {
    int err = 0;
    HBI_CUDA_TRY(cudaMemcpy(&err, h->mr->d_err, sizeof(int), cudaMemcpyDeviceToHost));
    if (err) {
        HBI_CUDA_TRY(cudaMemset(h->mr->d_err, 0, sizeof(int)));
        set_error("a multi-RHS product wait timed out");
        return HBI_ERR_TIMEOUT;
    }
    return HBI_OK;
}

hbi_status mr_args(hbi_handle *h, int k, int &kp) {
    if (!h) { set_error("handle is required"); return HBI_ERR_INVALID_ARG; }
    if (!h->mr) {
        set_error("the handle was built without the multi-RHS panels (hbi_build_params.multi_rhs = 0)");
        return HBI_ERR_INVALID_ARG;
    }
    if (k < 1 || k > MR_KP_MAX) { set_error("need 1 <= k <= 64 right-hand sides"); return HBI_ERR_INVALID_ARG; }
    kp = (int)mr_round(k, 16);
    if (h->num_sms <= 0) {
        int dev = 0;
        HBI_CUDA_TRY(cudaGetDevice(&dev));
        HBI_CUDA_TRY(cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, dev));
    }
    return mr_prepare(h, kp);
}
}  // namespace
}  // namespace hbi

using namespace hbi;

extern "C" hbi_status hbi_matvec_multi(hbi_handle *h, int k, const double *d_X, double *d_Y, hbi_stream stream) {
    if (!d_X || !d_Y) { set_error("X and Y are required"); return HBI_ERR_INVALID_ARG; }
    int kp = 0;
    hbi_status st = mr_args(h, k, kp);
    if (st) return st;
    cudaStream_t s = (cudaStream_t)stream;
    if ((st = mr_enqueue(h, k, kp, d_X, d_Y, s))) return st;
    HBI_CUDA_TRY(cudaStreamSynchronize(s));
    return mr_check(h);
}

extern "C" hbi_status hbi_time_multi(hbi_handle *h, int k, int n_rep, double *out3, hbi_stream stream) {
    if (!out3 || n_rep < 1) { set_error("out3 and n_rep >= 1 are required"); return HBI_ERR_INVALID_ARG; }
    int kp = 0;
    hbi_status st = mr_args(h, k, kp);
    if (st) return st;
    cudaStream_t s = (cudaStream_t)stream;
    cudaEvent_t e[4];
    for (auto &x : e) HBI_CUDA_TRY(cudaEventCreate(&x));
    double acc[3] = {0, 0, 0};
    for (int r = 0; r < n_rep && !st; ++r) {
        // the input already in xt (from the last call); the scales are recomputed from it
        HBI_CUDA_TRY(cudaEventRecord(e[0], s));
        st = mr_phase(h, kp, 0, s);
        if (!st) { HBI_CUDA_TRY(cudaEventRecord(e[1], s)); st = mr_phase(h, kp, 1, s); }
        if (!st) HBI_CUDA_TRY(cudaEventRecord(e[2], s));
        if (!st) HBI_CUDA_TRY(cudaEventSynchronize(e[2]));
        float a = 0, b = 0;
        if (!st) {
            HBI_CUDA_TRY(cudaEventElapsedTime(&a, e[0], e[1]));
            HBI_CUDA_TRY(cudaEventElapsedTime(&b, e[1], e[2]));
        }
        acc[0] += a; acc[1] += b; acc[2] += a + b;
    }
    for (auto &x : e) cudaEventDestroy(x);
    if (st) return st;
    for (int i = 0; i < 3; ++i) out3[i] = acc[i] / n_rep;
    return mr_check(h);
}

extern "C" hbi_status hbi_multi_stats(const hbi_handle *h, hbi_multi_stats_t *out) {
    if (!h || !out) { set_error("handle and out are required"); return HBI_ERR_INVALID_ARG; }
    if (!h->mr) { set_error("the handle was built without the multi-RHS panels"); return HBI_ERR_INVALID_ARG; }
    const MultiRhs *M = h->mr;
    out->panel_bytes = M->panel_bytes;
    out->bytes_panels_algorithmic = M->bytes_panels_alg;
    out->vector_bytes_per_rhs = M->vec_bytes_per_rhs;
    out->flops_per_rhs = M->flops_per_rhs;
    out->mma_flops_per_rhs = M->mma_flops_per_rhs;
    out->n_tasks_vt = M->n_vt;
    out->n_tasks_uy = M->n_uy;
    out->n_t = M->n_t;
    out->n_split_tiles = M->n_split;
    return HBI_OK;
}
