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
// One persistent CTA per SM slot, warp-specialised: a producer warp streams A chunks into a
// ring of MR_SA shared-memory stages (bulk copies on mbarriers), four warps convert B chunks
// into a ring of MR_SB stages and run the epilogue (tcgen05.ld, one TMEM lane per panel row),
// and one warp allocates tensor memory and issues the MMAs, releasing each stage with
// tcgen05.commit.  Every wait is bounded; a CTA that gives up raises the error flag, lets its
// copies and MMAs in flight finish and frees its tensor memory.
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <map>
#include <vector>

#include "hbi_internal.h"

namespace hbi {

constexpr int MR_CW = 32;                          // K columns per chunk
constexpr int MR_SA = 4;                           // A ring stages
constexpr int MR_SB = 2;                           // B ring stages
constexpr int MR_GW = 4;                           // gather / epilogue warps (TMEM lanes 0..127)
constexpr int MR_THREADS = 32 * (MR_GW + 2);       // + producer warp + MMA warp
constexpr int MR_ROWS = 128;                       // MMA M: panel rows of a task
constexpr int MR_A_STAGE = 2 * MR_ROWS * MR_CW * 2;   // bytes: hi + lo parts of a 128-row chunk
constexpr int MR_KP_MAX = 64;                      // right-hand sides per call (padded to 16)
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
    int pad_;
};

}  // namespace hbi

// Everything the handle keeps for the multi-RHS product.
struct hbi::MultiRhs {
    unsigned char *d_panels = nullptr;
    int64_t panel_bytes = 0;
    MrTask *d_vt = nullptr, *d_uy = nullptr;
    int n_vt = 0, n_uy = 0;
    int *d_gidx = nullptr;        // UY gather lists: row of xt, or -1 (zero)
    float *d_gsc = nullptr;       // UY gather scales (dense column scales, 1 for t entries)
    float *d_rowscale = nullptr;  // V^T output row scales (sv su)
    int64_t n_t = 0;              // rows of T
    int64_t nx = 0;               // rows of X (n_in N)
    float cmax = 1.0f;            // largest dense column scale
    int lo = 0;
    int grid = 0;
    // per-call buffers, sized for kp_cap right-hand sides
    int kp_cap = 0;
    float *d_xt = nullptr, *d_yp = nullptr;
    unsigned *d_vmax = nullptr;   // [0, 64): max |x| per right-hand side, [64, 128): max |t|
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

// Chunk c of a task: dense or factor, its first column in the task's K, width, panel bytes
// and byte offset (a dense chunk holds its hi part, then its lo part).
struct MrChunk {
    int dense, col0, w;
    unsigned bytes;
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
        k.bytes = (unsigned)(rg * k.w * 16 * parts);
    } else {
        const int cu = c - nchd;
        k.dense = 0;
        k.col0 = t.kd + cu * MR_CW;
        k.w = min(MR_CW, t.kl - cu * MR_CW);
        k.off = t.a_off + (int64_t)rg * t.kd * 16 * parts + (int64_t)cu * rg * MR_CW * 16;
        k.bytes = (unsigned)(rg * k.w * 16);
    }
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
template <int KP>
__global__ void __launch_bounds__(MR_THREADS, 1)
    mr_kernel(const MrTask *__restrict__ tasks, int ntasks, int vt, const unsigned char *__restrict__ panels,
              const int *__restrict__ gidx, const float *__restrict__ gsc, const float *__restrict__ rowscale,
              float *xt, float *out, unsigned *vmax, float cmax, int *err) {
    constexpr int BSTAGE = MR_CW * KP * 2;   // bytes of one FP16 B part (hi or lo)
    constexpr unsigned TCOLS = 2 * KP <= 32 ? 32 : (2 * KP <= 64 ? 64 : 128);
    extern __shared__ __align__(1024) unsigned char mr_sm[];
    unsigned char *sA = mr_sm;                            // MR_SA x MR_A_STAGE
    unsigned char *sB = mr_sm + MR_SA * MR_A_STAGE;       // MR_SB x (hi | lo)
    __shared__ uint64_t a_full[MR_SA], a_empty[MR_SA], b_full[MR_SB], b_empty[MR_SB], acc_full, acc_empty, fin;
    __shared__ unsigned s_taddr;
    __shared__ float s_scale[KP], s_inv[KP];
    __shared__ volatile int s_fail;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    if (threadIdx.x == 0) {
        s_fail = 0;
        for (int s = 0; s < MR_SA; ++s) { mr_bar_init(&a_full[s], 1); mr_bar_init(&a_empty[s], 1); }
        for (int s = 0; s < MR_SB; ++s) { mr_bar_init(&b_full[s], 32 * MR_GW); mr_bar_init(&b_empty[s], 1); }
        mr_bar_init(&acc_full, 1);
        mr_bar_init(&acc_empty, 32 * MR_GW);
        mr_bar_init(&fin, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (threadIdx.x < KP) {
        const int r = threadIdx.x;
        const float xm = __uint_as_float(vmax[r]);
        const float m = vt ? xm : fmaxf(xm * cmax, __uint_as_float(vmax[64 + r]));
        const float s = mr_scale_for(m);
        s_scale[r] = s;
        s_inv[r] = 1.0f / s;
    }
    if (warp == MR_GW + 1) {
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

    if (warp == MR_GW) {
        // ---------------------------------------------------------------- producer
        if (lane == 0) {
            unsigned ga = 0;
            for (int ti = blockIdx.x; ti < ntasks && !*fail; ti += gridDim.x) {
                const MrTask t = tasks[ti];
                const int nch = mr_nchunks(t);
                for (int c = 0; c < nch; ++c) {
                    const int s = ga % MR_SA;
                    if (ga >= MR_SA && !mr_wait(&a_empty[s], ((ga / MR_SA) - 1) & 1, fail)) break;
                    const MrChunk k = mr_chunk(t, c);
                    mr_expect_tx(&a_full[s], k.bytes);
                    mr_bulk(sA + (size_t)s * MR_A_STAGE, panels + k.off, k.bytes, &a_full[s]);
                    ++ga;
                }
            }
            if (*fail) {   // let the copies in flight land before the CTA exits
                for (int s = 0; s < MR_SA; ++s) {
                    const unsigned uses = ga / MR_SA + (s < (int)(ga % MR_SA) ? 1u : 0u);
                    if (uses == 0) continue;
                    const unsigned long long t0 = mr_ns();
                    while (!mr_try(&a_full[s], (uses - 1) & 1) && mr_ns() - t0 < MR_WAIT_NS) {
                    }
                }
            }
        }
    } else if (warp == MR_GW + 1) {
        // ---------------------------------------------------------------- MMA issuer
        if (lane == 0) {
            // D F32 (bits 4-5 = 1), A and B F16, A K-major, B MN-major (bit 16), N = KP, M = 128
            const unsigned idesc = (1u << 4) | (1u << 16) | ((unsigned)(KP >> 3) << 17) | ((unsigned)(MR_ROWS >> 4) << 24);
            const unsigned d1 = taddr, d2 = taddr + KP;
            unsigned ga = 0, gb = 0, nt = 0;
            for (int ti = blockIdx.x; ti < ntasks && !*fail; ti += gridDim.x) {
                const MrTask t = tasks[ti];
                if (nt > 0 && !mr_wait(&acc_empty, (nt - 1) & 1, fail)) break;
                mr_fence_after();
                const int nch = mr_nchunks(t);
                const int rg = (t.rows + 7) / 8;
                unsigned acc1 = 0, acc2 = 0;
                bool ok = true;
                for (int c = 0; c < nch && ok; ++c) {
                    const int sa = ga % MR_SA, sb = gb % MR_SB;
                    if (!mr_wait(&a_full[sa], (ga / MR_SA) & 1, fail) || !mr_wait(&b_full[sb], (gb / MR_SB) & 1, fail)) {
                        ok = false;
                        break;
                    }
                    mr_fence_after();
                    const MrChunk k = mr_chunk(t, c);
                    const unsigned a0 = mr_smem(sA + (size_t)sa * MR_A_STAGE);
                    const unsigned bh = mr_smem(sB + (size_t)sb * 2 * BSTAGE), bl = bh + BSTAGE;
                    const unsigned sbo_a = (unsigned)k.w * 16u;
                    for (int kk = 0; kk < k.w / 16; ++kk) {
                        const uint64_t ah = mr_desc(a0 + kk * 256u, 128u, sbo_a);
                        const uint64_t bhd = mr_desc(bh + kk * (unsigned)KP * 32u, (unsigned)KP * 16u, 128u);
                        const uint64_t bld = mr_desc(bl + kk * (unsigned)KP * 32u, (unsigned)KP * 16u, 128u);
                        mr_mma(d1, ah, bhd, idesc, acc1);
                        acc1 = 1;
                        mr_mma(d2, ah, bld, idesc, acc2);
                        acc2 = 1;
                        if (k.dense && t.lo) {
                            const uint64_t al = mr_desc(a0 + (unsigned)(rg * k.w * 16) + kk * 256u, 128u, sbo_a);
                            mr_mma(d2, al, bhd, idesc, 1u);
                        }
                    }
                    mr_commit(&a_empty[sa]);
                    mr_commit(&b_empty[sb]);
                    ++ga;
                    ++gb;
                }
                if (!ok) break;
                mr_commit(&acc_full);
                ++nt;
            }
            // every MMA issued so far has completed once this phase does
            mr_commit(&fin);
            const unsigned long long t0 = mr_ns();
            while (!mr_try(&fin, 0) && mr_ns() - t0 < MR_WAIT_NS) {
            }
        }
    } else {
        // ---------------------------------------------------------------- gather + epilogue
        const int tid = threadIdx.x;   // 0..127 = TMEM lane = panel row
        unsigned gb = 0, nt = 0;
        for (int ti = blockIdx.x; ti < ntasks; ti += gridDim.x) {
            const MrTask t = tasks[ti];
            const int nch = mr_nchunks(t);
            bool ok = true;
            for (int c = 0; c < nch; ++c) {
                const int sb = gb % MR_SB;
                if (gb >= MR_SB && !mr_warp_wait(&b_empty[sb], ((gb / MR_SB) - 1) & 1, fail)) { ok = false; break; }
                const MrChunk k = mr_chunk(t, c);
                unsigned char *bh = sB + (size_t)sb * 2 * BSTAGE, *bl = bh + BSTAGE;
                // vector v: K row kc = 8 kg + kr, right-hand sides 8 rq .. 8 rq + 7; eight
                // consecutive threads fill one 128-byte core matrix (no bank conflicts)
                const int nvec = k.w * (KP / 8);
                for (int v = tid; v < nvec; v += 32 * MR_GW) {
                    const int kr = v & 7, rq = (v >> 3) % (KP / 8), kg = (v >> 3) / (KP / 8);
                    const int kc = 8 * kg + kr, col = k.col0 + kc;
                    int64_t j;
                    float sc = 1.0f;
                    if (vt) {
                        j = col < t.kreal ? t.g_off + col : -1;
                    } else {
                        j = gidx[t.g_off + col];
                        sc = gsc[t.g_off + col];
                    }
                    float4 x0 = make_float4(0.f, 0.f, 0.f, 0.f), x1 = x0;
                    if (j >= 0) {
                        const float4 *src = reinterpret_cast<const float4 *>(xt + j * KP + 8 * rq);
                        x0 = __ldg(src);
                        x1 = __ldg(src + 1);
                    }
                    const float xs[8] = {x0.x, x0.y, x0.z, x0.w, x1.x, x1.y, x1.z, x1.w};
                    __align__(16) __half hi[8], lo[8];
#pragma unroll
                    for (int q = 0; q < 8; ++q) {
                        const float b = xs[q] * sc * s_scale[8 * rq + q];
                        hi[q] = __float2half_rn(b);
                        lo[q] = __float2half_rn((b - __half2float(hi[q])) * 2048.0f);
                    }
                    const int off = (kg * (KP / 8) + rq) * 128 + kr * 16;
                    *reinterpret_cast<uint4 *>(bh + off) = *reinterpret_cast<const uint4 *>(hi);
                    *reinterpret_cast<uint4 *>(bl + off) = *reinterpret_cast<const uint4 *>(lo);
                }
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                mr_arrive(&b_full[sb]);
                ++gb;
            }
            if (!ok || !mr_warp_wait(&acc_full, nt & 1, fail)) break;
            mr_fence_after();
            // epilogue: lane tid holds panel row tid; columns [0, KP) = D1, [KP, 2 KP) = D2
            const unsigned lane_base = taddr + ((unsigned)(32 * warp) << 16);
            const bool live = tid < t.rows;
            const float rs = (vt && live && rowscale) ? rowscale[t.s_off + tid] : 1.0f;
            float *orow = out + (t.out_off + tid) * KP;
#pragma unroll 1
            for (int c0 = 0; c0 < KP; c0 += 16) {
                float a[16], b[16];
                mr_ld16(lane_base + c0, a);
                mr_ld16(lane_base + KP + c0, b);
                mr_ld_wait();
                float y[16];
#pragma unroll
                for (int q = 0; q < 16; ++q) y[q] = (a[q] + b[q] * (1.0f / 2048.0f)) * s_inv[c0 + q] * rs;
                if (live) {
#pragma unroll
                    for (int q = 0; q < 16; q += 4)
                        *reinterpret_cast<float4 *>(orow + c0 + q) = make_float4(y[q], y[q + 1], y[q + 2], y[q + 3]);
                }
                if (vt) {
#pragma unroll
                    for (int q = 0; q < 16; ++q) {
                        float m = live ? fabsf(y[q]) : 0.0f;
                        if (!(m == m)) m = 0.0f;
#pragma unroll
                        for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
                        if (lane == 0 && m > 0.0f) atomicMax(vmax + 64 + c0 + q, __float_as_uint(m));
                    }
                }
            }
            mr_fence_before();
            mr_arrive(&acc_empty);
            ++nt;
        }
    }
    if (threadIdx.x == 0 && s_fail) atomicExch(err, 1);
    mr_fence_before();
    __syncthreads();
    mr_fence_after();
    if (warp == MR_GW + 1)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(TCOLS) : "memory");
}

// X (k right-hand sides, caller's order, component-major) -> xt rows (permuted, component-
// interleaved DOF) x KP FP32, zero for r >= k; max |x| per right-hand side.
__global__ void mr_in_kernel(const double *__restrict__ X, const int *__restrict__ perm, int n, int nin, int k, int KP,
                             float *__restrict__ xt, unsigned *__restrict__ vmax) {
    const int64_t nx = (int64_t)nin * n;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nx * KP; e += (int64_t)gridDim.x * blockDim.x) {
        const int r = (int)(e % KP);
        const int64_t row = e / KP;
        const int p = (int)(row / nin), c = (int)(row % nin);
        float v = 0.0f;
        if (r < k) v = (float)X[(int64_t)r * nx + (int64_t)c * n + perm[p]];
        xt[e] = v;
        const float a = fabsf(v);
        if (a > 0.0f && isfinite(a)) atomicMax(vmax + r, __float_as_uint(a));
    }
}

__global__ void mr_out_kernel(const float *__restrict__ yp, const int *__restrict__ perm, int n, int nout, int k, int KP,
                              double *__restrict__ Y) {
    const int64_t ny = (int64_t)nout * n;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < ny * k; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t row = e / k;
        const int r = (int)(e % k);
        const int p = (int)(row / nout), c = (int)(row % nout);
        Y[(int64_t)r * ny + (int64_t)c * n + perm[p]] = (double)yp[row * KP + r];
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
    HBI_CUDA_TRY(cudaMalloc((void **)dst, std::max<size_t>(1, v.size()) * sizeof(X)));
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
int mr_smem_bytes(int kp) { return MR_SA * MR_A_STAGE + MR_SB * 2 * MR_CW * kp * 2; }

}  // namespace

void multi_free(hbi_handle *h) {
    MultiRhs *m = h->mr;
    if (!m) return;
    void *ptrs[] = {m->d_panels, m->d_vt, m->d_uy, m->d_gidx, m->d_gsc, m->d_rowscale, m->d_xt, m->d_yp, m->d_vmax,
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
    if ((st = mr_upload(&d_inv_cs, inv_cs))) return st;
    M->cmax = 0.0f;
    for (size_t b = 0; b < blocks.size(); ++b)
        if (!blocks[b].lowrank)
            for (int64_t j = 0; j < blocks[b].nc; ++j) M->cmax = std::max(M->cmax, cs[soffD[b] + j]);
    if (M->cmax == 0.0f) M->cmax = 1.0f;

    // ---- V^T phase: column groups, 128-row tasks
    std::map<std::pair<int64_t, int64_t>, std::vector<int>> groups;
    for (size_t b = 0; b < blocks.size(); ++b)
        if (blocks[b].lowrank && blocks[b].rank > 0) groups[{blocks[b].col0, blocks[b].nc}].push_back((int)b);
    std::vector<int64_t> toff(blocks.size(), -1);
    std::vector<MrPackTask> pvt, puy;
    std::vector<MrRowSrc> vrows;
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
        for (int64_t q = 0; q < R; q += MR_ROWS) {
            MrPackTask P{};
            P.t.a_off = aoff;
            P.t.g_off = col0;
            P.t.out_off = M->nx + tbase + q;
            P.t.s_off = tbase + q;
            P.t.rows = (int)std::min<int64_t>(MR_ROWS, R - q);
            P.t.kd = 0;
            P.t.kl = (int)mr_round(nc, 16);
            P.t.kreal = (int)nc;
            P.t.lo = 0;
            P.src0 = (int)(vrows.size() + q);
            P.nsrc = P.t.rows;
            aoff += mr_round(mr_task_bytes(P.t), 256);
            mma += 2.0 * 2.0 * MR_ROWS * P.t.kl;
            pvt.push_back(P);
        }
        vrows.insert(vrows.end(), rs.begin(), rs.end());
        tcount += R;
    }
    M->n_t = tcount;

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
    std::vector<float> gsc;
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
                    T.inv_scales = d_inv_cs + soffD[b];
                    for (int64_t j = 0; j < B.nc; ++j) {
                        gidx.push_back((int)(B.col0 + j));
                        gsc.push_back(cs[soffD[b] + j]);
                    }
                    Cd += B.nc;
                    alg += R * B.nc * (lo ? 4 : 2) + 4 * B.nc;
                    flops += 2.0 * (double)R * B.nc;
                } else {
                    T.src = B.d_src; T.ld = B.m; T.width = B.rank; T.dense = 0; T.coloff = (int)Cl;
                    T.inv_scales = d_inv_cs + soffU[b];
                    for (int k = 0; k < B.rank; ++k) {
                        gidx.push_back((int)(M->nx + toff[b] + k));
                        gsc.push_back(1.0f);
                    }
                    Cl += B.rank;
                    alg += 2 * R * B.rank;
                    flops += 2.0 * (double)R * B.rank;
                }
                ut.push_back(T);
            }
            if (pass == 0)
                for (int64_t c = Cd; c < mr_round(Cd, 16); ++c) { gidx.push_back(-1); gsc.push_back(0.0f); }
        }
        for (int64_t c = Cl; c < mr_round(Cl, 16); ++c) { gidx.push_back(-1); gsc.push_back(0.0f); }
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
    if ((int64_t)gidx.size() > (int64_t)INT32_MAX || M->nx + tcount > (int64_t)INT32_MAX) {
        set_error("operator too large for the multi-RHS gather indices");
        return HBI_ERR_INVALID_ARG;
    }
    // every task's chunks lie inside the panel stream and fit one A stage; its rows fit the MMA
    for (const auto *L : {&pvt, &puy})
        for (const MrPackTask &P : *L) {
            const MrTask &t = P.t;
            const bool ok = t.rows >= 1 && t.rows <= MR_ROWS && t.kd % 16 == 0 && t.kl % 16 == 0 && t.kd + t.kl > 0 &&
                            t.a_off % 256 == 0 && t.a_off + mr_task_bytes(t) <= aoff &&
                            (int64_t)((t.rows + 7) / 8) * MR_CW * 16 * (1 + t.lo) <= MR_A_STAGE;
            if (!ok) {
                cudaFree(d_inv_cs);
                set_error("internal error: a multi-RHS task exceeds its buffers");
                return HBI_ERR_INVALID_ARG;
            }
        }

    // ---- device data and packing
    M->panel_bytes = aoff;
    HBI_CUDA_TRY(cudaMalloc(&M->d_panels, std::max<int64_t>(256, aoff)));
    HBI_CUDA_TRY(cudaMemset(M->d_panels, 0, std::max<int64_t>(256, aoff)));
    MrPackTask *d_pvt = nullptr, *d_puy = nullptr;
    MrRowSrc *d_rows = nullptr;
    MrTerm *d_terms = nullptr;
    if ((st = mr_upload(&d_pvt, pvt)) || (st = mr_upload(&d_puy, puy)) || (st = mr_upload(&d_rows, vrows)) ||
        (st = mr_upload(&d_terms, terms)))
        return st;
    if (!pvt.empty()) mr_pack_kernel<<<(unsigned)pvt.size(), 256>>>(d_pvt, 1, d_rows, d_terms, M->d_panels);
    HBI_CUDA_TRY(cudaGetLastError());
    if (!puy.empty()) mr_pack_kernel<<<(unsigned)puy.size(), 256>>>(d_puy, 0, d_rows, d_terms, M->d_panels);
    HBI_CUDA_TRY(cudaGetLastError());
    HBI_CUDA_TRY(cudaDeviceSynchronize());
    cudaFree(d_pvt); cudaFree(d_puy); cudaFree(d_rows); cudaFree(d_terms); cudaFree(d_inv_cs);

    std::vector<MrTask> tv, tu;
    for (auto &P : pvt) tv.push_back(P.t);
    for (auto &P : puy) tu.push_back(P.t);
    // V^T tasks largest first (they are independent); UY tasks in tree order, so that the
    // units running at the same time share far-field t entries in L2
    std::stable_sort(tv.begin(), tv.end(), [](const MrTask &a, const MrTask &b) { return mr_task_bytes(a) > mr_task_bytes(b); });
    M->n_vt = (int)tv.size();
    M->n_uy = (int)tu.size();
    if ((st = mr_upload(&M->d_vt, tv)) || (st = mr_upload(&M->d_uy, tu)) || (st = mr_upload(&M->d_gidx, gidx)) ||
        (st = mr_upload(&M->d_gsc, gsc)) || (st = mr_upload(&M->d_rowscale, rowscale)))
        return st;
    M->bytes_panels_alg = alg;
    M->vec_bytes_per_rhs = 4 * (M->nx + 2 * tcount + (int64_t)nout * n);
    M->flops_per_rhs = flops;
    M->mma_flops_per_rhs = mma;
    return HBI_OK;
}

namespace {
hbi_status mr_prepare(hbi_handle *h, int kp) {
    MultiRhs *M = h->mr;
    if (M->kp_cap < kp) {
        if (M->d_xt) cudaFree(M->d_xt);
        if (M->d_yp) cudaFree(M->d_yp);
        M->d_xt = M->d_yp = nullptr;
        M->kp_cap = 0;
        HBI_CUDA_TRY(cudaMalloc(&M->d_xt, (size_t)(M->nx + M->n_t) * kp * sizeof(float)));
        HBI_CUDA_TRY(cudaMalloc(&M->d_yp, (size_t)h->nout * h->n * kp * sizeof(float)));
        M->kp_cap = kp;
    }
    if (!M->d_vmax) {
        HBI_CUDA_TRY(cudaMalloc(&M->d_vmax, 128 * sizeof(unsigned)));
        HBI_CUDA_TRY(cudaMalloc(&M->d_err, sizeof(int)));
        HBI_CUDA_TRY(cudaMemset(M->d_err, 0, sizeof(int)));
    }
    const void *fn = mr_fn_for(kp);
    const int smem = mr_smem_bytes(kp);
    HBI_CUDA_TRY(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    int per_sm = 0;
    HBI_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, MR_THREADS, smem));
    // each CTA holds up to 128 tensor-memory columns of the SM's 512
    per_sm = std::max(1, std::min(per_sm, 4));
    int dev = 0, sms = 0;
    HBI_CUDA_TRY(cudaGetDevice(&dev));
    HBI_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    M->grid = sms * per_sm;
    return HBI_OK;
}

template <int KP>
hbi_status mr_launch_phase(hbi_handle *h, int phase, cudaStream_t s) {
    MultiRhs *M = h->mr;
    const int smem = mr_smem_bytes(KP);
    if (phase == 0 && M->n_vt)
        mr_kernel<KP><<<std::min(M->grid, M->n_vt), MR_THREADS, smem, s>>>(
            M->d_vt, M->n_vt, 1, M->d_panels, M->d_gidx, M->d_gsc, M->d_rowscale, M->d_xt, M->d_xt, M->d_vmax,
            M->cmax, M->d_err);
    if (phase == 1 && M->n_uy)
        mr_kernel<KP><<<std::min(M->grid, M->n_uy), MR_THREADS, smem, s>>>(
            M->d_uy, M->n_uy, 0, M->d_panels, M->d_gidx, M->d_gsc, M->d_rowscale, M->d_xt, M->d_yp, M->d_vmax,
            M->cmax, M->d_err);
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
    HBI_CUDA_TRY(cudaMemsetAsync(M->d_vmax, 0, 128 * sizeof(unsigned), s));
    const int g = std::max(1, std::min<int>((int)((M->nx * kp + 255) / 256), 8 * std::max(1, h->num_sms)));
    if (d_X) mr_in_kernel<<<g, 256, 0, s>>>(d_X, h->d_perm, h->n, h->nin, k, kp, M->d_xt, M->d_vmax);
    HBI_CUDA_TRY(cudaGetLastError());
    hbi_status st = mr_phase(h, kp, 0, s);
    if (st) return st;
    if ((st = mr_phase(h, kp, 1, s))) return st;
    if (d_Y) {
        const int64_t ny = (int64_t)h->nout * h->n;
        const int g2 = std::max(1, std::min<int>((int)((ny * k + 255) / 256), 8 * std::max(1, h->num_sms)));
        mr_out_kernel<<<g2, 256, 0, s>>>(M->d_yp, h->d_perm, h->n, h->nout, k, kp, d_Y);
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
    return HBI_OK;
}
