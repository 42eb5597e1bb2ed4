// Internal declarations of the hbi library (host orchestration + device kernels).
// Not part of the public ABI; see include/hbi.h for that.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <string>
#include <vector>

#include "../../include/hbi.h"
#include "hbi_tables.h"

namespace hbi {

// ------------------------------------------------------------------ errors
void set_error(const std::string &msg);
#define HBI_CUDA_TRY(expr)                                                        \
    do {                                                                          \
        cudaError_t e_ = (expr);                                                  \
        if (e_ != cudaSuccess) {                                                  \
            ::hbi::set_error(std::string(#expr) + ": " + cudaGetErrorString(e_)); \
            return HBI_ERR_CUDA;                                                  \
        }                                                                         \
    } while (0)

// Device allocation of the library: cudaMalloc, HBI_ERR_OOM when it (or an injected failure,
// hbi_inject_failure) fails.
hbi_status dev_malloc(void **p, size_t bytes);
#define HBI_ALLOC_TRY(pp, bytes)                                           \
    do {                                                                   \
        hbi_status s_ = ::hbi::dev_malloc((void **)(pp), (size_t)(bytes)); \
        if (s_) return s_;                                                 \
    } while (0)
// An injected ACA failure: true for the one ACA block result hbi_inject_failure selected.
bool inject_aca_failure();

// Device temporaries of one host function, freed when the holder goes out of scope (on every
// return path, failures included).
struct DevScratch {
    std::vector<void *> p;
    template <typename T> hbi_status alloc(T **out, size_t bytes) {
        void *q = nullptr;
        hbi_status s = dev_malloc(&q, bytes);
        if (s) return s;
        p.push_back(q);
        *out = static_cast<T *>(q);
        return HBI_OK;
    }
    template <typename T> hbi_status upload(T **out, const std::vector<T> &v) {
        hbi_status s = alloc(out, std::max<size_t>(1, v.size()) * sizeof(T));
        if (s) return s;
        if (!v.empty() && cudaMemcpy(*out, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice) != cudaSuccess) {
            set_error("copy of a build table to the device failed");
            return HBI_ERR_CUDA;
        }
        return HBI_OK;
    }
    DevScratch() = default;
    DevScratch(const DevScratch &) = delete;
    DevScratch &operator=(const DevScratch &) = delete;
    ~DevScratch() {
        for (void *q : p) cudaFree(q);
    }
};

// ------------------------------------------------------------ host geometry
struct Frames {
    // per element (original order): centre, normal, strike, dip
    std::vector<double> c, n, s, d;
};
Frames element_frames(int n, int nv, const double *verts);

// ------------------------------------------------------------ cluster tree
struct Cluster {
    int start, size, depth, child0, child1;
    double lo[3], hi[3];
};
struct Tree {
    std::vector<int> perm;        // permuted position -> original element
    std::vector<Cluster> cl;      // cl[0] = root
    std::vector<int> leaves;      // leaf cluster ids in index order
    std::vector<int> lattice;     // lattice cluster ids (depth L or earlier leaves)
};
Tree build_tree(const std::vector<double> &centres, int n, int leaf_size, int lattice_depth);

struct Block {
    int tau, sig;                 // cluster ids (-1 when imported)
    int64_t row0, m, col0, nc;    // DOF offsets and sizes
    int lowrank;                  // 1 = low-rank factors, 0 = dense
    int rank;
    const double *d_src;          // device FP64: U (m x rank, column-major) or dense (m x nc, row-major)
    const double *d_src2;         // device FP64: V (nc x rank, column-major), or null
    int dense_trans;              // 1: a dense block of the transposed operator, stored as its
                                  //    transpose (nc x m row-major) at d_src
};
std::vector<Block> build_partition(const Tree &T, int nin, int nout, double eta,
                                   std::vector<int> *lattice_ij = nullptr);

// ------------------------------------------------------------ HMVM layout
// One UY-phase work item (a leaf row unit): `rows` outputs, each the dot product of a stored
// row with an input vector gathered into shared memory.  A row has two segments: dense
// near-field columns (element type of the dense stream) followed by low-rank U columns
// (element type of the factor stream).  Both segments are row-major, 16-byte aligned and
// padded to whole 16-byte vectors.
struct GemvTask {
    int64_t data_off;     // low-rank segment: element offset in its stream
    int64_t data_off_d;   // dense segment: element offset in the dense stream
    int64_t out_off;      // first output index
    int64_t gather_off;   // offset into the gather index/scale arrays
    int rows;
    int cpad;             // padded length of the low-rank segment
    int cpad_d;           // padded length of the dense segment
    int model;            // model of an ensemble handle the rows belong to
};

// One VT-phase item: a row block x column chunk of the stacked V^T panel of a column group.
// The panel (rows x cpad, row-major) and the x slice xt[x_off, x_off + cpad) are copied to
// shared memory as they are; x_off is 16-byte aligned, so the group's columns sit at panel
// columns [lo, hi).  Chunks of one row block are consecutive items of one CTA (flags bit 0 =
// first chunk, bit 1 = last chunk).
struct VtItem {
    int64_t data_off;     // element offset of the panel in the V^T stream
    int64_t x_off;        // xt offset of panel column 0
    int64_t out_off;      // xt offset of the row block's first t entry
    int64_t scale_off;    // rowscale offset of the row block's first row, or -1
    int rows, cpad, lo, hi;
    int flags;
    int poff;             // panel offset inside its batch's shared-memory stage (elements)
    int zoff;             // x slice offset inside the stage's x area (accumulator words)
    int model;            // model of an ensemble handle the columns belong to
};

// Consecutive VT items of one CTA whose panels are contiguous in the V^T stream: one bulk
// copy of pbytes for the panels plus one per x slice fill one shared-memory stage.
struct VtBatch {
    int64_t data_off;     // element offset of the first panel
    int pbytes, xbytes;   // panel bytes, x slice bytes
    int item0, nitems;    // the batch's items
};

// Device-side control block of the adaptive Runge-Kutta loop of one model (an ensemble
// handle has one per model; each model keeps its own t, step size and decisions).
struct StepCtl {
    double t, dt, dt_used, eps;
    unsigned long long err_bits, vmax_bits;
    int accepted, target, rejects, stop, done_pending, status, accept_flag;
    int flags;      // bit 0: a trial had sigma <= 0, bit 1: a trial was non-finite
    int reuse_k0;   // the last attempt was rejected: y is unchanged, so k_1 = f(y) is still in stage slot 0
    int nelem;      // elements of the model
    long long mu_fix;   // sum over the model's elements of tau / sigma of the trial, fixed point 2^-40
};
// Flags shared by all models of a handle, read by the HMVM kernels of the attempt graph.
struct GlobalCtl {
    int stop;       // every model is done: all kernels of a replayed attempt return at once
    int skip0;      // stop, or every active model rejected its last attempt: skip the first product
    int commit_done;   // CTAs of the fused commit kernel that finished (the last one rearms it)
    int pad_;
};

template <typename T> struct StorageTraits;

// One FP64 factor or dense column (len entries at the given stride) for per-column scaling.
struct ColRef {
    const double *p;
    int64_t len, stride;
};
// Power-of-two scale of each column: max |entry| / scale lies in (2^13, 2^14] (1 for a zero
// column), the scaling of the 2-byte storage formats.
hbi_status column_scales(const std::vector<ColRef> &cols, std::vector<float> &out);

}  // namespace hbi

namespace hbi {
struct MultiRhs;   // tensor-core panels of the multi-RHS product (hbi_multi.cu)
}

// --------------------------------------------------------------- the handle
struct hbi_handle {
    int n = 0, nin = 1, nout = 1, op = 0, nv = 3, storage = HBI_FP32;
    double mu = 0, nu = 0;
    int half_space = 0;                // entries of the half space z < 0 (free surface z = 0)
    std::vector<int> perm;             // permuted position -> original element
    int *d_perm = nullptr;             // same, on the device
    double *d_geom = nullptr;          // permuted: per element c(3), n(3), s(3), d(3)
    double *d_verts = nullptr;         // permuted: per element nv x 3
    double *d_rake = nullptr;          // permuted rake angles (single-component operators)

    // partition summary
    int64_t n_clusters = 0, n_leaves = 0, n_lattice = 0;
    int64_t n_blocks = 0, n_lowrank = 0, n_dense = 0, max_rank = 0;
    double mean_rank = 0;
    int64_t entries_lr = 0, entries_dense = 0;

    // packed HMVM data
    size_t elem_bytes = 4, elem_bytes_d = 4;  // low-rank / dense storage element sizes
    void *d_data1 = nullptr, *d_data2 = nullptr, *d_data3 = nullptr;  // V^T, U, dense streams
    int64_t n_data1 = 0, n_data2 = 0, n_data3 = 0;                    // elements
    float *d_rowscale = nullptr;            // phase-1 output scales
    int *d_gidx = nullptr;                  // phase-2 gather indices into xt
    float *d_gscale = nullptr;              // phase-2 gather scales (FP16/BF16 only)
    int64_t n_gather = 0, n_rowscale = 0;
    hbi::VtItem *d_items1 = nullptr;        // VT items in CTA order
    hbi::VtBatch *d_batches1 = nullptr;     // VT stage batches in CTA order
    int *d_vt_begin = nullptr;              // first batch of each VT CTA (grid1 + 1 entries)
    hbi::GemvTask *d_tasks2 = nullptr;      // UY tasks, decreasing size
    int n_tasks1 = 0, n_tasks2 = 0;
    int64_t n_t = 0;
    int smem1 = 0, smem2 = 0;               // dynamic shared memory of the two phases
    int grid1 = 0, grid2 = 0;
    // launch configuration (defaults from the build; hbi_autotune may change them)
    int uy_rpw = 4;                         // UY rows per lane group and pass: 4 or 8
    int uy_occ[2] = {1, 1};                 // UY CTAs per SM that fit, for 4 / 8 rows per pass
    int uy_ctas_per_sm = 1;
    int vt_pass_cost = 8;                   // per-pass cost in the VT per-item shape choice
    void *d_xt = nullptr;                   // [x (nin N) | t (n_t) | 16 zero guards] in accumulation type
    void *d_xt2 = nullptr;                  // a second one: consecutive products of an attempt alternate
    void *d_yp = nullptr;                   // nout N accumulation type
    int *d_counters = nullptr;              // [0] UY work counter, [1] error flag of bounded device waits
    hbi::TableLimits lim;                   // the buffers the product's work tables index
    void *d_lim = nullptr;                  // bounds-checked build: the same limits on the device
    int64_t bytes_factors = 0, bytes_algorithmic = 0, bytes_alg_vt = 0, bytes_alg_uy = 0;
    double build_seconds = 0;

    // ODE state (permuted order)
    // (sized for the rake-free form: y, ys 4N; Vs, Vold 3N; D 2N; k 6 stages x 4N)
    double *d_y = nullptr, *d_D = nullptr, *d_ys = nullptr, *d_Vs = nullptr, *d_Vold = nullptr;
    double *d_dVs = nullptr, *d_dVold = nullptr;   // dV/dtau (Eq. 13a) at the stage state / at y
    double *d_k = nullptr;                  // 6 stages x 3N (x 4N rake-free)
    double *d_inv_a = nullptr, *d_inv_b = nullptr, *d_b_dc = nullptr;   // 1/a, 1/b, b/d_c (permuted)
    double *d_fcr = nullptr, *d_fsr = nullptr;                           // rake cosine, sine
    // models of an ensemble handle: contiguous element ranges (original = permuted order of
    // the model blocks); a plain handle has one model
    // a shard of the paper's lattice distribution (Sec. 3.2): the blocks of rank shard_rank on a
    // shard_rows x shard_cols process grid only (-1: the whole operator)
    int shard_rank = -1, shard_rows = 1, shard_cols = 1;
    int n_models = 1;
    std::vector<int> model_start;           // n_models + 1 element offsets
    int *d_model = nullptr;                 // model index of each (permuted) element
    hbi::StepCtl *d_ctl = nullptr;          // n_models control blocks
    hbi::StepCtl *h_ctl = nullptr;          // pinned mirror
    hbi::GlobalCtl *d_gctl = nullptr;
    int *d_mskip = nullptr;                 // 2 x n_models: models whose first / other stage products are skipped
    hbi::GlobalCtl *h_gctl = nullptr;       // pinned mirror
    int *h_flag = nullptr;                  // pinned mirror of the bounded-wait error flag
    hbi_step_record *d_rec = nullptr;       // n_models x rec_cap
    int rec_cap = 0;
    cudaStream_t cap_stream = nullptr;
    cudaGraphExec_t graph_exec = nullptr;   // one attempt, fixed-rake friction
    cudaGraphExec_t graph_exec_vec = nullptr;   // one attempt, rake-free friction
    double g_f0 = 0, g_V0 = 0, g_Vpl = 0, g_eta = 0;   // scalars baked into the graph
    int num_sms = 0;
    int64_t last_attempts = 0;              // attempt graphs launched by the last hbi_step
    int64_t last_kernels = 0;               // kernels launched by the last hbi_step
    hbi_handle *adj = nullptr;              // the transposed operator H^T (built on request)
    // adjoint work arrays (allocated on first use)
    double *d_stY = nullptr, *d_stS = nullptr;     // one step's stage states / product outputs
    double *d_Kbar = nullptr, *d_lam = nullptr;    // adjoints of the 6 stage slopes / of y
    double *d_gA = nullptr, *d_gDC = nullptr;      // parameter gradients (permuted)
    double *d_aux = nullptr;                       // N: target (permuted) / loss partial sums
    double *d_ckpt = nullptr, *d_segY = nullptr;   // checkpoints / stage data of one segment
    int64_t n_ckpt = 0, n_segY = 0;                // their capacities (doubles)
    hbi::MultiRhs *mr = nullptr;                   // multi-RHS panels (built on request)
};

namespace hbi {
struct OdeArgs;
// hbi_host.cpp / hbi_pack.cu / hbi_hmvm.cu / hbi_ode.cu entry points used by hbi_api.cu
hbi_status pack_operator(hbi_handle *h, const Tree *T, std::vector<Block> &blocks,
                         const std::vector<int> &leaf_starts);
// Pack H (into h) and, if with_transpose, H^T (into the internal handle h->adj) from the
// same blocks and factors.
hbi_status pack_operators(hbi_handle *h, std::vector<Block> &blocks, const std::vector<int> &leaf_starts,
                          int with_transpose, int multi_rhs = 0);
// The tensor-core panels of the multi-RHS product (hbi_multi.cu), from the same blocks.
hbi_status pack_multi(hbi_handle *h, std::vector<Block> &blocks, const std::vector<int> &leaf_starts);
void multi_free(hbi_handle *h);
// d_stop: the whole product returns at once while *d_stop != 0; d_mskip (optional, one int
// per model): the rows / columns of model m are skipped while d_mskip[m] != 0.
// reset_counter = false: leave out the reset of the UY work counter before the launch (every
// UY launch that runs to its end leaves the counter at zero; used inside the attempt graph).
// xt: the input buffer of the product (nullptr: h->d_xt; the attempt alternates h->d_xt and
// h->d_xt2).  fuse != nullptr: the UY phase also runs Cash-Karp stage `stage` (0..5, the last
// with the error maxima) of the law `law` (1 fixed rake, 2 rake-free) for the elements of
// each leaf row unit as soon as the unit's rows are written, with fuse->xt (the other buffer)
// receiving the next product's input; with *d_stop set it runs stages 0-4 alone.
hbi_status hmvm_launch(hbi_handle *h, cudaStream_t s, const int *d_stop, const int *d_mskip = nullptr,
                       bool reset_counter = true, void *xt = nullptr, const OdeArgs *fuse = nullptr, int stage = 0,
                       int law = 1);
void set_uy_grid(hbi_handle *h, int per_sm);
hbi_status hmvm_check(hbi_handle *h);   // after a stream sync: TIMEOUT if a device wait gave up
hbi_status stalled_wait_status(cudaStream_t s);
// phases separately (0 = VT, 1 = nothing, 2 = UY), for timing
hbi_status hmvm_phase(hbi_handle *h, int phase, cudaStream_t s, const int *d_stop);
hbi_status permute_x_in(hbi_handle *h, const double *d_x, cudaStream_t s);
hbi_status permute_y_out(hbi_handle *h, double *d_y, cudaStream_t s);
hbi_status device_build_factors(hbi_handle *h, const Tree &T, std::vector<Block> &blocks,
                                double eps, std::vector<void *> &owned);
hbi_status upload_geometry(hbi_handle *h, const double *h_verts, const double *h_rake);
hbi_status recompress_lowrank(std::vector<Block> &blocks, double tol);
hbi_status ode_alloc(hbi_handle *h, int rec_cap);
hbi_status ode_rk_fixed(hbi_handle *h, const double *h_dts, int n_steps, cudaStream_t s);
hbi_status ode_adj_alloc(hbi_handle *h, int n_ckpt, int n_seg);
// ncomp component arrays of N between the caller's order and the permuted order
hbi_status ode_gather(hbi_handle *h, const double *src, int ncomp, double *dst, cudaStream_t s);
hbi_status ode_scatter(hbi_handle *h, const double *src, int ncomp, double *dst, cudaStream_t s);
hbi_status ode_adjoint(hbi_handle *h, const double *h_dts, int n_steps, int every, const double *d_target,
                       double *h_loss, double *d_state_final, cudaStream_t s);
hbi_status ode_rhs_vjp(hbi_handle *h, const double *d_v, double *d_ybar, double *d_grad_a, double *d_grad_dc,
                       cudaStream_t s);
// vec != 0: rake-free friction (state phi, tau_s, tau_d, sigma | D_s, D_d; 2-component input)
hbi_status run_steps(hbi_handle *h, const hbi_friction *f, double *d_state, double *d_t, double *d_dt, double eps_rk,
                     int n_steps, hbi_step_record *h_records, int *n_done, cudaStream_t s, int vec = 0);
hbi_status ode_set_friction(hbi_handle *h, const hbi_friction *f, cudaStream_t s);
hbi_status ode_state_in(hbi_handle *h, const double *d_state, int with_slip, cudaStream_t s, int vec = 0);
hbi_status ode_state_out(hbi_handle *h, double *d_state, cudaStream_t s, int vec = 0);
hbi_status ode_rhs(hbi_handle *h, double *d_dydt, double *d_V, cudaStream_t s);
hbi_status ode_rhs_vec(hbi_handle *h, double *d_dydt, double *d_V, cudaStream_t s);
hbi_status ode_prep(hbi_handle *h, cudaStream_t s, int vec = 0);
hbi_status ode_attempt(hbi_handle *h, cudaStream_t s, int vec = 0);
hbi_status ode_attempt_profiled(hbi_handle *h, cudaStream_t s, cudaEvent_t *ev, int *cat, int &nev);
void drop_graphs(hbi_handle *h);   // the attempt graphs, after launch shapes or baked scalars changed
hbi_status steady_state_launch(int n, const double *V, const double *a, const double *b,
                               const double *sig, double f0, double V0, double *phi, double *tau,
                               cudaStream_t s);
}  // namespace hbi
