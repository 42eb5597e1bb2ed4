// The C ABI of include/hbi.h: argument checks, handle life cycle, orchestration of the
// host set-up (tree, partition), device build (entries, ACA, packing), the HMVM and the
// adaptive Runge-Kutta loop (a captured attempt graph replayed until enough steps are
// accepted; accept/reject is decided on the device).
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstring>
#include <map>

#include "hbi_internal.h"

namespace hbi {
const char *last_error();

hbi_status upload_geometry(hbi_handle *h, const double *h_verts, const double *h_rake) {
    const int n = h->n, nv = h->nv;
    Frames F = element_frames(n, nv, h_verts);
    std::vector<double> geom(12 * (size_t)n), verts((size_t)n * nv * 3), rake(n, 0.0);
    for (int p = 0; p < n; ++p) {
        const int e = h->perm[p];
        for (int k = 0; k < 3; ++k) {
            geom[12 * (size_t)p + k] = F.c[3 * (size_t)e + k];
            geom[12 * (size_t)p + 3 + k] = F.n[3 * (size_t)e + k];
            geom[12 * (size_t)p + 6 + k] = F.s[3 * (size_t)e + k];
            geom[12 * (size_t)p + 9 + k] = F.d[3 * (size_t)e + k];
        }
        std::memcpy(&verts[(size_t)p * nv * 3], h_verts + (size_t)e * nv * 3, sizeof(double) * nv * 3);
        rake[p] = h_rake ? h_rake[e] : 0.0;
    }
    HBI_ALLOC_TRY(&h->d_geom, geom.size() * sizeof(double));
    HBI_ALLOC_TRY(&h->d_verts, verts.size() * sizeof(double));
    HBI_ALLOC_TRY(&h->d_rake, rake.size() * sizeof(double));
    HBI_ALLOC_TRY(&h->d_perm, (size_t)n * sizeof(int));
    HBI_CUDA_TRY(cudaMemcpy(h->d_geom, geom.data(), geom.size() * sizeof(double), cudaMemcpyHostToDevice));
    HBI_CUDA_TRY(cudaMemcpy(h->d_verts, verts.data(), verts.size() * sizeof(double), cudaMemcpyHostToDevice));
    HBI_CUDA_TRY(cudaMemcpy(h->d_rake, rake.data(), rake.size() * sizeof(double), cudaMemcpyHostToDevice));
    HBI_CUDA_TRY(cudaMemcpy(h->d_perm, h->perm.data(), (size_t)n * sizeof(int), cudaMemcpyHostToDevice));
    return HBI_OK;
}

namespace {
int op_nin(int op) { return (op == HBI_OP_VEC_SHEAR || op == HBI_OP_VEC_FULL) ? 2 : 1; }
int op_nout(int op) { return op == HBI_OP_RAKE_SHEAR ? 1 : (op == HBI_OP_VEC_FULL ? 3 : 2); }

hbi_status check_common(const hbi_mesh *mesh, const hbi_elastic *ek, int storage) {
    if (!mesh || !ek || !mesh->h_verts || mesh->n_elem < 1) {
        set_error("mesh, elastic constants and vertices are required; n_elem >= 1");
        return HBI_ERR_INVALID_ARG;
    }
    if (mesh->kind != HBI_RECT && mesh->kind != HBI_TRI) { set_error("kind must be HBI_RECT or HBI_TRI"); return HBI_ERR_INVALID_ARG; }
    if (ek->op < 0 || ek->op > 3) { set_error("op out of range"); return HBI_ERR_INVALID_ARG; }
    if (storage < 0 || storage > 5) { set_error("storage out of range"); return HBI_ERR_INVALID_ARG; }
    if (!(ek->mu > 0) || !(ek->nu > -1.0 && ek->nu < 0.5)) { set_error("need mu > 0 and -1 < nu < 0.5"); return HBI_ERR_INVALID_ARG; }
    if (ek->half_space != 0 && ek->half_space != 1) { set_error("half_space must be 0 or 1"); return HBI_ERR_INVALID_ARG; }
    if (ek->half_space) {
        const int nv = mesh->kind;
        for (int e = 0; e < mesh->n_elem; ++e) {
            double zc = 0.0;
            for (int a = 0; a < nv; ++a) {
                const double z = mesh->h_verts[((size_t)e * nv + a) * 3 + 2];
                if (!(z <= 0.0)) { set_error("half space: every vertex needs z <= 0"); return HBI_ERR_INVALID_ARG; }
                zc += z;
            }
            if (!(zc < 0.0)) { set_error("half space: every element centre needs z < 0"); return HBI_ERR_INVALID_ARG; }
        }
    }
    return HBI_OK;
}

hbi_status check_friction(const hbi_friction *f) {
    if (!f || !f->d_a || !f->d_b || !f->d_dc || !(f->V0 > 0) || !(f->mu > 0) || !(f->cs > 0)) {
        set_error("friction arrays a, b, dc and V0, mu, cs > 0 are required");
        return HBI_ERR_INVALID_ARG;
    }
    return HBI_OK;
}

void free_owned(std::vector<void *> &owned) {
    for (void *p : owned) cudaFree(p);
    owned.clear();
}

hbi_handle *new_handle(const hbi_mesh *mesh, const hbi_elastic *ek, int storage) {
    hbi_handle *h = new hbi_handle();
    h->n = mesh->n_elem;
    h->nv = mesh->kind;
    h->op = ek->op;
    h->nin = op_nin(ek->op);
    h->nout = op_nout(ek->op);
    h->mu = ek->mu;
    h->nu = ek->nu;
    h->half_space = ek->half_space;
    h->storage = storage;
    h->model_start = {0, h->n};
    return h;
}
}  // namespace

// The adaptive RK loop of hbi_step / hbi_step_ensemble: per-model control blocks, one captured
// attempt graph (all models advance in it, each with its own step size and decisions)
// replayed in batches until every model has n_steps accepted steps or stopped on an error.
// d_t, d_dt: n_models doubles; h_records: n_models x n_steps or NULL; n_done: n_models or NULL.
namespace {
// The captured attempt graph of the handle (fixed-rake or rake-free friction), captured once.
hbi_status ensure_graph(hbi_handle *h, int vec) {
    cudaGraphExec_t &gexec = vec ? h->graph_exec_vec : h->graph_exec;
    if (gexec) return HBI_OK;
    if (!h->cap_stream) HBI_CUDA_TRY(cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking));
    cudaGraph_t g = nullptr;
    HBI_CUDA_TRY(cudaStreamBeginCapture(h->cap_stream, cudaStreamCaptureModeThreadLocal));
    hbi_status cst = ode_attempt(h, h->cap_stream, vec);
    cudaError_t ce = cudaStreamEndCapture(h->cap_stream, &g);
    if (cst) { if (g) cudaGraphDestroy(g); return cst; }
    if (ce != cudaSuccess) { set_error(std::string("graph capture: ") + cudaGetErrorString(ce)); return HBI_ERR_CUDA; }
    ce = cudaGraphInstantiate(&gexec, g, 0);
    cudaGraphDestroy(g);
    if (ce != cudaSuccess) { set_error(std::string("graph instantiate: ") + cudaGetErrorString(ce)); return HBI_ERR_CUDA; }
    return HBI_OK;
}
}  // namespace

hbi_status run_steps(hbi_handle *h, const hbi_friction *f, double *d_state, double *d_t, double *d_dt, double eps_rk,
                     int n_steps, hbi_step_record *h_records, int *n_done, cudaStream_t s, int vec) {
    hbi_status st = check_friction(f);
    if (st) return st;
    if (h->shard_rank >= 0) {
        set_error("a shard holds part of the operator; its product is partial and does not drive the integrator");
        return HBI_ERR_INVALID_ARG;
    }
    const int nm = h->n_models;
    if ((st = ode_alloc(h, n_steps)) || (st = ode_set_friction(h, f, s)) ||
        (st = ode_state_in(h, d_state, 1, s, vec)))
        return st;
    StepCtl c0;
    std::memset(&c0, 0, sizeof c0);
    c0.eps = eps_rk;
    c0.target = n_steps;
    for (int m = 0; m < nm; ++m) {
        h->h_ctl[m] = c0;
        h->h_ctl[m].nelem = h->model_start[m + 1] - h->model_start[m];
    }
    h->h_gctl->stop = 0;
    h->h_gctl->skip0 = 0;
    h->h_gctl->commit_done = 0;
    HBI_CUDA_TRY(cudaMemcpyAsync(h->d_ctl, h->h_ctl, nm * sizeof(StepCtl), cudaMemcpyHostToDevice, s));
    HBI_CUDA_TRY(cudaMemcpyAsync(h->d_gctl, h->h_gctl, sizeof(GlobalCtl), cudaMemcpyHostToDevice, s));
    HBI_CUDA_TRY(cudaMemsetAsync(h->d_mskip, 0, 2 * (size_t)nm * sizeof(int), s));
    // t and dt of every model into its control block (strided copies)
    HBI_CUDA_TRY(cudaMemcpy2DAsync(&h->d_ctl->t, sizeof(StepCtl), d_t, sizeof(double), sizeof(double), nm,
                                   cudaMemcpyDeviceToDevice, s));
    HBI_CUDA_TRY(cudaMemcpy2DAsync(&h->d_ctl->dt, sizeof(StepCtl), d_dt, sizeof(double), sizeof(double), nm,
                                   cudaMemcpyDeviceToDevice, s));
    if ((st = ode_prep(h, s, vec))) return st;
    if ((st = ensure_graph(h, vec))) return st;
    cudaGraphExec_t &gexec = vec ? h->graph_exec_vec : h->graph_exec;
    // replay attempts until every model reports n_steps accepted steps (or stopped on an error)
    int64_t launched = 0;
    const int64_t max_attempts = 200LL * n_steps + 10000;
    int batch = n_steps;
    int batches = 0;
    for (;;) {
        for (int b = 0; b < batch; ++b) HBI_CUDA_TRY(cudaGraphLaunch(gexec, s));
        launched += batch;
        ++batches;
        // the outputs, in case this batch completed every model (rewritten after a further
        // batch; the caller's state is read only at the start), then one host round trip for
        // the control blocks and the error flag of the bounded device waits
        if ((st = ode_state_out(h, d_state, s, vec))) return st;
        HBI_CUDA_TRY(cudaMemcpy2DAsync(d_t, sizeof(double), &h->d_ctl->t, sizeof(StepCtl), sizeof(double), nm,
                                       cudaMemcpyDeviceToDevice, s));
        HBI_CUDA_TRY(cudaMemcpy2DAsync(d_dt, sizeof(double), &h->d_ctl->dt, sizeof(StepCtl), sizeof(double), nm,
                                       cudaMemcpyDeviceToDevice, s));
        HBI_CUDA_TRY(cudaMemcpyAsync(h->h_ctl, h->d_ctl, nm * sizeof(StepCtl), cudaMemcpyDeviceToHost, s));
        HBI_CUDA_TRY(cudaMemcpyAsync(h->h_gctl, h->d_gctl, sizeof(GlobalCtl), cudaMemcpyDeviceToHost, s));
        HBI_CUDA_TRY(cudaMemcpyAsync(h->h_flag, h->d_counters + 1, sizeof(int), cudaMemcpyDeviceToHost, s));
        HBI_CUDA_TRY(cudaStreamSynchronize(s));
        if (*h->h_flag) {
            HBI_CUDA_TRY(cudaMemset(h->d_counters + 1, 0, sizeof(int)));
            set_error("an HMVM stage wait timed out");
            return HBI_ERR_TIMEOUT;
        }
        if (h->h_gctl->stop) break;
        if (launched >= max_attempts) { set_error("adaptive stepping did not finish"); return HBI_ERR_TIMEOUT; }
        // the slowest active model sets the next batch: its remaining steps plus as many again
        // times its rejection rate so far (replays past its target cost ~2 us per kernel)
        double need = 2.0;
        for (int m = 0; m < nm; ++m) {
            const StepCtl &c = h->h_ctl[m];
            if (c.stop) continue;
            const double rej = launched > 0 ? std::max(0.0, (double)(launched - c.accepted) / (double)launched) : 0.0;
            const double rem = (double)(c.target - c.accepted);
            need = std::max(need, rem + std::ceil(rem * rej));
        }
        batch = (int)std::min<double>(need, (double)max_attempts);
    }
    // kernels: friction, 2 gathers, prep; per attempt 6 x ([VT], UY) (the stages run inside
    // the UY launches) and the fused commit (fixed rake) or controller + commit + stop
    // (rake-free); 2 scatters per batch
    const int per_attempt = 6 * ((h->n_tasks1 ? 1 : 0) + 1) + (vec ? 3 : 1);
    h->last_attempts = launched;
    h->last_kernels = 4 + launched * per_attempt + 2 * batches;
    hbi_status status = HBI_OK;
    for (int m = 0; m < nm; ++m) {
        const StepCtl &c = h->h_ctl[m];
        const int acc = std::min(c.accepted, n_steps);
        if (h_records && acc > 0)
            HBI_CUDA_TRY(cudaMemcpy(h_records + (size_t)m * n_steps, h->d_rec + (size_t)m * h->rec_cap,
                                    (size_t)acc * sizeof(hbi_step_record), cudaMemcpyDeviceToHost));
        if (n_done) n_done[m] = acc;
        if (!status && c.status) status = c.status;
    }
    return status;
}
}  // namespace hbi

namespace hbi {
namespace {
std::atomic<long long> g_fail_alloc{0};   // > 0: the g_fail_alloc-th allocation from now fails
std::atomic<long long> g_fail_aca{0};     // > 0: the g_fail_aca-th ACA block result from now fails
}  // namespace

hbi_status dev_malloc(void **p, size_t bytes) {
    *p = nullptr;
    long long k = g_fail_alloc.load();
    while (k > 0 && !g_fail_alloc.compare_exchange_weak(k, k - 1)) {
    }
    if (k == 1) {
        set_error("device allocation of " + std::to_string(bytes) + " bytes failed (injected)");
        return HBI_ERR_OOM;
    }
    const cudaError_t e = cudaMalloc(p, bytes);
    if (e != cudaSuccess) {
        *p = nullptr;
        cudaGetLastError();   // a failed allocation leaves the context usable
        set_error("device allocation of " + std::to_string(bytes) + " bytes failed: " + cudaGetErrorString(e));
        return HBI_ERR_OOM;
    }
    return HBI_OK;
}

bool inject_aca_failure() {
    long long k = g_fail_aca.load();
    while (k > 0 && !g_fail_aca.compare_exchange_weak(k, k - 1)) {
    }
    return k == 1;
}
}  // namespace hbi

using namespace hbi;

extern "C" {

hbi_status hbi_inject_failure(int what, long long count) {
    if (what == HBI_INJECT_NONE) {
        g_fail_alloc = 0;
        g_fail_aca = 0;
        return HBI_OK;
    }
    if (count < 0 || (what != HBI_INJECT_ALLOC && what != HBI_INJECT_ACA)) {
        set_error("what must be HBI_INJECT_NONE, _ALLOC or _ACA and count >= 0");
        return HBI_ERR_INVALID_ARG;
    }
    (what == HBI_INJECT_ALLOC ? g_fail_alloc : g_fail_aca) = count;
    return HBI_OK;
}

const char *hbi_last_error(void) { return hbi::last_error(); }

const char *hbi_status_string(hbi_status s) {
    switch (s) {
        case HBI_OK: return "HBI_OK";
        case HBI_ERR_INVALID_ARG: return "HBI_ERR_INVALID_ARG";
        case HBI_ERR_OOM: return "HBI_ERR_OOM";
        case HBI_ERR_CUDA: return "HBI_ERR_CUDA";
        case HBI_ERR_ACA_FAIL: return "HBI_ERR_ACA_FAIL";
        case HBI_ERR_DT_UNDERFLOW: return "HBI_ERR_DT_UNDERFLOW";
        case HBI_ERR_NEG_NORMAL: return "HBI_ERR_NEG_NORMAL";
        case HBI_ERR_NONFINITE: return "HBI_ERR_NONFINITE";
        case HBI_ERR_TIMEOUT: return "HBI_ERR_TIMEOUT";
        case HBI_ERR_SINGULAR: return "HBI_ERR_SINGULAR";
        default: return "HBI_ERR_UNKNOWN";
    }
}

namespace {
// hbi_build, or with p_rows > 0 the shard of rank `rank` on a p_rows x p_cols grid: only the
// blocks of the lattice blocks that rank owns are computed and packed.
hbi_status build_impl(const hbi_mesh *mesh, const hbi_elastic *ek, const hbi_build_params *bp, int p_rows, int p_cols,
                      int rank, hbi_handle **out) {
    if (!out || !bp) { set_error("out and build params are required"); return HBI_ERR_INVALID_ARG; }
    *out = nullptr;
    hbi_status st = check_common(mesh, ek, bp->storage);
    if (st) return st;
    if (bp->leaf_size < 1 || bp->lattice_depth < 0 || !(bp->aca_eps > 0) || !(bp->eta > 0) ||
        !(bp->recompress_eps >= 0)) {
        set_error("need leaf_size >= 1, lattice_depth >= 0, aca_eps > 0, eta > 0, recompress_eps >= 0");
        return HBI_ERR_INVALID_ARG;
    }
    auto t0 = std::chrono::steady_clock::now();
    hbi_handle *h = new_handle(mesh, ek, bp->storage);
    Frames F = element_frames(h->n, h->nv, mesh->h_verts);
    Tree T = build_tree(F.c, h->n, bp->leaf_size, bp->lattice_depth);
    h->perm = T.perm;
    h->n_clusters = (int64_t)T.cl.size();
    h->n_leaves = (int64_t)T.leaves.size();
    h->n_lattice = (int64_t)T.lattice.size();
    std::vector<int> ij;
    std::vector<Block> blocks = build_partition(T, h->nin, h->nout, bp->eta, p_rows > 0 ? &ij : nullptr);
    if (p_rows > 0) {
        // the 2D-cyclic owner of lattice block (I, J) is rank (I mod p_rows) p_cols + J mod p_cols
        std::vector<Block> mine;
        for (size_t b = 0; b < blocks.size(); ++b)
            if ((ij[2 * b] % p_rows) * p_cols + ij[2 * b + 1] % p_cols == rank) mine.push_back(blocks[b]);
        blocks.swap(mine);
        h->shard_rank = rank;
        h->shard_rows = p_rows;
        h->shard_cols = p_cols;
    }
    std::vector<void *> owned;
    if ((st = upload_geometry(h, mesh->h_verts, mesh->h_rake)) ||
        (!blocks.empty() && (st = device_build_factors(h, T, blocks, bp->aca_eps, owned)))) {
        free_owned(owned);
        hbi_destroy(h);
        return st;
    }
    if (!blocks.empty() && bp->recompress_eps > 0 && (st = recompress_lowrank(blocks, bp->recompress_eps))) {
        free_owned(owned);
        hbi_destroy(h);
        return st;
    }
    std::vector<int> leaf_starts;
    for (int c : T.leaves) leaf_starts.push_back(T.cl[c].start);
    leaf_starts.push_back(h->n);
    st = pack_operators(h, blocks, leaf_starts, bp->with_transpose, bp->multi_rhs);
    free_owned(owned);
    if (st) { hbi_destroy(h); return st; }
    h->build_seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    *out = h;
    return HBI_OK;
}
}  // namespace

hbi_status hbi_build_shard(const hbi_mesh *mesh, const hbi_elastic *ek, const hbi_build_params *bp, int p_rows,
                           int p_cols, int rank, hbi_handle **out) {
    if (out) *out = nullptr;
    if (p_rows < 1 || p_cols < 1 || rank < 0 || rank >= p_rows * p_cols) {
        set_error("need a process grid of at least 1 x 1 and 0 <= rank < p_rows p_cols");
        return HBI_ERR_INVALID_ARG;
    }
    return build_impl(mesh, ek, bp, p_rows, p_cols, rank, out);
}

hbi_status hbi_build(const hbi_mesh *mesh, const hbi_elastic *ek, const hbi_build_params *bp, hbi_handle **out) {
    return build_impl(mesh, ek, bp, 0, 0, 0, out);
}

hbi_status hbi_build_ensemble(int n_models, const hbi_mesh *meshes, const hbi_elastic *ek,
                              const hbi_build_params *bp, hbi_handle **out) {
    if (!out || !bp || !meshes || n_models < 1) {
        set_error("out, build params, meshes and n_models >= 1 are required");
        return HBI_ERR_INVALID_ARG;
    }
    *out = nullptr;
    int64_t ntot = 0;
    for (int m = 0; m < n_models; ++m) {
        hbi_status st = check_common(&meshes[m], ek, bp->storage);
        if (st) return st;
        ntot += meshes[m].n_elem;
    }
    if (bp->leaf_size < 1 || bp->lattice_depth < 0 || !(bp->aca_eps > 0) || !(bp->eta > 0) ||
        !(bp->recompress_eps >= 0)) {
        set_error("need leaf_size >= 1, lattice_depth >= 0, aca_eps > 0, eta > 0, recompress_eps >= 0");
        return HBI_ERR_INVALID_ARG;
    }
    if (ntot > (int64_t)INT32_MAX / 4) { set_error("ensemble too large"); return HBI_ERR_INVALID_ARG; }
    auto t0 = std::chrono::steady_clock::now();
    hbi_mesh all = meshes[0];
    all.n_elem = (int)ntot;
    hbi_handle *h = new_handle(&all, ek, bp->storage);
    h->n_models = n_models;
    h->model_start.assign(1, 0);
    std::vector<Block> blocks;
    std::vector<int> leaf_starts;
    std::vector<void *> owned;
    hbi_status st = HBI_OK;
    int e0 = 0;
    h->perm.clear();
    // every model: its own tree, partition and ACA (entries from its own geometry); the
    // ensemble operator is block diagonal over the models, element ranges concatenated
    for (int m = 0; m < n_models && !st; ++m) {
        hbi_handle *hm = new_handle(&meshes[m], ek, bp->storage);
        Frames F = element_frames(hm->n, hm->nv, meshes[m].h_verts);
        Tree T = build_tree(F.c, hm->n, bp->leaf_size, bp->lattice_depth);
        hm->perm = T.perm;
        std::vector<Block> bm = build_partition(T, hm->nin, hm->nout, bp->eta);
        if ((st = upload_geometry(hm, meshes[m].h_verts, meshes[m].h_rake)) ||
            (st = device_build_factors(hm, T, bm, bp->aca_eps, owned))) {
            hbi_destroy(hm);
            break;
        }
        hbi_destroy(hm);   // geometry only; the factors live in `owned`
        for (Block B : bm) {
            B.tau = B.sig = -1;
            B.row0 += (int64_t)h->nout * e0;
            B.col0 += (int64_t)h->nin * e0;
            blocks.push_back(B);
        }
        for (int c : T.leaves) leaf_starts.push_back(e0 + T.cl[c].start);
        for (int p : T.perm) h->perm.push_back(e0 + p);
        h->n_clusters += (int64_t)T.cl.size();
        h->n_leaves += (int64_t)T.leaves.size();
        h->n_lattice += (int64_t)T.lattice.size();
        e0 += meshes[m].n_elem;
        h->model_start.push_back(e0);
    }
    leaf_starts.push_back(h->n);
    if (!st && bp->recompress_eps > 0) st = recompress_lowrank(blocks, bp->recompress_eps);
    if (!st) {
        st = dev_malloc((void **)&h->d_perm, (size_t)h->n * sizeof(int));
        if (!st) {
            cudaError_t e = cudaMemcpy(h->d_perm, h->perm.data(), (size_t)h->n * sizeof(int), cudaMemcpyHostToDevice);
            if (e != cudaSuccess) { set_error(std::string("ensemble permutation: ") + cudaGetErrorString(e)); st = HBI_ERR_CUDA; }
        }
    }
    if (!st) st = pack_operators(h, blocks, leaf_starts, bp->with_transpose, bp->multi_rhs);
    free_owned(owned);
    if (st) { hbi_destroy(h); return st; }
    h->build_seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    *out = h;
    return HBI_OK;
}

hbi_status hbi_plan(const hbi_mesh *mesh, const hbi_elastic *ek, const hbi_build_params *bp, int *h_perm,
                    int *h_leaf_starts, int *n_leaves, int64_t *h_blocks, int max_blocks, int *n_blocks) {
    if (!bp || !h_perm || !h_leaf_starts || !n_leaves || !n_blocks) {
        set_error("params, perm, leaf starts and counts are required");
        return HBI_ERR_INVALID_ARG;
    }
    hbi_status st = check_common(mesh, ek, bp->storage);
    if (st) return st;
    if (bp->leaf_size < 1 || bp->lattice_depth < 0 || !(bp->eta > 0)) {
        set_error("need leaf_size >= 1, lattice_depth >= 0, eta > 0");
        return HBI_ERR_INVALID_ARG;
    }
    const int n = mesh->n_elem;
    Frames F = element_frames(n, mesh->kind, mesh->h_verts);
    Tree T = build_tree(F.c, n, bp->leaf_size, bp->lattice_depth);
    std::vector<Block> blocks = build_partition(T, op_nin(ek->op), op_nout(ek->op), bp->eta);
    std::copy(T.perm.begin(), T.perm.end(), h_perm);
    *n_leaves = (int)T.leaves.size();
    for (size_t u = 0; u < T.leaves.size(); ++u) h_leaf_starts[u] = T.cl[T.leaves[u]].start;
    h_leaf_starts[T.leaves.size()] = n;
    *n_blocks = (int)blocks.size();
    if (h_blocks) {
        if ((int)blocks.size() > max_blocks) { set_error("max_blocks too small"); return HBI_ERR_INVALID_ARG; }
        for (size_t b = 0; b < blocks.size(); ++b) {
            int64_t *o = h_blocks + 6 * b;
            o[0] = blocks[b].row0; o[1] = blocks[b].m; o[2] = blocks[b].col0; o[3] = blocks[b].nc;
            o[4] = blocks[b].lowrank; o[5] = 0;
        }
    }
    return HBI_OK;
}

hbi_status hbi_lattice_owners(const hbi_mesh *mesh, const hbi_elastic *ek, const hbi_build_params *bp, int p_rows,
                              int p_cols, int *h_owner, int max_blocks, int *n_blocks) {
    if (!bp || !n_blocks || p_rows < 1 || p_cols < 1) {
        set_error("params, block count and a process grid of at least 1 x 1 are required");
        return HBI_ERR_INVALID_ARG;
    }
    hbi_status st = check_common(mesh, ek, bp->storage);
    if (st) return st;
    if (bp->leaf_size < 1 || bp->lattice_depth < 0 || !(bp->eta > 0)) {
        set_error("need leaf_size >= 1, lattice_depth >= 0, eta > 0");
        return HBI_ERR_INVALID_ARG;
    }
    const int n = mesh->n_elem;
    Frames F = element_frames(n, mesh->kind, mesh->h_verts);
    Tree T = build_tree(F.c, n, bp->leaf_size, bp->lattice_depth);
    std::vector<int> ij;
    std::vector<Block> blocks = build_partition(T, op_nin(ek->op), op_nout(ek->op), bp->eta, &ij);
    *n_blocks = (int)blocks.size();
    if (h_owner) {
        if ((int)blocks.size() > max_blocks) { set_error("max_blocks too small"); return HBI_ERR_INVALID_ARG; }
        for (size_t b = 0; b < blocks.size(); ++b)
            h_owner[b] = (ij[2 * b] % p_rows) * p_cols + ij[2 * b + 1] % p_cols;
    }
    return HBI_OK;
}

hbi_status hbi_build_from_factors(const hbi_mesh *mesh, const hbi_elastic *ek, int storage, const int *h_perm,
                                  int n_blocks, const int64_t *h_blocks, const int64_t *h_offsets,
                                  const double *h_data, int n_leaves, const int *h_leaf_starts, int with_transpose,
                                  hbi_handle **out) {
    if (!out) { set_error("out is required"); return HBI_ERR_INVALID_ARG; }
    *out = nullptr;
    hbi_status st = check_common(mesh, ek, storage);
    if (st) return st;
    if (!h_perm || n_blocks < 1 || !h_blocks || !h_offsets || !h_data || n_leaves < 1 || !h_leaf_starts) {
        set_error("perm, blocks, offsets, data and leaf starts are required");
        return HBI_ERR_INVALID_ARG;
    }
    const int n = mesh->n_elem;
    hbi_handle *h = new_handle(mesh, ek, storage);
    const int nin = h->nin, nout = h->nout;
    // permutation
    std::vector<char> seen(n, 0);
    for (int p = 0; p < n; ++p) {
        if (h_perm[p] < 0 || h_perm[p] >= n || seen[h_perm[p]]) {
            set_error("perm is not a permutation");
            hbi_destroy(h);
            return HBI_ERR_INVALID_ARG;
        }
        seen[h_perm[p]] = 1;
    }
    h->perm.assign(h_perm, h_perm + n);
    std::vector<int> leaf_starts(h_leaf_starts, h_leaf_starts + n_leaves + 1);
    if (leaf_starts.front() != 0 || leaf_starts.back() != n) {
        set_error("leaf starts must run from 0 to n_elem");
        hbi_destroy(h);
        return HBI_ERR_INVALID_ARG;
    }
    for (int u = 0; u < n_leaves; ++u)
        if (leaf_starts[u + 1] <= leaf_starts[u]) {
            set_error("leaf starts must increase");
            hbi_destroy(h);
            return HBI_ERR_INVALID_ARG;
        }
    std::vector<int> is_start(n + 1, 0);
    for (int u = 0; u <= n_leaves; ++u) is_start[leaf_starts[u]] = 1;
    // blocks: bounds, leaf alignment and an exact tiling (per leaf unit, column ranges tile)
    int64_t total = 0;
    std::vector<Block> blocks(n_blocks);
    std::vector<std::vector<std::pair<int64_t, int64_t>>> unit_cols(n_leaves);
    std::vector<int> leaf_of(n + 1, 0);
    for (int u = 0; u < n_leaves; ++u)
        for (int e = leaf_starts[u]; e < leaf_starts[u + 1]; ++e) leaf_of[e] = u;
    for (int b = 0; b < n_blocks; ++b) {
        const int64_t *q = h_blocks + 6 * (size_t)b;
        Block B{-1, -1, q[0], q[1], q[2], q[3], (int)q[4], (int)q[5], nullptr, nullptr};
        bool ok = B.m > 0 && B.nc > 0 && B.row0 >= 0 && B.col0 >= 0 && B.row0 % nout == 0 && B.m % nout == 0 &&
                  B.col0 % nin == 0 && B.nc % nin == 0 && B.row0 + B.m <= (int64_t)nout * n &&
                  B.col0 + B.nc <= (int64_t)nin * n && (B.lowrank == 0 || B.lowrank == 1) && B.rank >= 0 &&
                  h_offsets[b] >= 0;
        if (ok) ok = is_start[B.row0 / nout] && is_start[(B.row0 + B.m) / nout];
        if (!ok) {
            set_error("block " + std::to_string(b) + " is out of range or not aligned to leaf clusters");
            hbi_destroy(h);
            return HBI_ERR_INVALID_ARG;
        }
        for (int u = leaf_of[B.row0 / nout]; u < n_leaves && leaf_starts[u] < (B.row0 + B.m) / nout; ++u)
            unit_cols[u].push_back({B.col0, B.col0 + B.nc});
        total = std::max<int64_t>(total, h_offsets[b] + (B.lowrank ? (B.m + B.nc) * B.rank : B.m * B.nc));
        blocks[b] = B;
    }
    for (int u = 0; u < n_leaves; ++u) {
        auto &v = unit_cols[u];
        std::sort(v.begin(), v.end());
        int64_t pos = 0;
        for (auto &pr : v) {
            if (pr.first != pos) {
                set_error("blocks do not tile the matrix exactly once");
                hbi_destroy(h);
                return HBI_ERR_INVALID_ARG;
            }
            pos = pr.second;
        }
        if (pos != (int64_t)nin * n) {
            set_error("blocks do not tile the matrix exactly once");
            hbi_destroy(h);
            return HBI_ERR_INVALID_ARG;
        }
    }
    double *d_data = nullptr;
    if ((st = dev_malloc((void **)&d_data, std::max<int64_t>(1, total) * sizeof(double)))) {
        hbi_destroy(h);
        return st;
    }
    if (cudaMemcpy(d_data, h_data, total * sizeof(double), cudaMemcpyHostToDevice) != cudaSuccess) {
        cudaFree(d_data);
        set_error("copy of the imported factors failed");
        hbi_destroy(h);
        return HBI_ERR_CUDA;
    }
    for (int b = 0; b < n_blocks; ++b) {
        Block &B = blocks[b];
        B.d_src = d_data + h_offsets[b];
        B.d_src2 = B.lowrank ? d_data + h_offsets[b] + B.m * B.rank : nullptr;
    }
    st = upload_geometry(h, mesh->h_verts, mesh->h_rake);
    if (!st) st = pack_operators(h, blocks, leaf_starts, with_transpose);
    cudaFree(d_data);
    if (st) { hbi_destroy(h); return st; }
    h->n_leaves = n_leaves;
    *out = h;
    return HBI_OK;
}

hbi_status hbi_matvec_async(hbi_handle *h, const double *d_x, double *d_y, hbi_stream stream) {
    if (!h || !d_x || !d_y) { set_error("handle, x and y are required"); return HBI_ERR_INVALID_ARG; }
    cudaStream_t s = (cudaStream_t)stream;
    hbi_status st = permute_x_in(h, d_x, s);
    if (!st) st = hmvm_launch(h, s, nullptr);
    if (!st) st = permute_y_out(h, d_y, s);
    return st;
}

hbi_status hbi_matvec(hbi_handle *h, const double *d_x, double *d_y, hbi_stream stream) {
    hbi_status st = hbi_matvec_async(h, d_x, d_y, stream);
    if (st) return st;
    HBI_CUDA_TRY(cudaStreamSynchronize((cudaStream_t)stream));
    return hmvm_check(h);
}

hbi_status hbi_matvec_transpose(hbi_handle *h, const double *d_v, double *d_w, hbi_stream stream) {
    if (!h || !d_v || !d_w) { set_error("handle, v and w are required"); return HBI_ERR_INVALID_ARG; }
    if (!h->adj) { set_error("the handle was built without with_transpose"); return HBI_ERR_INVALID_ARG; }
    return hbi_matvec(h->adj, d_v, d_w, stream);
}

hbi_status hbi_steady_state(int n, const double *d_V, const double *d_a, const double *d_b, const double *d_sigma,
                            double f0, double V0, double *d_phi, double *d_tau, hbi_stream stream) {
    if (n < 1 || !d_V || !d_a || !d_b || !d_sigma || !d_phi || !d_tau || !(V0 > 0)) {
        set_error("n >= 1, all arrays and V0 > 0 are required");
        return HBI_ERR_INVALID_ARG;
    }
    hbi_status st = steady_state_launch(n, d_V, d_a, d_b, d_sigma, f0, V0, d_phi, d_tau, (cudaStream_t)stream);
    if (st) return st;
    HBI_CUDA_TRY(cudaStreamSynchronize((cudaStream_t)stream));
    return HBI_OK;
}


hbi_status hbi_rhs(hbi_handle *h, const hbi_friction *f, const double *d_state, double *d_dydt, double *d_V,
                   hbi_stream stream) {
    if (!h || !d_state || !d_dydt) { set_error("handle, state and dydt are required"); return HBI_ERR_INVALID_ARG; }
    hbi_status st = check_friction(f);
    if (st) return st;
    if (h->shard_rank >= 0) {
        set_error("a shard holds part of the operator; its product is partial and does not drive the integrator");
        return HBI_ERR_INVALID_ARG;
    }
    cudaStream_t s = (cudaStream_t)stream;
    if ((st = ode_alloc(h, 1)) || (st = ode_set_friction(h, f, s)) || (st = ode_state_in(h, d_state, 0, s)) ||
        (st = ode_rhs(h, d_dydt, d_V, s)))
        return st;
    HBI_CUDA_TRY(cudaStreamSynchronize(s));
    return hmvm_check(h);
}

hbi_status hbi_step(hbi_handle *h, const hbi_friction *f, double *d_state, double *d_t, double *d_dt, double eps_rk,
                    int n_steps, hbi_step_record *h_records, int *n_done, hbi_stream stream) {
    if (n_done) *n_done = 0;
    if (!h || !d_state || !d_t || !d_dt || n_steps < 1 || !(eps_rk > 0)) {
        set_error("handle, state, t, dt, n_steps >= 1 and eps_rk > 0 are required");
        return HBI_ERR_INVALID_ARG;
    }
    if (h->n_models != 1) {
        set_error("an ensemble handle steps with hbi_step_ensemble");
        return HBI_ERR_INVALID_ARG;
    }
    return run_steps(h, f, d_state, d_t, d_dt, eps_rk, n_steps, h_records, n_done, (cudaStream_t)stream);
}

hbi_status hbi_time_attempts(hbi_handle *h, const hbi_friction *f, const double *d_state, const double *d_t,
                             const double *d_dt, double eps_rk, int n_attempts, double *out8, hbi_stream stream) {
    if (!h || !d_state || !d_t || !d_dt || !out8 || n_attempts < 1 || !(eps_rk > 0)) {
        set_error("handle, state, t, dt, out8, n_attempts >= 1 and eps_rk > 0 are required");
        return HBI_ERR_INVALID_ARG;
    }
    if (h->n_models != 1) { set_error("single-model handles only"); return HBI_ERR_INVALID_ARG; }
    hbi_status st = check_friction(f);
    if (st) return st;
    if (h->shard_rank >= 0) {
        set_error("a shard holds part of the operator; its product is partial and does not drive the integrator");
        return HBI_ERR_INVALID_ARG;
    }
    cudaStream_t s = (cudaStream_t)stream;
    // the internal state from the caller's (the caller's arrays are not written)
    if ((st = ode_alloc(h, 1)) || (st = ode_set_friction(h, f, s)) ||
        (st = ode_state_in(h, d_state, 1, s, 0)))
        return st;
    StepCtl c0;
    std::memset(&c0, 0, sizeof c0);
    c0.eps = eps_rk;
    c0.target = 1 << 30;   // nothing stops
    c0.nelem = h->n;
    *h->h_ctl = c0;
    h->h_gctl->stop = 0;
    h->h_gctl->skip0 = 0;
    h->h_gctl->commit_done = 0;
    HBI_CUDA_TRY(cudaMemcpyAsync(h->d_ctl, h->h_ctl, sizeof(StepCtl), cudaMemcpyHostToDevice, s));
    HBI_CUDA_TRY(cudaMemcpyAsync(h->d_gctl, h->h_gctl, sizeof(GlobalCtl), cudaMemcpyHostToDevice, s));
    HBI_CUDA_TRY(cudaMemsetAsync(h->d_mskip, 0, 2 * sizeof(int), s));
    HBI_CUDA_TRY(cudaMemcpyAsync(&h->d_ctl->t, d_t, sizeof(double), cudaMemcpyDeviceToDevice, s));
    HBI_CUDA_TRY(cudaMemcpyAsync(&h->d_ctl->dt, d_dt, sizeof(double), cudaMemcpyDeviceToDevice, s));
    if ((st = ode_prep(h, s, 0)) || (st = ensure_graph(h, 0))) return st;
    cudaEvent_t ev[32];
    int cat[32];
    for (auto &e : ev) HBI_CUDA_TRY(cudaEventCreate(&e));
    double acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    for (int a = 0; a < n_attempts && !st; ++a) {
        int nev = 0;
        st = ode_attempt_profiled(h, s, ev, cat, nev);
        if (st) break;
        HBI_CUDA_TRY(cudaEventSynchronize(ev[nev - 1]));
        for (int k = 0; k + 1 < nev; ++k) {
            float ms = 0;
            HBI_CUDA_TRY(cudaEventElapsedTime(&ms, ev[k], ev[k + 1]));
            acc[cat[k]] += ms;
            acc[6] += ms;
        }
    }
    // the same number of attempts as graph replays
    if (!st) {
        HBI_CUDA_TRY(cudaEventRecord(ev[0], s));
        for (int a = 0; a < n_attempts; ++a) HBI_CUDA_TRY(cudaGraphLaunch(h->graph_exec, s));
        HBI_CUDA_TRY(cudaEventRecord(ev[1], s));
        HBI_CUDA_TRY(cudaEventSynchronize(ev[1]));
        float ms = 0;
        HBI_CUDA_TRY(cudaEventElapsedTime(&ms, ev[0], ev[1]));
        acc[7] = ms;
    }
    for (auto &e : ev) cudaEventDestroy(e);
    if (st || (st = hmvm_check(h))) return st;
    for (int k = 0; k < 8; ++k) out8[k] = acc[k] / n_attempts;
    return HBI_OK;
}

hbi_status hbi_step_ensemble(hbi_handle *h, const hbi_friction *f, double *d_state, double *d_t, double *d_dt,
                             double eps_rk, int n_steps, hbi_step_record *h_records, int *h_n_done,
                             hbi_stream stream) {
    if (!h || !d_state || !d_t || !d_dt || n_steps < 1 || !(eps_rk > 0) || !h_n_done) {
        set_error("handle, state, t, dt, n_done, n_steps >= 1 and eps_rk > 0 are required");
        return HBI_ERR_INVALID_ARG;
    }
    for (int m = 0; m < h->n_models; ++m) h_n_done[m] = 0;
    return run_steps(h, f, d_state, d_t, d_dt, eps_rk, n_steps, h_records, h_n_done, (cudaStream_t)stream);
}

hbi_status hbi_rhs_vec(hbi_handle *h, const hbi_friction *f, const double *d_state, double *d_dydt, double *d_V,
                       hbi_stream stream) {
    if (!h || !d_state || !d_dydt) { set_error("handle, state and dydt are required"); return HBI_ERR_INVALID_ARG; }
    if (h->nin != 2) { set_error("rake-free friction needs a two-component operator"); return HBI_ERR_INVALID_ARG; }
    hbi_status st = check_friction(f);
    if (st) return st;
    if (h->shard_rank >= 0) {
        set_error("a shard holds part of the operator; its product is partial and does not drive the integrator");
        return HBI_ERR_INVALID_ARG;
    }
    cudaStream_t s = (cudaStream_t)stream;
    if ((st = ode_alloc(h, 1)) || (st = ode_set_friction(h, f, s)) || (st = ode_state_in(h, d_state, 0, s, 1)) ||
        (st = ode_rhs_vec(h, d_dydt, d_V, s)))
        return st;
    HBI_CUDA_TRY(cudaStreamSynchronize(s));
    return hmvm_check(h);
}

hbi_status hbi_step_vector(hbi_handle *h, const hbi_friction *f, double *d_state, double *d_t, double *d_dt,
                           double eps_rk, int n_steps, hbi_step_record *h_records, int *h_n_done,
                           hbi_stream stream) {
    if (!h || !d_state || !d_t || !d_dt || n_steps < 1 || !(eps_rk > 0) || !h_n_done) {
        set_error("handle, state, t, dt, n_done, n_steps >= 1 and eps_rk > 0 are required");
        return HBI_ERR_INVALID_ARG;
    }
    for (int m = 0; m < h->n_models; ++m) h_n_done[m] = 0;
    if (h->nin != 2) { set_error("rake-free friction needs a two-component operator"); return HBI_ERR_INVALID_ARG; }
    return run_steps(h, f, d_state, d_t, d_dt, eps_rk, n_steps, h_records, h_n_done, (cudaStream_t)stream, 1);
}

hbi_status hbi_rhs_vjp(hbi_handle *h, const hbi_friction *f, const double *d_state, const double *d_v, double *d_ybar,
                       double *d_grad_a, double *d_grad_dc, hbi_stream stream) {
    if (!h || !d_state || !d_v || !d_ybar) { set_error("handle, state, v and ybar are required"); return HBI_ERR_INVALID_ARG; }
    if (!h->adj) { set_error("the handle was built without with_transpose"); return HBI_ERR_INVALID_ARG; }
    hbi_status st = check_friction(f);
    if (st) return st;
    if (h->shard_rank >= 0) {
        set_error("a shard holds part of the operator; its product is partial and does not drive the integrator");
        return HBI_ERR_INVALID_ARG;
    }
    cudaStream_t s = (cudaStream_t)stream;
    if ((st = ode_alloc(h, 1)) || (st = ode_set_friction(h, f, s)) || (st = ode_state_in(h, d_state, 0, s)) ||
        (st = ode_rhs_vjp(h, d_v, d_ybar, d_grad_a, d_grad_dc, s)))
        return st;
    HBI_CUDA_TRY(cudaStreamSynchronize(s));
    if ((st = hmvm_check(h))) return st;
    return hmvm_check(h->adj);
}

hbi_status hbi_rk_fixed(hbi_handle *h, const hbi_friction *f, double *d_state, const double *h_dts, int n_steps,
                        hbi_stream stream) {
    if (!h || !d_state || !h_dts || n_steps < 1) {
        set_error("handle, state, step sizes and n_steps >= 1 are required");
        return HBI_ERR_INVALID_ARG;
    }
    if (h->n_models != 1) { set_error("fixed steps need a single-model handle"); return HBI_ERR_INVALID_ARG; }
    for (int k = 0; k < n_steps; ++k)
        if (!(h_dts[k] > 0)) { set_error("step sizes must be > 0"); return HBI_ERR_INVALID_ARG; }
    hbi_status st = check_friction(f);
    if (st) return st;
    if (h->shard_rank >= 0) {
        set_error("a shard holds part of the operator; its product is partial and does not drive the integrator");
        return HBI_ERR_INVALID_ARG;
    }
    cudaStream_t s = (cudaStream_t)stream;
    if ((st = ode_alloc(h, 1)) || (st = ode_set_friction(h, f, s)) || (st = ode_state_in(h, d_state, 1, s)) ||
        (st = ode_rk_fixed(h, h_dts, n_steps, s)) || (st = ode_state_out(h, d_state, s)))
        return st;
    HBI_CUDA_TRY(cudaStreamSynchronize(s));
    return hmvm_check(h);
}

hbi_status hbi_adjoint(hbi_handle *h, const hbi_friction *f, const double *d_state0, const double *h_dts, int n_steps,
                       int checkpoint_every, const double *d_target, double *h_loss, double *d_grad_amb,
                       double *d_grad_dc, double *d_state_final, hbi_stream stream) {
    if (!h || !d_state0 || !h_dts || n_steps < 1 || checkpoint_every < 1 || !d_target || !d_grad_amb || !d_grad_dc) {
        set_error("handle, state, step sizes, target, gradients, n_steps >= 1, checkpoint_every >= 1 are required");
        return HBI_ERR_INVALID_ARG;
    }
    if (h->n_models != 1) { set_error("the adjoint needs a single-model handle"); return HBI_ERR_INVALID_ARG; }
    if (!h->adj) { set_error("the handle was built without with_transpose"); return HBI_ERR_INVALID_ARG; }
    for (int k = 0; k < n_steps; ++k)
        if (!(h_dts[k] > 0)) { set_error("step sizes must be > 0"); return HBI_ERR_INVALID_ARG; }
    hbi_status st = check_friction(f);
    if (st) return st;
    if (h->shard_rank >= 0) {
        set_error("a shard holds part of the operator; its product is partial and does not drive the integrator");
        return HBI_ERR_INVALID_ARG;
    }
    cudaStream_t s = (cudaStream_t)stream;
    if ((st = ode_alloc(h, 1)) || (st = ode_set_friction(h, f, s)) || (st = ode_state_in(h, d_state0, 1, s)))
        return st;
    // the target into the permuted order (the adjoint's auxiliary array)
    const int nseg = (n_steps + checkpoint_every - 1) / checkpoint_every;
    if ((st = ode_adj_alloc(h, nseg, checkpoint_every)) || (st = ode_gather(h, d_target, 1, h->d_aux, s))) return st;
    if ((st = ode_adjoint(h, h_dts, n_steps, checkpoint_every, h->d_aux, h_loss, d_state_final, s))) return st;
    if ((st = ode_scatter(h, h->d_gA, 1, d_grad_amb, s)) || (st = ode_scatter(h, h->d_gDC, 1, d_grad_dc, s))) return st;
    HBI_CUDA_TRY(cudaStreamSynchronize(s));
    if ((st = hmvm_check(h))) return st;
    return hmvm_check(h->adj);
}

hbi_status hbi_stats(const hbi_handle *h, hbi_stats_t *o) {
    if (!h || !o) { set_error("handle and output are required"); return HBI_ERR_INVALID_ARG; }
    std::memset(o, 0, sizeof *o);
    o->n_elem = h->n; o->n_in = h->nin; o->n_out = h->nout;
    o->n_clusters = h->n_clusters; o->n_leaves = h->n_leaves; o->n_lattice = h->n_lattice;
    o->n_blocks = h->n_blocks; o->n_lowrank = h->n_lowrank; o->n_dense = h->n_dense;
    o->max_rank = h->max_rank; o->mean_rank = h->mean_rank;
    o->entries_lowrank = h->entries_lr; o->entries_dense = h->entries_dense;
    o->bytes_factors = h->bytes_factors; o->bytes_algorithmic = h->bytes_algorithmic;
    o->n_tasks_vt = h->n_tasks1; o->n_tasks_uy = h->n_tasks2;
    o->storage = h->storage;
    o->build_seconds = h->build_seconds;
    o->bytes_alg_vt = h->bytes_alg_vt;
    o->bytes_alg_uy = h->bytes_alg_uy;
    o->last_step_attempts = h->last_attempts;
    o->last_step_kernels = h->last_kernels;
    o->n_models = h->n_models;
    return HBI_OK;
}

hbi_status hbi_time_hmvm(hbi_handle *h, int n_rep, double *out4, hbi_stream stream) {
    if (!h || !out4 || n_rep < 1) { set_error("handle, output and n_rep >= 1 are required"); return HBI_ERR_INVALID_ARG; }
    cudaStream_t s = (cudaStream_t)stream;
    cudaEvent_t ev[4];
    for (auto &e : ev) HBI_CUDA_TRY(cudaEventCreate(&e));
    double acc[3] = {0, 0, 0}, whole = 0;
    hbi_status st = HBI_OK;
    for (int r = 0; r < n_rep && !st; ++r) {
        HBI_CUDA_TRY(cudaEventRecord(ev[0], s));
        for (int ph = 0; ph < 3 && !st; ++ph) {
            st = hmvm_phase(h, ph, s, nullptr);
            HBI_CUDA_TRY(cudaEventRecord(ev[ph + 1], s));
        }
        HBI_CUDA_TRY(cudaEventSynchronize(ev[3]));
        float ms;
        for (int ph = 0; ph < 3; ++ph) {
            HBI_CUDA_TRY(cudaEventElapsedTime(&ms, ev[ph], ev[ph + 1]));
            acc[ph] += ms;
        }
    }
    // the whole product as hbi_matvec and hbi_step launch it
    for (int r = 0; r < n_rep && !st; ++r) {
        HBI_CUDA_TRY(cudaEventRecord(ev[0], s));
        st = hmvm_phase(h, -1, s, nullptr);
        HBI_CUDA_TRY(cudaEventRecord(ev[1], s));
        HBI_CUDA_TRY(cudaEventSynchronize(ev[1]));
        float ms;
        HBI_CUDA_TRY(cudaEventElapsedTime(&ms, ev[0], ev[1]));
        whole += ms;
    }
    for (auto &e : ev) cudaEventDestroy(e);
    if (st || (st = hmvm_check(h))) return st;
    for (int ph = 0; ph < 3; ++ph) out4[ph] = acc[ph] / n_rep;
    out4[3] = whole / n_rep;
    return HBI_OK;
}

hbi_status hbi_autotune(hbi_handle *h, int n_rep, int *out3, double *out_ms, hbi_stream stream) {
    if (!h || n_rep < 1) { set_error("handle and n_rep >= 1 are required"); return HBI_ERR_INVALID_ARG; }
    cudaStream_t s = (cudaStream_t)stream;
    cudaEvent_t e0, e1;
    HBI_CUDA_TRY(cudaEventCreate(&e0));
    HBI_CUDA_TRY(cudaEventCreate(&e1));
    hbi_status st = HBI_OK;
    // average device time of n_rep back-to-back launches of one phase (after one warm-up)
    auto time_phase = [&](int phase, double &ms_out) -> hbi_status {
        hbi_status r = hmvm_phase(h, phase, s, nullptr);
        if (r) return r;
        HBI_CUDA_TRY(cudaEventRecord(e0, s));
        for (int k = 0; k < n_rep && !r; ++k) r = hmvm_phase(h, phase, s, nullptr);
        HBI_CUDA_TRY(cudaEventRecord(e1, s));
        HBI_CUDA_TRY(cudaEventSynchronize(e1));
        float ms = 0.0f;
        HBI_CUDA_TRY(cudaEventElapsedTime(&ms, e0, e1));
        ms_out = ms / n_rep;
        return r;
    };
    double best_vt = 1e300, best_uy = 1e300, t = 0.0;
    int best_cost = h->vt_pass_cost, best_rpw = h->uy_rpw, best_per_sm = h->uy_ctas_per_sm;
    // V^T phase: the per-pass cost of its per-item shape choice
    if (h->n_tasks1) {
        const int costs[3] = {4, 8, 16};
        for (int c : costs) {
            h->vt_pass_cost = c;
            if ((st = time_phase(0, t))) break;
            if (t < best_vt) { best_vt = t; best_cost = c; }
        }
    } else {
        best_vt = 0.0;
    }
    // UY phase: rows per pass and CTAs per SM
    for (int v = 0; v < 2 && !st; ++v) {
        h->uy_rpw = v ? 8 : 4;
        const int occ = h->uy_occ[v];
        for (int per_sm = occ; per_sm >= std::max(1, occ - 2) && !st; --per_sm) {
            set_uy_grid(h, per_sm);
            if ((st = time_phase(2, t))) break;
            if (t < best_uy) { best_uy = t; best_rpw = h->uy_rpw; best_per_sm = per_sm; }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    h->vt_pass_cost = best_cost;
    h->uy_rpw = best_rpw;
    set_uy_grid(h, best_per_sm);
    drop_graphs(h);   // launch shapes changed
    if (st || (st = hmvm_check(h))) return st;
    if (out3) { out3[0] = h->uy_rpw; out3[1] = h->uy_ctas_per_sm; out3[2] = h->vt_pass_cost; }
    if (out_ms) *out_ms = best_vt + best_uy;
    // the transposed operator of the adjoint has its own blocks and launch shapes
    if (h->adj) return hbi_autotune(h->adj, n_rep, nullptr, nullptr, stream);
    return HBI_OK;
}

hbi_status hbi_stalled_wait_status(hbi_stream stream) { return stalled_wait_status((cudaStream_t)stream); }

void hbi_destroy(hbi_handle *h) {
    if (!h) return;
    if (h->adj) hbi_destroy(h->adj);
    multi_free(h);
    drop_graphs(h);
    if (h->cap_stream) cudaStreamDestroy(h->cap_stream);
    void *ptrs[] = {h->d_perm, h->d_geom, h->d_verts, h->d_rake, h->d_data1, h->d_data2, h->d_data3, h->d_rowscale, h->d_gidx,
                    h->d_gscale, h->d_items1, h->d_batches1, h->d_vt_begin, h->d_tasks2, h->d_xt, h->d_xt2, h->d_yp, h->d_counters,
                    h->d_y, h->d_D, h->d_ys, h->d_Vs, h->d_Vold, h->d_dVs, h->d_dVold, h->d_k, h->d_inv_a, h->d_inv_b, h->d_b_dc, h->d_fcr,
                    h->d_fsr, h->d_ctl, h->d_gctl, h->d_model, h->d_mskip, h->d_rec, h->d_stY, h->d_stS, h->d_Kbar,
                    h->d_lam, h->d_gA, h->d_gDC, h->d_aux, h->d_ckpt, h->d_segY, h->d_lim};
    for (void *p : ptrs)
        if (p) cudaFree(p);
    if (h->h_ctl) cudaFreeHost(h->h_ctl);
    if (h->h_gctl) cudaFreeHost(h->h_gctl);
    if (h->h_flag) cudaFreeHost(h->h_flag);
    delete h;
}

}  // extern "C"
