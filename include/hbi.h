/*
 * hbi.h -- C ABI of the GB300 (sm_103a) library for the hot path of the quasi-dynamic
 * earthquake-sequence BEM with lattice H-matrices of Ozawa, Ida, Hoshino & Ando
 * (arXiv 2110.12165): the H-matrix x slip-rate product (HMVM), the rate-and-state
 * right-hand side and the adaptive Runge-Kutta step.
 *
 * Conventions shared by every call
 * --------------------------------
 * - Elements are indexed 0..n-1 in the caller's (original) order.  Vectors with several
 *   components per element are COMPONENT-MAJOR: v[c * n + i].
 * - Slip components: 0 = along strike s = normalise(z x n), 1 = along d = n x s (up-dip when
 *   the normal n, given by the right-hand rule of the vertex order, points up).  Slip is the
 *   displacement of the + side (the side n points to) relative to the - side.
 * - Stress outputs per element: shear tractions s.sig.n, d.sig.n, and the normal stress
 *   change with compression positive (-n.sig.n).  The single-component operator forms
 *   project slip and shear onto a per-element rake direction cos(r) s + sin(r) d.
 * - "d_" pointers are device pointers (cudaMalloc / torch CUDA tensors) on the device that
 *   is current when the call is made; "h_" pointers are host pointers.  The caller owns all
 *   of them; nothing is retained after the call returns except inside an hbi_handle.
 * - Every call returns hbi_status (0 = success).  No C++ exception and no device trap
 *   crosses this interface; device-detected conditions are reported through a status word
 *   that the call reads back after synchronising the stream it was given.
 * - Calls taking a cudaStream_t enqueue their work on it and synchronise it before
 *   returning unless stated otherwise.
 * - A handle owns scratch buffers, control blocks and captured graphs that every call on
 *   it reuses: calls on one handle must not run concurrently (one thread, or external
 *   locking).  Different handles are independent.
 */
#ifndef HBI_H
#define HBI_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st *hbi_stream; /* a cudaStream_t; NULL = legacy default stream */

typedef int hbi_status;
#define HBI_OK 0
#define HBI_ERR_INVALID_ARG (-1)   /* bad pointer, size, enum or inconsistent arguments */
#define HBI_ERR_OOM (-2)           /* device or host allocation failed */
#define HBI_ERR_CUDA (-3)          /* a CUDA runtime call failed (message via hbi_last_error) */
#define HBI_ERR_ACA_FAIL (-4)      /* ACA did not converge within the rank limit of a block */
#define HBI_ERR_DT_UNDERFLOW (-5)  /* adaptive step fell below 1e-12 s */
#define HBI_ERR_NEG_NORMAL (-6)    /* effective normal stress became <= 0 */
#define HBI_ERR_NONFINITE (-7)     /* non-finite state or result */
#define HBI_ERR_TIMEOUT (-8)       /* a bounded device wait gave up */
#define HBI_ERR_SINGULAR (-9)      /* a receiver lies on an element edge (stress singular) */

/* Element shape (Sec. 2.1: rectangles with two horizontal sides, or triangles). */
typedef enum { HBI_RECT = 4, HBI_TRI = 3 } hbi_elem_kind;

/* Operator form: which slip components go in and which stress components come out
 * (Eqs. 5-6 are HBI_OP_RAKE_SHEAR_NORMAL; the two-component forms carry strike and dip
 * slip separately). */
typedef enum {
    HBI_OP_RAKE_SHEAR = 0,         /* in: V_r            out: tau_r                  (1 -> 1) */
    HBI_OP_RAKE_SHEAR_NORMAL = 1,  /* in: V_r            out: tau_r, sigma           (1 -> 2) */
    HBI_OP_VEC_SHEAR = 2,          /* in: V_s, V_d       out: tau_s, tau_d           (2 -> 2) */
    HBI_OP_VEC_FULL = 3            /* in: V_s, V_d       out: tau_s, tau_d, sigma    (2 -> 3) */
} hbi_operator;

/* Storage precision of the packed factors and dense blocks (accumulation is FP64 for
 * HBI_FP64 and FP32 otherwise; FP16/BF16 carry one FP32 scale per factor column).
 * HBI_MIXED stores the dense near-field blocks, which carry most of the operator's norm, in
 * FP32 and the low-rank factors of the far field in FP16 with per-column scales.
 * HBI_ADAPTIVE is HBI_MIXED with the leading pair (first column of U and of V) of every
 * low-rank block kept in FP32: after SVD recompression that is the block's dominant singular
 * pair, which carries most of its norm and so most of the FP16 rounding error (two more bytes
 * per entry of one rank of each block).  This mixed-precision storage is an extension of the
 * library; the paper stores FP64. */
typedef enum { HBI_FP64 = 0, HBI_FP32 = 1, HBI_FP16 = 2, HBI_BF16 = 3, HBI_MIXED = 4, HBI_ADAPTIVE = 5 } hbi_storage;

typedef struct {
    int n_elem;             /* number of elements N (>= 1) */
    int kind;               /* hbi_elem_kind */
    const double *h_verts;  /* host, [n_elem][kind][3] vertex coordinates in metres */
    const double *h_rake;   /* host, [n_elem] rake angles (rad) for the single-component
                               operator forms; NULL = 0 (pure strike slip) */
} hbi_mesh;

typedef struct {
    double mu;              /* rigidity (Pa) */
    double nu;              /* Poisson's ratio */
    int op;                 /* hbi_operator */
    int half_space;         /* 0: homogeneous full space.  1: elastic half space z < 0 with a
                               traction-free surface z = 0 (Sec. 2.1); every vertex must have
                               z <= 0 and every element centre z < 0.  The entries add to the
                               full-space ones Mindlin's (1936) point-force correction carried
                               over the source element (Volterra representation), integrated by
                               Radon's seven-point rule on a subdivision of the source whose
                               sub-triangles are at most 1/4 of their vertical distance to the
                               receiver's image (up to 4^7 of them per triangle), or by the
                               three-point rule when the source's diameter is at most 0.02 of
                               its distance to that image.  Entries agree with an independent
                               evaluation to about 1e-6 of a pair's largest entry.  The product
                               and the integrator are unchanged. */
} hbi_elastic;

typedef struct {
    double aca_eps;         /* Eq. 19 tolerance eps_ACA (e.g. 1e-4) */
    int leaf_size;          /* maximum cluster size of the binary tree (Sec. 3.1.1) */
    int lattice_depth;      /* L: tree truncation depth of the lattice (Sec. 3.2); 0 = normal H */
    double eta;             /* admissibility parameter of Eq. 17 (the paper uses 2) */
    int storage;            /* hbi_storage */
    double recompress_eps;  /* > 0: after ACA, reduce each low-rank block (rank <= 48) to the
                               smallest rank whose discarded singular values have Frobenius
                               norm <= recompress_eps x the block's norm (SVD of the factors);
                               0 = keep the ACA ranks (the paper's procedure) */
    int with_transpose;     /* 1: also pack the transposed operator H^T (hbi_matvec_transpose,
                               the adjoint), which doubles the factor memory; 0: H only */
    int multi_rhs;          /* 1: also pack the tensor-core panels of hbi_matvec_multi (storage
                               HBI_FP16 or HBI_MIXED; about the factor memory again); 0: none */
} hbi_build_params;

typedef struct hbi_handle hbi_handle;

/*
 * hbi_build -- build the lattice H-matrix of the elastic operator on the GPU.
 * Sec. 3.1.1-3.1.2 and 3.2 (cluster tree, Eq. 17 partition inside each lattice block,
 * ACA of Eqs. 18-19 on admissible blocks, dense near-field blocks); the entries are the
 * full-space stresses of uniform-slip elements collocated at element centres (Eqs. 3-6).
 * The tree and partition are built on the host; entries, ACA and packing run on the
 * device.  On success *out owns all device memory it needs; free it with hbi_destroy.
 * Errors: INVALID_ARG (NULL pointers, n_elem < 1, bad kind/op/storage, leaf_size < 1,
 * lattice_depth < 0, aca_eps <= 0), OOM, CUDA, ACA_FAIL, SINGULAR.
 */
hbi_status hbi_build(const hbi_mesh *mesh, const hbi_elastic *ek, const hbi_build_params *bp,
                     hbi_handle **out);

/*
 * hbi_plan -- the host part of hbi_build alone (no GPU needed): cluster tree on element
 * centres (Sec. 3.1.1), lattice truncation at depth L (Sec. 3.2) and the Eq. 17 block
 * partition.  h_perm[n_elem] receives permuted position -> original element;
 * h_leaf_starts[n_elem + 1] the element offsets of the leaf clusters (*n_leaves of them,
 * plus the final n_elem); h_blocks[max_blocks][6] (may be NULL) the blocks as
 * row0, m, col0, ncol, admissible (0/1), 0 in DOF units; *n_blocks the block count.
 * Errors: INVALID_ARG (as hbi_build, or max_blocks too small when h_blocks is given).
 */
hbi_status hbi_plan(const hbi_mesh *mesh, const hbi_elastic *ek, const hbi_build_params *bp, int *h_perm,
                    int *h_leaf_starts, int *n_leaves, int64_t *h_blocks, int max_blocks, int *n_blocks);

/*
 * hbi_lattice_owners -- the distribution of the lattice H-matrix over a P_r x P_c process grid
 * (Sec. 3.2): lattice block (I, J) belongs to rank (I mod P_r) P_c + (J mod P_c), and every
 * H-matrix block to the owner of its lattice block.  Host only (no GPU); the partition is that
 * of hbi_plan for the same arguments, in the same block order.  h_owner[max_blocks] (may be
 * NULL) receives the owner of each block, *n_blocks their number.  With it a rank computes
 * Eq. 20 over its own blocks; the partial products of each process row are reduced to the row's
 * first rank and the row sums combined and broadcast (the paper's one reduction and one
 * broadcast per product).  hbi_build_shard builds one rank's blocks by this map.
 * Errors: INVALID_ARG (as hbi_plan; P_r, P_c >= 1).
 */
hbi_status hbi_lattice_owners(const hbi_mesh *mesh, const hbi_elastic *ek, const hbi_build_params *bp, int p_rows,
                              int p_cols, int *h_owner, int max_blocks, int *n_blocks);

/*
 * hbi_build_shard -- one rank's share of the paper's distributed lattice H-matrix (Sec. 3.2):
 * the tree, lattice and Eq. 17 partition of hbi_build, of which only the blocks inside the
 * lattice blocks (I, J) with (I mod p_rows) p_cols + J mod p_cols == rank are computed (entries,
 * ACA, recompression) and packed, so the build work and the factor memory of a rank are its
 * share of the whole.  hbi_matvec on the shard gives that rank's partial product: Eq. 20 over
 * its blocks, every row (zero outside the lattice rows I = rank / p_cols mod p_rows).  The sum
 * of the partial products of all ranks is hbi_matvec of the whole operator; in the paper each
 * process row reduces its partial products and the row sums are then broadcast, one reduction
 * and one broadcast per product.  A shard does not drive the integrator (hbi_rhs, hbi_step and
 * the other time-stepping calls return INVALID_ARG on it).  This library runs one GPU per
 * process; the exchange between processes is the caller's.
 * Errors: INVALID_ARG (as hbi_build; p_rows, p_cols >= 1, 0 <= rank < p_rows p_cols), OOM,
 * CUDA, ACA_FAIL, SINGULAR.
 */
hbi_status hbi_build_shard(const hbi_mesh *mesh, const hbi_elastic *ek, const hbi_build_params *bp, int p_rows,
                           int p_cols, int rank, hbi_handle **out);

/*
 * hbi_build_from_factors -- build a handle from an externally computed H-matrix (same
 * partition and factors, FP64 on the host), e.g. to check the HMVM on given factors.
 * Layout, with DOFs in permuted, component-interleaved order (row DOF = n_out*p + c):
 *   h_perm[n_elem]        permuted position p -> original element index
 *   h_blocks[n_blocks][6] row0, m, col0, ncol, lowrank (0/1), rank   (DOF units)
 *   h_offsets[n_blocks]   offset of the block's data in h_data (doubles)
 *   h_data                dense block: m x ncol row-major; low-rank block: U (m x rank,
 *                         column-major) followed by V (ncol x rank, column-major), A ~ U V^T
 *   h_leaf_starts[n_leaves+1]  element offsets (in permuted order) of the leaf clusters;
 *                         every block row range must be a union of consecutive leaves.
 * The mesh is used for the geometry of the RHS only (entries are taken as given).
 * The blocks must tile the (n_out N) x (n_in N) matrix exactly once.  with_transpose != 0
 * also packs H^T from the same factors (as hbi_build_params.with_transpose), for
 * hbi_matvec_transpose, hbi_rhs_vjp and hbi_adjoint.
 * Errors: INVALID_ARG (inconsistent sizes or tiling), OOM, CUDA.
 */
hbi_status hbi_build_from_factors(const hbi_mesh *mesh, const hbi_elastic *ek, int storage,
                                  const int *h_perm, int n_blocks, const int64_t *h_blocks,
                                  const int64_t *h_offsets, const double *h_data,
                                  int n_leaves, const int *h_leaf_starts, int with_transpose,
                                  hbi_handle **out);

/*
 * hbi_matvec -- y = H x (Sec. 3.1.3, Eq. 20), the H-matrix x slip-rate product.
 * d_x: n_in * N doubles (component-major, original order); d_y: n_out * N doubles, same
 * layout.  Runs the persistent HMVM kernels on `stream` and synchronises it.
 * Errors: INVALID_ARG (NULL handle/pointers), CUDA.
 */
hbi_status hbi_matvec(hbi_handle *h, const double *d_x, double *d_y, hbi_stream stream);

/*
 * hbi_matvec_transpose -- w = H^T v, the transposed product (the adjoint of hbi_matvec:
 * <H x, v> = <x, H^T v>), for handles built with with_transpose = 1.  H^T is packed at build
 * time from the same partition and factors (a low-rank block U V^T contributes V (U^T v), a
 * dense block D contributes D^T v) and runs on the same two kernels.  d_v: n_out N doubles
 * (component-major, original order); d_w: n_in N doubles, same layout.  Synchronises the
 * stream.  The paper has no transposed product; it serves the adjoint (hbi_adjoint).
 * Errors: INVALID_ARG (NULL pointers, handle without the transpose), CUDA, TIMEOUT.
 */
hbi_status hbi_matvec_transpose(hbi_handle *h, const double *d_v, double *d_w, hbi_stream stream);

/* Asynchronous form of hbi_matvec: enqueues only, no synchronisation, no status read. */
hbi_status hbi_matvec_async(hbi_handle *h, const double *d_x, double *d_y, hbi_stream stream);

/*
 * hbi_matvec_noalloc -- the product of hbi_matvec for callers that cannot allocate device
 * memory when they need it: a host program that hands the whole device memory to its own
 * pool allocator at start-up, or code on a path where an allocation (which may synchronise
 * the device) is not allowed.  This call makes no cudaMalloc, cudaFree or other allocating
 * call, and it does not use the handle's own scratch buffers either.  The paper has no
 * counterpart of this call; it is an interface convenience of this library.
 * Scratch: one static device array of HBI_NOALLOC_SCRATCH_BYTES inside the library, which
 * every GPU that loads the library holds until the process exits.  One product needs
 * 3 int words (work counter, error flag, finish count) plus (n_in N + T + 16) and n_out N accumulation
 * words (8 bytes for HBI_FP64 storage, 4 otherwise; T = sum of the ranks), each part rounded
 * up to 256 bytes; larger operators are rejected with HBI_ERR_INVALID_ARG.
 * The first call on a device looks the array's device address up (cudaGetSymbolAddress)
 * with that device current; make that first call before any stream capture.  Every call
 * shares the array, which keeps the last call's contents (each call clears the work counters
 * it needs); calls that overlap on the GPU (other streams or threads) race on the array
 * and must be serialised by the caller.  The looked-up address is kept for the life of the
 * process: after cudaDeviceReset (which also invalidates every handle on that device) this
 * call must not be used again in the same process.  d_x, d_y and the synchronisation are as
 * in hbi_matvec.  Errors: INVALID_ARG, CUDA, TIMEOUT.
 */
#define HBI_NOALLOC_SCRATCH_BYTES ((size_t)16 << 20)
hbi_status hbi_matvec_noalloc(hbi_handle *h, const double *d_x, double *d_y, hbi_stream stream);

/*
 * hbi_matvec_multi -- Y = H X for k right-hand sides at once (Eq. 20 applied to k slip-rate
 * vectors), on the tensor cores.  Each stored entry of the operator then feeds k multiply-adds,
 * so the product is a dense contraction (two batched GEMMs: the V^T x products of the column
 * groups, then the [dense | U] row panels of the leaf row units times the gathered inputs),
 * run with tcgen05.mma (FP16 operands, FP32 accumulation in tensor memory).  The handle must
 * be built with hbi_build_params.multi_rhs = 1 and storage HBI_FP16 or HBI_MIXED: the panels
 * hold the same entries as the single-vector storage (FP16 with per-column power-of-two
 * scales; HBI_MIXED's FP32 near field as an FP16 pair hi + 2^-11 lo), and each input is
 * scaled per right-hand side and split into FP16 hi + 2^-11 lo (22 significant bits), so the
 * accuracy is that of the storage.  The paper multiplies one vector at a time; several
 * right-hand sides serve ensembles of slip-rate states on one fault (e.g. perturbed initial
 * conditions, or the stages of several runs).
 * d_X: k x n_in N doubles, right-hand side r at d_X[r n_in N + c N + i] (each one laid out
 * as the d_x of hbi_matvec); d_Y: k x n_out N doubles, the same way.  1 <= k <= 64 (k is
 * padded to a multiple of 16 internally).  Work buffers for k are allocated on the first
 * call with that size and kept by the handle.  Synchronises the stream.
 * Errors: INVALID_ARG (NULL pointers, k out of range, handle without the panels), CUDA,
 * TIMEOUT.
 */
hbi_status hbi_matvec_multi(hbi_handle *h, int k, const double *d_X, double *d_Y, hbi_stream stream);

/*
 * hbi_time_multi -- device time of the multi-RHS product on the input of the handle's last
 * hbi_matvec_multi call with the same k (call that first), averaged over n_rep back-to-back
 * products with CUDA events recorded on `stream`: out3[0] = V^T phase, out3[1] = U t + dense
 * phase, out3[2] = both (ms; the input and output permutations are not included).
 * Errors: INVALID_ARG, CUDA, TIMEOUT.
 */
hbi_status hbi_time_multi(hbi_handle *h, int k, int n_rep, double *out3, hbi_stream stream);

/* Sizes of the multi-RHS panels (hbi_matvec_multi). */
typedef struct {
    int64_t panel_bytes;              /* packed panel stream read per product (with padding) */
    int64_t bytes_panels_algorithmic; /* stored entries (4 bytes for a hi + lo pair, 2 for FP16)
                                         and their scales: the factor bytes of one product */
    int64_t vector_bytes_per_rhs;     /* FP32 words per right-hand side: x read, t written and
                                         read, y written (x 4 bytes) */
    double flops_per_rhs;             /* 2 x stored entries: the product's arithmetic per vector */
    double mma_flops_per_rhs;         /* as issued on the tensor cores per vector (128-row tiles,
                                         K padded to 16, hi / lo passes) */
    int64_t n_tasks_vt, n_tasks_uy, n_t;
    int64_t n_split_tiles;            /* V^T row tiles of column groups wider than 2048 columns,
                                         cut into K slices whose partial sums a reduction adds */
} hbi_multi_stats_t;

/* hbi_multi_stats -- sizes of the multi-RHS panels.  Errors: INVALID_ARG (also for a handle
 * built without them). */
hbi_status hbi_multi_stats(const hbi_handle *h, hbi_multi_stats_t *out);

/*
 * hbi_build_ensemble -- many independent fault models in one handle: model m is built
 * exactly as hbi_build would build meshes[m] (its own cluster tree, Eq. 17 partition, lattice
 * and ACA, with the shared elastic constants and build parameters), and the handle's
 * operator is block diagonal over the models, so one HMVM (two kernel launches) serves all
 * of them.  Elements are the models' elements concatenated in order (model m occupies
 * [sum_{k<m} N_k, sum_{k<=m} N_k)); every per-element array of hbi_matvec, hbi_rhs,
 * hbi_steady_state and hbi_step_ensemble (d_x, d_y, state, friction a, b, d_c, rake) uses
 * that order.  Batched execution of independent models is an extension of this library,
 * not a construct of the paper.  Errors: as hbi_build.
 */
hbi_status hbi_build_ensemble(int n_models, const hbi_mesh *meshes, const hbi_elastic *ek,
                              const hbi_build_params *bp, hbi_handle **out);

/* Rate-and-state friction parameters (Eqs. 7-8, 9-10, 21-22).  Arrays are device
 * pointers of length N in the original element order. */
typedef struct {
    const double *d_a;      /* direct-effect coefficient a */
    const double *d_b;      /* evolution-effect coefficient b */
    const double *d_dc;     /* characteristic slip distance d_c (m) */
    const double *d_rake;   /* slip direction angle (rad) in the (strike, dip) frame */
    double f0;              /* reference friction coefficient */
    double V0;              /* reference slip rate (m/s) */
    double Vpl;             /* plate rate of the backslip loading (m/s) */
    double mu;              /* rigidity for radiation damping mu/(2 c_s) (Pa) */
    double cs;              /* shear-wave speed (m/s) */
} hbi_friction;

/*
 * hbi_steady_state -- initial state at steady sliding (Eq. 8 = 0) and the shear stress of
 * Eq. 7 (read as tau = a sigma asinh(V/(2 V0) exp(phi/a))) for given slip rates.
 * All pointers device, length n.  Errors: INVALID_ARG, CUDA.
 */
hbi_status hbi_steady_state(int n, const double *d_V, const double *d_a, const double *d_b,
                            const double *d_sigma, double f0, double V0, double *d_phi,
                            double *d_tau, hbi_stream stream);

/*
 * hbi_rhs -- dy/dt of the 3N ODE system y = (phi, tau, sigma) (Eqs. 7-13 with the
 * backslip loading of Eqs. 21-22 folded into the HMVM input: H (V - V_pl) r).
 * d_state: 3N doubles (phi[N], tau[N], sigma[N], original order); d_dydt: 3N doubles;
 * d_V (optional, may be NULL): N doubles receiving the slip rate of Eq. 7.
 * Errors: INVALID_ARG, CUDA.
 */
hbi_status hbi_rhs(hbi_handle *h, const hbi_friction *f, const double *d_state, double *d_dydt,
                   double *d_V, hbi_stream stream);

/*
 * hbi_rhs_vjp -- vector-Jacobian product of hbi_rhs: for the right-hand side f of Eqs. 7-13
 * at the state y, ybar = (df/dy)^T v and the gradients of <v, f(y)> with respect to the
 * per-element friction parameter a (at fixed b; the gradient with respect to a - b) and d_c.
 * The coupling through the product is applied with H^T (handle built with_transpose = 1).
 * d_state: 3N (phi, tau, sigma); d_v, d_ybar: 3N; d_grad_a, d_grad_dc: N each (optional);
 * all device, original order.  The paper has no adjoint; see hbi_adjoint.
 * Errors: INVALID_ARG (also without the transpose), CUDA, TIMEOUT.
 */
hbi_status hbi_rhs_vjp(hbi_handle *h, const hbi_friction *f, const double *d_state, const double *d_v,
                       double *d_ybar, double *d_grad_a, double *d_grad_dc, hbi_stream stream);

/*
 * hbi_rk_fixed -- n_steps Cash-Karp steps of the given sizes h_dts[n_steps] (host array,
 * all > 0), each accepted without error control (the step sequence of an earlier adaptive
 * run, frozen).  The same product kernels and per-element stage arithmetic as hbi_step, with
 * each stage launched as a kernel of its own (hbi_step runs the stages inside the products'
 * UY launches), so replaying an adaptive run's accepted step sizes gives its states to the
 * last bit.  d_state: 4N (phi, tau, sigma, D), updated in place.  Single-model handles.
 * Errors: INVALID_ARG, CUDA, TIMEOUT.
 */
hbi_status hbi_rk_fixed(hbi_handle *h, const hbi_friction *f, double *d_state, const double *h_dts,
                        int n_steps, hbi_stream stream);

/*
 * hbi_adjoint -- loss and gradient of a sequence run by the discrete adjoint.  From d_state0
 * (4N) the run takes the fixed steps h_dts[n_steps] (as hbi_rk_fixed); the loss is
 * L = 1/2 sum_i (ln V_i(y_N) - target_i)^2 with V from Eq. 7 at the final state; the
 * gradients with respect to each element's a - b (at fixed b) and d_c are the exact
 * derivatives of this discrete map (the transposed Cash-Karp stage recursion, the
 * transposed element-wise right-hand side and H^T for the coupling).  States are kept every
 * checkpoint_every steps; in the reverse pass each segment is recomputed once from its
 * checkpoint, keeping every step's stage states and product outputs, and then swept back,
 * so the memory is n_steps / checkpoint_every states of 3N plus checkpoint_every x
 * (18 + 6 n_out) N doubles, and the work two forward runs plus one reverse run (six H^T
 * products per step).  d_target: N; h_loss: host double;
 * d_grad_amb, d_grad_dc: N each; d_state_final (optional): 4N, the state after the forward
 * run.  Requires with_transpose = 1 and a single-model handle.  The paper has no adjoint;
 * this is an extension of the library.  Errors: INVALID_ARG, CUDA, TIMEOUT.
 */
hbi_status hbi_adjoint(hbi_handle *h, const hbi_friction *f, const double *d_state0, const double *h_dts,
                       int n_steps, int checkpoint_every, const double *d_target, double *h_loss,
                       double *d_grad_amb, double *d_grad_dc, double *d_state_final, hbi_stream stream);

/* Per-accepted-step record written by hbi_step when h_records is not NULL. */
typedef struct {
    double t;        /* time after the step (s) */
    double dt;       /* step size used (s) */
    double vmax;     /* max slip rate after the step (m/s) */
    double rejects;  /* rejected attempts before this step was accepted */
    double mu_mean;  /* mean friction coefficient after the step: the mean over the model's
                        elements of tau / sigma (rake-free friction: |tau| / sigma), the
                        quantity the paper plots against time (Sec. 4.3); summed exactly (fixed
                        point, 2^-40), so it does not depend on the order of the elements */
} hbi_step_record;

/*
 * hbi_step -- advance n_steps accepted adaptive Runge-Kutta steps (Cash-Karp 4(5),
 * six HMVMs per attempt; Eqs. 14-15 step control read as (err/eps_RK)^-0.25 on rejection
 * and ^-0.2 on acceptance, clamped to [dt/2, 2 dt]; err = max_i |y5-y4|/|y5|; slip by the
 * trapezoid of Eq. 16).  Accept/reject is decided on the device; the attempt is a CUDA
 * graph replayed until n_steps steps are accepted, in which each stage's element-wise work
 * (Eqs. 7-13, the stage sums, the error norm) runs inside the U t + dense launch of the
 * product before it, leaf row unit by leaf row unit.
 * d_state: 4N doubles (phi, tau, sigma, D) in original order, updated in place.
 * d_t, d_dt: one double each on the device (time and next step size), updated in place.
 * h_records: optional host array of n_steps records.  *n_done (optional host int) receives
 * the number of accepted steps.  A rejected attempt leaves the state unchanged, so the next
 * attempt reuses k_1 = f(y) and skips its first HMVM (same results, fewer products).
 * Errors: INVALID_ARG (also for an ensemble handle: use hbi_step_ensemble), CUDA, TIMEOUT,
 * DT_UNDERFLOW, NEG_NORMAL, NONFINITE.
 */
hbi_status hbi_step(hbi_handle *h, const hbi_friction *f, double *d_state, double *d_t,
                    double *d_dt, double eps_rk, int n_steps, hbi_step_record *h_records,
                    int *n_done, hbi_stream stream);

/*
 * hbi_time_attempts -- where the time of an adaptive step goes: from the state d_state (4N:
 * phi, tau, sigma, D), time *d_t and step *d_dt (device), n_attempts Cash-Karp attempts of
 * hbi_step (single-model handle, eps_rk as there) are launched kernel by kernel with CUDA
 * events on `stream` between launches, then the same number as replays of the captured attempt
 * graph.  out8 (host, ms per attempt): [0] the six products (Eq. 20), [1] the five stage
 * kernels (Eqs. 7-13 and the stage sums), [2] the last stage with the error norm, [3] the
 * controller (Eqs. 14-15), [4] the commit (Eq. 16), [5] the stop flags, [6] the sum of [0..5]
 * launched eagerly, [7] one graph replay.  The eager launches run each stage as a kernel of
 * its own; the captured graph of the fixed-rake law runs every stage inside the UY phase of
 * the product before it, so [6] - [7] is what that saves.  The caller's arrays are not written.
 * Errors: INVALID_ARG, CUDA, TIMEOUT.
 */
hbi_status hbi_time_attempts(hbi_handle *h, const hbi_friction *f, const double *d_state, const double *d_t,
                             const double *d_dt, double eps_rk, int n_attempts, double *out8, hbi_stream stream);

typedef struct {
    int64_t n_elem, n_in, n_out;
    int64_t n_clusters, n_leaves, n_lattice;
    int64_t n_blocks, n_lowrank, n_dense;
    int64_t max_rank;
    double mean_rank;
    int64_t entries_lowrank;      /* sum (m + ncol) r over low-rank blocks */
    int64_t entries_dense;        /* sum m ncol over dense blocks */
    int64_t bytes_factors;        /* packed factor + dense bytes read per HMVM (with padding) */
    int64_t bytes_algorithmic;    /* per HMVM: stored entries x element size + scales +
                                     x, y and intermediate vectors, no padding */
    int64_t n_tasks_vt, n_tasks_uy; /* work items of the two HMVM phases */
    int storage;
    double build_seconds;
    int64_t bytes_alg_vt;         /* algorithmic bytes of the V^T x phase: V entries, V scales,
                                     x read once, t written */
    int64_t bytes_alg_uy;         /* algorithmic bytes of the U t + dense phase: U and dense
                                     entries, their scales, x and t read once, y written */
    int64_t last_step_attempts;   /* attempts (graph replays) launched by the last hbi_step,
                                     including no-op replays after the target was reached */
    int64_t last_step_kernels;    /* device kernels launched by the last hbi_step */
    int64_t n_models;             /* 1, or the number of models of an ensemble handle */
} hbi_stats_t;

/*
 * hbi_step_ensemble -- hbi_step for every model of an ensemble handle at once: each model
 * keeps its own time, step size, accept/reject decisions and step count; one captured
 * attempt graph advances all models (their HMVMs fused into one product) until each has
 * n_steps accepted steps or has stopped on an error.
 * d_state: 4 N_total doubles (phi, tau, sigma, D; each in the concatenated element order).
 * d_t, d_dt: n_models doubles each on the device, updated in place.
 * h_records: optional host array [n_models][n_steps].  h_n_done: host array of n_models ints
 * (accepted steps per model).  Returns HBI_OK, or the first model's error status.
 * Errors: INVALID_ARG, CUDA, TIMEOUT, DT_UNDERFLOW, NEG_NORMAL, NONFINITE.
 */
hbi_status hbi_step_ensemble(hbi_handle *h, const hbi_friction *f, double *d_state, double *d_t,
                             double *d_dt, double eps_rk, int n_steps, hbi_step_record *h_records,
                             int *h_n_done, hbi_stream stream);

/*
 * Rake-free friction.  The fixed-rake law (Eqs. 5-13) lets the shear traction act along a
 * prescribed rake.  With a two-component operator (HBI_OP_VEC_SHEAR or HBI_OP_VEC_FULL) the
 * shear traction is a vector (tau_s, tau_d) in the element's (strike, dip) frame and the slip
 * rate is parallel to it: V = g tau / |tau|, g the slip rate of Eq. 7 at |tau|.  The
 * radiation-damping balance of Eqs. 11-13 holds per component; it is solved per element
 * with dV/dtau = g' t t^T + (g / |tau|)(I - t t^T), t = tau / |tau| (along t when tau = 0:
 * the rake direction).  Loading is backslip at V_pl along the friction's rake (Eq. 4 with
 * the plate-rate vector V_pl (cos rake, sin rake)).  sigma evolves with the operator's
 * normal component (HBI_OP_VEC_FULL, Eq. 10) and stays constant with HBI_OP_VEC_SHEAR.
 * This form generalises the paper's fixed-rake law; it reduces to it on a single element
 * loaded along its rake.
 *
 * hbi_rhs_vec -- dy/dt and V for a state.  d_state: 4N (phi, tau_s, tau_d, sigma);
 * d_dydt: 4N; d_V: 2N (V_s, V_d), optional; device, original order.
 * Errors: INVALID_ARG (also for a one-component operator), CUDA, TIMEOUT.
 */
hbi_status hbi_rhs_vec(hbi_handle *h, const hbi_friction *f, const double *d_state, double *d_dydt,
                       double *d_V, hbi_stream stream);

/*
 * hbi_step_vector -- hbi_step / hbi_step_ensemble with rake-free friction: adaptive
 * Cash-Karp steps of the state d_state = 6N (phi, tau_s, tau_d, sigma, D_s, D_d; each in the
 * original (or concatenated ensemble) element order).  The element error of Eq. 14 is the
 * largest of the relative changes of phi, of the traction vector (|d tau| / |tau|) and of
 * sigma; a step record's vmax is the largest |V|.  Slip integrates each component by the
 * trapezoid of Eq. 16.  d_t, d_dt: one double per model (device), updated in place;
 * h_records: optional [n_models][n_steps]; h_n_done: n_models ints.
 * Errors: INVALID_ARG (also for a one-component operator), CUDA, TIMEOUT, DT_UNDERFLOW,
 * NEG_NORMAL, NONFINITE.
 */
hbi_status hbi_step_vector(hbi_handle *h, const hbi_friction *f, double *d_state, double *d_t,
                           double *d_dt, double eps_rk, int n_steps, hbi_step_record *h_records,
                           int *h_n_done, hbi_stream stream);

/* hbi_stats -- sizes of the built operator.  Errors: INVALID_ARG. */
hbi_status hbi_stats(const hbi_handle *h, hbi_stats_t *out);

/*
 * hbi_time_hmvm -- device time of the HMVM phases, averaged over n_rep back-to-back
 * products of the handle's current input, measured with CUDA events recorded on `stream`
 * around each phase: out4[0] = V^T x phase alone, out4[1] = 0 (kept for layout), out4[2] =
 * U t + dense phase alone, out4[3] = the whole product as hbi_matvec launches it (ms).
 * Synchronises `stream`.
 * Errors: INVALID_ARG (n_rep < 1, NULL pointers), CUDA.
 */
hbi_status hbi_time_hmvm(hbi_handle *h, int n_rep, double *out4, hbi_stream stream);

/*
 * hbi_autotune -- pick this handle's HMVM launch configuration by timing it on the GPU: the
 * per-pass cost used by the V^T kernel to choose rows per pass and lanes per row for each
 * item (4, 8 or 16), and for the U t + dense kernel the rows per lane group (4 or 8) and CTAs
 * per SM (up to three values below the occupancy limit).  Each phase is timed as the average
 * of n_rep back-to-back launches on `stream` with the handle's current input; the fastest
 * setting is kept (until hbi_destroy) and used by every later product and by hbi_step.  The
 * choice changes the order of the sums, so results change at rounding level (runs remain
 * reproducible for a given choice).  out3 (optional host int[3]) receives (UY rows per pass,
 * UY CTAs per SM, VT pass cost); out_ms (optional) the tuned product time in ms.  A handle
 * built with_transpose has H^T tuned the same way (its settings are not reported).
 * Errors: INVALID_ARG, CUDA, TIMEOUT.
 */
hbi_status hbi_autotune(hbi_handle *h, int n_rep, int *out3, double *out_ms, hbi_stream stream);

/*
 * hbi_stalled_wait_status -- failure-path check of the bounded device waits: runs one warp
 * waiting on an mbarrier phase that nothing will complete, through the same bounded wait as
 * the V^T kernel (about one second of wall time), and returns the status the library reports
 * for a stalled wait: HBI_ERR_TIMEOUT (the context stays usable).  Not part of the paper.
 * Errors: CUDA.
 */
hbi_status hbi_stalled_wait_status(hbi_stream stream);

/*
 * hbi_inject_failure -- failure injection for tests of the library's error paths, made on the
 * host (no GPU call fails for real).  HBI_INJECT_ALLOC: the count-th device allocation of the
 * library from now on (1 = the next one) fails as an out-of-memory cudaMalloc would, and the
 * call that made it returns HBI_ERR_OOM after freeing what it had allocated.  HBI_INJECT_ACA:
 * the count-th ACA block result of the builds from now on is reported as not converged within
 * the rank limit (HBI_ERR_ACA_FAIL).  HBI_INJECT_NONE clears both.  Process-wide; not for use
 * while other threads call the library.  Not part of the paper.  Errors: INVALID_ARG.
 */
#define HBI_INJECT_NONE 0
#define HBI_INJECT_ALLOC 1
#define HBI_INJECT_ACA 2
hbi_status hbi_inject_failure(int what, long long count);

/*
 * hbi_bounds_violations -- the count of table and index violations found by the bounds-checked
 * build of the library (compiled with HBI_BOUNDS_CHECK) since the last call, which clears it:
 * in that build the two product kernels check every work-table entry (stream segments, output
 * rows, gather ranges, shared-memory sizes, bulk-copy extents) and every gather index against
 * the buffers of the handle being multiplied, and count a violation instead of making the
 * access (the affected task or batch is skipped; nothing traps).  Synchronises the device.
 * The normal build sets *out = -1 and returns INVALID_ARG.  Not part of the paper.
 */
hbi_status hbi_bounds_violations(long long *out);

/* hbi_destroy -- free every resource owned by the handle (NULL is a no-op). */
void hbi_destroy(hbi_handle *h);

/* Human-readable name of a status code (static string). */
const char *hbi_status_string(hbi_status s);

/* Last error message recorded by this library in the calling thread (static storage). */
const char *hbi_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* HBI_H */
