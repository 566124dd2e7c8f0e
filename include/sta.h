/*
 * libsta: STA-FEM exact streaming assembly of the linear-elasticity stiffness matrix over a
 * fixed, preallocated superset tetrahedral mesh, on one CUDA GPU (sm_103a).
 *
 * The library maintains  A_t = sum_{tau in T_t} P_tau^T K^(tau) P_tau + eps I   (STA-FEM,
 * arXiv 2605.11673, Sec. 3.4, Eq. 8) for the active set T_t of a superset mesh, under a
 * per-frame stream of tetrahedron edits (Sec. 3.2: deleted set Delta^-, added set Delta^+;
 * Sec. 3.3: fracture/merge toggle existing tets, refinement activates preallocated children
 * and deactivates their parents).  Invariant (Sec. 3.3): after every call the values equal a
 * from-scratch rebuild on the current active set -- here bit for bit.
 *
 * Conventions shared by every call:
 *  - Return value: STA_OK (0) or a negative STA_E* code; sta_last_error() gives a message
 *    for the calling thread.  All argument and edit validation happens on the host before
 *    any device work, and a rejected call changes no state.
 *  - `stream` is a cudaStream_t passed as void* (NULL = the legacy default stream).  Device
 *    work is enqueued on it; calls return before it finishes unless stated otherwise.
 *  - Host arrays passed in are copied; the caller keeps ownership.  Device pointers handed
 *    out by sta_csr / sta_scatter_map are owned by the context and valid until sta_destroy.
 *  - Matrix layout: scalar CSR with 3n rows, DOF 3v + i (node v, component i).  Row 3a+i
 *    holds, for every node b sharing at least one SUPERSET tetrahedron with node a (a
 *    included), in ascending b, the three columns 3b, 3b+1, 3b+2.  The pattern is fixed at
 *    create; entries with no active contributor hold +0.0.  Indices are int32 (STA_ERANGE
 *    when they would overflow).
 *  - Summation order: each value is the left-to-right fold, from +0.0, of the contributions
 *    of its active tetrahedra in ascending tetrahedron id; eps is added to diagonal entries
 *    afterwards.  Element matrices follow the fixed evaluation order documented with
 *    sta_element_matrices.  Results are therefore deterministic and independent of launch
 *    configuration.
 */
#ifndef STA_H
#define STA_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct sta_ctx sta_ctx;

enum {
    STA_OK = 0,
    STA_EINVAL = -1, /* bad argument, bad mesh, bad edit list */
    STA_ESTATE = -2, /* call not valid in the context's current state */
    STA_ERANGE = -3, /* a count or index would overflow int32 */
    STA_ENOMEM = -4, /* device or pinned host allocation failed */
    STA_ECUDA = -5   /* a CUDA runtime call or kernel failed */
};

/* Edit operations (Sec. 3.2 Delta^-, Delta^+; Algorithm 1 "receive edit sets"). */
enum { STA_DEACTIVATE = 0, STA_ACTIVATE = 1, STA_SWAP = 2 };

/* One edit.  DEACTIVATE: tet leaves the active set (fracture, coarsening parent...).
 * ACTIVATE: tet joins it (merge, refinement child...).  SWAP: tet leaves and tet2 joins
 * (e.g. a connected tetrahedron replaced by its preallocated split copy).  tet2 is ignored
 * unless op == STA_SWAP.  Within one call every tetrahedron may appear at most once. */
typedef struct {
    int32_t op;
    int32_t tet;
    int32_t tet2;
} sta_edit;

typedef struct {
    double eps;             /* eps of Eq. 4 / Eq. 8, added to diagonal entries; default 0 */
    int32_t block_threads;  /* threads per CTA of the rebuild fold: 64, 128 or 256; 0 = 128 */
    int32_t blocks_per_sm;  /* CTAs per SM of the persistent rebuild grid; 0 = occupancy max */
} sta_options;

/* Fills defaults (eps 0, launch shape from the built-in table). */
void sta_default_options(sta_options *opt);

/*
 * sta_create -- set up a context for one superset mesh (Sec. 3, "three inputs": superset
 * vertex positions V, candidate pool of tetrahedra; Algorithm 1 inputs V, T).
 *  nodes   host, n_nodes x 3 doubles (x, y, z per node)
 *  tets    host, n_tets x 4 int32 node ids; ids in [0, n_nodes), distinct per tetrahedron,
 *          positively oriented (det[x1-x0, x2-x0, x3-x0] > 0)
 *  young, poisson  host, n_tets doubles each (isotropic material per tetrahedron)
 *  opt     may be NULL (defaults)
 * Builds on the device, once: the superset CSR pattern (row_ptr, col), the tet-to-nnz
 * scatter map (P_tau of Eq. 8 as indices), the per-block contributor lists in ascending
 * tetrahedron id, and the element-matrix cache of every superset tetrahedron.  The initial
 * active set is empty and all values are +0.0; call sta_full_rebuild with the initial mask
 * (Algorithm 1 "a_0").  Synchronises `stream`.  Errors: STA_EINVAL for a bad id, a repeated
 * node or a tetrahedron with det <= 0 (its index is in sta_last_error()); STA_ERANGE when
 * nnz or 16 * n_tets exceeds int32 or n_tets > 25,565,281 (84 n_tets < 2^31: 31-bit offsets
 * into the element cache); STA_ENOMEM; STA_ECUDA.
 */
int sta_create(const double *nodes, int64_t n_nodes, const int32_t *tets, int64_t n_tets,
               const double *young, const double *poisson, const sta_options *opt,
               void *stream, sta_ctx **out);

/* Releases all device and host memory of the context (synchronises its last stream). */
int sta_destroy(sta_ctx *ctx);

/*
 * sta_full_rebuild -- the full_rebuild policy (Sec. 3.5): set the active mask and recompute
 * every value of the pattern from scratch from the element cache.
 *  mask            n_tets bytes, nonzero = active; host memory if mask_on_device == 0,
 *                  else device memory
 * With a device mask the host mirror used for edit validation is refreshed by a
 * device-to-host copy, which synchronises `stream`.  Either way the context keeps the mask as
 * 0/1 bytes (sta_mask).
 */
int sta_full_rebuild(sta_ctx *ctx, const uint8_t *mask, int mask_on_device, void *stream);

/*
 * sta_refold -- the full_rebuild policy (Sec. 3.5) on the maintained mask: recompute every
 * value of the pattern from scratch from the current active mask and element cache (use it
 * after sta_set_params / sta_recompute_elements, or to time a rebuild without a mask copy).
 */
int sta_refold(sta_ctx *ctx, void *stream);

/* Change the rebuild fold's launch shape (same meaning as the sta_options fields; results do
 * not depend on it; the streaming fold always runs at occupancy maximum).  Not allowed while
 * graph mode is on (STA_ESTATE). */
int sta_set_launch(sta_ctx *ctx, int32_t block_threads, int32_t blocks_per_sm);

/* Operand loads each lane of the rebuild fold keeps in flight: 4 (default; the fold kernel
 * then fits 64 registers a thread, 32 resident warps per SM) or 6 (80 registers, 24 warps).
 * The fold is bound by load latency and which choice hides it better depends on the mesh and
 * mask; results do not depend on it.  A launch choice of the library with no counterpart in
 * the paper.  Not allowed while graph mode is on (STA_ESTATE); STA_EINVAL for another value. */
int sta_set_fold_depth(sta_ctx *ctx, int32_t operands_in_flight);

/*
 * sta_set_rebuild_form -- how the full rebuild (sta_full_rebuild, sta_refold; Sec. 3.5) writes
 * the values; the values are the same bits in every form.
 *  STA_REBUILD_FUSED:     one fold kernel writes every value, +0.0 for the entries without an
 *                         active contributor.  Suits a superset that is mostly active.
 *  STA_REBUILD_ZERO_FILL: a coalesced fill sets every value to +0.0 while the tiles of fold
 *                         units with an active contributor are flagged from the mask; the fold
 *                         then visits only the flagged tiles (and, when eps != 0, the diagonal
 *                         ones).  Suits a superset that is mostly inactive (preallocated
 *                         refinement children, split copies).  Takes 4 more bytes of device
 *                         memory per fold unit and 2 per tile of 32 fold entries (at create).
 *  STA_REBUILD_AUTO:      (default) ZERO_FILL while fewer than 40% of the tetrahedra are
 *                         active, else FUSED; decided when the rebuild is issued (in graph mode:
 *                         when sta_graph_enable captures it).
 * A launch choice of the library with no counterpart in the paper.  Not allowed while graph
 * mode is on (STA_ESTATE); STA_EINVAL for another value.
 */
#define STA_REBUILD_AUTO 0
#define STA_REBUILD_FUSED 1
#define STA_REBUILD_ZERO_FILL 2
int sta_set_rebuild_form(sta_ctx *ctx, int32_t form);

/* The form (STA_REBUILD_FUSED or STA_REBUILD_ZERO_FILL) a rebuild issued now would take, AUTO
 * resolved for the current mask. */
int sta_get_rebuild_form(const sta_ctx *ctx, int32_t *form);

/*
 * sta_apply_edits -- one frame of the streaming update (Sec. 3.2; Algorithm 1 receive /
 * update mask / per-tet update; Sec. 3.5 local_recompute made bitwise): applies the edits to
 * the mask, marks every block of the pattern touched by an edited tetrahedron (its 16 node
 * pairs, 144 entries), and re-folds exactly those entries over their active contributors in
 * the same canonical order as sta_full_rebuild, so the result is bit-identical to a rebuild.
 *  edits   host array of n_edits sta_edit, validated against the host mirror of the mask:
 *          op in {0,1,2}; ids in range; DEACTIVATE needs an active tet, ACTIVATE an
 *          inactive one, SWAP an active tet and an inactive tet2; no tetrahedron twice.
 *          On a bad edit nothing changes and STA_EINVAL is returned with its index.
 * n_edits == 0 is a valid no-op frame.
 */
int sta_apply_edits(sta_ctx *ctx, const sta_edit *edits, int64_t n_edits, void *stream);

/* Number of distinct CSR entries re-folded by the last sta_apply_edits (= 9 x touched node
 * pairs).  Reads a device counter: synchronises `stream`. */
int sta_last_touched(sta_ctx *ctx, int64_t *touched_nnz, void *stream);

/* Device pointers of the CSR arrays (owned by the context; pattern fixed for its lifetime).
 * row_ptr: n_rows + 1 int32; col: nnz int32; val: nnz doubles.  Any out-pointer may be
 * NULL. */
int sta_csr(const sta_ctx *ctx, const int32_t **row_ptr, const int32_t **col,
            const double **val, int64_t *n_rows, int64_t *nnz);

/* Device pointer to the scatter map, n_tets x 144 int32: scat[t][12p + q] is the CSR index
 * of the global entry (3 v_a + i, 3 v_b + j) for local p = 3a + i, q = 3b + j -- the
 * injection P_tau of Eq. 8 written as indices. */
int sta_scatter_map(const sta_ctx *ctx, const int32_t **scat);

/* Sizes: nodes, tets, node-pair blocks (nnz / 9), and device bytes held by the context. */
int sta_sizes(const sta_ctx *ctx, int64_t *n_nodes, int64_t *n_tets, int64_t *n_blocks,
              int64_t *device_bytes);

/* Device pointer to the current active mask (n_tets bytes, 0/1), owned by the context. */
int sta_mask(const sta_ctx *ctx, const uint8_t **mask);

/*
 * sta_recompute_elements -- recompute the element-matrix cache (the element part of the
 * paper's full_rebuild, Sec. 3.5), for active tetrahedra only (active_only != 0) or for the
 * whole superset.  Element matrix K^(tau) (Sec. 3.4, Sec. 5.2: standard linear-tetrahedron
 * elasticity), fixed evaluation order:
 *   d_k = x_k - x_0;  c_1 = d_2 x d_3, c_2 = d_3 x d_1, c_3 = d_1 x d_2 with
 *   (u x v).x = fma(u.y, v.z, -(u.z v.y)) and cyclic;  det = fma(d1.z, c1.z, fma(d1.y, c1.y,
 *   d1.x c1.x));  r = 1/det;  g_k = c_k r;  g_0 = -((g_1 + g_2) + g_3);  V = det / 6;
 *   lam = (E nu) / ((1 + nu)(1 - (nu + nu)));  mu = E / ((1 + nu) + (1 + nu));
 *   P_a = (V lam) g_a;  Q_a = (V mu) g_a;  D_ab = (V mu) fma(g_a.z, g_b.z, fma(g_a.y, g_b.y,
 *   g_a.x g_b.x));  for p = 3a+i <= q = 3b+j:  K = fma(P_a[i], g_b[j], Q_a[j] g_b[i]) if
 *   i != j, else fma(P_a[i], g_b[i], fma(Q_a[i], g_b[i], D_ab));  K[q][p] = K[p][q].
 * All other operations are separately rounded IEEE double operations.
 */
int sta_recompute_elements(sta_ctx *ctx, int active_only, void *stream);

/*
 * sta_set_params -- replace node positions and/or materials (any pointer may be NULL to
 * keep the current values) and recompute the element cache of the whole superset.  Arrays
 * are host memory unless on_device != 0 (then device memory of the same layout: nodes n x 3
 * doubles, young/poisson n_tets doubles).  Values are NOT re-folded: call
 * sta_full_rebuild afterwards.  Tetrahedra with det <= 0 make the call fail with STA_EINVAL
 * after the copy (synchronises `stream`); the context then holds the new parameters.
 */
int sta_set_params(sta_ctx *ctx, const double *nodes, const double *young,
                   const double *poisson, int on_device, void *stream);

/*
 * sta_element_matrices -- expand the cached element matrices of n tetrahedra to full 12x12
 * row-major doubles.  tet_ids: device, n int32 (each in range, checked on the device:
 * out-of-range ids give zero matrices); out: device, n x 144 doubles.
 */
int sta_element_matrices(sta_ctx *ctx, const int32_t *tet_ids, int64_t n, double *out,
                         void *stream);

/*
 * sta_adjoint -- reverse-mode derivative of the assembly (Eq. 8) with respect to the element
 * parameters, for the current active mask.  Given grad_val = dL/dA per CSR entry (device,
 * nnz doubles; entries of the same pattern as sta_csr), computes on the device
 *   dE  (n_tets doubles)  dL/dE_tau,   dnu (n_tets doubles)  dL/dnu_tau   (0 for inactive),
 *   dX  (n_nodes x 3 doubles)  dL/dx_v, summed over the active tetrahedra incident to v in
 *       ascending id (deterministic).
 * Element matrices are recomputed from positions and materials (not read from the cache).
 * The first call allocates a per-element scratch of 96 bytes per tetrahedron held by the
 * context.  All pointers are device memory.
 */
int sta_adjoint(sta_ctx *ctx, const double *grad_val, double *dE, double *dnu, double *dX,
                void *stream);

/* y = A x over the context's pattern (device vectors of n_rows doubles), with the values `val`
 * (device, nnz doubles) or, when val is NULL, the context's current values; each row is summed
 * in ascending column order.  For consumers such as the conjugate-gradient solve. */
int sta_spmv(sta_ctx *ctx, const double *val, const double *x, double *y, void *stream);

/*
 * sta_apply_edits_noalloc -- the same streaming update as sta_apply_edits, for callers that
 * must not allocate (no counterpart in the paper).  sta_apply_edits may grow a pinned host
 * buffer and a device buffer on its first call or when a frame edits more tetrahedra than
 * before; a frame loop that must never stall on cudaMalloc, or a process whose GPU memory is
 * held by a framework's caching allocator, cannot allow that.  This variant calls no
 * allocator: its per-call scratch (edited-tet list, touched-unit list, counters) is one
 * fixed device array of 44 x STA_NOALLOC_MAX_EDITED + 32 bytes (about 1.4 MB) that every GPU
 * loading the library holds until the process exits.  Arguments, validation, results and errors are those of
 * sta_apply_edits, plus:
 *  - at most STA_NOALLOC_MAX_EDITED edited tetrahedra per call (a swap counts two); more
 *    is rejected with STA_ERANGE before any device work;
 *  - the context's device must be current; the first call on each device looks up the
 *    array's device address (cudaGetSymbolAddress), so make that first call before any
 *    stream capture;
 *  - all calls, on every context and stream of a device, share the one array: calls that
 *    overlap on the GPU race and must be serialised by the caller;
 *  - the edit list is copied from pageable host memory, so the call returns only after that
 *    copy has been staged.
 */
#define STA_NOALLOC_MAX_EDITED 32768
int sta_apply_edits_noalloc(sta_ctx *ctx, const sta_edit *edits, int64_t n_edits, void *stream);

/*
 * Batched form: k independent superset meshes in one context.  Instance i's arrays (host) are
 * given by pointer; node ids are local to the instance.  The instances are concatenated with
 * disjoint id ranges (instance i's tetrahedra get global ids tet_offset_i + local id), so the
 * assembled matrix is block diagonal and each instance's values are bit-identical to those of
 * a context created for that instance alone.  sta_full_rebuild takes the concatenated mask
 * (sum of n_tets bytes, instances in order); sta_refold, sta_recompute_elements and
 * sta_graph_enable work on the whole batch; one call drives every instance with one launch
 * sequence (one persistent fold over the blocks of all instances).
 */
int sta_batch_create(int32_t k, const int64_t *n_nodes, const double *const *nodes,
                     const int64_t *n_tets, const int32_t *const *tets,
                     const double *const *young, const double *const *poisson,
                     const sta_options *opt, void *stream, sta_ctx **out);

/* Number of instances of a batched context (0 for a plain context). */
int sta_batch_size(const sta_ctx *ctx, int32_t *k);

/* Instance i's CSR in its own numbering: row_ptr (3 n_i + 1, from 0) and col (local DOFs) are
 * device index arrays owned by the context; val points at the instance's slice of the batch
 * values.  tet_offset is the global id of the instance's first tetrahedron. */
int sta_batch_instance(const sta_ctx *ctx, int32_t i, const int32_t **row_ptr,
                       const int32_t **col, const double **val, int64_t *n_rows, int64_t *nnz,
                       int64_t *tet_offset);

/* One streaming frame for every instance: counts[i] edits of instance i (tet ids local to the
 * instance) follow each other in `edits`.  Same validation and results as sta_apply_edits. */
int sta_batch_apply_edits(sta_ctx *ctx, const int64_t *counts, const sta_edit *edits,
                          void *stream);

/*
 * sta_graph_enable -- capture the per-frame device work of the context into CUDA graphs: the
 * streaming update (mask and activity update, touched-block dedupe, fold; the edit count and
 * list read from the staging block below, grids sized for max_edited), the refold, and the
 * fold of a full rebuild.  Afterwards sta_apply_edits (frames of at most max_edited edited tetrahedra; a
 * swap counts two), sta_refold and sta_full_rebuild replay them with one cudaGraphLaunch each;
 * results are unchanged.  A frame is staged in one of two host-mapped pinned blocks (used in
 * turn) that the captured kernels read directly, so it costs no copy call; the block is
 * reused once the frame two calls back has finished.  Allocates those blocks and two sets of
 * device counters (each frame's last kernel zeroes the set of the frame after it) and
 * synchronises `stream`.  sta_graph_disable releases them and returns to plain
 * launches.
 */
int sta_graph_enable(sta_ctx *ctx, int64_t max_edited, void *stream);
int sta_graph_disable(sta_ctx *ctx, void *stream);

/*
 * sta_set_policy -- how sta_apply_edits maintains the values, and what a rebuild computes.
 *  STA_POLICY_REFOLD (default): every touched entry is re-folded from +0.0 over its active
 *    contributions in ascending tetrahedron id (the local_recompute policy of Sec. 3.5 made
 *    bitwise); values are the canonical FP64 fold.
 *  STA_POLICY_FIXED: the streaming_update of Sec. 3.4 / 3.5 (add or subtract the edited
 *    tetrahedra's contributions, O(|Delta|)) made exact in fixed point: each entry k has a
 *    binary exponent e_k fixed by its superset contributions (2^-62 of the largest, times the
 *    contributor count rounded up to a power of two), each contribution is quantised once to
 *    the nearest integer multiple of 2^e_k, the context keeps the exact integer sum per entry
 *    and a value is that sum converted once (+ eps on the diagonal).  Streaming equals the
 *    fixed-point rebuild bit for bit; values are within about 2^-56 of each entry's largest
 *    contribution of the FP64 fold.
 * Switching computes what the policy needs (exponents and quantised contributions, about
 * 8.5 bytes per nnz and 672 bytes per tetrahedron on first use) and rebuilds every value from
 * the current mask.  Not allowed while graph mode is on (STA_ESTATE); graphs enabled afterwards
 * capture the current policy.  sta_set_params / sta_recompute_elements recompute the
 * fixed-point inputs under STA_POLICY_FIXED (values are not re-folded; call sta_refold).
 */
#define STA_POLICY_REFOLD 0
#define STA_POLICY_FIXED 1
int sta_set_policy(sta_ctx *ctx, int32_t policy, void *stream);

/*
 * Graph-Laplacian proxy operator (Sec. 3.1 Eqs. 1-4, Sec. 3.2 Eqs. 5-7, Sec. 3.3,
 * Algorithm 1).  sta_proxy_create makes a context for the scalar n x n matrix
 *     A_t = L_t + eps I,   L_t(u, v) = -a_t(u, v) (u != v),   L_t(u, u) = sum_{w != u} a_t(u, w),
 *     a_t(u, v) = 1[c_t(u, v) > 0],   c_t(u, v) = #active tetrahedra with edge {u, v},
 * over the same superset mesh and edit model as the elasticity operator.
 *  - Layout: node-level CSR, n rows; row u holds every node sharing a SUPERSET tetrahedron
 *    with u (u included), ascending.  Inactive edges keep their slot and hold +0.0, active
 *    ones -1.0; the diagonal is (double) degree + eps.  A node of no tetrahedron has an empty
 *    row.  sta_csr returns this CSR (n_rows = n, nnz = n_blocks of sta_sizes).
 *  - State: the edge multiplicities c_t and node degrees, int32 (sta_proxy_state), the mask
 *    and the values.  All of it is integer arithmetic, so values are exact.
 *  - Calls: sta_full_rebuild (count c over the active set, then Eqs. 2-4), sta_refold (the
 *    same from the current mask), sta_apply_edits / sta_apply_edits_noalloc (the streaming
 *    rule: +-1 on the multiplicity of each edge of each edited tetrahedron, off-diagonal
 *    entries set or cleared and the end nodes' degrees moved where a multiplicity moves
 *    between 0 and > 0), sta_last_touched (entries the last frame visited: both entries of
 *    each edge and the diagonal entry of each node of the edited tetrahedra), sta_graph_*,
 *    sta_mask, sta_sizes, sta_spmv, sta_solve, sta_destroy.  The streamed state equals a
 *    rebuild on the same mask bit for bit.  sta_set_policy chooses the update:
 *    STA_POLICY_FIXED (the default for the proxy: the maintained multiplicities updated by
 *    +-1, Sec. 3.2) or STA_POLICY_REFOLD (the paper's local_recompute: each touched edge
 *    recounted over the tetrahedra incident to it, each touched node's degree over its row);
 *    same values and state.  Calls of the elasticity operator (sta_set_params,
 *    sta_recompute_elements, sta_element_matrices, sta_scatter_map, sta_adjoint) return
 *    STA_ESTATE.
 * Create: tets (n_tets x 4 int32, host) as for sta_create; every tetrahedron starts inactive
 * (A = eps I on the nodes of the mesh).  Limits: n_tets < 2^27, nnz < 2^31.
 */
int sta_proxy_create(int64_t n_nodes, const int32_t *tets, int64_t n_tets, double eps,
                     void *stream, sta_ctx **out);
/* Device pointers (context-owned): mult[g] = c_t of the edge of block g for each upper block
 * (col[g] > row node); 0 at every other block; degree[u] = sum_{w != u} a_t(u, w).
 * STA_ESTATE for an elasticity context.  Either pointer argument may be NULL. */
int sta_proxy_state(const sta_ctx *ctx, const int32_t **mult, const int32_t **degree);

/*
 * Implicit-Euler dynamic loop on the maintained operator (Sec. 6.2, Eq. 9): each step solves
 *     (M_t + h^2 K_t) u_{t+1} = M_t (u_t + h v_t) + h^2 f,   v_{t+1} = (u_{t+1} - u_t) / h,
 * with K_t the context's current values (eps included) and M_t a lumped mass maintained with
 * the mask.  Elasticity contexts only (STA_ESTATE otherwise).
 *  - Lumped mass (the paper gives no formula): each active tetrahedron gives (rho V) / 4 to
 *    each of its four nodes (all three DOFs), V = det / 6 in the element matrix's fixed order,
 *    folded per node from +0.0 in ascending tetrahedron id; after every sta_apply_edits (the
 *    nodes of the edited tetrahedra are re-folded), sta_full_rebuild, sta_refold and
 *    sta_set_params it equals a from-scratch evaluation bit for bit.  A node of no active
 *    tetrahedron has mass +0.0.
 *  - Free DOFs: those of nodes that are not clamped and have mass.  A clamped DOF is held at
 *    0; a DOF of a node without mass keeps its displacement, with velocity 0.
 *  - Solve: Jacobi-preconditioned CG from x = u_t until ||r|| <= tol ||b|| or max_iter
 *    iterations, deterministic (fixed-order reductions).
 * sta_dyn_setup: rho, h > 0; f (3n, host, NULL = 0) and clamped (n, host, NULL = none) are
 * copied; u = v = 0; computes the per-tetrahedron quarter masses and the lumped mass of the
 * current mask.  Not allowed in graph mode (STA_ESTATE); graphs enabled afterwards include
 * the mass update.  May be called again to change rho, h, f or clamped (resets u and v).
 * sta_dyn_step: one step; synchronises `stream`; *iters = CG iterations, *rel_res =
 * ||r|| / ||b|| at exit (0 when b = 0); either may be NULL.  Reaching max_iter is not an error.
 * sta_dyn_apply: y = (M_t + h^2 K_t) x on the free DOFs, 0 elsewhere (x read on the free DOFs
 * only); x and y are device arrays of 3n doubles, y must not overlap x; asynchronous on
 * `stream`.  The operator the step's CG applies, for a caller's own solver.
 * sta_dyn_state: device pointers (context-owned): u, v (3n) and the lumped mass (n).
 * sta_dyn_set_state: overwrite u and/or v (3n each, host or device; NULL = keep).
 */
int sta_dyn_setup(sta_ctx *ctx, double rho, double h, const double *f, const uint8_t *clamped,
                  void *stream);
int sta_dyn_step(sta_ctx *ctx, double tol, int32_t max_iter, int32_t *iters, double *rel_res,
                 void *stream);
int sta_dyn_apply(sta_ctx *ctx, const double *x, double *y, void *stream);
int sta_dyn_state(const sta_ctx *ctx, const double **u, const double **v, const double **mass);
int sta_dyn_set_state(sta_ctx *ctx, const double *u, const double *v, int on_device, void *stream);

/*
 * sta_solve -- the consumer of the assembly (the paper's solver, Sec. 4: conjugate gradients
 * with diagonal preconditioning) for a static problem A_ff x_f = b_f: Jacobi-PCG on the DOFs
 * with free[i] != 0 (and a nonzero diagonal), x = 0 elsewhere, from the initial guess in x,
 * until ||r|| <= tol ||b_f||, max_iter iterations, or no halving of the residual for 1000
 * iterations (the attainable accuracy).  val: device nnz values of the context's pattern
 * (NULL = the current values); b, x: device n_rows doubles; free: device n_rows bytes
 * (n_rows of sta_csr: 3n for elasticity, n for the proxy operator, whose solve is the paper's
 * per-frame solve of Algorithm 1).  Same kernels as the implicit-Euler step (fixed-order
 * reductions: deterministic).  Synchronises `stream`.  *iters and *rel_res (||r|| / ||b_f||
 * from the recurrence) may be NULL.  Both operators.
 *
 * sta_outer_grad -- the adjoint rule of such a solve: grad_val[k] = -lam[row(k)] u[col(k)]
 * for entries k between free DOFs, 0 elsewhere (lam, u: device nrows doubles; free: device
 * nrows bytes; grad_val: device nnz doubles).  Asynchronous on `stream`.
 */
int sta_solve(sta_ctx *ctx, const double *val, const double *b, const uint8_t *free, double tol,
              int32_t max_iter, double *x, int32_t *iters, double *rel_res, void *stream);
int sta_outer_grad(sta_ctx *ctx, const double *lam, const double *u, const uint8_t *free,
                   double *grad_val, void *stream);

/* Human-readable message of the last error on the calling thread. */
const char *sta_last_error(void);
const char *sta_status_string(int status);

#ifdef __cplusplus
}
#endif

#endif /* STA_H */
