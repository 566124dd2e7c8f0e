// Internal declarations of libsta: context layout, device helpers shared by the fold
// kernels, launch helpers.  Not part of the public ABI (see include/sta.h).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "sta.h"

namespace sta {

// ------------------------------------------------------------------------------------
// Error plumbing
// ------------------------------------------------------------------------------------
void set_error(const std::string &msg);
int fail(int code, const std::string &msg);

#define STA_CUDA_TRY(expr)                                                                   \
    do {                                                                                     \
        cudaError_t _e = (expr);                                                             \
        if (_e != cudaSuccess)                                                               \
            return ::sta::fail(_e == cudaErrorMemoryAllocation ? STA_ENOMEM : STA_ECUDA,     \
                               std::string(#expr) + ": " + cudaGetErrorString(_e));         \
    } while (0)

#define STA_TRY(expr)                                                                        \
    do {                                                                                     \
        int _s = (expr);                                                                     \
        if (_s != STA_OK) return _s;                                                         \
    } while (0)

// ------------------------------------------------------------------------------------
// Element cache: the 78 unique entries of each symmetric 12x12 element matrix, grouped by 3x3
// node-pair block into runs, stored as two row arrays in one allocation of 84 T doubles:
//   Kd = Ke[0 .. 24T):   row 4t + a (6 doubles, 48 B): diagonal block (a, a), entries i <= j
//                        row-major: (0,0) (0,1) (0,2) (1,1) (1,2) (2,2)
//   Kp = Ke[24T .. 84T): row 6t + pair(a, b) (10 doubles, 80 B: 9 entries + a +0.0 pad), a < b
//                        local indices: the block row-major over the node with the LOWER global
//                        id, i.e. K[3a+i][3b+j] at 3i+j if id(a) < id(b), else at 3j+i
// with pair(0,1..3) = 0..2, pair(1,2..3) = 3..4, pair(2,3) = 5.  Every run starts on a 16-byte
// boundary.  Oriented this way, the contribution of any tetrahedron to the node-pair block
// (a, b), id(a) < id(b), is one row read as is (the folds never transpose), and the rows of
// one kind have one width (whole-row gathers).  A tet's record is computed in the order
// diagonal runs then pair runs (84 doubles, KE_STRIDE), then split between the two arrays.
// ------------------------------------------------------------------------------------
constexpr int KE_STRIDE = 84;
constexpr int KE_DIAG = 24;   // doubles of a tet's 4 diagonal runs (Kd)
constexpr int KE_PAIR = 60;   // doubles of a tet's 6 pair runs (Kp)

__host__ __device__ inline int ke_diag_off(int a) { return 6 * a; }
__host__ __device__ inline int ke_pair(int a, int b) {  // a < b
    return a == 0 ? b - 1 : (a == 1 ? b + 1 : 5);
}
__host__ __device__ inline int ke_off_off(int a, int b) { return 24 + 10 * ke_pair(a, b); }
// Ke offset of tet t's diagonal run a, and of its pair run p
__host__ __device__ inline int64_t ke_diag_at(int64_t T, int64_t t, int a) {
    (void)T;
    return KE_DIAG * t + 6 * a;
}
__host__ __device__ inline int64_t ke_pair_at(int64_t T, int64_t t, int p) {
    return KE_DIAG * T + KE_PAIR * t + 10 * p;
}
// index of (i, j), i <= j, inside a diagonal 6-run
__host__ __device__ inline int ke_tri(int i, int j) {
    return i == 0 ? j : (i == 1 ? 2 + j : 5);
}

// Contributor code of a fold unit (node pair a <= b): tetrahedron id and the local indices of
// the unit's nodes a (la) and b (lb) inside that tetrahedron; bit 31 holds the tetrahedron's
// current activity (kept equal to the mask by every call that changes it).
constexpr uint32_t CODE_ACTIVE = 0x80000000u;
__host__ __device__ inline int32_t contrib_code(int32_t t, int la, int lb) {
    return (t << 4) | (la << 2) | lb;
}
__host__ __device__ inline int32_t code_tet(int32_t code) { return (code >> 4) & 0x07ffffff; }

// Contributor word of a unit list (ccode after create): the element-cache offset of the
// contributor's run for the unit (ke_diag_at / ke_pair_at) | active << 31.
__host__ __device__ inline uint32_t word_offset(uint32_t w) { return w & 0x7fffffffu; }
__host__ __device__ inline int32_t word_tet(uint32_t w, int64_t T) {
    const int64_t off = word_offset(w);
    return (int32_t)(off < KE_DIAG * T ? off / KE_DIAG : (off - KE_DIAG * T) / KE_PAIR);
}
// the run of tet t for unit slot s (0..3 diagonal, 4..9 pairs)
__host__ __device__ inline int64_t ke_slot_at(int64_t T, int64_t t, int s) {
    return s < 4 ? ke_diag_at(T, t, s) : ke_pair_at(T, t, s - 4);
}

// The 10 unit slots of a tetrahedron: 0..3 diagonal (la, la), 4..9 the pairs (0,1) (0,2) (0,3)
// (1,2) (1,3) (2,3).
__host__ __device__ inline int slot_la(int s) { return s < 4 ? s : (s < 7 ? 0 : (s < 9 ? 1 : 2)); }
__host__ __device__ inline int slot_lb(int s) {
    return s < 4 ? s : (s == 4 ? 1 : (s == 5 ? 2 : (s == 6 ? 3 : (s == 7 ? 2 : 3))));
}
__host__ __device__ inline int slot_of(int la, int lb) {  // unordered local pair -> slot
    if (la == lb) return la;
    const int lo = la < lb ? la : lb, hi = la < lb ? lb : la;
    return 4 + (lo == 0 ? hi - 1 : (lo == 1 ? hi + 1 : 5));
}

// Lanes of the rebuild fold per unit (one fold entry each): a diagonal unit folds its 6
// distinct entries, an off-diagonal unit its 9.
constexpr int FOLD_TASKS_DIAG = 6;
constexpr int FOLD_TASKS_PAIR = 9;

// Frame block: what one streaming frame moves to the device in a single transfer -- the
// edited count, the frame's counters (zeroed by the host) and the edited list (tet id | new
// state << 31) right after the header.
struct FrameHeader {
    int64_t m;                     // edited tetrahedra
    unsigned long long cnt[3];     // touched units, unused, touched CSR entries (the FP64
                                   // re-fold counts its units as diagonal | pair << 32)
};
static_assert(sizeof(FrameHeader) == 32, "frame header layout");
// counter view with the indices of Ctx::counters: [1] touched units, [3] touched entries
inline unsigned long long *frame_counters(FrameHeader *f) {
    return reinterpret_cast<unsigned long long *>(f);
}
inline int32_t *frame_edited(FrameHeader *f) { return reinterpret_cast<int32_t *>(f + 1); }
inline size_t frame_bytes(int64_t m) { return sizeof(FrameHeader) + sizeof(int32_t) * (size_t)m; }

// ------------------------------------------------------------------------------------
// Context
// ------------------------------------------------------------------------------------
// Operator of a context: the elasticity operator (sta_create, sta_batch_create) or the
// graph-Laplacian proxy (sta_proxy_create).
constexpr int STA_OP_ELASTICITY = 0;
constexpr int STA_OP_PROXY = 1;

struct Ctx {
    int op = STA_OP_ELASTICITY;
    int64_t n = 0, T = 0, nblocks = 0, nnz = 0, nrows = 0;
    double eps = 0.0;
    int block_threads = 256;
    int blocks_per_sm = 0;
    int fold_depth = 4;            // operand loads in flight per lane of the rebuild fold: 4 or 6
    int rebuild_form = STA_REBUILD_AUTO;  // sta_set_rebuild_form
    int64_t n_active = 0;                 // active tetrahedra (host mirror count)
    int num_sms = 0;
    int device = 0;

    // inputs
    double4_32a *X = nullptr;   // n, (x, y, z, 0)
    int4 *tets = nullptr;   // T
    double2 *mat = nullptr; // T, (E, nu)

    // pattern
    int32_t *adj_ptr = nullptr;    // n + 1: first block of node a
    int32_t *adj = nullptr;        // nblocks: neighbour node of each block (ascending per node)
    int32_t *block_node = nullptr; // nblocks: owner node of each block
    int32_t *row_ptr = nullptr;    // 3n + 1
    int32_t *col = nullptr;        // nnz
    int32_t *tblk = nullptr;       // T x 16: block of local pair (la, lb) = 4 la + lb
    int32_t *scat = nullptr;       // T x 144: CSR index of local entry (p, q)
    int2 *boff = nullptr;          // nblocks: {first value index, row stride}
    // Fold units: unordered node pairs {a <= b}.  Entry (3a+i, 3b+j) and its mirror
    // (3b+j, 3a+i) fold the same operands in the same order (the element matrices are exactly
    // symmetric), so one fold per unit writes both blocks.
    int64_t nunits = 0;
    int64_t ntiles = 0;
    int4 *ftile = nullptr;         // ntiles: rebuild fold tiles {first unit, q0 | diag << 4 |
                                   //   entries << 5, code range of the tile's units}
    // zero-fill rebuild (sta_rebuild.cu): per unit its first tile | reaches the next << 31;
    // per tile whether its units are diagonal, and its flag "fold this tile"
    int32_t *utile = nullptr;      // nunits
    uint8_t *tdiag = nullptr;      // ntiles
    uint8_t *tflag = nullptr;      // ntiles: zero-fill flags, all zero between rebuilds
    int4 *bmeta = nullptr;         // nunits: {value offset of (a,b), rs_a << 1 | diagonal, c0, c1}
    int2 *bmirror = nullptr;       // nunits: {value offset of (b,a), rs_b}
    int32_t *ccode = nullptr;      // 10 T: unit contributor words (word_offset), ascending tet id
    int32_t *cslot = nullptr;      // T x 10: position in ccode of tet t's unit slot
    int32_t *tunit = nullptr;      // T x 10: unit of tet t's slot (4 diagonal, 6 pairs)
    int32_t *nt_ptr = nullptr;     // n + 1: node -> incident tetrahedra
    int32_t *nt_list = nullptr;    // 4 T: incident tetrahedra, ascending id
    double *dXe = nullptr;         // T x 12: per-element position gradients (adjoint, lazily)
    int32_t *act_list = nullptr;   // T: active tets, unordered (element / adjoint kernels, lazily)
    unsigned long long *act_count = nullptr;

    // state
    double *Ke = nullptr;       // 84 T: element cache, diagonal runs then pair runs (KE_DIAG, KE_PAIR)
    // update policy (STA_POLICY_*) and the fixed-point state (sta_fixed.cu), allocated on first use
    int policy = STA_POLICY_REFOLD;
    long long *fx_q = nullptr;  // 84 T: quantised contributions at the element-cache offsets
    int16_t *fx_e = nullptr;    // nnz: exponent of each entry (keyed by its upper-block index)
    long long *fx_s = nullptr;  // nnz: exact integer sum of each entry's active contributions
    uint8_t *mask = nullptr;    // T
    double *val = nullptr;      // nnz
    int32_t *owner = nullptr;   // nunits: streaming dedupe slot, INT32_MAX when free
    int32_t *touched = nullptr; // nunits: list of units touched by the current frame
    // [0] bad elements, [1] touched units, [2] first bad element, [3] touched CSR entries
    unsigned long long *counters = nullptr;

    // streaming staging: one frame block on the device and its pinned host copy
    FrameHeader *d_frame = nullptr, *h_frame = nullptr;
    int64_t edit_cap = 0;         // edited tetrahedra a frame block holds
    int64_t last_edited = 0;
    unsigned long long *last_counters = nullptr;  // device counters of the last frame
    // host-mapped pinned word the re-fold streaming frame's fold kernel stores its touched-entry
    // count into (h: host address, d: its device address); count_on_host: the last frame did
    unsigned long long *h_count_mapped = nullptr, *d_count_mapped = nullptr;
    bool count_on_host = false;
    uint8_t stamp_gen = 0;        // the sta_apply_edits call's stamp (1 .. 127), see tstate

    // graph-Laplacian proxy operator (sta_proxy.cu); its CSR is the node-level pattern
    // (row_ptr = adj_ptr, col = adj, nrows = n, nnz = nblocks)
    int32_t *ptblk = nullptr;   // T x 10: block of tet t's unit slot s (diagonal; upper edge block)
    int32_t *pmir = nullptr;    // nblocks: block (b, a) of block (a, b)
    int32_t *pup = nullptr;     // nblocks: upper block of the block's edge, -1 on the diagonal
    int32_t *pdiag = nullptr;   // n: diagonal block of each node, -1 for a node of no tetrahedron
    int32_t *pmult = nullptr;   // nblocks + n: edge multiplicity at the upper block, then degrees
    uint32_t *pflag = nullptr;  // nblocks: claim flags of the frame's touched blocks
    int32_t *plist = nullptr;   // nblocks: the frame's touched blocks

    // implicit-Euler loop (sta_dyn.cu), allocated by the first sta_dyn_setup
    bool dyn = false;
    double dyn_rho = 0.0, dyn_h = 0.0;
    double *qmass = nullptr;    // T: (rho V) / 4 of each tetrahedron
    double *mass = nullptr;     // n: lumped mass per node, maintained with the mask
    double *du = nullptr, *dv = nullptr, *df = nullptr;  // 3n: displacement, velocity, load
    uint8_t *clamped = nullptr; // n
    double *cg = nullptr;       // 7 x 3n: x, b, r, z, p, q, D^-1
    uint8_t *cg_free = nullptr; // 3n: DOF solved for
    double *cg_part = nullptr;  // 3 x cg_grid: per-CTA partial sums
    unsigned char *cg_state = nullptr;  // the solve's device scalars
    int32_t *dyn_perm = nullptr;  // n: the CG SpMV's node order (ascending row length)
    double *cg_zero = nullptr;    // n zeros: the mass term of a static solve (sta_solve)
    int cg_grid = 0;
    cudaGraphExec_t g_cg = nullptr;     // one captured chunk of CG iterations

    // CUDA-graph mode (sta_graph_enable): captured frame sequences and fixed staging
    bool graph_on = false;
    cudaGraphExec_t g_refold = nullptr, g_rebuild = nullptr;
    // graph mode stages frames in two host-mapped pinned blocks that the captured kernels read
    // directly (no copy call per frame), used alternately; each has its own captured sequence,
    // its own device counters (zeroed by the other sequence's last kernel) and an event
    // recorded after its launch, waited on before the block is written again
    int64_t gcap = 0;
    cudaGraphExec_t g_streams[2] = {nullptr, nullptr};
    FrameHeader *h_gframe[2] = {nullptr, nullptr};  // host-mapped pinned, gcap entries each
    FrameHeader *m_gframe[2] = {nullptr, nullptr};  // their device addresses
    unsigned long long *d_gcnt = nullptr;           // 2 x 4 counters
    cudaEvent_t g_done[2] = {nullptr, nullptr};
    bool g_pending[2] = {false, false};
    int g_next = 0;

    // batched form (sta_batch_create): instance offsets and per-instance CSR index arrays
    int32_t n_inst = 0;
    std::vector<int64_t> node_off, tet_off, nnz_off;
    int32_t *local_rp = nullptr;   // sum_i (3 n_i + 1): instance i at 3 node_off[i] + i
    int32_t *local_col = nullptr;  // nnz: column minus the instance's first DOF

    // host mirror of every tetrahedron, one byte: bit 7 = active (the mask), bits 0..6 = the
    // stamp of the last sta_apply_edits call that named it (duplicate check); one random
    // access per edited tetrahedron serves both checks
    std::vector<uint8_t> tstate;
    std::vector<uint8_t> seen;  // per-tet scratch for edit validation (all zero at rest)
    int64_t device_bytes = 0;
    std::vector<void *> allocations;
};

constexpr uint8_t TS_ACTIVE = 0x80;
constexpr uint8_t TS_STAMP = 0x7f;
inline bool ts_active(const Ctx *c, int64_t t) { return (c->tstate[t] & TS_ACTIVE) != 0; }
inline void ts_set_active(Ctx *c, int64_t t, bool on) {
    c->tstate[t] = (uint8_t)((c->tstate[t] & TS_STAMP) | (on ? TS_ACTIVE : 0));
}

template <typename T> int dev_alloc(Ctx *c, T **p, int64_t count) {
    size_t bytes = sizeof(T) * (size_t)(count > 0 ? count : 1);
    cudaError_t e = cudaMalloc((void **)p, bytes);
    if (e != cudaSuccess) {
        *p = nullptr;
        return fail(STA_ENOMEM, std::string("cudaMalloc failed: ") + cudaGetErrorString(e));
    }
    c->allocations.push_back((void *)*p);
    c->device_bytes += (int64_t)bytes;
    return STA_OK;
}

// Persistent grid for an item count: min(ceil(items / threads), SMs * CTAs per SM), CTAs per
// SM = the context's blocks_per_sm (the rebuild's tuned shape) if `tuned` and it is set, else
// the occupancy maximum.
int persistent_grid(const Ctx *c, const void *kernel, int threads, int64_t items,
                    bool tuned = false);

// ------------------------------------------------------------------------------------
// Kernel launchers (each returns STA_OK or STA_ECUDA on a launch error)
// ------------------------------------------------------------------------------------
int build_pattern(Ctx *c, cudaStream_t s);                       // sta_create.cu
int launch_elements(Ctx *c, bool active_only, cudaStream_t s);   // sta_element.cu
int launch_expand_elements(Ctx *c, const int32_t *ids, int64_t n, double *out, cudaStream_t s);
int launch_adjoint(Ctx *c, const double *gval, double *dE, double *dnu, double *dX, cudaStream_t s);
int launch_spmv(Ctx *c, const double *val, const double *x, double *y, cudaStream_t s);
int launch_rebuild(Ctx *c, cudaStream_t s);                      // sta_rebuild.cu
int rebuild_form_of(const Ctx *c);  // the form the next rebuild takes (AUTO resolved)
int launch_stream_frame(Ctx *c, FrameHeader *frame, int64_t cap, cudaStream_t s);  // sta_stream.cu
// whether a streaming frame of this context stores its touched count into h_count_mapped
bool frame_counts_to_host(const Ctx *c);
// the same with the edited list, its count and the counters at separate addresses (the graph
// mode's host-mapped frames keep their counters in device memory); next_cnt: the counters the
// frame's last kernel zeroes for the next frame, or nullptr
int launch_stream_frame(Ctx *c, const int32_t *edited, const int64_t *m_dev,
                        unsigned long long *cnt, int64_t cap, cudaStream_t s,
                        unsigned long long *next_cnt);
int launch_fx_prepare(Ctx *c, cudaStream_t s);                   // sta_fixed.cu
int launch_fx_frame(Ctx *c, const int32_t *edited, int64_t m, const int64_t *m_dev, int64_t cap,
                    int32_t *touched, unsigned long long *counters, cudaStream_t s,
                    unsigned long long *next_cnt);
int launch_mask_bits(Ctx *c, cudaStream_t s);                    // codes <- mask
int launch_values(Ctx *c, cudaStream_t s);  // the operator's rebuild (elasticity or proxy)
int launch_dyn_qmass(Ctx *c, cudaStream_t s);     // sta_dyn.cu (no-ops unless set up)
int launch_dyn_mass_all(Ctx *c, cudaStream_t s);
int launch_dyn_mass_edited(Ctx *c, const int32_t *edited, int64_t m, const int64_t *m_dev,
                           int64_t cap, cudaStream_t s);
int launch_dyn_step(Ctx *c, double tol, int32_t max_iter, int32_t *iters, double *rel_res,
                    cudaStream_t s);
int build_proxy_maps(Ctx *c, const int32_t *tblk, cudaStream_t s);  // sta_proxy.cu
int launch_proxy_rebuild(Ctx *c, cudaStream_t s);
int launch_proxy_frame(Ctx *c, const int32_t *edited, int64_t m, const int64_t *m_dev,
                       int64_t cap, int32_t *list, unsigned long long *counters, cudaStream_t s,
                       unsigned long long *next_cnt);
int launch_stream_scratch(Ctx *c, int64_t m, const int32_t *d_edited, int32_t *touched,
                          unsigned long long *counters, cudaStream_t s);

int create_impl(const double *nodes, int64_t n_nodes, const int32_t *tets, int64_t n_tets,
                const double *young, const double *poisson, const sta_options *opt, void *stream,
                sta_ctx **out);
void graph_release(Ctx *c);  // sta_graph.cu

}  // namespace sta

// The opaque handle of the C-ABI.
struct sta_ctx {
    sta::Ctx c;
    cudaEvent_t h2d_done = nullptr;
    bool h2d_pending = false;
    uint8_t *h_mask = nullptr;  // pinned staging for host masks, T bytes
    unsigned long long *h_count = nullptr;  // pinned word: sta_last_touched's read-back
};
