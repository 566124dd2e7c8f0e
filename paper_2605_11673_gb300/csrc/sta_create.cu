// One-time construction of the superset pattern and index maps on the device (sta_create).
//
// STA-FEM (arXiv 2605.11673) Sec. 3.3 keeps "precomputed tetrahedron-to-edge incidence" and
// the sparse matrix pattern; Eq. 8's P_tau injects the 12 local DOFs of a tetrahedron.  For
// the elasticity operator these become, built once here and never changed:
//   node -> incident tetrahedra (ascending id)       nt_ptr / nt_list (scratch)
//   node-pair blocks: sorted neighbour list per node adj_ptr / adj / block_node
//   scalar CSR                                        row_ptr / col
//   tet -> block of each local node pair              tblk   (T x 16)
//   tet -> CSR index of each local entry              scat   (T x 144)
//   fold units (node pairs a <= b) with their contributors in ascending tet id, and each
//   tetrahedron's 10 unit slots                      bmeta / bmirror / ccode / cslot / tunit
// Lists filled with atomics are sorted afterwards, so every array is deterministic.
#include <algorithm>
#include <climits>

#include "sta_internal.cuh"

namespace sta {
namespace {

constexpr int TPB = 256;

inline unsigned grid_for(int64_t items, int threads = TPB) {
    int64_t g = (items + threads - 1) / threads;
    return (unsigned)(g < 1 ? 1 : g);
}

// ---------------------------------------------------------------- exclusive scan (int64)
// out[0] = 0, out[i + 1] = sum_{k <= i} in[k].  Three phases: per-CTA sums, a single-CTA
// scan of the CTA sums, and a fix-up pass.

constexpr int SCAN_TPB = 1024;

__device__ __forceinline__ int64_t cta_inclusive_scan(int64_t v, int64_t *warp_sums) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int o = 1; o < 32; o <<= 1) {
        int64_t y = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += y;
    }
    if (lane == 31) warp_sums[wid] = v;
    __syncthreads();
    if (wid == 0) {
        int64_t w = (lane < (int)(blockDim.x >> 5)) ? warp_sums[lane] : 0;
        for (int o = 1; o < 32; o <<= 1) {
            int64_t y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += y;
        }
        warp_sums[lane] = w;
    }
    __syncthreads();
    if (wid > 0) v += warp_sums[wid - 1];
    return v;
}

template <typename In>
__global__ void k_scan_tiles(const In *in, int64_t m, int64_t *out, int64_t *tile_sums) {
    __shared__ int64_t ws[32];
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int64_t v = i < m ? (int64_t)in[i] : 0;
    int64_t inc = cta_inclusive_scan(v, ws);
    if (i < m) out[i + 1] = inc;
    if (threadIdx.x == blockDim.x - 1) tile_sums[blockIdx.x] = inc;
}

// Second pass of the exclusive scan: one CTA turns the per-tile totals, in tile order, into
// exclusive tile offsets.
__global__ void k_scan_sums(int64_t *tile_sums, int64_t ntiles) {
    __shared__ int64_t ws[32];
    __shared__ int64_t carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int64_t base = 0; base < ntiles; base += blockDim.x) {
        int64_t i = base + threadIdx.x;
        int64_t v = i < ntiles ? tile_sums[i] : 0;
        int64_t inc = cta_inclusive_scan(v, ws);
        int64_t c = carry;
        if (i < ntiles) tile_sums[i] = c + inc - v;  // exclusive offset of tile i
        __syncthreads();
        if (threadIdx.x == blockDim.x - 1) carry = c + inc;
        __syncthreads();
    }
}

// Third pass: each element gets its tile's offset; out[0] = 0.
__global__ void k_scan_fix(int64_t *out, int64_t m, const int64_t *tile_off) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < m) out[i + 1] += tile_off[blockIdx.x];
    if (i == 0) out[0] = 0;
}

template <typename In>
int exclusive_scan(Ctx *c, const In *in, int64_t m, int64_t *out, int64_t *tmp_tiles,
                   cudaStream_t s) {
    int64_t ntiles = (m + SCAN_TPB - 1) / SCAN_TPB;
    if (ntiles < 1) ntiles = 1;
    k_scan_tiles<In><<<(unsigned)ntiles, SCAN_TPB, 0, s>>>(in, m, out, tmp_tiles);
    k_scan_sums<<<1, SCAN_TPB, 0, s>>>(tmp_tiles, ntiles);
    k_scan_fix<<<(unsigned)ntiles, SCAN_TPB, 0, s>>>(out, m, tmp_tiles);
    STA_CUDA_TRY(cudaGetLastError());
    (void)c;
    return STA_OK;
}

// ---------------------------------------------------------------- node -> tetrahedra

// Number of superset tetrahedra incident to each node (the incidence the paper precomputes,
// Sec. 3.3).
__global__ void k_count_node_tets(const int4 *tets, int64_t T, int32_t *cnt) {
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < T;
         t += (int64_t)gridDim.x * blockDim.x) {
        int4 q = tets[t];
        atomicAdd(&cnt[q.x], 1);
        atomicAdd(&cnt[q.y], 1);
        atomicAdd(&cnt[q.z], 1);
        atomicAdd(&cnt[q.w], 1);
    }
}

// Node -> tetrahedra lists: each tetrahedron appends its id to its four nodes' lists; the
// append order is arbitrary, so the lists are sorted afterwards (k_sort_segments).
__global__ void k_fill_node_tets(const int4 *tets, int64_t T, const int64_t *nt_ptr,
                                 int32_t *fill, int32_t *nt_list) {
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < T;
         t += (int64_t)gridDim.x * blockDim.x) {
        int4 q = tets[t];
        int v[4] = {q.x, q.y, q.z, q.w};
        for (int k = 0; k < 4; ++k) {
            int32_t slot = atomicAdd(&fill[v[k]], 1);
            nt_list[nt_ptr[v[k]] + slot] = (int32_t)t;
        }
    }
}

// insertion sort of each segment [ptr[i], ptr[i+1]) of int32 keys, one thread per segment
__global__ void k_sort_segments(const int64_t *ptr, int64_t nseg, int32_t *keys) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nseg;
         i += (int64_t)gridDim.x * blockDim.x) {
        int64_t b = ptr[i], e = ptr[i + 1];
        for (int64_t k = b + 1; k < e; ++k) {
            int32_t x = keys[k];
            int64_t j = k - 1;
            while (j >= b && keys[j] > x) {
                keys[j + 1] = keys[j];
                --j;
            }
            keys[j + 1] = x;
        }
    }
}

// ---------------------------------------------------------------- neighbour sets

// Sorted, de-duplicated nodes of the tetrahedra incident to node a, built by insertion into
// scratch[4 nt_ptr[a] ...] (capacity 4 x incident count).
__global__ void k_node_neighbors(const int4 *tets, int64_t n, const int64_t *nt_ptr,
                                 const int32_t *nt_list, int32_t *scratch, int32_t *deg) {
    for (int64_t a = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; a < n;
         a += (int64_t)gridDim.x * blockDim.x) {
        int32_t *buf = scratch + 4 * nt_ptr[a];
        int32_t cnt = 0;
        for (int64_t e = nt_ptr[a]; e < nt_ptr[a + 1]; ++e) {
            int4 q = tets[nt_list[e]];
            int v[4] = {q.x, q.y, q.z, q.w};
            for (int k = 0; k < 4; ++k) {
                int32_t x = v[k];
                int32_t j = cnt - 1;
                while (j >= 0 && buf[j] > x) --j;
                if (j >= 0 && buf[j] == x) continue;
                for (int32_t m = cnt - 1; m > j; --m) buf[m + 1] = buf[m];
                buf[j + 1] = x;
                ++cnt;
            }
        }
        deg[a] = cnt;
    }
}

// Node adjacency in CSR form (adj_ptr, adj) from the per-node neighbour sets, and the row
// node of every block.
__global__ void k_adj_fill(int64_t n, const int64_t *nt_ptr, const int32_t *scratch,
                           const int64_t *adj_ptr64, int32_t *adj_ptr, int32_t *adj,
                           int32_t *block_node) {
    for (int64_t a = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; a <= n;
         a += (int64_t)gridDim.x * blockDim.x) {
        adj_ptr[a] = (int32_t)adj_ptr64[a];
        if (a == n) continue;
        const int32_t *buf = scratch + 4 * nt_ptr[a];
        int64_t b = adj_ptr64[a], d = adj_ptr64[a + 1] - b;
        for (int64_t k = 0; k < d; ++k) {
            adj[b + k] = buf[k];
            block_node[b + k] = (int32_t)a;
        }
    }
}

// row 3a+i starts at 9 adj_ptr[a] + 3 i deg(a)
__global__ void k_row_ptr(int64_t n, const int32_t *adj_ptr, int32_t *row_ptr) {
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r <= 3 * n;
         r += (int64_t)gridDim.x * blockDim.x) {
        if (r == 3 * n) {
            row_ptr[r] = 9 * adj_ptr[n];
            continue;
        }
        int64_t a = r / 3, i = r % 3;
        int32_t s = adj_ptr[a], d = adj_ptr[a + 1] - s;
        row_ptr[r] = 9 * s + 3 * (int32_t)i * d;
    }
}

// Column indices: block g = (a, b) fills columns 3b .. 3b+2 of the three rows of node a.
__global__ void k_col(int64_t nblocks, const int32_t *block_node, const int32_t *adj_ptr,
                      const int32_t *adj, int32_t *col) {
    for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < nblocks;
         g += (int64_t)gridDim.x * blockDim.x) {
        int32_t a = block_node[g], s = adj_ptr[a], d = adj_ptr[a + 1] - s;
        int32_t p = (int32_t)g - s, b = adj[g];
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) col[9 * s + 3 * i * d + 3 * p + j] = 3 * b + j;
    }
}

// tblk[16 t + 4 la + lb] = block of (v_la, v_lb); scat[144 t + 12 (3la+i) + 3lb + j] = CSR
// index of (3 v_la + i, 3 v_lb + j) (skipped when scat is NULL).  Position of v_lb in v_la's
// sorted list by bisection.
__global__ void k_tet_maps(const int4 *tets, int64_t T, const int32_t *adj_ptr,
                           const int32_t *adj, int32_t *tblk, int32_t *scat) {
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < T;
         t += (int64_t)gridDim.x * blockDim.x) {
        int4 q = tets[t];
        int v[4] = {q.x, q.y, q.z, q.w};
        for (int la = 0; la < 4; ++la) {
            int32_t s = adj_ptr[v[la]], d = adj_ptr[v[la] + 1] - s;
            for (int lb = 0; lb < 4; ++lb) {
                int32_t lo = 0, hi = d;  // first position with adj >= v[lb]
                while (lo < hi) {
                    int32_t mid = (lo + hi) >> 1;
                    if (adj[s + mid] < v[lb]) lo = mid + 1; else hi = mid;
                }
                tblk[16 * t + 4 * la + lb] = s + lo;
                if (!scat) continue;  // proxy operator: blocks only
                for (int i = 0; i < 3; ++i)
                    for (int j = 0; j < 3; ++j)
                        scat[144 * t + 12 * (3 * la + i) + 3 * lb + j] =
                            9 * s + 3 * i * d + 3 * lo + j;
            }
        }
    }
}

// ---------------------------------------------------------------- fold units
// A unit is an unordered node pair {a <= b} of the pattern: the block (a, b) of an "upper"
// block g (adj[g] >= block_node[g]); the lower block (b, a) is its mirror.

__global__ void k_block_off(int64_t nblocks, const int32_t *block_node, const int32_t *adj_ptr,
                            int2 *boff, int32_t *upper) {
    for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < nblocks;
         g += (int64_t)gridDim.x * blockDim.x) {
        const int32_t a = block_node[g], s = adj_ptr[a], d = adj_ptr[a + 1] - s;
        boff[g] = make_int2(9 * s + 3 * ((int32_t)g - s), 3 * d);
        upper[g] = 0;  // set by k_upper_flags
    }
}

// 1 for the blocks (a, b) with b >= a: the blocks that own a fold unit.
__global__ void k_upper_flags(int64_t nblocks, const int32_t *block_node, const int32_t *adj,
                              int32_t *upper) {
    for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < nblocks;
         g += (int64_t)gridDim.x * blockDim.x)
        upper[g] = adj[g] >= block_node[g] ? 1 : 0;
}

__device__ __forceinline__ int32_t find_block(const int32_t *adj_ptr, const int32_t *adj,
                                              int32_t a, int32_t b) {
    int32_t lo = adj_ptr[a], hi = adj_ptr[a + 1];  // first position with adj >= b
    while (lo < hi) {
        const int32_t mid = (lo + hi) >> 1;
        if (adj[mid] < b) lo = mid + 1; else hi = mid;
    }
    return lo;
}

// unit of every block (upper: its own prefix index; lower: its mirror's)
__global__ void k_unit_of_block(int64_t nblocks, const int32_t *block_node, const int32_t *adj,
                                const int32_t *adj_ptr, const int64_t *uid, int32_t *ublk) {
    for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < nblocks;
         g += (int64_t)gridDim.x * blockDim.x) {
        const int32_t a = block_node[g], b = adj[g];
        const int64_t gu = b >= a ? g : find_block(adj_ptr, adj, b, a);
        ublk[g] = (int32_t)uid[gu];
    }
}

// diagonal flag of every unit (upper blocks with a == b)
__global__ void k_unit_diag(int64_t nblocks, const int32_t *block_node, const int32_t *adj,
                            const int32_t *upper, const int64_t *uid, uint8_t *diag) {
    for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < nblocks;
         g += (int64_t)gridDim.x * blockDim.x)
        if (upper[g]) diag[uid[g]] = block_node[g] == adj[g] ? 1 : 0;
}

// lowest contributing tetrahedron of every unit
__global__ void k_unit_min_tet(const int32_t *tunit, int64_t T, int32_t *umin) {
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < 10 * T;
         k += (int64_t)gridDim.x * blockDim.x)
        atomicMin(&umin[tunit[k]], (int32_t)(k / 10));
}

// apply a unit renumbering rn (old id -> new id) to the block -> unit maps
__global__ void k_unit_renumber(int64_t nblocks, const int32_t *upper, const int32_t *rn,
                                int64_t *uid, int32_t *ublk) {
    for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < nblocks;
         g += (int64_t)gridDim.x * blockDim.x) {
        ublk[g] = rn[ublk[g]];
        if (upper[g]) uid[g] = rn[uid[g]];
    }
}

// tunit[10 t + s] = unit of slot s of tetrahedron t; counts per unit
__global__ void k_unit_count(const int32_t *tblk, const int32_t *ublk, int64_t T, int32_t *tunit,
                             int32_t *cnt) {
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < 10 * T;
         k += (int64_t)gridDim.x * blockDim.x) {
        const int64_t t = k / 10;
        const int s = (int)(k % 10);
        const int32_t u = ublk[tblk[16 * t + 4 * slot_la(s) + slot_lb(s)]];
        tunit[k] = u;
        atomicAdd(&cnt[u], 1);
    }
}

// codes in each unit's list: (t, la, lb) with la the local index of the unit's lower node
__global__ void k_unit_fill(const int4 *tets, const int32_t *tunit, int64_t T, const int64_t *uptr,
                            int32_t *fill, int32_t *ccode) {
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < 10 * T;
         k += (int64_t)gridDim.x * blockDim.x) {
        const int64_t t = k / 10;
        const int s = (int)(k % 10);
        const int4 q = tets[t];
        const int v[4] = {q.x, q.y, q.z, q.w};
        int la = slot_la(s), lb = slot_lb(s);
        if (v[la] > v[lb]) {
            const int x = la;
            la = lb;
            lb = x;
        }
        const int32_t u = tunit[k];
        const int32_t slot = atomicAdd(&fill[u], 1);
        ccode[uptr[u] + slot] = contrib_code((int32_t)t, la, lb);
    }
}

// cslot[10 t + s] = position of tetrahedron t's slot-s contribution in its unit's list
__global__ void k_unit_slots(const int32_t *ccode, int64_t T, int32_t *cslot) {
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < 10 * T;
         k += (int64_t)gridDim.x * blockDim.x) {
        const int32_t code = ccode[k];
        cslot[10 * (int64_t)code_tet(code) + slot_of((code >> 2) & 3, code & 3)] = (int32_t)k;
    }
}

// contributor codes (t, la, lb) -> contributor words: offset of the element-cache run the
// contributor supplies to its unit (word_offset), active bit clear
__global__ void k_code_words(int32_t *ccode, int64_t n, int64_t T) {
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n;
         k += (int64_t)gridDim.x * blockDim.x) {
        const int32_t code = ccode[k];
        const int la = (code >> 2) & 3, lb = code & 3;
        ccode[k] = (int32_t)ke_slot_at(T, code_tet(code), slot_of(la, lb));
    }
}

// unit records: value offset and row stride of (a, b) and of its mirror (b, a), contributors
__global__ void k_unit_meta(int64_t nblocks, const int32_t *block_node, const int32_t *adj,
                            const int32_t *adj_ptr, const int2 *boff, const int64_t *uid,
                            const int32_t *upper, const int64_t *uptr, int4 *umeta, int2 *umirror) {
    for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < nblocks;
         g += (int64_t)gridDim.x * blockDim.x) {
        if (!upper[g]) continue;
        const int32_t a = block_node[g], b = adj[g];
        const int64_t u = uid[g];
        const int2 o = boff[g], m = boff[find_block(adj_ptr, adj, b, a)];
        umeta[u] = make_int4(o.x, o.y << 1 | (a == b ? 1 : 0), (int32_t)uptr[u], (int32_t)uptr[u + 1]);
        umirror[u] = m;
    }
}

// Narrowing copy of node -> tetrahedron offsets (at most 4 n_tets < 2^29: they fit int32).
__global__ void k_to_i32(const int64_t *in, int64_t m, int32_t *out) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m;
         i += (int64_t)gridDim.x * blockDim.x)
        out[i] = (int32_t)in[i];
}

// p[0 .. m) = v.
__global__ void k_fill_i32(int32_t *p, int64_t m, int32_t v) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m;
         i += (int64_t)gridDim.x * blockDim.x)
        p[i] = v;
}

struct Scratch {
    std::vector<void *> ptrs;
    ~Scratch() {
        for (void *p : ptrs) cudaFree(p);
    }
    template <typename T> int get(T **p, int64_t count) {
        cudaError_t e = cudaMalloc((void **)p, sizeof(T) * (size_t)(count > 0 ? count : 1));
        if (e != cudaSuccess)
            return fail(STA_ENOMEM, std::string("cudaMalloc (scratch): ") + cudaGetErrorString(e));
        ptrs.push_back(*p);
        return STA_OK;
    }
};

// Unit order and fold tiles.  The units (node order) are cut into windows of UNIT_WINDOW;
// inside a window the diagonal units come first, then the off-diagonal ones, each group with
// the longest contributor lists first.  The rebuild (k_fold_flat) gives every fold entry a
// lane -- 6 entries per diagonal unit, 9 per off-diagonal unit -- and takes 32 consecutive
// entries of one group per warp tile, so tiles never mix the two kinds, neighbouring units
// have lists of equal length (the tile waits for its longest), and a window's values are
// written close together in time.  Any order gives the same values: each unit folds its own
// list in its own order.
// Tile record: {first unit, entry offset in it | diagonal << 4 | entries in the tile << 5,
// first code of the tile's units, end of their codes}.
#ifndef STA_UNIT_WINDOW
#define STA_UNIT_WINDOW 2048
#endif

void unit_order(const std::vector<int32_t> &cnt, const std::vector<int32_t> &umin,
                const std::vector<uint8_t> &diag, std::vector<int32_t> &rn, std::vector<int4> &tiles) {
    const int64_t m = (int64_t)cnt.size();
    const int64_t W = STA_UNIT_WINDOW > 1 ? STA_UNIT_WINDOW : 1;
    std::vector<int32_t> order;
    order.reserve(m);
    rn.assign(m, 0);
    tiles.clear();
    for (int64_t w0 = 0; w0 < m; w0 += W) {
        const int64_t w1 = std::min(m, w0 + W);
        for (int cls = 1; cls >= 0; --cls) {
            const size_t first = order.size();
            for (int64_t u = w0; u < w1; ++u)
                if (diag[u] == cls) order.push_back((int32_t)u);
            std::stable_sort(order.begin() + first, order.end(), [&](int32_t a, int32_t b) {
                return cnt[a] != cnt[b] ? cnt[a] > cnt[b] : umin[a] < umin[b];
            });
            const int64_t per = cls ? FOLD_TASKS_DIAG : FOLD_TASKS_PAIR;
            const int64_t nent = per * (int64_t)(order.size() - first);
            for (int64_t e = 0; e < nent; e += 32) {
                const int64_t k = std::min<int64_t>(32, nent - e);
                // code range filled in below, once every unit's list position is known
                tiles.push_back(make_int4((int32_t)(first + e / per),
                                          (int32_t)(e % per) | cls << 4 | (int32_t)k << 5,
                                          (int32_t)(first + (e + k - 1) / per), 0));
            }
        }
    }
    for (int64_t k = 0; k < m; ++k) rn[order[k]] = (int32_t)k;
    // lists are stored in new-id order: unit k's codes start at the sum of the earlier counts
    std::vector<int64_t> cs(m + 1, 0);
    for (int64_t k = 0; k < m; ++k) cs[k + 1] = cs[k] + cnt[order[k]];
    for (auto &t : tiles) {
        const int64_t last = t.z;
        t.z = (int32_t)cs[t.x];
        t.w = (int32_t)cs[last + 1];
    }
}

}  // namespace

int build_pattern(Ctx *c, cudaStream_t s) {
    const int64_t n = c->n, T = c->T;
    Scratch sc;
    int32_t *cnt = nullptr, *nt_list = nullptr, *scratch = nullptr, *deg = nullptr;
    int64_t *nt_ptr = nullptr, *adj_ptr64 = nullptr, *tiles = nullptr;
    int64_t max_m = (n > 16 * T ? n : 16 * T) + 1;
    STA_TRY(sc.get(&cnt, max_m));
    STA_TRY(sc.get(&nt_ptr, n + 1));
    STA_TRY(sc.get(&nt_list, 4 * T));
    STA_TRY(sc.get(&scratch, 16 * T));
    STA_TRY(sc.get(&deg, n));
    STA_TRY(sc.get(&adj_ptr64, n + 1));
    STA_TRY(sc.get(&tiles, max_m / SCAN_TPB + 2));

    // node -> incident tetrahedra, ascending
    STA_CUDA_TRY(cudaMemsetAsync(cnt, 0, sizeof(int32_t) * n, s));
    k_count_node_tets<<<grid_for(T), TPB, 0, s>>>(c->tets, T, cnt);
    STA_TRY(exclusive_scan(c, cnt, n, nt_ptr, tiles, s));
    STA_CUDA_TRY(cudaMemsetAsync(cnt, 0, sizeof(int32_t) * n, s));
    k_fill_node_tets<<<grid_for(T), TPB, 0, s>>>(c->tets, T, nt_ptr, cnt, nt_list);
    k_sort_segments<<<grid_for(n), TPB, 0, s>>>(nt_ptr, n, nt_list);

    // neighbour sets -> blocks
    k_node_neighbors<<<grid_for(n), TPB, 0, s>>>(c->tets, n, nt_ptr, nt_list, scratch, deg);
    STA_TRY(exclusive_scan(c, deg, n, adj_ptr64, tiles, s));
    int64_t nblocks = 0;
    STA_CUDA_TRY(cudaMemcpyAsync(&nblocks, adj_ptr64 + n, sizeof(int64_t),
                                 cudaMemcpyDeviceToHost, s));
    STA_CUDA_TRY(cudaStreamSynchronize(s));
    STA_CUDA_TRY(cudaGetLastError());
    if (c->op == STA_OP_PROXY) {  // node-level pattern, slot blocks and mirrors only
        if (nblocks > INT32_MAX)
            return fail(STA_ERANGE, "nnz = " + std::to_string(nblocks) + " exceeds int32");
        c->nblocks = nblocks;
        int32_t *tblk = nullptr;
        STA_TRY(sc.get(&tblk, 16 * T));
        STA_TRY(dev_alloc(c, &c->adj_ptr, n + 1));
        STA_TRY(dev_alloc(c, &c->adj, nblocks));
        STA_TRY(dev_alloc(c, &c->block_node, nblocks));
        k_adj_fill<<<grid_for(n + 1), TPB, 0, s>>>(n, nt_ptr, scratch, adj_ptr64, c->adj_ptr,
                                                   c->adj, c->block_node);
        k_tet_maps<<<grid_for(T), TPB, 0, s>>>(c->tets, T, c->adj_ptr, c->adj, tblk, nullptr);
        // node -> incident tetrahedra, kept for the local-recompute policy
        STA_TRY(dev_alloc(c, &c->nt_ptr, n + 1));
        STA_TRY(dev_alloc(c, &c->nt_list, 4 * T));
        k_to_i32<<<grid_for(n + 1), TPB, 0, s>>>(nt_ptr, n + 1, c->nt_ptr);
        STA_CUDA_TRY(cudaMemcpyAsync(c->nt_list, nt_list, sizeof(int32_t) * 4 * T,
                                     cudaMemcpyDeviceToDevice, s));
        STA_TRY(build_proxy_maps(c, tblk, s));
        STA_CUDA_TRY(cudaGetLastError());
        STA_CUDA_TRY(cudaStreamSynchronize(s));  // the scratch is freed on return
        return STA_OK;
    }
    if (9 * nblocks > INT32_MAX)
        return fail(STA_ERANGE, "nnz = " + std::to_string(9 * nblocks) + " exceeds int32");
    c->nblocks = nblocks;
    c->nnz = 9 * nblocks;
    c->nrows = 3 * n;

    STA_TRY(dev_alloc(c, &c->adj_ptr, n + 1));
    STA_TRY(dev_alloc(c, &c->adj, nblocks));
    STA_TRY(dev_alloc(c, &c->block_node, nblocks));
    STA_TRY(dev_alloc(c, &c->row_ptr, 3 * n + 1));
    STA_TRY(dev_alloc(c, &c->col, c->nnz));
    STA_TRY(dev_alloc(c, &c->tblk, 16 * T));
    STA_TRY(dev_alloc(c, &c->scat, 144 * T));
    STA_TRY(dev_alloc(c, &c->boff, nblocks));

    STA_TRY(dev_alloc(c, &c->nt_ptr, n + 1));
    STA_TRY(dev_alloc(c, &c->nt_list, 4 * T));
    k_to_i32<<<grid_for(n + 1), TPB, 0, s>>>(nt_ptr, n + 1, c->nt_ptr);
    STA_CUDA_TRY(cudaMemcpyAsync(c->nt_list, nt_list, sizeof(int32_t) * 4 * T,
                                 cudaMemcpyDeviceToDevice, s));
    k_adj_fill<<<grid_for(n + 1), TPB, 0, s>>>(n, nt_ptr, scratch, adj_ptr64, c->adj_ptr,
                                               c->adj, c->block_node);
    k_row_ptr<<<grid_for(3 * n + 1), TPB, 0, s>>>(n, c->adj_ptr, c->row_ptr);
    k_col<<<grid_for(nblocks), TPB, 0, s>>>(nblocks, c->block_node, c->adj_ptr, c->adj, c->col);
    k_tet_maps<<<grid_for(T), TPB, 0, s>>>(c->tets, T, c->adj_ptr, c->adj, c->tblk, c->scat);

    // fold units and their contributor lists, ascending tetrahedron id (the codes carry the id
    // in their high bits)
    int32_t *upper = nullptr, *ublk = nullptr;
    int64_t *uid = nullptr;
    STA_TRY(sc.get(&upper, nblocks));
    STA_TRY(sc.get(&ublk, nblocks));
    STA_TRY(sc.get(&uid, nblocks + 1));
    k_block_off<<<grid_for(nblocks), TPB, 0, s>>>(nblocks, c->block_node, c->adj_ptr, c->boff, upper);
    k_upper_flags<<<grid_for(nblocks), TPB, 0, s>>>(nblocks, c->block_node, c->adj, upper);
    STA_TRY(exclusive_scan(c, upper, nblocks, uid, tiles, s));
    int64_t nunits = 0;
    STA_CUDA_TRY(cudaMemcpyAsync(&nunits, uid + nblocks, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    STA_CUDA_TRY(cudaStreamSynchronize(s));
    c->nunits = nunits;
    STA_TRY(dev_alloc(c, &c->bmeta, nunits));
    STA_TRY(dev_alloc(c, &c->bmirror, nunits));
    STA_TRY(dev_alloc(c, &c->ccode, 10 * T));
    STA_TRY(dev_alloc(c, &c->cslot, 10 * T));
    STA_TRY(dev_alloc(c, &c->tunit, 10 * T));
    STA_TRY(dev_alloc(c, &c->owner, nunits));
    STA_TRY(dev_alloc(c, &c->touched, nunits));
    k_unit_of_block<<<grid_for(nblocks), TPB, 0, s>>>(nblocks, c->block_node, c->adj, c->adj_ptr,
                                                      uid, ublk);
    int64_t *uptr = nullptr;
    STA_TRY(sc.get(&uptr, nunits + 1));
    STA_CUDA_TRY(cudaMemsetAsync(cnt, 0, sizeof(int32_t) * (nunits > 0 ? nunits : 1), s));
    k_unit_count<<<grid_for(10 * T), TPB, 0, s>>>(c->tblk, ublk, T, c->tunit, cnt);
    if (nunits > 0) {  // renumber (windows: diagonal units first, longest lists first)
        uint8_t *udiag = nullptr;
        int32_t *rn_dev = nullptr;
        STA_TRY(sc.get(&udiag, nunits));
        STA_TRY(sc.get(&rn_dev, nunits));
        k_unit_diag<<<grid_for(nblocks), TPB, 0, s>>>(nblocks, c->block_node, c->adj, upper, uid,
                                                      udiag);
        std::vector<int32_t> hcnt(nunits), hmin(nunits), rn;
        std::vector<uint8_t> hdiag(nunits);
        std::vector<int4> htiles;
        k_fill_i32<<<grid_for(nunits), TPB, 0, s>>>(rn_dev, nunits, INT32_MAX);
        k_unit_min_tet<<<grid_for(10 * T), TPB, 0, s>>>(c->tunit, T, rn_dev);
        STA_CUDA_TRY(cudaMemcpyAsync(hmin.data(), rn_dev, sizeof(int32_t) * nunits,
                                     cudaMemcpyDeviceToHost, s));
        STA_CUDA_TRY(cudaMemcpyAsync(hcnt.data(), cnt, sizeof(int32_t) * nunits,
                                     cudaMemcpyDeviceToHost, s));
        STA_CUDA_TRY(cudaMemcpyAsync(hdiag.data(), udiag, nunits, cudaMemcpyDeviceToHost, s));
        STA_CUDA_TRY(cudaStreamSynchronize(s));
        unit_order(hcnt, hmin, hdiag, rn, htiles);
        c->ntiles = (int64_t)htiles.size();
        STA_TRY(dev_alloc(c, &c->ftile, c->ntiles));
        // per unit (new ids) its first tile | (it also reaches the next tile) << 31, and per
        // tile whether it is of diagonal units: the zero-fill rebuild's tile flags
        {
            std::vector<int32_t> hut(nunits, -1);
            std::vector<uint8_t> htd(c->ntiles);
            for (int64_t ti = 0; ti < c->ntiles; ++ti) {
                const int4 t = htiles[ti];
                const int per = (t.y >> 4) & 1 ? FOLD_TASKS_DIAG : FOLD_TASKS_PAIR;
                const int64_t ulast = t.x + ((t.y & 15) + (t.y >> 5) - 1) / per;
                htd[ti] = (uint8_t)((t.y >> 4) & 1);
                for (int64_t u = t.x; u <= ulast; ++u)
                    hut[u] = hut[u] < 0 ? (int32_t)ti : (int32_t)(hut[u] | INT32_MIN);
            }
            STA_TRY(dev_alloc(c, &c->utile, nunits));
            STA_TRY(dev_alloc(c, &c->tdiag, c->ntiles));
            STA_TRY(dev_alloc(c, &c->tflag, c->ntiles));
            STA_CUDA_TRY(cudaMemcpyAsync(c->utile, hut.data(), sizeof(int32_t) * nunits,
                                         cudaMemcpyHostToDevice, s));
            STA_CUDA_TRY(cudaMemcpyAsync(c->tdiag, htd.data(), (size_t)c->ntiles,
                                         cudaMemcpyHostToDevice, s));
            // zero between rebuilds (the zero-fill fold clears each flag it reads)
            STA_CUDA_TRY(cudaMemsetAsync(c->tflag, 0, (size_t)c->ntiles, s));
            STA_CUDA_TRY(cudaStreamSynchronize(s));  // host vectors go out of scope
        }
        STA_CUDA_TRY(cudaMemcpyAsync(c->ftile, htiles.data(), sizeof(int4) * c->ntiles,
                                     cudaMemcpyHostToDevice, s));
        STA_CUDA_TRY(cudaMemcpyAsync(rn_dev, rn.data(), sizeof(int32_t) * nunits,
                                     cudaMemcpyHostToDevice, s));
        k_unit_renumber<<<grid_for(nblocks), TPB, 0, s>>>(nblocks, upper, rn_dev, uid, ublk);
        STA_CUDA_TRY(cudaMemsetAsync(cnt, 0, sizeof(int32_t) * nunits, s));
        k_unit_count<<<grid_for(10 * T), TPB, 0, s>>>(c->tblk, ublk, T, c->tunit, cnt);
        STA_CUDA_TRY(cudaStreamSynchronize(s));  // host vectors go out of scope
    }
    STA_TRY(exclusive_scan(c, cnt, nunits, uptr, tiles, s));
    STA_CUDA_TRY(cudaMemsetAsync(cnt, 0, sizeof(int32_t) * (nunits > 0 ? nunits : 1), s));
    k_unit_fill<<<grid_for(10 * T), TPB, 0, s>>>(c->tets, c->tunit, T, uptr, cnt, c->ccode);
    k_sort_segments<<<grid_for(nunits), TPB, 0, s>>>(uptr, nunits, c->ccode);
    k_unit_slots<<<grid_for(10 * T), TPB, 0, s>>>(c->ccode, T, c->cslot);
    k_code_words<<<grid_for(10 * T), TPB, 0, s>>>(c->ccode, 10 * T, T);
    k_unit_meta<<<grid_for(nblocks), TPB, 0, s>>>(nblocks, c->block_node, c->adj, c->adj_ptr,
                                                  c->boff, uid, upper, uptr, c->bmeta, c->bmirror);
    k_fill_i32<<<grid_for(nunits), TPB, 0, s>>>(c->owner, nunits, INT32_MAX);
    STA_CUDA_TRY(cudaGetLastError());
    STA_CUDA_TRY(cudaStreamSynchronize(s));
    return STA_OK;
}

}  // namespace sta
