// Graph-Laplacian proxy operator (STA-FEM Sec. 3.1 Eqs. 1-4, Sec. 3.2 Eqs. 5-7, Sec. 3.3,
// Algorithm 1): the scalar n x n matrix A_t = L_t + eps I on the node-level superset pattern
// (row u: the sorted neighbour set of u, u included), L_t the unweighted Laplacian of the
// edges that at least one active tetrahedron has.  Persistent state: the edge multiplicity
// c_t (int32 at the edge's upper block), the node degrees (int32) and the values (FP64).
//
// full_rebuild: zero c and the degrees, count c over the active tetrahedra (6 integer atomics
// a tetrahedron), threshold every off-diagonal entry while counting the degrees, write the
// diagonal.
// streaming_update: one thread per (edited tetrahedron, unit slot).  An edge slot adds +-1 to
// the edge's multiplicity with an integer atomic; the thread whose atomic moves it between 0
// and > 0 moves the degrees of both end nodes by the same +-1.  Every slot's block (6 edges,
// 4 diagonals) is claimed once per frame into a touched list, and a second kernel writes the
// touched entries from the final counts.  The atomics on one counter are totally ordered, so
// the transitions they report sum to the net change of the edge's activity whatever the
// order: the streamed state is bit-identical to the rebuild's.
// Under STA_POLICY_REFOLD a frame instead recounts each touched edge over the tetrahedra
// incident to it and each touched node's degree over its row (the paper's local_recompute,
// O(|Delta| kappa)); same values and state.
#include "sta_claim.cuh"

namespace sta {
namespace {

constexpr int PX_TPB = 256;

inline unsigned px_grid(const Ctx *c, int64_t items, int per_sm = 8) {
    int64_t g = (items + PX_TPB - 1) / PX_TPB;
    const int64_t cap = (int64_t)c->num_sms * per_sm;
    if (g > cap) g = cap;
    return (unsigned)(g < 1 ? 1 : g);
}

// ptblk[10 t + s]: block of tet t's unit slot s -- the diagonal block of local node s (s < 4),
// the upper block (lower global id first) of the edge slot_la(s)-slot_lb(s) (s >= 4).
__global__ void k_proxy_slots(const int4 *__restrict__ tets, int64_t T,
                              const int32_t *__restrict__ tblk, int32_t *__restrict__ ptblk) {
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < T;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int4 q = tets[t];
        const int v[4] = {q.x, q.y, q.z, q.w};
        for (int s = 0; s < 10; ++s) {
            const int la = slot_la(s), lb = slot_lb(s);
            const int lo = v[la] < v[lb] ? la : lb, hi = v[la] < v[lb] ? lb : la;
            ptblk[10 * t + s] = tblk[16 * t + 4 * lo + hi];
        }
    }
}

// pmir[g]: the block (b, a) of block g = (a, b) (a diagonal block is its own); pup[g]: the
// upper block of g's edge (g itself or its mirror), -1 for a diagonal block; pdiag[a]: the
// diagonal block of node a (left at -1 for a node of no tetrahedron).
__global__ void k_proxy_block_maps(int64_t nblocks, const int32_t *__restrict__ block_node,
                                   const int32_t *__restrict__ adj,
                                   const int32_t *__restrict__ adj_ptr, int32_t *__restrict__ pmir,
                                   int32_t *__restrict__ pup, int32_t *__restrict__ pdiag) {
    for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < nblocks;
         g += (int64_t)gridDim.x * blockDim.x) {
        const int32_t a = block_node[g], b = adj[g];
        if (a == b) {
            pmir[g] = (int32_t)g;
            pup[g] = -1;
            pdiag[a] = (int32_t)g;
            continue;
        }
        int32_t lo = adj_ptr[b], hi = adj_ptr[b + 1];  // position of a in b's sorted row
        while (lo < hi) {
            const int32_t mid = (lo + hi) >> 1;
            if (adj[mid] < a) lo = mid + 1; else hi = mid;
        }
        pmir[g] = lo;
        pup[g] = b > a ? (int32_t)g : lo;
    }
}

// Eq. 1 over the active set: +1 on the multiplicity of each of the six edges.  The edge
// blocks are loaded together with the mask byte (not after it), so one memory round trip
// serves each tetrahedron.
__global__ void k_proxy_count(const uint8_t *__restrict__ mask, const int32_t *__restrict__ ptblk,
                              int64_t T, int32_t *__restrict__ mult) {
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < T;
         t += (int64_t)gridDim.x * blockDim.x) {
        // the six edge blocks: ints 10 t + 4 .. 10 t + 9, an 8-byte aligned run
        const int2 *e = reinterpret_cast<const int2 *>(ptblk + 10 * t + 4);
        const uint8_t on = __ldg(mask + t);
        const int2 e0 = __ldg(e), e1 = __ldg(e + 1), e2 = __ldg(e + 2);
        if (!on) continue;
        atomicAdd(&mult[e0.x], 1);
        atomicAdd(&mult[e0.y], 1);
        atomicAdd(&mult[e1.x], 1);
        atomicAdd(&mult[e1.y], 1);
        atomicAdd(&mult[e2.x], 1);
        atomicAdd(&mult[e2.y], 1);
    }
}

// Eqs. 2-3 for every off-diagonal block: -a_t, and the degree of the row's node (Eq. 3's
// diagonal sum) as a count of the active entries, added once per node and warp.
__global__ void k_proxy_offdiag(int64_t nblocks, const int32_t *__restrict__ block_node,
                                const int32_t *__restrict__ pup, const int32_t *__restrict__ mult,
                                int32_t *__restrict__ deg, double *__restrict__ val) {
    const int lane = threadIdx.x & 31;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31); base < nblocks;
         base += stride) {
        const int64_t g = base + lane;
        int32_t a = -1;
        bool on = false;
        if (g < nblocks) {
            a = block_node[g];
            const int32_t up = pup[g];
            if (up >= 0) {
                on = mult[up] > 0;
                val[g] = on ? -1.0 : 0.0;
            }
        }
        const unsigned same = __match_any_sync(0xffffffffu, a);
        const unsigned act = __ballot_sync(0xffffffffu, on) & same;
        if (a >= 0 && act && lane == __ffs(same) - 1) atomicAdd(&deg[a], __popc(act));
    }
}

// Eq. 4: the diagonal, degree + eps.
__global__ void k_proxy_diag(int64_t n, const int32_t *__restrict__ pdiag,
                             const int32_t *__restrict__ deg, double eps, double *__restrict__ val) {
    for (int64_t a = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; a < n;
         a += (int64_t)gridDim.x * blockDim.x) {
        const int32_t g = pdiag[a];
        if (g >= 0) val[g] = (double)deg[a] + eps;
    }
}

// Streaming, part 1 (Eqs. 5-7, Algorithm 1): one thread per (edited tet, slot).  Writes the
// mask, moves multiplicities and degrees, and claims each touched block once into `list`
// (counters[1]: blocks, counters[3]: entries -- 2 per edge, 1 per diagonal; one atomic on
// each per CTA).
__global__ void __launch_bounds__(PX_TPB)
k_proxy_claim(const int32_t *__restrict__ edited, int64_t m,
                              const int64_t *__restrict__ m_dev, const int4 *__restrict__ tets,
                              const int32_t *__restrict__ ptblk, int32_t *__restrict__ mult,
                              int32_t *__restrict__ deg, uint32_t *__restrict__ flag,
                              uint8_t *__restrict__ mask, int32_t *__restrict__ list,
                              unsigned long long *__restrict__ counters, bool count) {
    const int64_t items = 10 * (m_dev ? *m_dev : m);
    const int lane = threadIdx.x & 31;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i0 = (int64_t)blockIdx.x * blockDim.x; i0 < items; i0 += stride) {  // CTA-uniform
        const int64_t i = i0 + threadIdx.x;
        bool won = false, edge = false;
        int32_t g = 0;
        if (i < items) {
            const int64_t k = i / 10;
            const int s = (int)(i - 10 * k);
            const uint32_t e = (uint32_t)edited[k];
            const int64_t t = e & 0x7fffffffu;
            const bool on = (e >> 31) != 0u;
            g = ptblk[10 * t + s];
            edge = s >= 4;
            if (edge && count) {
                const int step = on ? 1 : -1;
                const int32_t before = atomicAdd(&mult[g], step);
                if ((before == 0) != (before + step == 0)) {  // 0 <-> > 0
                    const int4 q = tets[t];
                    const int v[4] = {q.x, q.y, q.z, q.w};
                    atomicAdd(&deg[v[slot_la(s)]], step);
                    atomicAdd(&deg[v[slot_lb(s)]], step);
                }
            } else if (s == 0) {
                mask[t] = on ? 1 : 0;
            }
            won = atomicExch(&flag[g], 1u) == 0u;
        }
        const unsigned ball = __ballot_sync(0xffffffffu, won);
        const unsigned eball = __ballot_sync(0xffffffffu, won && edge);
        const unsigned long long pos =
            cta_append<PX_TPB>(counters, __popc(ball), __popc(ball) + __popc(eball));
        if (won) list[pos + __popc(ball & ((1u << lane) - 1u))] = g;
    }
}

// Streaming, part 2: each touched block from the final state (an edge: both of its entries
// from its multiplicity; a diagonal: degree + eps), and its claim released.
__global__ void k_proxy_write(const int32_t *__restrict__ list,
                              const unsigned long long *__restrict__ count,
                              const int32_t *__restrict__ block_node, const int32_t *__restrict__ adj,
                              const int32_t *__restrict__ pmir, const int32_t *__restrict__ mult,
                              int32_t *__restrict__ deg, double eps,
                              uint32_t *__restrict__ flag, double *__restrict__ val,
                              const int32_t *__restrict__ adj_ptr, const int32_t *__restrict__ pup,
                              unsigned long long *next_count) {
    if (next_count && blockIdx.x == 0 && threadIdx.x == 0) {  // the next graph frame's counts
        next_count[0] = 0;
        next_count[2] = 0;
    }
    const int64_t cnt = (int64_t)*count;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < cnt;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int32_t g = list[i];
        const int32_t a = block_node[g];
        if (adj[g] == a) {
            if (adj_ptr) {  // local recompute: the degree from the row's (final) multiplicities
                int32_t d = 0;
                for (int32_t b = adj_ptr[a]; b < adj_ptr[a + 1]; ++b) {
                    const int32_t up = pup[b];
                    d += up >= 0 && mult[up] > 0;
                }
                deg[a] = d;
            }
            val[g] = (double)deg[a] + eps;
        } else {
            const double v = mult[g] > 0 ? -1.0 : 0.0;
            val[g] = v;
            val[pmir[g]] = v;
        }
        flag[g] = 0u;
    }
}

// Local recompute (STA_POLICY_REFOLD, the paper's local_recompute for the proxy): each claimed
// edge's multiplicity counted from scratch over the active tetrahedra incident to its lower
// node that also hold its upper node (O(|Delta| kappa)); diagonals are left to k_proxy_write.
__global__ void k_proxy_recount(const int32_t *__restrict__ list,
                                const unsigned long long *__restrict__ count,
                                const int32_t *__restrict__ block_node,
                                const int32_t *__restrict__ adj, const int32_t *__restrict__ nt_ptr,
                                const int32_t *__restrict__ nt_list, const int4 *__restrict__ tets,
                                const uint8_t *__restrict__ mask, int32_t *__restrict__ mult) {
    const int64_t cnt = (int64_t)*count;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < cnt;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int32_t g = list[i];
        const int32_t u = block_node[g], v = adj[g];
        if (u == v) continue;
        int32_t c = 0;
        for (int32_t e = nt_ptr[u]; e < nt_ptr[u + 1]; ++e) {
            const int32_t t = nt_list[e];
            if (!mask[t]) continue;
            const int4 q = tets[t];
            c += q.x == v || q.y == v || q.z == v || q.w == v;
        }
        mult[g] = c;
    }
}

}  // namespace

int build_proxy_maps(Ctx *c, const int32_t *tblk, cudaStream_t s) {
    const int64_t n = c->n, T = c->T, nb = c->nblocks;
    STA_TRY(dev_alloc(c, &c->ptblk, 10 * T));
    STA_TRY(dev_alloc(c, &c->pmir, nb));
    STA_TRY(dev_alloc(c, &c->pup, nb));
    STA_TRY(dev_alloc(c, &c->pdiag, n));
    STA_TRY(dev_alloc(c, &c->pmult, nb + n));
    STA_TRY(dev_alloc(c, &c->pflag, nb));
    STA_TRY(dev_alloc(c, &c->plist, nb));
    STA_CUDA_TRY(cudaMemsetAsync(c->pdiag, 0xff, sizeof(int32_t) * (size_t)(n > 0 ? n : 1), s));
    STA_CUDA_TRY(cudaMemsetAsync(c->pflag, 0, sizeof(uint32_t) * (size_t)(nb > 0 ? nb : 1), s));
    STA_CUDA_TRY(cudaMemsetAsync(c->pmult, 0, sizeof(int32_t) * (size_t)(nb + n > 0 ? nb + n : 1), s));
    if (T > 0) k_proxy_slots<<<px_grid(c, T, 16), PX_TPB, 0, s>>>(c->tets, T, tblk, c->ptblk);
    if (nb > 0)
        k_proxy_block_maps<<<px_grid(c, nb, 16), PX_TPB, 0, s>>>(nb, c->block_node, c->adj,
                                                                 c->adj_ptr, c->pmir, c->pup,
                                                                 c->pdiag);
    STA_CUDA_TRY(cudaGetLastError());
    // the node-level pattern is the proxy's CSR (sta_csr, sta_spmv)
    c->row_ptr = c->adj_ptr;
    c->col = c->adj;
    c->nrows = n;
    c->nnz = nb;
    return STA_OK;
}

int launch_proxy_rebuild(Ctx *c, cudaStream_t s) {
    const int64_t n = c->n, T = c->T, nb = c->nblocks;
    int32_t *deg = c->pmult + nb;
    STA_CUDA_TRY(cudaMemsetAsync(c->pmult, 0, sizeof(int32_t) * (size_t)(nb + n > 0 ? nb + n : 1), s));
    if (T > 0) k_proxy_count<<<px_grid(c, T), PX_TPB, 0, s>>>(c->mask, c->ptblk, T, c->pmult);
    if (nb > 0)
        k_proxy_offdiag<<<px_grid(c, nb), PX_TPB, 0, s>>>(nb, c->block_node, c->pup, c->pmult,
                                                          deg, c->val);
    if (n > 0) k_proxy_diag<<<px_grid(c, n), PX_TPB, 0, s>>>(n, c->pdiag, deg, c->eps, c->val);
    STA_CUDA_TRY(cudaGetLastError());
    return STA_OK;
}

// One streaming frame of the proxy: `edited` holds m tetrahedra (or *m_dev of them, grids
// sized for `cap`); `list` has room for min(10 cap, nblocks) blocks; counters[1] and [3] are
// zero on entry.
int launch_proxy_frame(Ctx *c, const int32_t *edited, int64_t m, const int64_t *m_dev,
                       int64_t cap, int32_t *list, unsigned long long *counters, cudaStream_t s,
                       unsigned long long *next_cnt) {
    const int64_t items = 10 * (cap > 0 ? cap : 1);
    int32_t *deg = c->pmult + c->nblocks;
    const bool rescan = c->policy == STA_POLICY_REFOLD;  // local recompute instead of +-1
    k_proxy_claim<<<px_grid(c, items, 16), PX_TPB, 0, s>>>(edited, m, m_dev, c->tets, c->ptblk,
                                                           c->pmult, deg, c->pflag, c->mask, list,
                                                           counters, !rescan);
    const int64_t most = items < c->nblocks ? items : c->nblocks;
    if (rescan)
        k_proxy_recount<<<px_grid(c, most, 16), PX_TPB, 0, s>>>(list, counters + 1, c->block_node,
                                                                c->adj, c->nt_ptr, c->nt_list,
                                                                c->tets, c->mask, c->pmult);
    k_proxy_write<<<px_grid(c, most, 16), PX_TPB, 0, s>>>(list, counters + 1, c->block_node,
                                                          c->adj, c->pmir, c->pmult, deg, c->eps,
                                                          c->pflag, c->val,
                                                          rescan ? c->adj_ptr : nullptr, c->pup,
                                                          next_cnt ? next_cnt + 1 : nullptr);
    STA_CUDA_TRY(cudaGetLastError());
    return STA_OK;
}

}  // namespace sta

using namespace sta;

extern "C" int sta_proxy_state(const sta_ctx *x, const int32_t **mult, const int32_t **degree) {
    if (!x) return fail(STA_EINVAL, "ctx is NULL");
    if (x->c.op != STA_OP_PROXY) return fail(STA_ESTATE, "not a proxy-operator context");
    if (mult) *mult = x->c.pmult;
    if (degree) *degree = x->c.pmult + x->c.nblocks;
    return STA_OK;
}
