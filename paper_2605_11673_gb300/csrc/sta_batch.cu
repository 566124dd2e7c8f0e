// Batched form: k independent superset meshes in one context.
//
// The instances are concatenated with disjoint node and tetrahedron id ranges, so the pattern
// of the union is block diagonal and every CSR entry keeps exactly the contributor list (in
// the same ascending order) it has in a context of its own instance: results are bit-identical
// to per-instance runs.  A full rebuild or a frame of streaming edits of all instances is then
// one launch sequence of the same kernels (one persistent fold over the blocks of every
// instance), which balances uneven instance sizes and uneven per-instance edit counts.
#include <algorithm>

#include "sta_internal.cuh"

namespace sta {
namespace {

__device__ __forceinline__ int find_instance(const int64_t *off, int k, int64_t x) {
    int lo = 0, hi = k;  // largest i with off[i] <= x
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (off[mid] <= x) lo = mid; else hi = mid;
    }
    return lo;
}

// Per-instance CSR index arrays: instance i's row_ptr (3 n_i + 1 entries, starting at 0) is
// stored at 3 node_off[i] + i; columns are shifted to the instance's own DOF numbering.
__global__ void k_local_rowptr(const int32_t *row_ptr, int64_t nrows, const int64_t *row_off,
                               const int64_t *nnz_off, int k, int32_t *local_rp) {
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < nrows + k;
         r += (int64_t)gridDim.x * blockDim.x) {
        if (r < nrows) {
            const int i = find_instance(row_off, k, r);
            local_rp[r + i] = (int32_t)(row_ptr[r] - nnz_off[i]);
        } else {
            const int i = (int)(r - nrows);
            local_rp[row_off[i + 1] + i] = (int32_t)(nnz_off[i + 1] - nnz_off[i]);
        }
    }
}

// Instance-local column indices: each entry's column less its instance's first DOF.
__global__ void k_local_col(const int32_t *col, int64_t nnz, const int64_t *nnz_off,
                            const int64_t *row_off, int k, int32_t *local_col) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < nnz;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int i = find_instance(nnz_off, k, e);
        local_col[e] = (int32_t)(col[e] - row_off[i]);
    }
}

}  // namespace
}  // namespace sta

using namespace sta;

extern "C" {

int sta_batch_create(int32_t k, const int64_t *n_nodes, const double *const *nodes,
                     const int64_t *n_tets, const int32_t *const *tets,
                     const double *const *young, const double *const *poisson,
                     const sta_options *opt, void *stream, sta_ctx **out) {
    if (!out) return fail(STA_EINVAL, "out is NULL");
    *out = nullptr;
    if (k < 1 || !n_nodes || !nodes || !n_tets || !tets || !young || !poisson)
        return fail(STA_EINVAL, "bad batch arguments");
    std::vector<int64_t> node_off(k + 1, 0), tet_off(k + 1, 0);
    for (int i = 0; i < k; ++i) {
        if (n_nodes[i] < 0 || n_tets[i] < 0) return fail(STA_EINVAL, "negative size");
        if ((n_nodes[i] > 0 && !nodes[i]) ||
            (n_tets[i] > 0 && (!tets[i] || !young[i] || !poisson[i])))
            return fail(STA_EINVAL, "NULL instance array");
        for (int64_t t = 0; t < 4 * n_tets[i]; ++t)
            if (tets[i][t] < 0 || tets[i][t] >= n_nodes[i])
                return fail(STA_EINVAL, "instance " + std::to_string(i) + ": node id out of range");
        node_off[i + 1] = node_off[i] + n_nodes[i];
        tet_off[i + 1] = tet_off[i] + n_tets[i];
    }
    if (node_off[k] > INT32_MAX / 3) return fail(STA_ERANGE, "too many nodes in the batch");
    std::vector<double> X(3 * (size_t)std::max<int64_t>(node_off[k], 1)),
        E((size_t)std::max<int64_t>(tet_off[k], 1)), NU((size_t)std::max<int64_t>(tet_off[k], 1));
    std::vector<int32_t> TT(4 * (size_t)std::max<int64_t>(tet_off[k], 1));
    for (int i = 0; i < k; ++i) {
        std::copy(nodes[i], nodes[i] + 3 * n_nodes[i], X.begin() + 3 * node_off[i]);
        std::copy(young[i], young[i] + n_tets[i], E.begin() + tet_off[i]);
        std::copy(poisson[i], poisson[i] + n_tets[i], NU.begin() + tet_off[i]);
        for (int64_t t = 0; t < 4 * n_tets[i]; ++t)
            TT[4 * tet_off[i] + t] = tets[i][t] + (int32_t)node_off[i];
    }
    sta_ctx *x = nullptr;
    int rc = create_impl(X.data(), node_off[k], TT.data(), tet_off[k], E.data(), NU.data(), opt,
                         stream, &x);
    if (rc != STA_OK) return rc;
    Ctx *c = &x->c;
    cudaStream_t s = (cudaStream_t)stream;
    c->n_inst = k;
    c->node_off = node_off;
    c->tet_off = tet_off;
    // nnz offsets: instance i's rows are [3 node_off[i], 3 node_off[i+1])
    std::vector<int32_t> rp(3 * (size_t)node_off[k] + 1);
    std::vector<int64_t> row_off(k + 1);
    auto cleanup = [&](int code) {
        sta_destroy(x);
        return code;
    };
    if (cudaMemcpyAsync(rp.data(), c->row_ptr, sizeof(int32_t) * rp.size(), cudaMemcpyDeviceToHost, s) ||
        cudaStreamSynchronize(s))
        return cleanup(fail(STA_ECUDA, "row_ptr copy"));
    c->nnz_off.assign(k + 1, 0);
    for (int i = 0; i <= k; ++i) {
        row_off[i] = 3 * node_off[i];
        c->nnz_off[i] = rp[row_off[i]];
    }
    int64_t *d_row_off = nullptr, *d_nnz_off = nullptr;
    if ((rc = dev_alloc(c, &d_row_off, k + 1)) || (rc = dev_alloc(c, &d_nnz_off, k + 1)) ||
        (rc = dev_alloc(c, &c->local_rp, c->nrows + k)) || (rc = dev_alloc(c, &c->local_col, c->nnz)))
        return cleanup(rc);
    if (cudaMemcpyAsync(d_row_off, row_off.data(), sizeof(int64_t) * (k + 1), cudaMemcpyHostToDevice, s) ||
        cudaMemcpyAsync(d_nnz_off, c->nnz_off.data(), sizeof(int64_t) * (k + 1), cudaMemcpyHostToDevice, s))
        return cleanup(fail(STA_ECUDA, "offset copy"));
    const unsigned g = (unsigned)std::min<int64_t>(std::max<int64_t>((c->nrows + k + 255) / 256, 1),
                                                    (int64_t)c->num_sms * 16);
    k_local_rowptr<<<g, 256, 0, s>>>(c->row_ptr, c->nrows, d_row_off, d_nnz_off, k, c->local_rp);
    const unsigned g2 = (unsigned)std::min<int64_t>(std::max<int64_t>((c->nnz + 255) / 256, 1),
                                                     (int64_t)c->num_sms * 16);
    k_local_col<<<g2, 256, 0, s>>>(c->col, c->nnz, d_nnz_off, d_row_off, k, c->local_col);
    if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(s) != cudaSuccess)
        return cleanup(fail(STA_ECUDA, "local index kernels"));
    *out = x;
    return STA_OK;
}

int sta_batch_size(const sta_ctx *x, int32_t *k) {
    if (!x || !k) return fail(STA_EINVAL, "NULL argument");
    *k = x->c.n_inst;
    return STA_OK;
}

int sta_batch_instance(const sta_ctx *x, int32_t i, const int32_t **row_ptr, const int32_t **col,
                       const double **val, int64_t *n_rows, int64_t *nnz, int64_t *tet_offset) {
    if (!x) return fail(STA_EINVAL, "ctx is NULL");
    const Ctx *c = &x->c;
    if (c->n_inst == 0) return fail(STA_ESTATE, "not a batched context");
    if (i < 0 || i >= c->n_inst) return fail(STA_EINVAL, "instance index out of range");
    if (row_ptr) *row_ptr = c->local_rp + 3 * c->node_off[i] + i;
    if (col) *col = c->local_col + c->nnz_off[i];
    if (val) *val = c->val + c->nnz_off[i];
    if (n_rows) *n_rows = 3 * (c->node_off[i + 1] - c->node_off[i]);
    if (nnz) *nnz = c->nnz_off[i + 1] - c->nnz_off[i];
    if (tet_offset) *tet_offset = c->tet_off[i];
    return STA_OK;
}

int sta_batch_apply_edits(sta_ctx *x, const int64_t *counts, const sta_edit *edits, void *stream) {
    if (!x || !counts) return fail(STA_EINVAL, "NULL argument");
    Ctx *c = &x->c;
    if (c->n_inst == 0) return fail(STA_ESTATE, "not a batched context");
    int64_t total = 0;
    for (int i = 0; i < c->n_inst; ++i) {
        if (counts[i] < 0) return fail(STA_EINVAL, "negative edit count");
        total += counts[i];
    }
    if (total > 0 && !edits) return fail(STA_EINVAL, "edits is NULL");
    std::vector<sta_edit> g((size_t)total);
    int64_t e = 0;
    for (int i = 0; i < c->n_inst; ++i) {
        const int64_t Ti = c->tet_off[i + 1] - c->tet_off[i], off = c->tet_off[i];
        for (int64_t j = 0; j < counts[i]; ++j, ++e) {
            sta_edit E = edits[e];
            const bool two = E.op == STA_SWAP;
            if (E.tet < 0 || E.tet >= Ti || (two && (E.tet2 < 0 || E.tet2 >= Ti)))
                return fail(STA_EINVAL, "instance " + std::to_string(i) + ", edit " +
                                            std::to_string(j) + ": tet out of the instance's range");
            E.tet += (int32_t)off;
            if (two) E.tet2 += (int32_t)off;
            g[e] = E;
        }
    }
    return sta_apply_edits(x, g.data(), total, stream);
}

}  // extern "C"
