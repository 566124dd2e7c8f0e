// Element stiffness kernel: the 12x12 linear-tetrahedron elasticity matrix K^(tau)
// (STA-FEM Sec. 3.4 and Sec. 5.2; the standard P1 isotropic small-strain element,
// K = V B^T D B), 78 unique entries per tetrahedron written to the element cache.
//
// The evaluation order is fixed (see include/sta.h, sta_recompute_elements) and this file
// is compiled with --fmad=false: every fma below is an explicit __fma_rn, every other
// operation is a separately rounded IEEE double operation.  On GB300 the FP64 pipe is the
// scarce unit (about 0.5 Top/s against 35 Top/s of int32), so the order is also chosen to
// need few FP64 operations: about 300 per tetrahedron.
#include "sta_internal.cuh"

namespace sta {
namespace {

constexpr int EL_TPB = 128;

struct V3 {
    double x, y, z;
};

__device__ __forceinline__ V3 sub(const double4_32a &a, const double4_32a &b) {
    return {a.x - b.x, a.y - b.y, a.z - b.z};
}

// (u x v) with each component fma(u1, v2, -(u2 * v1))
__device__ __forceinline__ V3 cross_fma(const V3 &u, const V3 &v) {
    return {__fma_rn(u.y, v.z, -(u.z * v.y)), __fma_rn(u.z, v.x, -(u.x * v.z)),
            __fma_rn(u.x, v.y, -(u.y * v.x))};
}

__device__ __forceinline__ double gc(const V3 &g, int i) { return i == 0 ? g.x : (i == 1 ? g.y : g.z); }

// Computes the 78-entry record of one tetrahedron (node ids q) into rec[] (registers or shared
// memory).  Returns false when det <= 0 (record filled with zeros).
__device__ __forceinline__ bool element_record(double4_32a x0, double4_32a x1, double4_32a x2, double4_32a x3,
                                               double E, double nu, int4 q, double *rec) {
    const int gid[4] = {q.x, q.y, q.z, q.w};
    V3 d1 = sub(x1, x0), d2 = sub(x2, x0), d3 = sub(x3, x0);
    V3 c1 = cross_fma(d2, d3), c2 = cross_fma(d3, d1), c3 = cross_fma(d1, d2);
    double det = __fma_rn(d1.z, c1.z, __fma_rn(d1.y, c1.y, d1.x * c1.x));
    if (!(det > 0.0)) {
#pragma unroll
        for (int k = 0; k < KE_STRIDE; ++k) rec[k] = 0.0;
        return false;
    }
    double r = 1.0 / det;
    V3 g[4];
    g[1] = {c1.x * r, c1.y * r, c1.z * r};
    g[2] = {c2.x * r, c2.y * r, c2.z * r};
    g[3] = {c3.x * r, c3.y * r, c3.z * r};
    g[0] = {-((g[1].x + g[2].x) + g[3].x), -((g[1].y + g[2].y) + g[3].y),
            -((g[1].z + g[2].z) + g[3].z)};
    double V = det / 6.0;
    double onu = 1.0 + nu;
    double lam = (E * nu) / (onu * (1.0 - (nu + nu)));
    double mu = E / (onu + onu);
    double Vl = V * lam, Vm = V * mu;
    double P[4][3], Q[4][3];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            P[a][i] = Vl * gc(g[a], i);
            Q[a][i] = Vm * gc(g[a], i);
        }
    // diagonal blocks (a, a), entries i <= j
#pragma unroll
    for (int a = 0; a < 4; ++a) {
        double D = Vm * __fma_rn(g[a].z, g[a].z, __fma_rn(g[a].y, g[a].y, g[a].x * g[a].x));
        double *o = rec + ke_diag_off(a);
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
            for (int j = i; j < 3; ++j) {
                double v = (i != j)
                               ? __fma_rn(P[a][i], gc(g[a], j), Q[a][j] * gc(g[a], i))
                               : __fma_rn(P[a][i], gc(g[a], i), __fma_rn(Q[a][i], gc(g[a], i), D));
                o[ke_tri(i, j)] = v;
            }
    }
    // off-diagonal blocks (a, b), a < b, all (i, j)
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = a + 1; b < 4; ++b) {
            double D = Vm * __fma_rn(g[a].z, g[b].z, __fma_rn(g[a].y, g[b].y, g[a].x * g[b].x));
            double *o = rec + ke_off_off(a, b);
            const bool tr = gid[a] > gid[b];  // run stored with the lower node id's rows
#pragma unroll
            for (int i = 0; i < 3; ++i)
#pragma unroll
                for (int j = 0; j < 3; ++j) {
                    double v = (i != j)
                                   ? __fma_rn(P[a][i], gc(g[b], j), Q[a][j] * gc(g[b], i))
                                   : __fma_rn(P[a][i], gc(g[b], i), __fma_rn(Q[a][i], gc(g[b], i), D));
                    o[tr ? 3 * j + i : 3 * i + j] = v;
                }
            o[9] = 0.0;  // pad to a 16-byte aligned run
        }
    return true;
}

// One thread per tetrahedron; a warp stages its 32 records in shared memory and writes
// each record of an updated tetrahedron as one contiguous 624-byte run (coalesced).
// active_only: tetrahedra with mask == 0 keep their cached record untouched.
// Active tetrahedra, unordered (warp-aggregated append): the FP64 kernels below run over this
// list so that every FP64 instruction carries full lanes when part of the superset is inactive.
// With dE non-null, the adjoint outputs of inactive tets are zeroed on the way.
__global__ void k_active_list(const uint8_t *__restrict__ mask, int64_t T, int32_t *__restrict__ list,
                              unsigned long long *count, double *__restrict__ dE,
                              double *__restrict__ dnu, double *__restrict__ dXe) {
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i0 = (int64_t)blockIdx.x * blockDim.x; i0 < T; i0 += stride) {  // warp-uniform
        const int64_t t = i0 + threadIdx.x;
        const bool act = t < T && mask[t];
        if (dE && t < T && !act) {
            dE[t] = 0.0;
            dnu[t] = 0.0;
#pragma unroll
            for (int k = 0; k < 12; ++k) dXe[12 * t + k] = 0.0;
        }
        const unsigned m = __ballot_sync(FULL, act);
        unsigned long long base = 0;
        if (lane == 0 && m) base = atomicAdd(count, (unsigned long long)__popc(m));
        base = __shfl_sync(FULL, base, 0);
        if (act) list[base + __popc(m & ((1u << lane) - 1u))] = (int32_t)t;
    }
}

// Element records of tets list[0 .. *count) (or of all tets 0 .. T-1 when list is null), one
// per thread, staged per warp in shared memory and written out as contiguous records.
__global__ void __launch_bounds__(EL_TPB)
k_elements(const double4_32a *__restrict__ X, const int4 *__restrict__ tets,
           const double2 *__restrict__ mat, const int32_t *__restrict__ list,
           const unsigned long long *__restrict__ count, int64_t T, double *__restrict__ Ke,
           unsigned long long *bad) {
    extern __shared__ double smem[];
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    double *wrec = smem + (size_t)wid * 32 * KE_STRIDE;
    const int64_t n = list ? (int64_t)*count : T;
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < n;
         base += (int64_t)gridDim.x * blockDim.x) {  // block-uniform
        const int64_t i = base + threadIdx.x;
        const bool doit = i < n;
        const int32_t t = doit ? (list ? list[i] : (int32_t)i) : 0;
        if (doit) {
            const int4 q = tets[t];
            const double2 m = mat[t];
            const bool ok = element_record(X[q.x], X[q.y], X[q.z], X[q.w], m.x, m.y, q,
                                           wrec + (size_t)lane * KE_STRIDE);
            if (!ok) {
                atomicAdd(&bad[0], 1ull);
                atomicMin(&bad[2], (unsigned long long)t);
            }
        }
        unsigned todo = __ballot_sync(FULL, doit);
        __syncwarp();
        while (todo) {  // coalesced copy-out, one record at a time, to its diagonal and pair rows
            const int r = __ffs(todo) - 1;
            todo &= todo - 1;
            const int32_t tr = __shfl_sync(FULL, t, r);
            const double2 *src = reinterpret_cast<const double2 *>(wrec + (size_t)r * KE_STRIDE);
            double2 *dd = reinterpret_cast<double2 *>(Ke + ke_diag_at(T, tr, 0));
            double2 *dp = reinterpret_cast<double2 *>(Ke + ke_pair_at(T, tr, 0));
            for (int k = lane; k < KE_STRIDE / 2; k += 32) {
                if (k < KE_DIAG / 2)
                    dd[k] = src[k];
                else
                    dp[k - KE_DIAG / 2] = src[k];
            }
        }
        __syncwarp();
    }
}


// ------------------------------------------------------------------------------------------
// Adjoint: dL/dE, dL/dnu and per-element dL/dx for an upstream gradient dL/dA given per
// CSR entry.  With G = dL/dK^(tau) gathered through the node-pair blocks of the tetrahedron and
// K = V (lam A + mu B), A[ai][bj] = g_a[i] g_b[j], B[ai][bj] = g_a[j] g_b[i] + d_ij g_a.g_b:
//   SA = sum_ab g_a^T G_ab g_b,   SB = sum_ab (g_b^T G_ab g_a + tr(G_ab) g_a.g_b)
//   dL/dE  = V (lam_E SA + mu_E SB),  dL/dnu = V (lam_nu SA + mu_nu SB)
//   dL/dx_c = V [ (lam SA + mu SB) g_c - sum_a (h_a . g_c) g_a ],  h_a = d(lam SA + mu SB)/dg_a
// using dV/dx_c = V g_c and dg_a = -(g_a . dx_c) g_c (barycentric gradients of a P1
// tetrahedron).  Element matrices are recomputed here, not stored.
// ------------------------------------------------------------------------------------------
__global__ void __launch_bounds__(128)
k_adjoint(const double4_32a *__restrict__ X, const int4 *__restrict__ tets,
          const double2 *__restrict__ mat, const int32_t *__restrict__ list,
          const unsigned long long *__restrict__ count, const int32_t *__restrict__ tblk,
          const int2 *__restrict__ boff, const double *__restrict__ gval,
          double *__restrict__ dE, double *__restrict__ dnu, double *__restrict__ dXe) {
    const int64_t n = (int64_t)*count;  // active tets (inactive ones were zeroed beforehand)
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t t = list[i];
        const int4 q = tets[t];
        const double4_32a x0 = X[q.x], x1 = X[q.y], x2 = X[q.z], x3 = X[q.w];
        V3 d1 = sub(x1, x0), d2 = sub(x2, x0), d3 = sub(x3, x0);
        V3 c1 = cross_fma(d2, d3), c2 = cross_fma(d3, d1), c3 = cross_fma(d1, d2);
        const double det = __fma_rn(d1.z, c1.z, __fma_rn(d1.y, c1.y, d1.x * c1.x));
        const double r = 1.0 / det;
        double g[4][3] = {{0, 0, 0}, {c1.x * r, c1.y * r, c1.z * r},
                          {c2.x * r, c2.y * r, c2.z * r}, {c3.x * r, c3.y * r, c3.z * r}};
#pragma unroll
        for (int m = 0; m < 3; ++m) g[0][m] = -((g[1][m] + g[2][m]) + g[3][m]);
        const double V = det / 6.0;
        const double2 em = mat[t];
        const double E = em.x, nu = em.y;
        const double onu = 1.0 + nu, omn = 1.0 - (nu + nu);
        const double lam = (E * nu) / (onu * omn), mu = E / (onu + onu);
        double SA = 0.0, SB = 0.0, hA[4][3], hB[4][3];
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int m = 0; m < 3; ++m) hA[a][m] = hB[a][m] = 0.0;
        // node pairs a <= b: for a < b the blocks (a,b) and (b,a) enter every sum through
        // H = G_ab + G_ba^T (g_a^T G_ab g_b + g_b^T G_ba g_a = g_a^T H g_b, and likewise for
        // SB and the h terms), so each unordered pair costs one set of products
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int b = a; b < 4; ++b) {
                double M[3][3];
                {
                    const int2 bo = boff[tblk[16 * t + 4 * a + b]];
                    const double *G = gval + bo.x;
#pragma unroll
                    for (int i = 0; i < 3; ++i)
#pragma unroll
                        for (int j = 0; j < 3; ++j) M[i][j] = G[i * bo.y + j];
                }
                if (a != b) {
                    const int2 bo = boff[tblk[16 * t + 4 * b + a]];
                    const double *G = gval + bo.x;
#pragma unroll
                    for (int i = 0; i < 3; ++i)
#pragma unroll
                        for (int j = 0; j < 3; ++j) M[i][j] += G[j * bo.y + i];
                }
                const double tr = M[0][0] + M[1][1] + M[2][2];
                // (the adjoint needs no fixed evaluation order: every product-sum below is an
                // explicit FMA chain, which halves its FP64 instructions under --fmad=false)
                double Mgb[3], Mtga[3], Mtgb[3], Mga[3];
#pragma unroll
                for (int i = 0; i < 3; ++i) {
                    Mgb[i] = __fma_rn(M[i][2], g[b][2], __fma_rn(M[i][1], g[b][1], M[i][0] * g[b][0]));
                    Mga[i] = __fma_rn(M[i][2], g[a][2], __fma_rn(M[i][1], g[a][1], M[i][0] * g[a][0]));
                    Mtga[i] = __fma_rn(M[2][i], g[a][2], __fma_rn(M[1][i], g[a][1], M[0][i] * g[a][0]));
                    Mtgb[i] = __fma_rn(M[2][i], g[b][2], __fma_rn(M[1][i], g[b][1], M[0][i] * g[b][0]));
                }
                const double gab = __fma_rn(g[a][2], g[b][2], __fma_rn(g[a][1], g[b][1], g[a][0] * g[b][0]));
                SA = __fma_rn(g[a][2], Mgb[2], __fma_rn(g[a][1], Mgb[1], __fma_rn(g[a][0], Mgb[0], SA)));
                SB = __fma_rn(tr, gab, __fma_rn(g[b][2], Mga[2], __fma_rn(g[b][1], Mga[1],
                                                                         __fma_rn(g[b][0], Mga[0], SB))));
#pragma unroll
                for (int m = 0; m < 3; ++m) {
                    hA[a][m] += Mgb[m];
                    hA[b][m] += Mtga[m];
                    hB[a][m] = __fma_rn(tr, g[b][m], hB[a][m] + Mtgb[m]);
                    hB[b][m] = __fma_rn(tr, g[a][m], hB[b][m] + Mga[m]);
                }
            }
        const double lamE = nu / (onu * omn), muE = 1.0 / (onu + onu);
        const double lamN = E * (1.0 + 2.0 * nu * nu) / (onu * onu * omn * omn);
        const double muN = -E / (2.0 * onu * onu);
        dE[t] = V * __fma_rn(lamE, SA, muE * SB);
        dnu[t] = V * __fma_rn(lamN, SA, muN * SB);
        const double S = __fma_rn(lam, SA, mu * SB);
        double hh[4][3];  // lam hA + mu hB, once per node
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int m = 0; m < 3; ++m) hh[a][m] = __fma_rn(lam, hA[a][m], mu * hB[a][m]);
#pragma unroll
        for (int cidx = 0; cidx < 4; ++cidx) {
            double o[3] = {S * g[cidx][0], S * g[cidx][1], S * g[cidx][2]};
#pragma unroll
            for (int a = 0; a < 4; ++a) {
                const double hg = __fma_rn(hh[a][2], g[cidx][2],
                                           __fma_rn(hh[a][1], g[cidx][1], hh[a][0] * g[cidx][0]));
#pragma unroll
                for (int m = 0; m < 3; ++m) o[m] = __fma_rn(-hg, g[a][m], o[m]);
            }
#pragma unroll
            for (int m = 0; m < 3; ++m) dXe[12 * t + 3 * cidx + m] = V * o[m];
        }
    }
}

// dL/dX of each node: fold over its incident tetrahedra in ascending id (deterministic).
__global__ void k_node_grad(const int32_t *__restrict__ nt_ptr, const int32_t *__restrict__ nt_list,
                            const int4 *__restrict__ tets, const double *__restrict__ dXe,
                            int64_t n, double *__restrict__ dX) {
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n;
         v += (int64_t)gridDim.x * blockDim.x) {
        double s0 = 0.0, s1 = 0.0, s2 = 0.0;
        for (int32_t e = nt_ptr[v]; e < nt_ptr[v + 1]; ++e) {
            const int32_t t = nt_list[e];
            const int4 q = tets[t];
            const int k = q.x == v ? 0 : (q.y == v ? 1 : (q.z == v ? 2 : 3));
            const double *p = dXe + 12 * (int64_t)t + 3 * k;
            s0 += p[0];
            s1 += p[1];
            s2 += p[2];
        }
        dX[3 * v] = s0;
        dX[3 * v + 1] = s1;
        dX[3 * v + 2] = s2;
    }
}

// y = A x over the context's CSR (one thread per row, ascending columns).
__global__ void k_spmv(const int32_t *__restrict__ row_ptr, const int32_t *__restrict__ col,
                       const double *__restrict__ val, const double *__restrict__ x, int64_t nrows,
                       double *__restrict__ y) {
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < nrows;
         r += (int64_t)gridDim.x * blockDim.x) {
        double s = 0.0;
        for (int32_t k = row_ptr[r]; k < row_ptr[r + 1]; ++k) s += val[k] * x[col[k]];
        y[r] = s;
    }
}

// Expand cached records of selected tetrahedra to full 12x12 row-major matrices.
__global__ void k_expand(const double *__restrict__ Ke, const int4 *__restrict__ tets, int64_t T,
                         const int32_t *ids, int64_t n, double *out) {
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < 144 * n;
         k += (int64_t)gridDim.x * blockDim.x) {
        int64_t e = k / 144;
        int pq = (int)(k % 144), p = pq / 12, q = pq % 12;
        int32_t t = ids[e];
        if (t < 0 || t >= T) {
            out[k] = 0.0;
            continue;
        }
        int a = p / 3, i = p % 3, b = q / 3, j = q % 3;
        if (a > b || (a == b && i > j)) {  // mirror into the stored upper triangle
            int ta = a, ti = i;
            a = b; i = j; b = ta; j = ti;
        }
        const int4 tq = tets[t];
        const int gid[4] = {tq.x, tq.y, tq.z, tq.w};
        const double *dg = Ke + ke_diag_at(T, t, a), *pr = Ke + ke_pair_at(T, t, ke_pair(a, b));
        out[k] = (a == b)             ? dg[ke_tri(i, j)]
                 : gid[a] < gid[b] ? pr[3 * i + j]
                                   : pr[3 * j + i];
    }
}

}  // namespace

namespace {

// The unordered list of active tets (c->act_list, count in c->act_count), allocated on first use.
int launch_active_list(Ctx *c, double *dE, double *dnu, double *dXe, cudaStream_t s) {
    if (!c->act_list) {
        STA_TRY(dev_alloc(c, &c->act_list, c->T));
        STA_TRY(dev_alloc(c, &c->act_count, 1));
    }
    STA_CUDA_TRY(cudaMemsetAsync(c->act_count, 0, sizeof(unsigned long long), s));
    int64_t grid = (c->T + 255) / 256;
    const int64_t cap = (int64_t)c->num_sms * 16;
    if (grid > cap) grid = cap;
    k_active_list<<<(unsigned)grid, 256, 0, s>>>(c->mask, c->T, c->act_list, c->act_count, dE,
                                                 dnu, dXe);
    STA_CUDA_TRY(cudaGetLastError());
    return STA_OK;
}

}  // namespace

int launch_elements(Ctx *c, bool active_only, cudaStream_t s) {
    if (c->T == 0) return STA_OK;
    size_t smem = (size_t)EL_TPB * KE_STRIDE * sizeof(double);  // 84 KB
    STA_CUDA_TRY(cudaFuncSetAttribute(k_elements, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)smem));
    if (active_only) STA_TRY(launch_active_list(c, nullptr, nullptr, nullptr, s));
    int64_t blocks = (c->T + EL_TPB - 1) / EL_TPB;
    int per_sm = 0;
    STA_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_elements, EL_TPB, smem));
    if (per_sm < 1) per_sm = 1;
    int64_t cap = (int64_t)per_sm * c->num_sms;
    if (blocks > cap) blocks = cap;
    k_elements<<<(unsigned)blocks, EL_TPB, smem, s>>>(c->X, c->tets, c->mat,
                                                      active_only ? c->act_list : nullptr,
                                                      active_only ? c->act_count : nullptr, c->T,
                                                      c->Ke, c->counters);
    STA_CUDA_TRY(cudaGetLastError());
    return STA_OK;
}

int launch_adjoint(Ctx *c, const double *gval, double *dE, double *dnu, double *dX,
                   cudaStream_t s) {
    if (!c->dXe) STA_TRY(dev_alloc(c, &c->dXe, 12 * c->T));
    if (c->T > 0) {
        STA_TRY(launch_active_list(c, dE, dnu, c->dXe, s));
        int64_t grid = (c->T + 127) / 128;
        const int64_t cap = (int64_t)c->num_sms * 16;
        if (grid > cap) grid = cap;
        k_adjoint<<<(unsigned)grid, 128, 0, s>>>(c->X, c->tets, c->mat, c->act_list, c->act_count,
                                                c->tblk, c->boff, gval, dE, dnu, c->dXe);
    }
    if (c->n > 0) {
        int64_t grid = (c->n + 255) / 256;
        const int64_t cap = (int64_t)c->num_sms * 16;
        if (grid > cap) grid = cap;
        k_node_grad<<<(unsigned)grid, 256, 0, s>>>(c->nt_ptr, c->nt_list, c->tets, c->dXe, c->n, dX);
    }
    STA_CUDA_TRY(cudaGetLastError());
    return STA_OK;
}

int launch_spmv(Ctx *c, const double *val, const double *x, double *y, cudaStream_t s) {
    if (c->nrows == 0) return STA_OK;
    int64_t grid = (c->nrows + 255) / 256;
    const int64_t cap = (int64_t)c->num_sms * 16;
    if (grid > cap) grid = cap;
    k_spmv<<<(unsigned)grid, 256, 0, s>>>(c->row_ptr, c->col, val, x, c->nrows, y);
    STA_CUDA_TRY(cudaGetLastError());
    return STA_OK;
}

int launch_expand_elements(Ctx *c, const int32_t *ids, int64_t n, double *out, cudaStream_t s) {
    if (n == 0) return STA_OK;
    int64_t items = 144 * n;
    int64_t blocks = (items + 255) / 256;
    if (blocks > 65535LL * 16) blocks = 65535LL * 16;
    k_expand<<<(unsigned)blocks, 256, 0, s>>>(c->Ke, c->tets, c->T, ids, n, out);
    STA_CUDA_TRY(cudaGetLastError());
    return STA_OK;
}

}  // namespace sta
