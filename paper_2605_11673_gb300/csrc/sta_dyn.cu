// Implicit-Euler dynamic loop on the maintained operator (STA-FEM Sec. 6.2, Eq. 9):
//     (M_t + h^2 K_t) u_{t+1} = M_t (u_t + h v_t) + h^2 f,   v_{t+1} = (u_{t+1} - u_t) / h,
// K_t the context's maintained values (eps included), M_t a maintained lumped mass.
//
// Lumped mass (the paper gives no formula): row-sum lumping of the consistent P1 mass, each
// active tetrahedron gives (rho V) / 4 to each of its nodes (every DOF of the node), folded per
// node from +0.0 in ascending tetrahedron id -- the canonical order of the stiffness, so the
// maintained mass equals a rebuild bit for bit.  V = det / 6 with det in the element matrix's
// fixed order.  The per-tet quarter masses are computed once (sta_dyn_setup, sta_set_params);
// a streaming frame re-folds the nodes of its edited tetrahedra after the mask update; a
// rebuild re-folds every node.
//
// Solve: conjugate gradients with the Jacobi preconditioner (the paper's solver: CG with
// diagonal preconditioning), on the free DOFs -- not clamped, of a node with mass; a clamped
// DOF stays 0, a DOF of a node without mass keeps its displacement with velocity 0.  Start:
// x = u_t.  Stop: ||r|| <= tol ||b|| or max_iter.  A x = m x + h^2 (K x) is applied without
// forming the matrix, one thread per node over its three rows (they share their columns).
// Every dot product is a fixed-order reduction (warp tree, warps in order, CTAs in order by the
// last CTA to arrive), so a solve is deterministic for a given context.  Iterations run in
// captured chunks of CG_CHUNK (2 launches each: the SpMV of z also forms p = z + beta p and
// q = A z + beta q = A p, then the update); the host reads the state between chunks.
#include <algorithm>
#include <cmath>
#include <vector>

#include "sta_internal.cuh"

namespace sta {
namespace {

constexpr int DYN_TPB = 256;
constexpr int DYN_WARPS = DYN_TPB / 32;
constexpr int CG_CHUNK = 8;

// Device state of one step's solve.
struct CgState {
    double rz, pq, rr, bb, alpha, beta, tol2, pad0;
    int32_t iters, max_iter, done, pad1;
    unsigned int arrive[4];  // last-CTA counters: spmv, r0, update, spare
};

// -------------------------------------------------------------------------------- mass

__global__ void k_dyn_qmass(const double4_32a *__restrict__ X, const int4 *__restrict__ tets,
                            int64_t T, double rho, double *__restrict__ qmass) {
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < T;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int4 q = tets[t];
        const double4_32a x0 = X[q.x], x1 = X[q.y], x2 = X[q.z], x3 = X[q.w];
        const double d1x = x1.x - x0.x, d1y = x1.y - x0.y, d1z = x1.z - x0.z;
        const double d2x = x2.x - x0.x, d2y = x2.y - x0.y, d2z = x2.z - x0.z;
        const double d3x = x3.x - x0.x, d3y = x3.y - x0.y, d3z = x3.z - x0.z;
        // c_1 = d_2 x d_3, det = d_1 . c_1 (the element matrix's order)
        const double cx = __fma_rn(d2y, d3z, -(d2z * d3y));
        const double cy = __fma_rn(d2z, d3x, -(d2x * d3z));
        const double cz = __fma_rn(d2x, d3y, -(d2y * d3x));
        const double det = __fma_rn(d1z, cz, __fma_rn(d1y, cy, d1x * cx));
        qmass[t] = (rho * (det / 6.0)) * 0.25;
    }
}

__device__ __forceinline__ double node_mass(int32_t a, const int32_t *__restrict__ nt_ptr,
                                            const int32_t *__restrict__ nt_list,
                                            const uint8_t *__restrict__ mask,
                                            const double *__restrict__ qmass) {
    double m = 0.0;
    for (int32_t q = nt_ptr[a]; q < nt_ptr[a + 1]; ++q) {
        const int32_t t = nt_list[q];
        if (mask[t]) m += qmass[t];
    }
    return m;
}

// Lumped mass of every node: the fold of its active tetrahedra's quarter masses, ascending
// tetrahedron id, from +0.0.
__global__ void k_dyn_mass_all(int64_t n, const int32_t *__restrict__ nt_ptr,
                               const int32_t *__restrict__ nt_list, const uint8_t *__restrict__ mask,
                               const double *__restrict__ qmass, double *__restrict__ mass) {
    for (int64_t a = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; a < n;
         a += (int64_t)gridDim.x * blockDim.x)
        mass[a] = node_mass((int32_t)a, nt_ptr, nt_list, mask, qmass);
}

// The nodes of the frame's edited tetrahedra, after the mask update.  A node shared by several
// edited tetrahedra is re-folded by each of them; all read the same mask and write the same
// value.
__global__ void k_dyn_mass_edited(const int32_t *__restrict__ edited, int64_t m,
                                  const int64_t *__restrict__ m_dev, const int4 *__restrict__ tets,
                                  const int32_t *__restrict__ nt_ptr,
                                  const int32_t *__restrict__ nt_list,
                                  const uint8_t *__restrict__ mask,
                                  const double *__restrict__ qmass, double *__restrict__ mass) {
    const int64_t items = 4 * (m_dev ? *m_dev : m);
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < items;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t t = (uint32_t)edited[i >> 2] & 0x7fffffffu;
        const int4 q = tets[t];
        const int j = (int)(i & 3);
        const int32_t a = j == 0 ? q.x : (j == 1 ? q.y : (j == 2 ? q.z : q.w));
        mass[a] = node_mass(a, nt_ptr, nt_list, mask, qmass);
    }
}

// -------------------------------------------------------------------------------- CG

// Sum over the CTA in a fixed order; the result is valid in thread 0.
__device__ __forceinline__ double cta_sum(double v, double *sh) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
    __syncthreads();
    double t = 0.0;
    if (threadIdx.x == 0)
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += sh[w];
    __syncthreads();
    return t;
}

// Thread 0 has stored this CTA's partials; true (in every thread) in the last CTA to arrive,
// once all partials are visible.  The last CTA resets the counter for the next use.
__device__ __forceinline__ bool last_cta(unsigned int *arrive) {
    __shared__ bool last;
    __threadfence();
    if (threadIdx.x == 0) last = atomicAdd(arrive, 1u) == gridDim.x - 1;
    __syncthreads();
    if (last) __threadfence();
    return last;
}

// In the last CTA (every thread calls it): the sum of the n per-CTA partials, each thread over
// a fixed stride of them, then the CTA tree; valid in thread 0.
__device__ __forceinline__ double sum_parts(const double *part, int n, double *sh) {
    double t = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) t += __ldcg(part + i);
    return cta_sum(t, sh);
}

__device__ __forceinline__ bool cg_stopped(const CgState *st) {
    return st->done || st->iters >= st->max_iter;
}

// b, x0 = u, Jacobi inverse diagonal and the free flags, per DOF.
__global__ void k_cg_init(int64_t n3, const int32_t *__restrict__ adj_ptr,
                          const int32_t *__restrict__ adj, const int32_t *__restrict__ row_ptr,
                          const double *__restrict__ val, const double *__restrict__ mass,
                          const uint8_t *__restrict__ clamped, const double *__restrict__ u,
                          const double *__restrict__ v, const double *__restrict__ f, double h,
                          double *__restrict__ x, double *__restrict__ b,
                          double *__restrict__ dinv, uint8_t *__restrict__ fr) {
    const double h2 = h * h;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n3;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int32_t a = (int32_t)(i / 3), k = (int32_t)(i - 3 * (int64_t)a);
        const double m = mass[a];
        const bool free = !clamped[a] && m > 0.0;
        fr[i] = free ? 1 : 0;
        if (!free) {
            x[i] = 0.0;
            b[i] = 0.0;
            dinv[i] = 0.0;
            continue;
        }
        int32_t lo = adj_ptr[a], hi = adj_ptr[a + 1];  // the diagonal block of node a
        while (lo < hi) {
            const int32_t mid = (lo + hi) >> 1;
            if (adj[mid] < a) lo = mid + 1; else hi = mid;
        }
        const double kii = val[row_ptr[i] + 3 * (lo - adj_ptr[a]) + k];
        x[i] = u[i];
        b[i] = m * (u[i] + h * v[i]) + h2 * f[i];
        dinv[i] = 1.0 / (m + h2 * kii);
    }
}

// q = A x on the free DOFs (0 elsewhere), four lanes per node over its three rows (they share
// their columns): lane j of the quad takes the entries j, j + 4, ... of each row, ascending,
// and the quad adds its four partial sums as (s0 + s1) + (s2 + s3).  GB300 issues an FP64
// instruction for a whole warp whatever its active lanes, and the FP64 pipe is the scarce unit
// here, so every lane works on its own entries and the only cross-lane adds are the two quad
// levels.  The nodes are taken in the order `perm` (ascending row length), so that the eight
// nodes of a warp have rows of nearly one length.  With `dots`, the last CTA forms p.q and
// alpha = rz / pq.
__global__ void __launch_bounds__(DYN_TPB)
k_cg_spmv(int64_t n, const int32_t *__restrict__ perm, const int32_t *__restrict__ row_ptr,
          const int32_t *__restrict__ col, const double *__restrict__ val,
          const double *__restrict__ mass, double h2, const uint8_t *__restrict__ fr,
          const double *__restrict__ xin, double *__restrict__ qout, double *__restrict__ part,
          CgState *st, bool dots, double *__restrict__ p) {
    __shared__ double sh[DYN_WARPS];
    if (dots && cg_stopped(st)) return;
    const double beta = p ? st->beta : 0.0;
    const int lane = threadIdx.x & 31, qd = lane & 3;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    double pq = 0.0;
    for (int64_t base = 8 * warp; base < n; base += 8 * nwarps) {  // warp-uniform
        const int64_t j = base + (lane >> 2);
        double s0 = 0.0, s1 = 0.0, s2 = 0.0;
        int64_t a = -1;
        if (j < n) {
            a = perm[j];
            const int32_t r0 = row_ptr[3 * a], len = (row_ptr[3 * a + 3] - r0) / 3;
            const int32_t r1 = r0 + len, r2 = r1 + len;
            int32_t k = qd;
            for (; k + 12 < len; k += 16) {
                int32_t cj[4];
                double v0[4], v1[4], v2[4], xj[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    cj[u] = col[r0 + k + 4 * u];
                    v0[u] = val[r0 + k + 4 * u];
                    v1[u] = val[r1 + k + 4 * u];
                    v2[u] = val[r2 + k + 4 * u];
                }
#pragma unroll
                for (int u = 0; u < 4; ++u) xj[u] = xin[cj[u]];
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    s0 = __fma_rn(v0[u], xj[u], s0);
                    s1 = __fma_rn(v1[u], xj[u], s1);
                    s2 = __fma_rn(v2[u], xj[u], s2);
                }
            }
            for (; k < len; k += 4) {
                const double xj = xin[col[r0 + k]];
                s0 = __fma_rn(val[r0 + k], xj, s0);
                s1 = __fma_rn(val[r1 + k], xj, s1);
                s2 = __fma_rn(val[r2 + k], xj, s2);
            }
        }
        for (int o = 1; o <= 2; o <<= 1) {
            s0 += __shfl_xor_sync(0xffffffffu, s0, o);
            s1 += __shfl_xor_sync(0xffffffffu, s1, o);
            s2 += __shfl_xor_sync(0xffffffffu, s2, o);
        }
        if (a >= 0 && qd < 3) {
            const int64_t d = 3 * a + qd;
            const double xd = xin[d];
            const double sd = qd == 0 ? s0 : (qd == 1 ? s1 : s2);
            double q = fr[d] ? __fma_rn(mass[a], xd, h2 * sd) : 0.0;
            if (p) {  // CG step: xin = z, p = z + beta p, q = A z + beta q = A p
                const double pd = __fma_rn(beta, p[d], xd);
                q = __fma_rn(beta, qout[d], q);
                p[d] = pd;
                qout[d] = q;
                pq = __fma_rn(pd, q, pq);
            } else {
                qout[d] = q;
                pq = __fma_rn(xd, q, pq);
            }
        }
    }
    if (!dots) return;
    const double t = cta_sum(pq, sh);
    if (threadIdx.x == 0) part[blockIdx.x] = t;
    if (last_cta(&st->arrive[0])) {
        const double s = sum_parts(part, gridDim.x, sh);
        if (threadIdx.x == 0) {
            st->pq = s;
            if (s > 0.0) st->alpha = st->rz / s;
            else st->done = 1;  // breakdown: p = 0 (already converged) or A not positive definite
            st->arrive[0] = 0u;
        }
    }
}

// r = b - q, z = D^-1 r, p = q = 0; rz, rr, bb; the convergence test.
__global__ void __launch_bounds__(DYN_TPB)
k_cg_r0(int64_t n3, const double *__restrict__ b, double *__restrict__ q,
        const double *__restrict__ dinv, double *__restrict__ r, double *__restrict__ z,
        double *__restrict__ p, double *__restrict__ part, CgState *st) {
    __shared__ double sh[DYN_WARPS];
    double rz = 0.0, rr = 0.0, bb = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n3;
         i += (int64_t)gridDim.x * blockDim.x) {
        const double ri = b[i] - q[i], zi = dinv[i] * ri;
        r[i] = ri;
        z[i] = zi;
        p[i] = 0.0;  // with beta = 0 the first step forms p = z and q = A z
        q[i] = 0.0;
        rz = __fma_rn(ri, zi, rz);
        rr = __fma_rn(ri, ri, rr);
        bb = __fma_rn(b[i], b[i], bb);
    }
    const double a0 = cta_sum(rz, sh), a1 = cta_sum(rr, sh), a2 = cta_sum(bb, sh);
    if (threadIdx.x == 0) {
        part[blockIdx.x] = a0;
        part[gridDim.x + blockIdx.x] = a1;
        part[2 * gridDim.x + blockIdx.x] = a2;
    }
    if (last_cta(&st->arrive[1])) {
        const double s0 = sum_parts(part, gridDim.x, sh);
        const double s1 = sum_parts(part + gridDim.x, gridDim.x, sh);
        const double s2 = sum_parts(part + 2 * gridDim.x, gridDim.x, sh);
        if (threadIdx.x == 0) {
            st->rz = s0;
            st->rr = s1;
            st->bb = s2;
            st->beta = 0.0;
            st->iters = 0;
            st->done = s1 <= st->tol2 * s2 ? 1 : 0;
            st->arrive[1] = 0u;
        }
    }
}

// x += alpha p, r -= alpha q, z = D^-1 r; rz, rr; beta, the iteration count, the test.
__global__ void __launch_bounds__(DYN_TPB)
k_cg_update(int64_t n3, double *__restrict__ x, double *__restrict__ r, double *__restrict__ z,
            const double *__restrict__ p, const double *__restrict__ q,
            const double *__restrict__ dinv, double *__restrict__ part, CgState *st) {
    __shared__ double sh[DYN_WARPS];
    if (cg_stopped(st)) return;
    const double alpha = st->alpha;
    double rz = 0.0, rr = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n3;
         i += (int64_t)gridDim.x * blockDim.x) {
        x[i] = __fma_rn(alpha, p[i], x[i]);
        const double ri = __fma_rn(-alpha, q[i], r[i]), zi = dinv[i] * ri;
        r[i] = ri;
        z[i] = zi;
        rz = __fma_rn(ri, zi, rz);
        rr = __fma_rn(ri, ri, rr);
    }
    const double a0 = cta_sum(rz, sh), a1 = cta_sum(rr, sh);
    if (threadIdx.x == 0) {
        part[blockIdx.x] = a0;
        part[gridDim.x + blockIdx.x] = a1;
    }
    if (last_cta(&st->arrive[2])) {
        const double rzn = sum_parts(part, gridDim.x, sh);
        const double rrn = sum_parts(part + gridDim.x, gridDim.x, sh);
        if (threadIdx.x == 0) {
            st->rr = rrn;
            st->beta = st->rz != 0.0 ? rzn / st->rz : 0.0;
            st->rz = rzn;
            st->iters += 1;
            if (rrn <= st->tol2 * st->bb) st->done = 1;
            st->arrive[2] = 0u;
        }
    }
}


// Static solve (sta_solve): b, x0 and the Jacobi inverse diagonal on the caller's free DOFs.
__global__ void k_cg_init_static(int64_t n3, const int32_t *__restrict__ adj_ptr,
                                 const int32_t *__restrict__ adj,
                                 const int32_t *__restrict__ row_ptr,
                                 const double *__restrict__ val, const uint8_t *__restrict__ free_in,
                                 const double *__restrict__ b_in, const double *__restrict__ x_in,
                                 double *__restrict__ x, double *__restrict__ b,
                                 double *__restrict__ dinv, uint8_t *__restrict__ fr) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n3;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int32_t a = (int32_t)(i / 3), k = (int32_t)(i - 3 * (int64_t)a);
        double kii = 0.0;
        if (free_in[i] && adj_ptr[a + 1] > adj_ptr[a]) {
            int32_t lo = adj_ptr[a], hi = adj_ptr[a + 1];  // the diagonal block of node a
            while (lo < hi) {
                const int32_t mid = (lo + hi) >> 1;
                if (adj[mid] < a) lo = mid + 1; else hi = mid;
            }
            kii = val[row_ptr[i] + 3 * (lo - adj_ptr[a]) + k];
        }
        const bool free = free_in[i] && kii != 0.0;  // a free DOF needs a diagonal
        fr[i] = free ? 1 : 0;
        x[i] = free ? x_in[i] : 0.0;
        b[i] = free ? b_in[i] : 0.0;
        dinv[i] = free ? 1.0 / kii : 0.0;
    }
}

// Static solve of the scalar proxy operator (one row per node): b, x0 and the inverse diagonal.
__global__ void k_cg_init_scalar(int64_t n, const int32_t *__restrict__ pdiag,
                                 const double *__restrict__ val, const uint8_t *__restrict__ free_in,
                                 const double *__restrict__ b_in, const double *__restrict__ x_in,
                                 double *__restrict__ x, double *__restrict__ b,
                                 double *__restrict__ dinv, uint8_t *__restrict__ fr) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int32_t g = pdiag[i];
        const double kii = free_in[i] && g >= 0 ? val[g] : 0.0;
        const bool free = kii != 0.0;
        fr[i] = free ? 1 : 0;
        x[i] = free ? x_in[i] : 0.0;
        b[i] = free ? b_in[i] : 0.0;
        dinv[i] = free ? 1.0 / kii : 0.0;
    }
}

// q = A x on the free rows of a scalar operator, four lanes per row (rows in the order `perm`,
// ascending length), each row's lanes adding their partial sums as (s0 + s1) + (s2 + s3).
// With `dots`, the last CTA forms p.q and alpha = rz / pq.
__global__ void __launch_bounds__(DYN_TPB)
k_cg_spmv_scalar(int64_t n, const int32_t *__restrict__ perm, const int32_t *__restrict__ row_ptr,
                 const int32_t *__restrict__ col, const double *__restrict__ val,
                 const uint8_t *__restrict__ fr, const double *__restrict__ xin,
                 double *__restrict__ qout, double *__restrict__ part, CgState *st, bool dots,
                 double *__restrict__ p) {
    __shared__ double sh[DYN_WARPS];
    if (dots && cg_stopped(st)) return;
    const double beta = p ? st->beta : 0.0;
    const int lane = threadIdx.x & 31, qd = lane & 3;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    double pq = 0.0;
    for (int64_t base = 8 * warp; base < n; base += 8 * nwarps) {  // warp-uniform
        const int64_t j = base + (lane >> 2);
        double acc = 0.0;
        int64_t a = -1;
        if (j < n) {
            a = perm[j];
            const int32_t r0 = row_ptr[a], r1 = row_ptr[a + 1];
            for (int32_t k = r0 + qd; k < r1; k += 4) acc = __fma_rn(val[k], xin[col[k]], acc);
        }
        acc += __shfl_xor_sync(0xffffffffu, acc, 1);
        acc += __shfl_xor_sync(0xffffffffu, acc, 2);
        if (a >= 0 && qd == 0) {
            double q = fr[a] ? acc : 0.0;
            if (p) {  // CG step: xin = z, p = z + beta p, q = A z + beta q = A p
                const double pa = __fma_rn(beta, p[a], xin[a]);
                q = __fma_rn(beta, qout[a], q);
                p[a] = pa;
                qout[a] = q;
                pq = __fma_rn(pa, q, pq);
            } else {
                qout[a] = q;
                pq = __fma_rn(xin[a], q, pq);
            }
        }
    }
    if (!dots) return;
    const double t = cta_sum(pq, sh);
    if (threadIdx.x == 0) part[blockIdx.x] = t;
    if (last_cta(&st->arrive[0])) {
        const double s = sum_parts(part, gridDim.x, sh);
        if (threadIdx.x == 0) {
            st->pq = s;
            if (s > 0.0) st->alpha = st->rz / s;
            else st->done = 1;
            st->arrive[0] = 0u;
        }
    }
}

// The adjoint rule of a solve (A_ff u_f = f_f): dL/dA_ij = -lam_i u_j on entries between free
// DOFs, 0 elsewhere.  One thread per row.
__global__ void k_outer_grad(int64_t nrows, const int32_t *__restrict__ row_ptr,
                             const int32_t *__restrict__ col, const double *__restrict__ lam,
                             const double *__restrict__ u, const uint8_t *__restrict__ free,
                             double *__restrict__ g) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nrows;
         i += (int64_t)gridDim.x * blockDim.x) {
        const bool fi = free[i] != 0;
        const double li = -lam[i];
        for (int32_t k = row_ptr[i]; k < row_ptr[i + 1]; ++k) {
            const int32_t j = col[k];
            g[k] = fi && free[j] ? li * u[j] : 0.0;
        }
    }
}

// x restricted to the free DOFs (0 elsewhere), with the free flags from mass and clamping.
__global__ void k_dyn_restrict(int64_t n3, const double *__restrict__ mass,
                               const uint8_t *__restrict__ clamped, const double *__restrict__ x,
                               double *__restrict__ xf, uint8_t *__restrict__ fr) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n3;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t a = i / 3;
        const bool free = !clamped[a] && mass[a] > 0.0;
        fr[i] = free ? 1 : 0;
        xf[i] = free ? x[i] : 0.0;
    }
}

// u, v from the solution.
__global__ void k_dyn_advance(int64_t n3, double *__restrict__ u, double *__restrict__ v,
                              const double *__restrict__ x, const uint8_t *__restrict__ fr,
                              const uint8_t *__restrict__ clamped, double h) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n3;
         i += (int64_t)gridDim.x * blockDim.x) {
        if (fr[i]) {
            v[i] = (x[i] - u[i]) / h;
            u[i] = x[i];
        } else {
            v[i] = 0.0;
            if (clamped[i / 3]) u[i] = 0.0;
        }
    }
}

unsigned dyn_grid(const Ctx *c, int64_t items, int per_sm = 4) {
    int64_t g = (items + DYN_TPB - 1) / DYN_TPB;
    const int64_t cap = (int64_t)c->num_sms * per_sm;
    if (g > cap) g = cap;
    return (unsigned)(g < 1 ? 1 : g);
}

}  // namespace

// ------------------------------------------------------------------------------ launchers

int launch_dyn_mass_all(Ctx *c, cudaStream_t s) {
    if (!c->dyn || c->n == 0) return STA_OK;
    k_dyn_mass_all<<<dyn_grid(c, c->n), DYN_TPB, 0, s>>>(c->n, c->nt_ptr, c->nt_list, c->mask,
                                                         c->qmass, c->mass);
    STA_CUDA_TRY(cudaGetLastError());
    return STA_OK;
}

int launch_dyn_mass_edited(Ctx *c, const int32_t *edited, int64_t m, const int64_t *m_dev,
                           int64_t cap, cudaStream_t s) {
    if (!c->dyn) return STA_OK;
    k_dyn_mass_edited<<<dyn_grid(c, 4 * (cap > 0 ? cap : 1), 8), DYN_TPB, 0, s>>>(
        edited, m, m_dev, c->tets, c->nt_ptr, c->nt_list, c->mask, c->qmass, c->mass);
    STA_CUDA_TRY(cudaGetLastError());
    return STA_OK;
}

int launch_dyn_qmass(Ctx *c, cudaStream_t s) {
    if (!c->dyn || c->T == 0) return STA_OK;
    k_dyn_qmass<<<dyn_grid(c, c->T, 8), DYN_TPB, 0, s>>>(c->X, c->tets, c->T, c->dyn_rho, c->qmass);
    STA_CUDA_TRY(cudaGetLastError());
    return STA_OK;
}

namespace {

// One chunk of CG_CHUNK iterations (2 launches each) of A = diag(mass) + h2 K(val), launched
// or captured on s.
int cg_chunk(Ctx *c, const double *val, const double *mass, double h2, cudaStream_t s) {
    const int64_t n3 = c->nrows;  // DOFs: 3 per node, or 1 for the scalar proxy operator
    const unsigned gv = c->cg_grid;
    double *x = c->cg, *b = x + n3, *r = b + n3, *z = r + n3, *p = z + n3, *q = p + n3;
    double *dinv = q + n3;
    CgState *st = reinterpret_cast<CgState *>(c->cg_state);
    for (int it = 0; it < CG_CHUNK; ++it) {
        if (c->op == STA_OP_PROXY)
            k_cg_spmv_scalar<<<gv, DYN_TPB, 0, s>>>(c->n, c->dyn_perm, c->row_ptr, c->col, val,
                                                    c->cg_free, z, q, c->cg_part, st, true, p);
        else
            k_cg_spmv<<<gv, DYN_TPB, 0, s>>>(c->n, c->dyn_perm, c->row_ptr, c->col, val, mass, h2,
                                            c->cg_free, z, q, c->cg_part, st, true, p);
        k_cg_update<<<gv, DYN_TPB, 0, s>>>(n3, x, r, z, p, q, dinv, c->cg_part, st);
    }
    STA_CUDA_TRY(cudaGetLastError());
    return STA_OK;
}

}  // namespace

namespace {

// CG iterations in chunks until converged or max_iter: the captured chunk `g` if given, else
// direct launches of the chunk for (val, mass, h2).  The host reads the state between chunks;
// with `stagnate`, it also stops once the residual has not halved for 1000 iterations (the
// attainable accuracy reached).
int cg_iterate(Ctx *c, cudaGraphExec_t g, const double *val, const double *mass, double h2,
               int32_t max_iter, bool stagnate, cudaStream_t s, CgState *hs) {
    CgState *st = reinterpret_cast<CgState *>(c->cg_state);
    double best = -1.0;
    int32_t best_it = 0;
    // the first chunk goes out with the initial residual (its kernels return at once if that is
    // already converged or max_iter is 0): one host round trip fewer per solve
    if (c->n > 0) {
        if (g) STA_CUDA_TRY(cudaGraphLaunch(g, s));
        else STA_TRY(cg_chunk(c, val, mass, h2, s));
    }
    for (;;) {
        if (c->n > 0) {
            STA_CUDA_TRY(cudaMemcpyAsync(hs, st, sizeof *hs, cudaMemcpyDeviceToHost, s));
            STA_CUDA_TRY(cudaStreamSynchronize(s));
        }
        if (c->n == 0 || hs->done || hs->iters >= max_iter) break;
        if (stagnate) {
            if (best < 0.0 || hs->rr < 0.25 * best) {
                best = hs->rr;
                best_it = hs->iters;
            } else if (hs->iters - best_it > 1000) {
                break;
            }
        }
        if (g) STA_CUDA_TRY(cudaGraphLaunch(g, s));
        else STA_TRY(cg_chunk(c, val, mass, h2, s));
    }
    return STA_OK;
}

}  // namespace

// The CG buffers shared by the implicit-Euler step and the static solve, allocated once.
int cg_alloc(Ctx *c) {
    if (c->cg) return STA_OK;
    const int64_t n = c->n, n3 = c->nrows;  // DOFs
    const int rows = c->op == STA_OP_PROXY ? 1 : 3;  // rows per node
    c->cg_grid = (int)dyn_grid(c, n3 > 0 ? n3 : 1);
    STA_TRY(dev_alloc(c, &c->cg, 7 * n3));
    STA_TRY(dev_alloc(c, &c->cg_free, n3));
    STA_TRY(dev_alloc(c, &c->cg_part, 3 * (int64_t)c->cg_grid));
    STA_TRY(dev_alloc(c, &c->cg_state, (int64_t)sizeof(CgState)));
    STA_TRY(dev_alloc(c, &c->cg_zero, n));
    STA_CUDA_TRY(cudaMemset(c->cg_zero, 0, sizeof(double) * (size_t)(n > 0 ? n : 1)));
    // the SpMV's node order: ascending row length (ties by node id)
    STA_TRY(dev_alloc(c, &c->dyn_perm, n));
    std::vector<int32_t> rp(rows * n + 1), perm(n);
    STA_CUDA_TRY(cudaMemcpy(rp.data(), c->row_ptr, sizeof(int32_t) * (rows * n + 1),
                            cudaMemcpyDeviceToHost));
    for (int64_t a = 0; a < n; ++a) perm[a] = (int32_t)a;
    std::stable_sort(perm.begin(), perm.end(), [&](int32_t p, int32_t q) {
        return rp[rows * p + rows] - rp[rows * p] < rp[rows * q + rows] - rp[rows * q];
    });
    STA_CUDA_TRY(cudaMemcpy(c->dyn_perm, perm.data(), sizeof(int32_t) * n, cudaMemcpyHostToDevice));
    return STA_OK;
}

int launch_dyn_step(Ctx *c, double tol, int32_t max_iter, int32_t *iters, double *rel_res,
                    cudaStream_t s) {
    const int64_t n3 = 3 * c->n;
    const unsigned gv = c->cg_grid;
    double *x = c->cg, *b = x + n3, *r = b + n3, *z = r + n3, *p = z + n3, *q = p + n3;
    double *dinv = q + n3;
    CgState *st = reinterpret_cast<CgState *>(c->cg_state);
    CgState h0 = {};
    h0.tol2 = tol * tol;
    h0.max_iter = max_iter;
    STA_CUDA_TRY(cudaMemcpyAsync(st, &h0, sizeof h0, cudaMemcpyHostToDevice, s));
    if (n3 > 0) {
        k_cg_init<<<gv, DYN_TPB, 0, s>>>(n3, c->adj_ptr, c->adj, c->row_ptr, c->val, c->mass,
                                         c->clamped, c->du, c->dv, c->df, c->dyn_h, x, b, dinv,
                                         c->cg_free);
        k_cg_spmv<<<gv, DYN_TPB, 0, s>>>(c->n, c->dyn_perm, c->row_ptr, c->col, c->val, c->mass,
                                        c->dyn_h * c->dyn_h, c->cg_free, x, q, c->cg_part, st, false, nullptr);
        k_cg_r0<<<gv, DYN_TPB, 0, s>>>(n3, b, q, dinv, r, z, p, c->cg_part, st);
        STA_CUDA_TRY(cudaGetLastError());
    }
    if (!c->g_cg) {  // capture the chunk once (the context's buffers never move)
        cudaStream_t cs = nullptr;
        STA_CUDA_TRY(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
        cudaGraph_t g = nullptr;
        cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
        int rc = e == cudaSuccess ? cg_chunk(c, c->val, c->mass, c->dyn_h * c->dyn_h, cs) : STA_ECUDA;
        cudaError_t e2 = cudaStreamEndCapture(cs, &g);
        if (rc == STA_OK && e == cudaSuccess && e2 == cudaSuccess)
            e2 = cudaGraphInstantiate(&c->g_cg, g, 0);
        if (g) cudaGraphDestroy(g);
        cudaStreamDestroy(cs);
        if (rc != STA_OK || e != cudaSuccess || e2 != cudaSuccess) {
            c->g_cg = nullptr;
            return fail(STA_ECUDA, "CG chunk capture failed");
        }
    }
    CgState hs = {};
    STA_TRY(cg_iterate(c, c->g_cg, nullptr, nullptr, 0.0, max_iter, false, s, &hs));
    if (n3 > 0) {
        k_dyn_advance<<<gv, DYN_TPB, 0, s>>>(n3, c->du, c->dv, x, c->cg_free, c->clamped, c->dyn_h);
        STA_CUDA_TRY(cudaGetLastError());
        STA_CUDA_TRY(cudaStreamSynchronize(s));
    }
    if (iters) *iters = hs.iters;
    if (rel_res) *rel_res = hs.bb > 0.0 ? std::sqrt(hs.rr / hs.bb) : 0.0;
    return STA_OK;
}

}  // namespace sta

using namespace sta;

extern "C" int sta_dyn_setup(sta_ctx *x, double rho, double h, const double *f,
                             const uint8_t *clamped, void *stream) {
    if (!x) return fail(STA_EINVAL, "ctx is NULL");
    Ctx *c = &x->c;
    if (c->op != STA_OP_ELASTICITY) return fail(STA_ESTATE, "not an elasticity context");
    if (c->graph_on) return fail(STA_ESTATE, "disable graph mode before setting up the dynamics");
    if (!(rho > 0.0) || !(h > 0.0) || !std::isfinite(rho) || !std::isfinite(h))
        return fail(STA_EINVAL, "rho and h must be positive and finite");
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t n = c->n, n3 = 3 * n;
    if (!c->qmass) {
        STA_TRY(dev_alloc(c, &c->qmass, c->T));
        STA_TRY(dev_alloc(c, &c->mass, n));
        STA_TRY(dev_alloc(c, &c->du, n3));
        STA_TRY(dev_alloc(c, &c->dv, n3));
        STA_TRY(dev_alloc(c, &c->df, n3));
        STA_TRY(dev_alloc(c, &c->clamped, n));
    }
    STA_TRY(cg_alloc(c));
    std::vector<double> hf(n3 > 0 ? n3 : 1, 0.0);
    std::vector<uint8_t> hc(n > 0 ? n : 1, 0);
    if (f) std::copy(f, f + n3, hf.begin());
    if (clamped)
        for (int64_t a = 0; a < n; ++a) hc[a] = clamped[a] ? 1 : 0;
    STA_CUDA_TRY(cudaMemcpyAsync(c->df, hf.data(), sizeof(double) * n3, cudaMemcpyHostToDevice, s));
    STA_CUDA_TRY(cudaMemcpyAsync(c->clamped, hc.data(), (size_t)n, cudaMemcpyHostToDevice, s));
    STA_CUDA_TRY(cudaMemsetAsync(c->du, 0, sizeof(double) * (size_t)(n3 > 0 ? n3 : 1), s));
    STA_CUDA_TRY(cudaMemsetAsync(c->dv, 0, sizeof(double) * (size_t)(n3 > 0 ? n3 : 1), s));
    if (c->g_cg) {  // the captured CG chunk holds h^2: capture again on the next step
        cudaGraphExecDestroy(c->g_cg);
        c->g_cg = nullptr;
    }
    c->dyn = true;
    c->dyn_rho = rho;
    c->dyn_h = h;
    STA_TRY(launch_dyn_qmass(c, s));
    STA_TRY(launch_dyn_mass_all(c, s));
    STA_CUDA_TRY(cudaStreamSynchronize(s));  // the host vectors go out of scope
    return STA_OK;
}

extern "C" int sta_dyn_step(sta_ctx *x, double tol, int32_t max_iter, int32_t *iters,
                            double *rel_res, void *stream) {
    if (!x) return fail(STA_EINVAL, "ctx is NULL");
    Ctx *c = &x->c;
    if (!c->dyn) return fail(STA_ESTATE, "call sta_dyn_setup first");
    if (!(tol >= 0.0) || max_iter < 0) return fail(STA_EINVAL, "tol and max_iter must be >= 0");
    return launch_dyn_step(c, tol, max_iter, iters, rel_res, (cudaStream_t)stream);
}

extern "C" int sta_dyn_apply(sta_ctx *x, const double *xv, double *y, void *stream) {
    if (!x) return fail(STA_EINVAL, "ctx is NULL");
    Ctx *c = &x->c;
    if (!c->dyn) return fail(STA_ESTATE, "call sta_dyn_setup first");
    const int64_t n3 = 3 * c->n;
    if (n3 == 0) return STA_OK;
    if (!xv || !y) return fail(STA_EINVAL, "NULL argument");
    cudaStream_t s = (cudaStream_t)stream;
    double *xf = c->cg + 4 * n3;  // the CG's p buffer (free between steps)
    const unsigned gv = (unsigned)c->cg_grid;
    k_dyn_restrict<<<gv, DYN_TPB, 0, s>>>(n3, c->mass, c->clamped, xv, xf, c->cg_free);
    k_cg_spmv<<<gv, DYN_TPB, 0, s>>>(c->n, c->dyn_perm, c->row_ptr, c->col, c->val, c->mass,
                                    c->dyn_h * c->dyn_h, c->cg_free, xf, y, c->cg_part,
                                    reinterpret_cast<CgState *>(c->cg_state), false, nullptr);
    STA_CUDA_TRY(cudaGetLastError());
    return STA_OK;
}

extern "C" int sta_solve(sta_ctx *x, const double *val, const double *b, const uint8_t *free,
                         double tol, int32_t max_iter, double *xv, int32_t *iters,
                         double *rel_res, void *stream) {
    if (!x) return fail(STA_EINVAL, "ctx is NULL");
    Ctx *c = &x->c;
    if (!(tol >= 0.0) || max_iter < 0) return fail(STA_EINVAL, "tol and max_iter must be >= 0");
    const int64_t n3 = c->nrows;  // DOFs: 3 per node, or 1 for the proxy operator
    if (n3 > 0 && (!b || !free || !xv)) return fail(STA_EINVAL, "NULL argument");
    cudaStream_t s = (cudaStream_t)stream;
    STA_TRY(cg_alloc(c));
    const double *A = val ? val : c->val;
    double *xw = c->cg, *bw = xw + n3, *r = bw + n3, *z = r + n3, *p = z + n3, *q = p + n3;
    double *dinv = q + n3;
    CgState *st = reinterpret_cast<CgState *>(c->cg_state);
    CgState h0 = {};
    h0.tol2 = tol * tol;
    h0.max_iter = max_iter;
    STA_CUDA_TRY(cudaMemcpyAsync(st, &h0, sizeof h0, cudaMemcpyHostToDevice, s));
    CgState hs = {};
    if (n3 > 0) {
        const unsigned gv = (unsigned)c->cg_grid;
        if (c->op == STA_OP_PROXY) {
            k_cg_init_scalar<<<gv, DYN_TPB, 0, s>>>(n3, c->pdiag, A, free, b, xv, xw, bw, dinv,
                                                    c->cg_free);
            k_cg_spmv_scalar<<<gv, DYN_TPB, 0, s>>>(c->n, c->dyn_perm, c->row_ptr, c->col, A,
                                                    c->cg_free, xw, q, c->cg_part, st, false, nullptr);
        } else {
            k_cg_init_static<<<gv, DYN_TPB, 0, s>>>(n3, c->adj_ptr, c->adj, c->row_ptr, A, free, b,
                                                    xv, xw, bw, dinv, c->cg_free);
            k_cg_spmv<<<gv, DYN_TPB, 0, s>>>(c->n, c->dyn_perm, c->row_ptr, c->col, A, c->cg_zero,
                                            1.0, c->cg_free, xw, q, c->cg_part, st, false, nullptr);
        }
        k_cg_r0<<<gv, DYN_TPB, 0, s>>>(n3, bw, q, dinv, r, z, p, c->cg_part, st);
        STA_CUDA_TRY(cudaGetLastError());
        STA_TRY(cg_iterate(c, nullptr, A, c->cg_zero, 1.0, max_iter, true, s, &hs));
        STA_CUDA_TRY(cudaMemcpyAsync(xv, xw, sizeof(double) * n3, cudaMemcpyDeviceToDevice, s));
        STA_CUDA_TRY(cudaStreamSynchronize(s));
    }
    if (iters) *iters = hs.iters;
    if (rel_res) *rel_res = hs.bb > 0.0 ? std::sqrt(hs.rr / hs.bb) : 0.0;
    return STA_OK;
}

extern "C" int sta_outer_grad(sta_ctx *x, const double *lam, const double *u,
                              const uint8_t *free, double *grad_val, void *stream) {
    if (!x) return fail(STA_EINVAL, "ctx is NULL");
    Ctx *c = &x->c;
    if (c->nrows > 0 && (!lam || !u || !free || !grad_val)) return fail(STA_EINVAL, "NULL argument");
    if (c->nrows == 0) return STA_OK;
    const unsigned g = dyn_grid(c, c->nrows, 8);
    k_outer_grad<<<g, DYN_TPB, 0, (cudaStream_t)stream>>>(c->nrows, c->row_ptr, c->col, lam, u,
                                                          free, grad_val);
    STA_CUDA_TRY(cudaGetLastError());
    return STA_OK;
}

extern "C" int sta_dyn_state(const sta_ctx *x, const double **u, const double **v,
                             const double **mass) {
    if (!x) return fail(STA_EINVAL, "ctx is NULL");
    if (!x->c.dyn) return fail(STA_ESTATE, "call sta_dyn_setup first");
    if (u) *u = x->c.du;
    if (v) *v = x->c.dv;
    if (mass) *mass = x->c.mass;
    return STA_OK;
}

extern "C" int sta_dyn_set_state(sta_ctx *x, const double *u, const double *v, int on_device,
                                 void *stream) {
    if (!x) return fail(STA_EINVAL, "ctx is NULL");
    Ctx *c = &x->c;
    if (!c->dyn) return fail(STA_ESTATE, "call sta_dyn_setup first");
    const size_t bytes = sizeof(double) * 3 * (size_t)c->n;
    const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    cudaStream_t s = (cudaStream_t)stream;
    if (u) STA_CUDA_TRY(cudaMemcpyAsync(c->du, u, bytes, kind, s));
    if (v) STA_CUDA_TRY(cudaMemcpyAsync(c->dv, v, bytes, kind, s));
    if (!on_device) STA_CUDA_TRY(cudaStreamSynchronize(s));
    return STA_OK;
}
