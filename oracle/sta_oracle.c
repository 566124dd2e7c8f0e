/*
 * STA-FEM oracle: plain, slow, serial FP64 CPU implementation of the assembly that the
 * GPU path computes.  TEST INFRASTRUCTURE ONLY: the product path never links, loads or
 * calls this file.  Only the tests, the smoke check and the benchmark's CPU-baseline leg
 * use it.  It shares no code, header, table or helper with the CUDA library.
 *
 * Build: gcc -O2 -ffp-contract=off -fPIC -shared (no fast-math, no contraction), so every
 * `a*b + c` below is two IEEE roundings and every fma() call is one.
 *
 * What it follows (STA-FEM, arXiv 2605.11673):
 *   - Eq. 8 (Sec. 3.4): the element-assembled operator  A_t = sum_{tau in T_t} P_tau^T K^(tau) P_tau + eps I.
 *   - Sec. 3.4 / Sec. 5.2: K^(tau) is the standard vector-valued linear-tetrahedron
 *     elasticity matrix (P1, isotropic, small strain).  The paper does not print the formula;
 *     the closed form and its fixed evaluation order are the reading stated in the header of
 *     orc_element() below.
 *   - Sec. 3.3: the maintained matrix must equal a from-scratch rebuild on the active set.
 *   - Sec. 3.5 (Proposition 1): full_rebuild, local_recompute (rescan every incident active
 *     tetrahedron of each touched entry) and streaming_update (add / subtract element
 *     contributions of the edited tetrahedra), the latter also in fixed point (orc_fx_*:
 *     per-entry exponents, contributions quantised once, exact integer sums).
 *   - Sec. 3.1-3.3, Eqs. 1-7, Algorithm 1: the graph-Laplacian proxy operator (orc_proxy_*:
 *     edge multiplicities, thresholded adjacency, degrees, L + eps I).
 *   - Sec. 6.2, Eq. 9: the lumped mass of the implicit-Euler loop (orc_lumped_mass).
 *   - The adjoint (not in the paper): element parameter gradients, complex-step position
 *     gradients (orc_element_param_grad, orc_element_x_grad_cs, orc_grad_all).
 *
 * Summation order (reading of "rebuild from scratch", Sec. 3.3): every CSR value is the
 * left-to-right fold, starting at +0.0, of the contributions of its active tetrahedra in
 * ascending tetrahedron id; eps is added afterwards, to diagonal entries only.
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------------------- */
/* Element matrix                                                                          */
/* ------------------------------------------------------------------------------------- */

/*
 * orc_element: 12x12 stiffness of one linear tetrahedron (Sec. 3.4, Sec. 5.2).
 *
 * Local DOF p = 3a + i  (node a = 0..3, component i = 0..2).  With g_a the gradient of the
 * barycentric coordinate of node a and V the volume,
 *     K[3a+i][3b+j] = V * ( lam g_a[i] g_b[j] + mu g_a[j] g_b[i] + delta_ij mu (g_a . g_b) ),
 * which is V * B^T D B for Voigt strain with engineering shear (cross-checked against the
 * literal product in orc_element_btdb).  Fixed evaluation order (both implementations of
 * this library follow it; fma = one rounding):
 *   1. d_k = x_k - x_0, k = 1..3.
 *   2. c_1 = d_2 x d_3, c_2 = d_3 x d_1, c_3 = d_1 x d_2 with
 *      (u x v).x = fma(u.y, v.z, -(u.z*v.y)), (u x v).y = fma(u.z, v.x, -(u.x*v.z)),
 *      (u x v).z = fma(u.x, v.y, -(u.y*v.x)).
 *   3. det = fma(d_1.z, c_1.z, fma(d_1.y, c_1.y, d_1.x*c_1.x)); must be > 0.
 *   4. r = 1/det; g_k = c_k * r (k = 1..3); g_0 = -((g_1 + g_2) + g_3); V = det / 6.
 *   5. lam = (E*nu) / ((1+nu) * (1-(nu+nu))),  mu = E / ((1+nu) + (1+nu)).
 *   6. Vl = V*lam, Vm = V*mu;  P_a[i] = Vl*g_a[i];  Q_a[i] = Vm*g_a[i];
 *      D_ab = Vm * fma(g_a.z, g_b.z, fma(g_a.y, g_b.y, g_a.x*g_b.x)).
 *   7. for p = 3a+i <= q = 3b+j:
 *        i != j:  K[p][q] = fma(P_a[i], g_b[j], Q_a[j]*g_b[i])
 *        i == j:  K[p][q] = fma(P_a[i], g_b[i], fma(Q_a[i], g_b[i], D_ab))
 *      and K[q][p] = K[p][q] (exactly symmetric by construction).
 * Returns 0, or -1 when det <= 0 (inverted or degenerate tetrahedron).
 */
int orc_element(const double x[12], double E, double nu, double K[144])
{
    double d[3][3], c[3][3], g[4][3];
    for (int k = 1; k <= 3; ++k)
        for (int m = 0; m < 3; ++m) d[k - 1][m] = x[3 * k + m] - x[m];
    /* c_1 = d_2 x d_3, c_2 = d_3 x d_1, c_3 = d_1 x d_2 */
    const int cu[3] = {1, 2, 0}, cv[3] = {2, 0, 1};
    for (int k = 0; k < 3; ++k) {
        const double *u = d[cu[k]], *v = d[cv[k]];
        c[k][0] = fma(u[1], v[2], -(u[2] * v[1]));
        c[k][1] = fma(u[2], v[0], -(u[0] * v[2]));
        c[k][2] = fma(u[0], v[1], -(u[1] * v[0]));
    }
    double det = fma(d[0][2], c[0][2], fma(d[0][1], c[0][1], d[0][0] * c[0][0]));
    if (!(det > 0.0)) return -1;
    double r = 1.0 / det;
    for (int k = 0; k < 3; ++k)
        for (int m = 0; m < 3; ++m) g[k + 1][m] = c[k][m] * r;
    for (int m = 0; m < 3; ++m) g[0][m] = -((g[1][m] + g[2][m]) + g[3][m]);
    double V = det / 6.0;
    double onu = 1.0 + nu;
    double lam = (E * nu) / (onu * (1.0 - (nu + nu)));
    double mu = E / (onu + onu);
    double Vl = V * lam, Vm = V * mu;
    double P[4][3], Q[4][3], D[4][4];
    for (int a = 0; a < 4; ++a)
        for (int i = 0; i < 3; ++i) {
            P[a][i] = Vl * g[a][i];
            Q[a][i] = Vm * g[a][i];
        }
    for (int a = 0; a < 4; ++a)
        for (int b = a; b < 4; ++b)
            D[a][b] = Vm * fma(g[a][2], g[b][2], fma(g[a][1], g[b][1], g[a][0] * g[b][0]));
    for (int p = 0; p < 12; ++p)
        for (int q = p; q < 12; ++q) {
            int a = p / 3, i = p % 3, b = q / 3, j = q % 3;
            double v;
            if (i != j)
                v = fma(P[a][i], g[b][j], Q[a][j] * g[b][i]);
            else
                v = fma(P[a][i], g[b][i], fma(Q[a][i], g[b][i], D[a][b]));
            K[p * 12 + q] = v;
            K[q * 12 + p] = v;
        }
    return 0;
}

/*
 * orc_element_btdb: the same element matrix formed literally as V * B^T D B with the 6x12
 * strain-displacement matrix B (Voigt order xx, yy, zz, yz, xz, xy; engineering shear) and
 * the isotropic 6x6 D = lam * 1 1^T (upper 3x3) + mu * diag(2,2,2,1,1,1).  Different
 * rounding from orc_element; used only as an independent cross-check of its formula.
 */
int orc_element_btdb(const double x[12], double E, double nu, double K[144])
{
    /* g_a from the inverse of Dm = [x1-x0, x2-x0, x3-x0] (columns), by cofactors. */
    double Dm[3][3], inv[3][3];
    for (int m = 0; m < 3; ++m)
        for (int k = 0; k < 3; ++k) Dm[m][k] = x[3 * (k + 1) + m] - x[m];
    double det = Dm[0][0] * (Dm[1][1] * Dm[2][2] - Dm[1][2] * Dm[2][1]) -
                 Dm[0][1] * (Dm[1][0] * Dm[2][2] - Dm[1][2] * Dm[2][0]) +
                 Dm[0][2] * (Dm[1][0] * Dm[2][1] - Dm[1][1] * Dm[2][0]);
    if (!(det > 0.0)) return -1;
    for (int r = 0; r < 3; ++r)
        for (int cidx = 0; cidx < 3; ++cidx) {
            int r1 = (cidx + 1) % 3, r2 = (cidx + 2) % 3, c1 = (r + 1) % 3, c2 = (r + 2) % 3;
            inv[r][cidx] = (Dm[r1][c1] * Dm[r2][c2] - Dm[r1][c2] * Dm[r2][c1]) / det;
        }
    double g[4][3];
    for (int k = 0; k < 3; ++k)
        for (int m = 0; m < 3; ++m) g[k + 1][m] = inv[k][m]; /* row k of Dm^{-1} */
    for (int m = 0; m < 3; ++m) g[0][m] = -(g[1][m] + g[2][m] + g[3][m]);
    double B[6][12];
    memset(B, 0, sizeof B);
    for (int a = 0; a < 4; ++a) {
        double gx = g[a][0], gy = g[a][1], gz = g[a][2];
        B[0][3 * a + 0] = gx;
        B[1][3 * a + 1] = gy;
        B[2][3 * a + 2] = gz;
        B[3][3 * a + 1] = gz; B[3][3 * a + 2] = gy; /* yz */
        B[4][3 * a + 0] = gz; B[4][3 * a + 2] = gx; /* xz */
        B[5][3 * a + 0] = gy; B[5][3 * a + 1] = gx; /* xy */
    }
    double lam = E * nu / ((1.0 + nu) * (1.0 - 2.0 * nu));
    double mu = E / (2.0 * (1.0 + nu));
    double Dmat[6][6];
    memset(Dmat, 0, sizeof Dmat);
    for (int r = 0; r < 3; ++r)
        for (int s = 0; s < 3; ++s) Dmat[r][s] = lam;
    for (int r = 0; r < 3; ++r) Dmat[r][r] += 2.0 * mu;
    for (int r = 3; r < 6; ++r) Dmat[r][r] = mu;
    double V = det / 6.0;
    double DB[6][12];
    for (int r = 0; r < 6; ++r)
        for (int q = 0; q < 12; ++q) {
            double s = 0.0;
            for (int k = 0; k < 6; ++k) s += Dmat[r][k] * B[k][q];
            DB[r][q] = s;
        }
    for (int p = 0; p < 12; ++p)
        for (int q = 0; q < 12; ++q) {
            double s = 0.0;
            for (int k = 0; k < 6; ++k) s += B[k][p] * DB[k][q];
            K[p * 12 + q] = V * s;
        }
    return 0;
}

static void gather_x(const double *X, const int32_t *tet, double x[12])
{
    for (int a = 0; a < 4; ++a)
        for (int m = 0; m < 3; ++m) x[3 * a + m] = X[3 * (int64_t)tet[a] + m];
}

/* Element matrices of all tetrahedra (T x 144, row-major).  Returns the number of
 * tetrahedra with det <= 0 (their matrices are left zero). */
int64_t orc_element_all(const double *X, int64_t T, const int32_t *tets, const double *E,
                        const double *nu, double *Ke)
{
    int64_t bad = 0;
    for (int64_t t = 0; t < T; ++t) {
        double x[12];
        gather_x(X, tets + 4 * t, x);
        if (orc_element(x, E[t], nu[t], Ke + 144 * t) != 0) {
            memset(Ke + 144 * t, 0, 144 * sizeof(double));
            ++bad;
        }
    }
    return bad;
}

/* ------------------------------------------------------------------------------------- */
/* Superset sparsity pattern and scatter map (P_tau of Eq. 8)                              */
/* ------------------------------------------------------------------------------------- */

/*
 * Scalar CSR with 3n rows, DOF 3v + i.  Row 3a+i holds, for every node b that shares at
 * least one superset tetrahedron with node a (a itself included), in ascending b, the three
 * columns 3b, 3b+1, 3b+2.  The pattern is that of the whole superset and never changes;
 * entries with no active contributor hold +0.0.
 * scat[t][12p + q] = CSR index of global entry (3 v_a + i, 3 v_b + j), p = 3a+i, q = 3b+j:
 * the injection P_tau of Eq. 8 written as an index map.
 */
typedef struct {
    int64_t n, T, nrows, nnz;
    int32_t *tets;    /* copy, T x 4 */
    int64_t *nt_ptr;  /* node -> incident tetrahedra, n + 1 */
    int32_t *nt_list; /* ascending tetrahedron ids */
    int64_t *deg;     /* neighbours per node */
    int32_t *row_ptr; /* 3n + 1 */
    int32_t *col;     /* nnz */
    int32_t *scat;    /* T x 144 */
    int64_t *nptr;    /* node-level pattern: row u = sorted neighbour set of u, n + 1 */
    int32_t *ncol;    /* neighbour node of each node-level entry */
} orc_pattern_t;

static int cmp_i32(const void *a, const void *b)
{
    int32_t x = *(const int32_t *)a, y = *(const int32_t *)b;
    return (x > y) - (x < y);
}

void orc_pattern_free(orc_pattern_t *p)
{
    if (!p) return;
    free(p->tets); free(p->nt_ptr); free(p->nt_list); free(p->deg);
    free(p->row_ptr); free(p->col); free(p->scat);
    free(p->nptr); free(p->ncol);
    free(p);
}

/* Returns NULL on bad input (node id out of range, repeated node in a tetrahedron) or when
 * nnz does not fit int32. */
orc_pattern_t *orc_pattern_create(int64_t n, int64_t T, const int32_t *tets)
{
    for (int64_t t = 0; t < T; ++t)
        for (int a = 0; a < 4; ++a) {
            int32_t v = tets[4 * t + a];
            if (v < 0 || v >= n) return NULL;
            for (int b = 0; b < a; ++b)
                if (tets[4 * t + b] == v) return NULL;
        }
    orc_pattern_t *p = calloc(1, sizeof *p);
    p->n = n; p->T = T; p->nrows = 3 * n;
    p->tets = malloc(sizeof(int32_t) * 4 * (T > 0 ? T : 1));
    memcpy(p->tets, tets, sizeof(int32_t) * 4 * T);
    /* node -> tetrahedra, ascending tet id (counting sort over tets in ascending order) */
    p->nt_ptr = calloc(n + 1, sizeof(int64_t));
    for (int64_t t = 0; t < T; ++t)
        for (int a = 0; a < 4; ++a) p->nt_ptr[tets[4 * t + a] + 1]++;
    for (int64_t v = 0; v < n; ++v) p->nt_ptr[v + 1] += p->nt_ptr[v];
    p->nt_list = malloc(sizeof(int32_t) * (4 * T > 0 ? 4 * T : 1));
    int64_t *fill = malloc(sizeof(int64_t) * (n > 0 ? n : 1));
    for (int64_t v = 0; v < n; ++v) fill[v] = p->nt_ptr[v];
    for (int64_t t = 0; t < T; ++t)
        for (int a = 0; a < 4; ++a) p->nt_list[fill[tets[4 * t + a]]++] = (int32_t)t;
    free(fill);
    /* neighbour sets: union of the nodes of the incident tetrahedra, sorted, unique */
    p->deg = calloc(n > 0 ? n : 1, sizeof(int64_t));
    int64_t total_blocks = 0;
    int32_t **nbr = malloc(sizeof(int32_t *) * (n > 0 ? n : 1));
    for (int64_t v = 0; v < n; ++v) {
        int64_t m = p->nt_ptr[v + 1] - p->nt_ptr[v];
        int32_t *tmp = malloc(sizeof(int32_t) * (4 * m > 0 ? 4 * m : 1));
        int64_t k = 0;
        for (int64_t e = p->nt_ptr[v]; e < p->nt_ptr[v + 1]; ++e)
            for (int a = 0; a < 4; ++a) tmp[k++] = tets[4 * (int64_t)p->nt_list[e] + a];
        qsort(tmp, k, sizeof(int32_t), cmp_i32);
        int64_t u = 0;
        for (int64_t e = 0; e < k; ++e)
            if (u == 0 || tmp[e] != tmp[u - 1]) tmp[u++] = tmp[e];
        nbr[v] = tmp;
        p->deg[v] = u;
        total_blocks += u;
    }
    if (9 * total_blocks > INT32_MAX) {
        for (int64_t v = 0; v < n; ++v) free(nbr[v]);
        free(nbr);
        orc_pattern_free(p);
        return NULL;
    }
    p->nnz = 9 * total_blocks;
    p->row_ptr = malloc(sizeof(int32_t) * (3 * n + 1));
    p->col = malloc(sizeof(int32_t) * (p->nnz > 0 ? p->nnz : 1));
    int64_t k = 0;
    p->row_ptr[0] = 0;
    for (int64_t v = 0; v < n; ++v)
        for (int i = 0; i < 3; ++i) {
            for (int64_t e = 0; e < p->deg[v]; ++e)
                for (int j = 0; j < 3; ++j) p->col[k++] = 3 * nbr[v][e] + j;
            p->row_ptr[3 * v + i + 1] = (int32_t)k;
        }
    /* scatter map: position of v_b in the sorted neighbour list of v_a, by linear scan */
    p->scat = malloc(sizeof(int32_t) * (144 * T > 0 ? 144 * T : 1));
    for (int64_t t = 0; t < T; ++t) {
        const int32_t *tv = tets + 4 * t;
        for (int a = 0; a < 4; ++a)
            for (int b = 0; b < 4; ++b) {
                int64_t pos = -1;
                for (int64_t e = 0; e < p->deg[tv[a]]; ++e)
                    if (nbr[tv[a]][e] == tv[b]) { pos = e; break; }
                for (int i = 0; i < 3; ++i)
                    for (int j = 0; j < 3; ++j)
                        p->scat[144 * t + 12 * (3 * a + i) + 3 * b + j] =
                            p->row_ptr[3 * tv[a] + i] + (int32_t)(3 * pos + j);
            }
    }
    /* node-level pattern (the proxy operator's): the neighbour sets themselves */
    p->nptr = malloc(sizeof(int64_t) * (n + 1));
    p->ncol = malloc(sizeof(int32_t) * (total_blocks > 0 ? total_blocks : 1));
    p->nptr[0] = 0;
    for (int64_t v = 0; v < n; ++v) {
        for (int64_t e = 0; e < p->deg[v]; ++e) p->ncol[p->nptr[v] + e] = nbr[v][e];
        p->nptr[v + 1] = p->nptr[v] + p->deg[v];
    }
    for (int64_t v = 0; v < n; ++v) free(nbr[v]);
    free(nbr);
    return p;
}

int64_t orc_pattern_nnz(const orc_pattern_t *p) { return p->nnz; }
int64_t orc_pattern_nrows(const orc_pattern_t *p) { return p->nrows; }
void orc_pattern_copy(const orc_pattern_t *p, int32_t *row_ptr, int32_t *col, int32_t *scat)
{
    if (row_ptr) memcpy(row_ptr, p->row_ptr, sizeof(int32_t) * (p->nrows + 1));
    if (col) memcpy(col, p->col, sizeof(int32_t) * p->nnz);
    if (scat) memcpy(scat, p->scat, sizeof(int32_t) * 144 * p->T);
}

/* ------------------------------------------------------------------------------------- */
/* full_rebuild (Sec. 3.5; Eq. 8)                                                           */
/* ------------------------------------------------------------------------------------- */

/* val := sum over active tau, in ascending tau, of P^T K^(tau) P, then + eps on the
 * diagonal.  Ke is T x 144 (orc_element_all).  Written as the scatter-add of Eq. 8 in
 * ascending tetrahedron order, which is exactly the per-entry ascending fold from +0.0. */
void orc_rebuild(const orc_pattern_t *p, const double *Ke, const uint8_t *mask, double eps,
                 double *val)
{
    for (int64_t k = 0; k < p->nnz; ++k) val[k] = 0.0;
    for (int64_t t = 0; t < p->T; ++t) {
        if (!mask[t]) continue;
        for (int pq = 0; pq < 144; ++pq) val[p->scat[144 * t + pq]] += Ke[144 * t + pq];
    }
    if (eps != 0.0)
        for (int64_t r = 0; r < p->nrows; ++r)
            for (int64_t k = p->row_ptr[r]; k < p->row_ptr[r + 1]; ++k)
                if (p->col[k] == r) val[k] += eps;
}

/* Value of one CSR entry (row r, column c) from scratch: the fold over the active
 * tetrahedra containing both nodes r/3 and c/3, in ascending id (the rescan of
 * local_recompute, Sec. 3.5), plus eps when r == c.  Ke of each contributor is computed
 * on the spot from the inputs. */
double orc_entry(const orc_pattern_t *p, const double *X, const double *E, const double *nu,
                 const uint8_t *mask, double eps, int64_t r, int64_t c)
{
    int64_t va = r / 3, vb = c / 3;
    int i = (int)(r % 3), j = (int)(c % 3);
    double acc = 0.0;
    for (int64_t e = p->nt_ptr[va]; e < p->nt_ptr[va + 1]; ++e) {
        int64_t t = p->nt_list[e];
        if (!mask[t]) continue;
        const int32_t *tv = p->tets + 4 * t;
        int la = -1, lb = -1;
        for (int a = 0; a < 4; ++a) {
            if (tv[a] == va) la = a;
            if (tv[a] == vb) lb = a;
        }
        if (lb < 0) continue;
        double x[12], K[144];
        gather_x(X, tv, x);
        orc_element(x, E[t], nu[t], K);
        acc += K[12 * (3 * la + i) + 3 * lb + j];
    }
    if (r == c) acc += eps;
    return acc;
}

/* ------------------------------------------------------------------------------------- */
/* Edits and the two exact local policies of Sec. 3.5                                      */
/* ------------------------------------------------------------------------------------- */

/* An edit: op 0 = deactivate tet, 1 = activate tet, 2 = swap (deactivate tet, activate
 * tet2).  Sets Delta^- and Delta^+ of Sec. 3.2. */
typedef struct { int32_t op, tet, tet2; } orc_edit;

/* Checks an edit list against the current mask without changing anything.  Returns 0 or
 * the 1-based index of the first bad edit (bad op, id out of range, deactivating an
 * inactive or activating an active tetrahedron, a tetrahedron named twice). */
int64_t orc_validate_edits(int64_t T, const uint8_t *mask, const orc_edit *ed, int64_t n)
{
    uint8_t *seen = calloc(T > 0 ? T : 1, 1);
    int64_t bad = 0;
    for (int64_t e = 0; e < n && !bad; ++e) {
        int32_t op = ed[e].op, t = ed[e].tet, t2 = ed[e].tet2;
        if (op < 0 || op > 2 || t < 0 || t >= T) { bad = e + 1; break; }
        if (seen[t]) { bad = e + 1; break; }
        seen[t] = 1;
        if (op == 0 && !mask[t]) bad = e + 1;
        if (op == 1 && mask[t]) bad = e + 1;
        if (op == 2) {
            if (t2 < 0 || t2 >= T || seen[t2] || !mask[t] || mask[t2]) { bad = e + 1; break; }
            seen[t2] = 1;
        }
    }
    free(seen);
    return bad;
}

/* local_recompute (Sec. 3.5, Algorithm 1 receive/update steps): apply the edits to the
 * mask, collect every entry touched by an edited tetrahedron (its 144 scatter slots), and
 * recompute each touched entry from scratch with orc_entry's fold over the current active
 * set.  Ke (T x 144) replaces the on-the-spot element evaluation of orc_entry; values are
 * identical.  Returns the number of distinct touched entries, or -(1 + bad index) when the
 * edit list is invalid (nothing is changed then). */
int64_t orc_local_recompute(const orc_pattern_t *p, const double *Ke, uint8_t *mask,
                            const orc_edit *ed, int64_t n, double eps, double *val)
{
    int64_t bad = orc_validate_edits(p->T, mask, ed, n);
    if (bad) return -(bad + 1);
    for (int64_t e = 0; e < n; ++e) {
        if (ed[e].op == 0) mask[ed[e].tet] = 0;
        if (ed[e].op == 1) mask[ed[e].tet] = 1;
        if (ed[e].op == 2) { mask[ed[e].tet] = 0; mask[ed[e].tet2] = 1; }
    }
    uint8_t *touched = calloc(p->nnz > 0 ? p->nnz : 1, 1);
    int32_t *list = malloc(sizeof(int32_t) * (288 * n > 0 ? 288 * n : 1));
    int64_t count = 0;
    for (int64_t e = 0; e < n; ++e) {
        int32_t ts[2] = {ed[e].tet, ed[e].op == 2 ? ed[e].tet2 : -1};
        for (int s = 0; s < 2; ++s) {
            if (ts[s] < 0) continue;
            for (int pq = 0; pq < 144; ++pq) {
                int32_t k = p->scat[144 * (int64_t)ts[s] + pq];
                if (!touched[k]) { touched[k] = 1; list[count++] = k; }
            }
        }
    }
    /* recompute each touched entry: its row by binary search in row_ptr, contributors by
     * rescanning the tetrahedra incident to the row's node */
    for (int64_t e = 0; e < count; ++e) {
        int64_t k = list[e], lo = 0, hi = p->nrows; /* largest r with row_ptr[r] <= k */
        while (hi - lo > 1) {
            int64_t mid = (lo + hi) / 2;
            if (p->row_ptr[mid] <= k) lo = mid; else hi = mid;
        }
        int64_t r = lo, c = p->col[k], va = r / 3, vb = c / 3;
        int i = (int)(r % 3), j = (int)(c % 3);
        double acc = 0.0;
        for (int64_t q = p->nt_ptr[va]; q < p->nt_ptr[va + 1]; ++q) {
            int64_t t = p->nt_list[q];
            if (!mask[t]) continue;
            const int32_t *tv = p->tets + 4 * t;
            int la = -1, lb = -1;
            for (int a = 0; a < 4; ++a) {
                if (tv[a] == va) la = a;
                if (tv[a] == vb) lb = a;
            }
            if (lb < 0) continue;
            acc += Ke[144 * t + 12 * (3 * la + i) + 3 * lb + j];
        }
        if (r == c) acc += eps;
        val[k] = acc;
        touched[k] = 0;
    }
    free(touched);
    free(list);
    return count;
}

/* streaming_update as the paper states it (Sec. 3.4, Sec. 3.5): persistent values, each
 * edited tetrahedron adds (activation) or subtracts (deactivation) its element matrix at
 * its scatter slots, edits taken in list order, a swap as its deactivation then its
 * activation.  O(|Delta|).  Not bit-identical to a rebuild in FP64 (it is exact only up to
 * rounding); kept as the record of that.  Same return convention as orc_local_recompute. */
int64_t orc_additive_update(const orc_pattern_t *p, const double *Ke, uint8_t *mask,
                            const orc_edit *ed, int64_t n, double *val)
{
    int64_t bad = orc_validate_edits(p->T, mask, ed, n);
    if (bad) return -(bad + 1);
    for (int64_t e = 0; e < n; ++e) {
        int32_t off = -1, on = -1;
        if (ed[e].op == 0) off = ed[e].tet;
        if (ed[e].op == 1) on = ed[e].tet;
        if (ed[e].op == 2) { off = ed[e].tet; on = ed[e].tet2; }
        if (off >= 0) {
            mask[off] = 0;
            for (int pq = 0; pq < 144; ++pq)
                val[p->scat[144 * (int64_t)off + pq]] -= Ke[144 * (int64_t)off + pq];
        }
        if (on >= 0) {
            mask[on] = 1;
            for (int pq = 0; pq < 144; ++pq)
                val[p->scat[144 * (int64_t)on + pq]] += Ke[144 * (int64_t)on + pq];
        }
    }
    return 0;
}

/* ------------------------------------------------------------------------------------- */
/* Exact additive streaming in fixed point                                                  */
/* ------------------------------------------------------------------------------------- */

/*
 * The paper's streaming_update (Sec. 3.4, Sec. 3.5: add or subtract the edited tetrahedra's
 * element contributions, O(|Delta|)) is exact only up to rounding in floating point.  Reading
 * that makes it exact: every CSR entry k gets a fixed binary exponent e_k from its superset
 * contributions; every contribution c to k is quantised once, q = c * 2^-e_k rounded to the
 * nearest integer (ties to even); the entry keeps the exact integer sum S_k over its active
 * contributors and its value is that sum converted once, val_k = double(S_k) * 2^e_k, plus
 * eps on the diagonal.  Integer addition is associative, so adding and subtracting q in any
 * order gives the S_k of a rebuild.
 *   E(x)   unbiased exponent field of x (floor(log2|x|) for normal x; -1023 for 0 / subnormal)
 *   m_k    maximum of E over the entry's superset contributions
 *   L_k    ceil(log2(kappa_k)), kappa_k = number of superset contributions to k
 *   e_k    m_k + 1 + L_k - 62, limited to [-1022, 1023]; 0 when every contribution is 0
 * so |q| < 2^(62 - L_k), |S_k| < 2^62, and |val_k - sum of active c| <= kappa_k 2^(e_k - 1)
 * plus the rounding of the final conversion.
 */
static int exp_field(double x)
{
    uint64_t u;
    memcpy(&u, &x, sizeof u);
    return (int)((u >> 52) & 0x7ff) - 1023;
}

void orc_fx_exponents(const orc_pattern_t *p, const double *Ke, int32_t *e)
{
    int32_t *mk = malloc(sizeof(int32_t) * (p->nnz > 0 ? p->nnz : 1));
    int64_t *kap = calloc(p->nnz > 0 ? p->nnz : 1, sizeof(int64_t));
    for (int64_t k = 0; k < p->nnz; ++k) mk[k] = -1023;
    for (int64_t t = 0; t < p->T; ++t)
        for (int pq = 0; pq < 144; ++pq) {
            int64_t k = p->scat[144 * t + pq];
            int ex = exp_field(Ke[144 * t + pq]);
            if (ex > mk[k]) mk[k] = ex;
            kap[k] += 1;
        }
    for (int64_t k = 0; k < p->nnz; ++k) {
        if (mk[k] == -1023) {
            e[k] = 0;
            continue;
        }
        int L = 0;
        while (((int64_t)1 << L) < kap[k]) ++L;
        int ek = mk[k] + 1 + L - 62;
        e[k] = ek < -1022 ? -1022 : (ek > 1023 ? 1023 : ek);
    }
    free(mk);
    free(kap);
}

static int64_t fx_quant(double c, int32_t e) { return llrint(ldexp(c, -e)); }

static double fx_value(int64_t S, int32_t e) { return ldexp((double)S, e); }

/* S and val from scratch over the active set (plus eps on the diagonal). */
void orc_fx_rebuild(const orc_pattern_t *p, const double *Ke, const int32_t *e,
                    const uint8_t *mask, double eps, int64_t *S, double *val)
{
    for (int64_t k = 0; k < p->nnz; ++k) S[k] = 0;
    for (int64_t t = 0; t < p->T; ++t) {
        if (!mask[t]) continue;
        for (int pq = 0; pq < 144; ++pq) {
            int64_t k = p->scat[144 * t + pq];
            S[k] += fx_quant(Ke[144 * t + pq], e[k]);
        }
    }
    for (int64_t r = 0; r < p->nrows; ++r)
        for (int64_t k = p->row_ptr[r]; k < p->row_ptr[r + 1]; ++k) {
            val[k] = fx_value(S[k], e[k]);
            if (eps != 0.0 && p->col[k] == r) val[k] += eps;
        }
}

/* One frame of the additive update on S (O(|Delta|)): each edited tetrahedron subtracts
 * (deactivation) or adds (activation) its quantised contributions, edits in list order, a
 * swap as its deactivation then its activation; then the values of its entries are
 * converted again.  Same return convention as orc_local_recompute. */
int64_t orc_fx_update(const orc_pattern_t *p, const double *Ke, const int32_t *e, uint8_t *mask,
                      const orc_edit *ed, int64_t n, double eps, int64_t *S, double *val)
{
    int64_t bad = orc_validate_edits(p->T, mask, ed, n);
    if (bad) return -(bad + 1);
    for (int64_t i = 0; i < n; ++i) {
        int32_t off = -1, on = -1;
        if (ed[i].op == 0) off = ed[i].tet;
        if (ed[i].op == 1) on = ed[i].tet;
        if (ed[i].op == 2) { off = ed[i].tet; on = ed[i].tet2; }
        for (int side = 0; side < 2; ++side) {
            int32_t t = side == 0 ? off : on;
            if (t < 0) continue;
            mask[t] = side == 0 ? 0 : 1;
            for (int pq = 0; pq < 144; ++pq) {
                int64_t k = p->scat[144 * (int64_t)t + pq];
                int64_t q = fx_quant(Ke[144 * (int64_t)t + pq], e[k]);
                S[k] += side == 0 ? -q : q;
            }
        }
    }
    for (int64_t i = 0; i < n; ++i)
        for (int side = 0; side < 2; ++side) {
            int32_t t = side == 0 ? ed[i].tet : (ed[i].op == 2 ? ed[i].tet2 : -1);
            if (t < 0) continue;
            for (int pq = 0; pq < 144; ++pq) {  /* a local diagonal entry is a global one */
                int64_t k = p->scat[144 * (int64_t)t + pq];
                val[k] = fx_value(S[k], e[k]);
                if (eps != 0.0 && pq / 12 == pq % 12) val[k] += eps;
            }
        }
    return 0;
}

/* ------------------------------------------------------------------------------------- */
/* Graph-Laplacian proxy operator (Sec. 3.1 Eqs. 1-4; Sec. 3.2 Eqs. 5-7; Sec. 3.3;          */
/* Algorithm 1)                                                                             */
/* ------------------------------------------------------------------------------------- */

/*
 * A scalar n x n operator on the node-level superset pattern: row u holds the sorted
 * neighbour set of u, u included (the node pairs whose 3x3 blocks make the elasticity CSR).
 *   c_t(u, v) = number of active tetrahedra having {u, v} among their six edges   (Eq. 1)
 *   a_t(u, v) = 1[c_t(u, v) > 0]                                                  (Eq. 2)
 *   A_t(u, v) = -a_t(u, v) for u != v,  A_t(u, u) = sum_{w != u} a_t(u, w) + eps  (Eqs. 3, 4)
 * Readings: a superset edge that is not active keeps its slot and holds +0.0 (the paper
 * inserts and removes entries; a fixed slot holding +0.0 is the same matrix); an active one
 * holds -1.0; the diagonal is (double) degree + eps, one IEEE addition; a node of no
 * superset tetrahedron has an empty row (no eps entry), as in the elasticity pattern.  c_t is kept at
 * both entries (u, v) and (v, u) of an edge, the degree per node.
 */
int64_t orc_proxy_nnz(const orc_pattern_t *p) { return p->nptr[p->n]; }

void orc_proxy_pattern(const orc_pattern_t *p, int32_t *row_ptr, int32_t *col)
{
    for (int64_t v = 0; v <= p->n; ++v) row_ptr[v] = (int32_t)p->nptr[v];
    memcpy(col, p->ncol, sizeof(int32_t) * p->nptr[p->n]);
}

/* node-level entry (u, v), by a linear scan of u's neighbour set; -1 if absent */
static int64_t proxy_pos(const orc_pattern_t *p, int32_t u, int32_t v)
{
    for (int64_t k = p->nptr[u]; k < p->nptr[u + 1]; ++k)
        if (p->ncol[k] == v) return k;
    return -1;
}

/* full_rebuild of the proxy (Sec. 3.5): Eq. 1 by counting over the active tetrahedra, then
 * Eqs. 2-4 entry by entry. */
void orc_proxy_rebuild(const orc_pattern_t *p, const uint8_t *mask, double eps, int32_t *mult,
                       int32_t *deg, double *val)
{
    const int64_t nb = p->nptr[p->n];
    for (int64_t k = 0; k < nb; ++k) mult[k] = 0;
    for (int64_t t = 0; t < p->T; ++t) {
        if (!mask[t]) continue;
        const int32_t *tv = p->tets + 4 * t;
        for (int a = 0; a < 4; ++a)
            for (int b = a + 1; b < 4; ++b) {
                mult[proxy_pos(p, tv[a], tv[b])] += 1;
                mult[proxy_pos(p, tv[b], tv[a])] += 1;
            }
    }
    for (int64_t u = 0; u < p->n; ++u) {
        deg[u] = 0;
        for (int64_t k = p->nptr[u]; k < p->nptr[u + 1]; ++k) {
            if (p->ncol[k] == u) continue;
            int a = mult[k] > 0;
            val[k] = a ? -1.0 : 0.0;
            deg[u] += a;
        }
        int64_t kd = proxy_pos(p, (int32_t)u, (int32_t)u);
        if (kd >= 0) val[kd] = (double)deg[u] + eps;  /* a node of no tetrahedron has no row */
    }
}

/* streaming_update of the proxy (Sec. 3.2, Algorithm 1): the edits in list order (a swap as
 * its deactivation then its activation), each edited tetrahedron adding +-1 to the
 * multiplicity of its six edges (Eqs. 5-7); where a multiplicity moves between 0 and > 0,
 * the edge's two off-diagonal entries are set (inserted: -1.0) or cleared (removed: +0.0)
 * and the degrees of both end nodes and their diagonal entries follow.  mask, mult, deg and
 * val are updated in place.  Returns the number of distinct entries the update visits (the
 * two entries of each edge of an edited tetrahedron and the diagonal entry of each of their
 * nodes), or -(1 + bad index) for an invalid edit list (nothing is changed then). */
int64_t orc_proxy_update(const orc_pattern_t *p, uint8_t *mask, const orc_edit *ed, int64_t n,
                         double eps, int32_t *mult, int32_t *deg, double *val)
{
    int64_t bad = orc_validate_edits(p->T, mask, ed, n);
    if (bad) return -(bad + 1);
    const int64_t nb = p->nptr[p->n];
    uint8_t *seen = calloc(nb > 0 ? nb : 1, 1);
    int64_t visited = 0;
    for (int64_t i = 0; i < n; ++i) {
        int32_t off = -1, on = -1;
        if (ed[i].op == 0) off = ed[i].tet;
        if (ed[i].op == 1) on = ed[i].tet;
        if (ed[i].op == 2) { off = ed[i].tet; on = ed[i].tet2; }
        for (int side = 0; side < 2; ++side) {
            int32_t t = side == 0 ? off : on;
            if (t < 0) continue;
            int32_t step = side == 0 ? -1 : 1;
            mask[t] = side == 0 ? 0 : 1;
            const int32_t *tv = p->tets + 4 * (int64_t)t;
            for (int a = 0; a < 4; ++a) {
                int64_t kd = proxy_pos(p, tv[a], tv[a]);
                if (!seen[kd]) { seen[kd] = 1; ++visited; }
            }
            for (int a = 0; a < 4; ++a)
                for (int b = a + 1; b < 4; ++b) {
                    int32_t u = tv[a], v = tv[b];
                    int64_t kuv = proxy_pos(p, u, v), kvu = proxy_pos(p, v, u);
                    if (!seen[kuv]) { seen[kuv] = 1; ++visited; }
                    if (!seen[kvu]) { seen[kvu] = 1; ++visited; }
                    int32_t before = mult[kuv], after = before + step;
                    mult[kuv] = after;
                    mult[kvu] = after;
                    if ((before == 0) != (after == 0)) {
                        int32_t d = after > 0 ? 1 : -1;
                        val[kuv] = after > 0 ? -1.0 : 0.0;
                        val[kvu] = val[kuv];
                        deg[u] += d;
                        deg[v] += d;
                        val[proxy_pos(p, u, u)] = (double)deg[u] + eps;
                        val[proxy_pos(p, v, v)] = (double)deg[v] + eps;
                    }
                }
        }
    }
    free(seen);
    return visited;
}

/* ------------------------------------------------------------------------------------- */
/* Lumped mass of the implicit-Euler loop (Sec. 6.2, Eq. 9)                                 */
/* ------------------------------------------------------------------------------------- */

/*
 * M_t of Eq. 9, the "maintained lumped mass matrix" (the paper gives no formula).  Reading:
 * row-sum lumping of the consistent P1 mass, so every active tetrahedron gives a quarter of
 * its mass to each of its four nodes, for each of the node's three DOFs:
 *     m_v = sum over active tau containing v, in ascending tau, of (rho * V_tau) * 0.25,
 * folded from +0.0 (the summation-order reading of the stiffness); V_tau = det / 6 with det
 * evaluated as in orc_element (d_k = x_k - x_0, c_1 = d_2 x d_3 with the fma order there,
 * det = fma(d_1.z, c_1.z, fma(d_1.y, c_1.y, d_1.x c_1.x))).  A node of no active tetrahedron
 * has mass +0.0.
 */
static double tet_volume(const double *X, const int32_t *tv)
{
    double d[3][3];
    for (int k = 1; k <= 3; ++k)
        for (int m = 0; m < 3; ++m) d[k - 1][m] = X[3 * (int64_t)tv[k] + m] - X[3 * (int64_t)tv[0] + m];
    double c0 = fma(d[1][1], d[2][2], -(d[1][2] * d[2][1]));
    double c1 = fma(d[1][2], d[2][0], -(d[1][0] * d[2][2]));
    double c2 = fma(d[1][0], d[2][1], -(d[1][1] * d[2][0]));
    double det = fma(d[0][2], c2, fma(d[0][1], c1, d[0][0] * c0));
    return det / 6.0;
}

void orc_lumped_mass(const orc_pattern_t *p, const double *X, double rho, const uint8_t *mask,
                     double *mass)
{
    for (int64_t v = 0; v < p->n; ++v) {
        double m = 0.0;
        for (int64_t q = p->nt_ptr[v]; q < p->nt_ptr[v + 1]; ++q) {
            int64_t t = p->nt_list[q];
            if (!mask[t]) continue;
            m += (rho * tet_volume(X, p->tets + 4 * t)) * 0.25;
        }
        mass[v] = m;
    }
}

/* ------------------------------------------------------------------------------------- */
/* Gradient reference (adjoint form)                                                        */
/* ------------------------------------------------------------------------------------- */

/*
 * dL/dE and dL/dnu of one element for a given upstream G = dL/dK^(tau) (12x12):
 *   K = V (lam A + mu B),  A[ai][bj] = g_ai g_bj,  B[ai][bj] = g_aj g_bi + delta_ij g_a.g_b,
 *   dlam/dE = nu/((1+nu)(1-2nu)),  dmu/dE = 1/(2(1+nu)),
 *   dlam/dnu = E(1+2nu^2)/((1+nu)^2 (1-2nu)^2),  dmu/dnu = -E/(2(1+nu)^2).
 * A and B are formed here from g directly (no shared code with orc_element).
 */
int orc_element_param_grad(const double x[12], double E, double nu, const double G[144],
                           double *dE, double *dnu)
{
    double Dm[3][3];
    for (int m = 0; m < 3; ++m)
        for (int k = 0; k < 3; ++k) Dm[m][k] = x[3 * (k + 1) + m] - x[m];
    double det = Dm[0][0] * (Dm[1][1] * Dm[2][2] - Dm[1][2] * Dm[2][1]) -
                 Dm[0][1] * (Dm[1][0] * Dm[2][2] - Dm[1][2] * Dm[2][0]) +
                 Dm[0][2] * (Dm[1][0] * Dm[2][1] - Dm[1][1] * Dm[2][0]);
    if (!(det > 0.0)) return -1;
    double g[4][3];
    for (int r = 0; r < 3; ++r)
        for (int cidx = 0; cidx < 3; ++cidx) {
            int r1 = (cidx + 1) % 3, r2 = (cidx + 2) % 3, c1 = (r + 1) % 3, c2 = (r + 2) % 3;
            g[r + 1][cidx] = (Dm[r1][c1] * Dm[r2][c2] - Dm[r1][c2] * Dm[r2][c1]) / det;
        }
    for (int m = 0; m < 3; ++m) g[0][m] = -(g[1][m] + g[2][m] + g[3][m]);
    double V = det / 6.0, sa = 0.0, sb = 0.0;
    for (int a = 0; a < 4; ++a)
        for (int i = 0; i < 3; ++i)
            for (int b = 0; b < 4; ++b)
                for (int j = 0; j < 3; ++j) {
                    double A = g[a][i] * g[b][j];
                    double Bv = g[a][j] * g[b][i];
                    if (i == j) Bv += g[a][0] * g[b][0] + g[a][1] * g[b][1] + g[a][2] * g[b][2];
                    double w = G[12 * (3 * a + i) + 3 * b + j];
                    sa += w * A;
                    sb += w * Bv;
                }
    double onu = 1.0 + nu, omn = 1.0 - 2.0 * nu;
    *dE = V * (sa * nu / (onu * omn) + sb / (2.0 * onu));
    *dnu = V * (sa * E * (1.0 + 2.0 * nu * nu) / (onu * onu * omn * omn) - sb * E / (2.0 * onu * onu));
    return 0;
}

/* The element formula again, in complex arithmetic, for complex-step differentiation with
 * respect to node positions: dK/dx_m = Im K(x + i h e_m) / h, free of subtractive error. */
static int element_cplx(const double complex x[12], double E, double nu, double complex K[144])
{
    double complex d[3][3], c[3][3], g[4][3];
    for (int k = 1; k <= 3; ++k)
        for (int m = 0; m < 3; ++m) d[k - 1][m] = x[3 * k + m] - x[m];
    const int cu[3] = {1, 2, 0}, cv[3] = {2, 0, 1};
    for (int k = 0; k < 3; ++k) {
        const double complex *u = d[cu[k]], *v = d[cv[k]];
        c[k][0] = u[1] * v[2] - u[2] * v[1];
        c[k][1] = u[2] * v[0] - u[0] * v[2];
        c[k][2] = u[0] * v[1] - u[1] * v[0];
    }
    double complex det = d[0][0] * c[0][0] + d[0][1] * c[0][1] + d[0][2] * c[0][2];
    if (!(creal(det) > 0.0)) return -1;
    for (int k = 0; k < 3; ++k)
        for (int m = 0; m < 3; ++m) g[k + 1][m] = c[k][m] / det;
    for (int m = 0; m < 3; ++m) g[0][m] = -(g[1][m] + g[2][m] + g[3][m]);
    double complex V = det / 6.0;
    double lam = E * nu / ((1.0 + nu) * (1.0 - 2.0 * nu)), mu = E / (2.0 * (1.0 + nu));
    for (int a = 0; a < 4; ++a)
        for (int i = 0; i < 3; ++i)
            for (int b = 0; b < 4; ++b)
                for (int j = 0; j < 3; ++j) {
                    double complex v = lam * g[a][i] * g[b][j] + mu * g[a][j] * g[b][i];
                    if (i == j) v += mu * (g[a][0] * g[b][0] + g[a][1] * g[b][1] + g[a][2] * g[b][2]);
                    K[12 * (3 * a + i) + 3 * b + j] = V * v;
                }
    return 0;
}

/* dL/dx of one element's 12 node coordinates for upstream G = dL/dK^(tau), by complex
 * step with h = 1e-30. */
int orc_element_x_grad_cs(const double x[12], double E, double nu, const double G[144],
                          double dx[12])
{
    const double h = 1e-30;
    double complex xc[12], K[144];
    for (int m = 0; m < 12; ++m) {
        for (int q = 0; q < 12; ++q) xc[q] = x[q];
        xc[m] += h * I;
        if (element_cplx(xc, E, nu, K) != 0) return -1;
        double s = 0.0;
        for (int pq = 0; pq < 144; ++pq) s += G[pq] * (cimag(K[pq]) / h);
        dx[m] = s;
    }
    return 0;
}

/* Per-element reference gradients for a whole mesh.  G is given per CSR entry
 * (grad_val, nnz) and gathered through the scatter map: G^(tau)[pq] = grad_val[scat[tau][pq]].
 * Inactive tetrahedra get zero gradients.  dX (n x 3) accumulates over elements. */
int orc_grad_all(const orc_pattern_t *p, const double *X, const double *E, const double *nu,
                 const uint8_t *mask, const double *grad_val, double *dE, double *dnu,
                 double *dX)
{
    for (int64_t v = 0; v < 3 * p->n; ++v) dX[v] = 0.0;
    for (int64_t t = 0; t < p->T; ++t) {
        dE[t] = 0.0;
        dnu[t] = 0.0;
        if (!mask[t]) continue;
        double x[12], G[144], dx[12];
        gather_x(X, p->tets + 4 * t, x);
        for (int pq = 0; pq < 144; ++pq) G[pq] = grad_val[p->scat[144 * t + pq]];
        if (orc_element_param_grad(x, E[t], nu[t], G, &dE[t], &dnu[t]) != 0) return -1;
        if (orc_element_x_grad_cs(x, E[t], nu[t], G, dx) != 0) return -1;
        for (int a = 0; a < 4; ++a)
            for (int m = 0; m < 3; ++m) dX[3 * (int64_t)p->tets[4 * t + a] + m] += dx[3 * a + m];
    }
    return 0;
}
