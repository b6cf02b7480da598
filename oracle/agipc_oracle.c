/*
 * CPU FP64 oracle of the in-solve algebraic coarsening step (AGIPC, Sec. 4.1
 * and Sec. 4.3 of the paper; supplement Sec. 1 and Sec. 2).
 *
 * TEST INFRASTRUCTURE.  This file is the plain, slow, obviously-correct
 * statement of what the GPU path computes.  Only the test suite, the smoke
 * check in __graft_entry__ and the CPU-baseline leg of bench.py may build,
 * load or call it.  It shares no code, header, table or helper with the CUDA
 * library: every routine below is written from the paper's definitions.
 *
 * Conventions shared with the inputs (not with the GPU code):
 *   - 3x3 blocks are 9 doubles, row-major.
 *   - The fine Hessian arrives as an upper-triangular BSR matrix (column >=
 *     row; Sec. 5.2 keeps only the diagonal and upper triangle of the
 *     symmetric Hessians) plus barrier stencils of 4 vertices with 10 packed upper
 *     blocks in the local order (0,0),(0,1),(0,2),(0,3),(1,1),(1,2),(1,3),
 *     (2,2),(2,3),(3,3).
 *   - Return values: 0 = ok, negative = invalid input (-1), singular block
 *     (-2), capacity too small (-3), not converged (-5).
 *
 * Parity pins for every function live in tests/test_oracle_pins.py.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------ */
/* Aggregation: fine -> coarse labels                                        */
/* ------------------------------------------------------------------------ */

static int32_t uf_find(int32_t *parent, int32_t v)
{
    int32_t root = v;
    while (parent[root] != root) root = parent[root];
    while (parent[v] != root) { /* path compression */
        int32_t next = parent[v];
        parent[v] = root;
        v = next;
    }
    return root;
}

/*
 * Sec. 4.1: fine nodes are coalesced into super-nodes only across paths of
 * edges whose tag is 1; the supplement (Sec. 1) shows the limit of the
 * hierarchical hashing is one node per connected body when every tag is 1.
 * The exact result is therefore the connected components of the graph
 * (V, {e : tau_e = 1}).  Coarse indices follow the supplement's ordering:
 * inside a group, a node's coarse index is the position of the first set
 * bit of its hash (its component's smallest member) and groups are offset
 * by a prefix sum in index order, which is the rank of each component's
 * minimum fine index.  labels[f] = that rank; returns n_c, or -1.
 */
int32_t oracle_labels(int32_t n, int64_t n_edges, const int32_t *edges, const uint8_t *tags,
                      int32_t *labels)
{
    if (n < 0 || n_edges < 0) return -1;
    int32_t *parent = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    int32_t *root_label = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    if (!parent || !root_label) { free(parent); free(root_label); return -1; }
    for (int32_t v = 0; v < n; ++v) { parent[v] = v; root_label[v] = -1; }
    for (int64_t e = 0; e < n_edges; ++e) {
        int32_t u = edges[2 * e], v = edges[2 * e + 1];
        if (u < 0 || v < 0 || u >= n || v >= n) { free(parent); free(root_label); return -1; }
        if (!tags[e] || u == v) continue;
        int32_t ru = uf_find(parent, u), rv = uf_find(parent, v);
        if (ru != rv) parent[ru > rv ? ru : rv] = ru < rv ? ru : rv;
    }
    int32_t next = 0;
    for (int32_t f = 0; f < n; ++f) {
        int32_t r = uf_find(parent, f);
        if (root_label[r] < 0) root_label[r] = next++;
        labels[f] = root_label[r];
    }
    free(parent);
    free(root_label);
    return next;
}

/* ------------------------------------------------------------------------ */
/* Coarse gradient                                                           */
/* ------------------------------------------------------------------------ */

/* Sec. 4.1: g_c = sum over children f of c of g_f  (g_c = U g). */
int oracle_coarse_gradient(int32_t n, int32_t n_c, const int32_t *labels, const double *g, double *g_c)
{
    for (int64_t k = 0; k < 3 * (int64_t)n_c; ++k) g_c[k] = 0.0;
    for (int32_t f = 0; f < n; ++f) {
        int32_t c = labels[f];
        if (c < 0 || c >= n_c) return -1;
        for (int k = 0; k < 3; ++k) g_c[3 * c + k] += g[3 * f + k];
    }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Full fine Hessian from upper storage + stencils                           */
/* ------------------------------------------------------------------------ */

static const int STENCIL_S[10] = {0, 0, 0, 0, 1, 1, 1, 2, 2, 3};
static const int STENCIL_T[10] = {0, 1, 2, 3, 1, 2, 3, 2, 3, 3};

typedef struct {
    int32_t n;
    int64_t *row_start; /* [n+1] */
    int32_t *col;       /* [nnz], duplicates allowed */
    double *val;        /* [nnz][9] */
} full_rows;

static void put_block(full_rows *H, int64_t *cursor, int32_t r, int32_t c, const double *B, int transpose)
{
    int64_t k = cursor[r]++;
    H->col[k] = c;
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) H->val[9 * k + 3 * a + b] = transpose ? B[3 * b + a] : B[3 * a + b];
}

/*
 * The symmetric fine Hessian H in full storage, as per-row lists of
 * (column, 3x3 block) with repeated columns left unsummed.  An upper block
 * B at (i, j), i != j, stands for B at (i, j) and B^T at (j, i); a stencil
 * block B_st (s < t) on vertices (v_s, v_t) stands for B_st at (v_s, v_t)
 * and B_st^T at (v_t, v_s).  Contact Hessians join the fine system before
 * coarsening (Sec. 4.3).
 */
static int build_full(int32_t n, const int32_t *rp, const int32_t *ci, const double *val,
                      int64_t n_pairs, const int32_t *pidx, const double *pblk, full_rows *H)
{
    int64_t *cnt = (int64_t *)calloc((size_t)n + 1, sizeof(int64_t));
    if (!cnt) return -1;
    for (int32_t i = 0; i < n; ++i)
        for (int32_t k = rp[i]; k < rp[i + 1]; ++k) {
            int32_t j = ci[k];
            if (j < 0 || j >= n) { free(cnt); return -1; }
            cnt[i]++;
            if (j != i) cnt[j]++;
        }
    for (int64_t p = 0; p < n_pairs; ++p)
        for (int q = 0; q < 10; ++q) {
            int32_t vs = pidx[4 * p + STENCIL_S[q]], vt = pidx[4 * p + STENCIL_T[q]];
            if (vs < 0 || vs >= n || vt < 0 || vt >= n) { free(cnt); return -1; }
            cnt[vs]++;
            if (STENCIL_S[q] != STENCIL_T[q]) cnt[vt]++;
        }
    H->n = n;
    H->row_start = (int64_t *)malloc(sizeof(int64_t) * ((size_t)n + 1));
    int64_t *cursor = (int64_t *)malloc(sizeof(int64_t) * ((size_t)n + 1));
    H->row_start[0] = 0;
    for (int32_t i = 0; i < n; ++i) H->row_start[i + 1] = H->row_start[i] + cnt[i];
    int64_t nnz = H->row_start[n];
    H->col = (int32_t *)malloc(sizeof(int32_t) * (size_t)(nnz > 0 ? nnz : 1));
    H->val = (double *)malloc(sizeof(double) * 9 * (size_t)(nnz > 0 ? nnz : 1));
    for (int32_t i = 0; i <= n; ++i) cursor[i] = H->row_start[i];
    for (int32_t i = 0; i < n; ++i)
        for (int32_t k = rp[i]; k < rp[i + 1]; ++k) {
            int32_t j = ci[k];
            put_block(H, cursor, i, j, val + 9 * (int64_t)k, 0);
            if (j != i) put_block(H, cursor, j, i, val + 9 * (int64_t)k, 1);
        }
    for (int64_t p = 0; p < n_pairs; ++p)
        for (int q = 0; q < 10; ++q) {
            int s = STENCIL_S[q], t = STENCIL_T[q];
            int32_t vs = pidx[4 * p + s], vt = pidx[4 * p + t];
            const double *B = pblk + 90 * p + 9 * q;
            put_block(H, cursor, vs, vt, B, 0);
            if (s != t) put_block(H, cursor, vt, vs, B, 1);
        }
    free(cnt);
    free(cursor);
    return 0;
}

static void free_full(full_rows *H)
{
    free(H->row_start);
    free(H->col);
    free(H->val);
}

/* Number of (row, column, block) terms of the full fine Hessian before any
 * summation: an upper bound on the number of nonzero blocks of H and of
 * H_c = U H U^T.  Callers use it to size outputs. */
int64_t oracle_full_terms(int32_t n, const int32_t *rp, const int32_t *ci, int64_t n_pairs)
{
    int64_t t = 0;
    for (int32_t i = 0; i < n; ++i)
        for (int32_t k = rp[i]; k < rp[i + 1]; ++k) t += (ci[k] == i) ? 1 : 2;
    return t + 16 * n_pairs;
}

static int cmp_i32(const void *a, const void *b)
{
    int32_t x = *(const int32_t *)a, y = *(const int32_t *)b;
    return (x > y) - (x < y);
}

/*
 * Coarse Hessian H_c = U H U^T (Sec. 4.1), with U the n_c x n aggregation
 * operator (3x3 identity block at (labels[f], f)).  Entry (a, b) of H_c is
 * the sum of every fine block H_ij with labels[i] = a and labels[j] = b,
 * so coarse row a is the sum of the fine rows of a's children with their
 * columns relabelled.  Output: full storage (both triangles), columns sorted
 * ascending within each row.  Returns nnz_c, or a negative status.
 */
int64_t oracle_galerkin(int32_t n, int32_t n_c, const int32_t *labels,
                        const int32_t *rp, const int32_t *ci, const double *val,
                        int64_t n_pairs, const int32_t *pidx, const double *pblk,
                        int32_t *crp, int32_t *cci, double *cval, int64_t cap)
{
    full_rows H;
    if (build_full(n, rp, ci, val, n_pairs, pidx, pblk, &H) != 0) return -1;
    for (int32_t f = 0; f < n; ++f)
        if (labels[f] < 0 || labels[f] >= n_c) { free_full(&H); return -1; }

    /* children of each coarse node, in increasing fine index */
    int64_t *cstart = (int64_t *)calloc((size_t)n_c + 1, sizeof(int64_t));
    int32_t *child = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    for (int32_t f = 0; f < n; ++f) cstart[labels[f] + 1]++;
    for (int32_t c = 0; c < n_c; ++c) cstart[c + 1] += cstart[c];
    int64_t *cfill = (int64_t *)malloc(sizeof(int64_t) * ((size_t)n_c + 1));
    memcpy(cfill, cstart, sizeof(int64_t) * ((size_t)n_c + 1));
    for (int32_t f = 0; f < n; ++f) child[cfill[labels[f]]++] = f;

    /* sparse accumulator over coarse columns */
    int32_t *marker = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n_c > 0 ? n_c : 1));
    double *acc = (double *)malloc(sizeof(double) * 9 * (size_t)(n_c > 0 ? n_c : 1));
    int32_t *cols = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n_c > 0 ? n_c : 1));
    for (int32_t b = 0; b < n_c; ++b) marker[b] = -1;
    int64_t nnz = 0;
    int status = 0;
    crp[0] = 0;
    for (int32_t a = 0; a < n_c && status == 0; ++a) {
        int32_t ncols = 0;
        for (int64_t q = cstart[a]; q < cstart[a + 1]; ++q) {
            int32_t i = child[q];
            for (int64_t k = H.row_start[i]; k < H.row_start[i + 1]; ++k) {
                int32_t b = labels[H.col[k]];
                if (marker[b] != a) {
                    marker[b] = a;
                    cols[ncols++] = b;
                    for (int e = 0; e < 9; ++e) acc[9 * (int64_t)b + e] = 0.0;
                }
                for (int e = 0; e < 9; ++e) acc[9 * (int64_t)b + e] += H.val[9 * k + e];
            }
        }
        qsort(cols, (size_t)ncols, sizeof(int32_t), cmp_i32);
        if (nnz + ncols > cap) { status = -3; break; }
        for (int32_t t = 0; t < ncols; ++t) {
            cci[nnz] = cols[t];
            for (int e = 0; e < 9; ++e) cval[9 * nnz + e] = acc[9 * (int64_t)cols[t] + e];
            nnz++;
        }
        crp[a + 1] = (int32_t)nnz;
    }
    free(marker); free(acc); free(cols); free(cstart); free(cfill); free(child);
    free_full(&H);
    return status ? status : nnz;
}

/* ------------------------------------------------------------------------ */
/* Block-Jacobi preconditioner                                               */
/* ------------------------------------------------------------------------ */

/* Inverse of a 3x3 matrix by Gauss-Jordan elimination with partial pivoting;
 * returns -2 when a pivot vanishes. */
static int inv3(const double *A, double *Ainv)
{
    double M[3][6];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 6; ++j) M[i][j] = j < 3 ? A[3 * i + j] : (j - 3 == i ? 1.0 : 0.0);
    for (int c = 0; c < 3; ++c) {
        int piv = c;
        for (int r = c + 1; r < 3; ++r)
            if (fabs(M[r][c]) > fabs(M[piv][c])) piv = r;
        if (M[piv][c] == 0.0) return -2;
        if (piv != c)
            for (int j = 0; j < 6; ++j) { double t = M[c][j]; M[c][j] = M[piv][j]; M[piv][j] = t; }
        double d = M[c][c];
        for (int j = 0; j < 6; ++j) M[c][j] /= d;
        for (int r = 0; r < 3; ++r)
            if (r != c) {
                double f = M[r][c];
                for (int j = 0; j < 6; ++j) M[r][j] -= f * M[c][j];
            }
    }
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) Ainv[3 * i + j] = M[i][j + 3];
    return 0;
}

/* The 3x3 block-Jacobi preconditioner of the paper's diagonal option (Sec. 5.1,
 * Preconditioners): dinv[a] = (H[a,a])^{-1}. */
int oracle_block_jacobi(int32_t n, const int32_t *rp, const int32_t *ci, const double *val, double *dinv)
{
    for (int32_t a = 0; a < n; ++a) {
        int found = 0;
        for (int32_t k = rp[a]; k < rp[a + 1]; ++k)
            if (ci[k] == a) {
                if (inv3(val + 9 * (int64_t)k, dinv + 9 * (int64_t)a) != 0) return -2;
                found = 1;
                break;
            }
        if (!found) return -2;
    }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Sparse matrix-vector product and PCG                                      */
/* ------------------------------------------------------------------------ */

/* y = A x for a full-storage 3x3 BSR matrix. */
void oracle_spmv(int32_t n, const int32_t *rp, const int32_t *ci, const double *val, const double *x, double *y)
{
    for (int32_t i = 0; i < n; ++i) {
        double s[3] = {0.0, 0.0, 0.0};
        for (int32_t k = rp[i]; k < rp[i + 1]; ++k) {
            const double *B = val + 9 * (int64_t)k;
            const double *xj = x + 3 * (int64_t)ci[k];
            for (int a = 0; a < 3; ++a) s[a] += B[3 * a] * xj[0] + B[3 * a + 1] * xj[1] + B[3 * a + 2] * xj[2];
        }
        for (int a = 0; a < 3; ++a) y[3 * (int64_t)i + a] = s[a];
    }
}

static double dot(int64_t m, const double *a, const double *b)
{
    double s = 0.0;
    for (int64_t k = 0; k < m; ++k) s += a[k] * b[k];
    return s;
}

static void apply_dinv(int32_t n, const double *dinv, const double *r, double *z)
{
    for (int32_t i = 0; i < n; ++i) {
        const double *D = dinv + 9 * (int64_t)i;
        const double *ri = r + 3 * (int64_t)i;
        for (int a = 0; a < 3; ++a) z[3 * (int64_t)i + a] = D[3 * a] * ri[0] + D[3 * a + 1] * ri[1] + D[3 * a + 2] * ri[2];
    }
}

/*
 * d_c = -H_c^{-1} g_c by preconditioned conjugate gradients (Algorithm 1,
 * the coarse solve; Sec. 5: PCG stopped on a relative residual norm).
 * This is the textbook PCG recurrence (Saad, Iterative Methods for Sparse
 * Linear Systems, Algorithm 9.1) with x0 given (NULL = 0), stopping when
 * ||b - A x||_2 (the recurrence residual) <= tol * ||b||_2.  When b = 0 the
 * answer x = 0 is returned after 0 iterations.  iters = number of SpMVs
 * with the search direction; relres = ||r||_2 / ||b||_2 at exit.
 * Returns 0, or -5 when max_iter was reached first (x is still written).
 */
int oracle_pcg(int32_t n, const int32_t *rp, const int32_t *ci, const double *val, const double *dinv,
               const double *b, double *x, const double *x0, double tol, int32_t max_iter,
               int32_t *iters, double *relres)
{
    int64_t m = 3 * (int64_t)n;
    double *r = (double *)malloc(sizeof(double) * (size_t)(m > 0 ? m : 1));
    double *z = (double *)malloc(sizeof(double) * (size_t)(m > 0 ? m : 1));
    double *p = (double *)malloc(sizeof(double) * (size_t)(m > 0 ? m : 1));
    double *q = (double *)malloc(sizeof(double) * (size_t)(m > 0 ? m : 1));
    double bnorm = sqrt(dot(m, b, b));
    int status = 0;
    if (x0) {
        memcpy(x, x0, sizeof(double) * (size_t)m);
        oracle_spmv(n, rp, ci, val, x, q);
        for (int64_t k = 0; k < m; ++k) r[k] = b[k] - q[k];
    } else {
        for (int64_t k = 0; k < m; ++k) { x[k] = 0.0; r[k] = b[k]; }
    }
    *iters = 0;
    if (bnorm == 0.0) {
        for (int64_t k = 0; k < m; ++k) x[k] = 0.0;
        *relres = 0.0;
        free(r); free(z); free(p); free(q);
        return 0;
    }
    apply_dinv(n, dinv, r, z);
    memcpy(p, z, sizeof(double) * (size_t)m);
    double rz = dot(m, r, z);
    double rnorm = sqrt(dot(m, r, r));
    int32_t it = 0;
    while (rnorm > tol * bnorm) {
        if (it >= max_iter) { status = -5; break; }
        oracle_spmv(n, rp, ci, val, p, q);
        double alpha = rz / dot(m, p, q);
        for (int64_t k = 0; k < m; ++k) { x[k] += alpha * p[k]; r[k] -= alpha * q[k]; }
        apply_dinv(n, dinv, r, z);
        double rz_new = dot(m, r, z);
        double beta = rz_new / rz;
        rz = rz_new;
        for (int64_t k = 0; k < m; ++k) p[k] = z[k] + beta * p[k];
        rnorm = sqrt(dot(m, r, r));
        ++it;
    }
    *iters = it;
    *relres = rnorm / bnorm;
    free(r); free(z); free(p); free(q);
    return status;
}

/* ------------------------------------------------------------------------ */
/* Prolongation                                                              */
/* ------------------------------------------------------------------------ */

/* Sec. 4.3: d_f = U^T d_c, i.e. dx[f] = y[labels[f]]. */
int oracle_prolongate(int32_t n, int32_t n_c, const int32_t *labels, const double *y, double *dx)
{
    for (int32_t f = 0; f < n; ++f) {
        int32_t c = labels[f];
        if (c < 0 || c >= n_c) return -1;
        for (int k = 0; k < 3; ++k) dx[3 * (int64_t)f + k] = y[3 * (int64_t)c + k];
    }
    return 0;
}
