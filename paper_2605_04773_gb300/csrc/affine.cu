// Adaptive affine embedding (Sec. 4.2, Eq. 4, and the supplement's affine
// mapping): a coarse node whose aggregate holds more than `threshold` fine
// nodes gets 12 DoF.  Fine node f of such a node moves by
// dx_f = A_f^T y_c, A_f = Xbar_f (x) I3 with Xbar_f = (X_f, 1) its homogeneous
// rest position, so y_c is four 3-vectors and dx_f = sum_k Xbar_f[k] y_c[k];
// other coarse nodes keep dx_f = y_c.  Coarse 3-rows: every 3-DoF node first
// (label order), then every 12-DoF node as 4 consecutive rows (label order).
// The coarse system is the Galerkin product with that prolongation P:
// g_c = P^T g, H_c = P^T H P, i.e. a fine block B_ij adds
// Xbar_i[k] Xbar_j[l] B_ij to coarse block (row_i + k, row_j + l).
//
// GB300 design.  The expanded structure follows from the label-level coarse
// structure (agipc_assemble_coarse's output): row (c, k) holds, for every
// neighbour c' of c, the columns of c' (1 or 4), and because both classes
// keep label order and every 3-DoF row precedes every 12-DoF row, a label
// row's neighbours written 3-DoF first then 12-DoF are already sorted.
// Values are summed with FP64 atomics at the L2 (one thread per fine block
// or stencil block, up to 16 sub-blocks each, binary search in the row).
#include "agipc_common.cuh"

namespace {

__device__ __forceinline__ double weight(const double *__restrict__ Xr, int64_t f, int kdim, int k)
{
    if (kdim == 1) return 1.0;
    return k < 3 ? Xr[3 * f + k] : 1.0;
}

__device__ __forceinline__ int64_t find_in_row(const int32_t *__restrict__ rp, const int32_t *__restrict__ col,
                                               int64_t cap, int32_t r, int32_t c)
{
    int64_t lo = rp[r], hi = (int64_t)rp[r + 1] - 1;
    if (lo < 0 || hi >= cap) return -1;
    while (lo <= hi) {
        const int64_t mid = (lo + hi) >> 1;
        const int32_t v = col[mid];
        if (v == c) return mid;
        if (v < c) lo = mid + 1;
        else hi = mid - 1;
    }
    return -1;
}

__global__ void count_kernel(int32_t n, const int32_t *__restrict__ labels, const int32_t *__restrict__ n_c_dev,
                             int32_t *cnt, uint32_t *status)
{
    const int32_t nc = *n_c_dev;
    for (int64_t f = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; f < n; f += (int64_t)gridDim.x * blockDim.x) {
        const int32_t c = labels[f];
        if ((unsigned)c >= (unsigned)nc) {
            set_status(status, ST_BAD_INDEX);
            continue;
        }
        atomicAdd(cnt + c, 1);
    }
}

// a[c] = 1 for 3-DoF nodes, b[c] = 1 for 12-DoF nodes (0 past n_c)
__global__ void classify_kernel(int32_t n, const int32_t *__restrict__ n_c_dev, const int32_t *__restrict__ cnt,
                                int32_t threshold, int32_t *__restrict__ a, int32_t *__restrict__ b)
{
    const int32_t nc = *n_c_dev;
    for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < n; c += (int64_t)gridDim.x * blockDim.x) {
        const bool valid = c < nc;
        const bool aff = valid && cnt[c] > threshold;
        a[c] = valid && !aff ? 1 : 0;
        b[c] = aff ? 1 : 0;
    }
}

// base[c] and k[c] from the two ranks; n_rows = n3 + 4 nA
__global__ void base_kernel(int32_t n, const int32_t *__restrict__ n_c_dev, const int32_t *__restrict__ pos3,
                            const int32_t *__restrict__ posA, const int32_t *__restrict__ cnt, int32_t threshold,
                            int32_t *__restrict__ base, int32_t *__restrict__ kdim, int32_t *__restrict__ n_rows_dev)
{
    const int32_t nc = *n_c_dev;
    const int32_t n3 = pos3[n], nA = posA[n];
    for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < nc; c += (int64_t)gridDim.x * blockDim.x) {
        const bool aff = cnt[c] > threshold;
        base[c] = aff ? n3 + 4 * posA[c] : pos3[c];
        kdim[c] = aff ? 4 : 1;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) *n_rows_dev = n3 + 4 * nA;
}

// length of every expanded row: sum of the neighbours' widths
__global__ void rowlen_kernel(const int32_t *__restrict__ n_c_dev, const int32_t *__restrict__ lrp,
                              const int32_t *__restrict__ lcol, const int32_t *__restrict__ base,
                              const int32_t *__restrict__ kdim, int32_t *__restrict__ lens, uint32_t *status)
{
    const int32_t nc = *n_c_dev;
    for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < nc; c += (int64_t)gridDim.x * blockDim.x) {
        int32_t L = 0;
        for (int32_t q = lrp[c]; q < lrp[c + 1]; ++q) {
            const int32_t cc = lcol[q];
            if ((unsigned)cc >= (unsigned)nc) {
                set_status(status, ST_BAD_INDEX);
                continue;
            }
            L += kdim[cc];
        }
        for (int k = 0; k < kdim[c]; ++k) lens[base[c] + k] = L;
    }
}

__global__ void fill_cols_kernel(const int32_t *__restrict__ n_c_dev, const int32_t *__restrict__ lrp,
                                 const int32_t *__restrict__ lcol, const int32_t *__restrict__ base,
                                 const int32_t *__restrict__ kdim, const int32_t *__restrict__ rp, int64_t cap,
                                 int32_t *__restrict__ col, uint32_t *status)
{
    const int32_t nc = *n_c_dev;
    for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < nc; c += (int64_t)gridDim.x * blockDim.x) {
        for (int k = 0; k < kdim[c]; ++k) {
            int64_t dst = rp[base[c] + k];
            const int64_t end = rp[base[c] + k + 1];
            if (end > cap) {
                set_status(status, ST_CAPACITY);
                break;
            }
            for (int pass = 0; pass < 2; ++pass)
                for (int32_t q = lrp[c]; q < lrp[c + 1]; ++q) {
                    const int32_t cc = lcol[q];
                    if ((unsigned)cc >= (unsigned)nc) continue;
                    const int kk = kdim[cc];
                    if ((pass == 0) != (kk == 1)) continue;
                    for (int l = 0; l < kk && dst < end; ++l) col[dst++] = base[cc] + l;
                }
        }
    }
}

__global__ void zero_kernel(const int32_t *__restrict__ n_rows_dev, const int32_t *__restrict__ rp, int64_t cap,
                            double *__restrict__ val, double *__restrict__ g_c)
{
    const int32_t nr = *n_rows_dev;
    const int64_t nnz = min64(rp[nr], cap);
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < 9 * nnz; k += (int64_t)gridDim.x * blockDim.x)
        val[k] = 0.0;
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < 3 * (int64_t)nr;
         k += (int64_t)gridDim.x * blockDim.x)
        g_c[k] = 0.0;
}

struct Expand {
    const int32_t *labels;
    const double *Xr;
    const int32_t *base;
    const int32_t *kdim;
    const int32_t *rp;
    const int32_t *col;
    int64_t cap;
    double *val;
    uint32_t *status;

    // B (3x3 row-major, transposed when tr) weighted into every sub-block of
    // fine nodes (i, j)
    __device__ void add(int32_t i, int32_t j, const double B[9], bool tr) const
    {
        const int32_t ci = labels[i], cj = labels[j];
        const int ki = kdim[ci], kj = kdim[cj];
        for (int k = 0; k < ki; ++k) {
            const double wi = weight(Xr, i, ki, k);
            for (int l = 0; l < kj; ++l) {
                const double w = wi * weight(Xr, j, kj, l);
                const int64_t pos = find_in_row(rp, col, cap, base[ci] + k, base[cj] + l);
                if (pos < 0) {
                    set_status(status, ST_BAD_INDEX);
                    continue;
                }
                double *d = val + 9 * pos;
#pragma unroll
                for (int r = 0; r < 3; ++r)
#pragma unroll
                    for (int c = 0; c < 3; ++c) atomicAdd(d + 3 * r + c, w * (tr ? B[3 * c + r] : B[3 * r + c]));
            }
        }
    }
};

__global__ void numeric_fine_kernel(Expand X, int32_t n, const int32_t *__restrict__ frp,
                                    const int32_t *__restrict__ fcol, const double *__restrict__ fval, int64_t nnzb,
                                    const int32_t *__restrict__ n_c_dev)
{
    const int32_t nc = *n_c_dev;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        if ((unsigned)X.labels[i] >= (unsigned)nc) continue;  // reported by the plan
        const int32_t k0 = frp[i], k1 = frp[i + 1];
        if (k0 < 0 || k1 < k0 || k1 > nnzb) {
            set_status(X.status, ST_BAD_INDEX);
            continue;
        }
        for (int32_t q = k0; q < k1; ++q) {
            const int32_t j = fcol[q];
            if ((unsigned)j >= (unsigned)n || (unsigned)X.labels[j] >= (unsigned)nc) {
                set_status(X.status, ST_BAD_INDEX);
                continue;
            }
            double B[9];
#pragma unroll
            for (int e = 0; e < 9; ++e) B[e] = fval[9 * (int64_t)q + e];
            X.add((int32_t)i, j, B, false);
            if (j != i) X.add(j, (int32_t)i, B, true);
        }
    }
}

__constant__ int kS[10] = {0, 0, 0, 0, 1, 1, 1, 2, 2, 3};
__constant__ int kT[10] = {0, 1, 2, 3, 1, 2, 3, 2, 3, 3};

__global__ void numeric_pair_kernel(Expand X, int32_t n, int64_t n_pairs, const int32_t *__restrict__ pidx,
                                    const double *__restrict__ pblk, const int32_t *__restrict__ n_c_dev)
{
    const int32_t nc = *n_c_dev;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < 10 * n_pairs;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t pr = t / 10;
        const int q = (int)(t - 10 * pr);
        const int32_t va = pidx[4 * pr + kS[q]], vb = pidx[4 * pr + kT[q]];
        if ((unsigned)va >= (unsigned)n || (unsigned)vb >= (unsigned)n || (unsigned)X.labels[va] >= (unsigned)nc ||
            (unsigned)X.labels[vb] >= (unsigned)nc) {
            set_status(X.status, ST_BAD_INDEX);
            continue;
        }
        double B[9];
#pragma unroll
        for (int e = 0; e < 9; ++e) B[e] = pblk[90 * pr + 9 * q + e];
        X.add(va, vb, B, false);
        if (kS[q] != kT[q]) X.add(vb, va, B, true);
    }
}

__global__ void gradient_kernel(int32_t n, const int32_t *__restrict__ labels, const int32_t *__restrict__ n_c_dev,
                                const double *__restrict__ Xr, const int32_t *__restrict__ base,
                                const int32_t *__restrict__ kdim, const double *__restrict__ g, double *g_c)
{
    const int32_t nc = *n_c_dev;
    for (int64_t f = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; f < n; f += (int64_t)gridDim.x * blockDim.x) {
        const int32_t c = labels[f];
        if ((unsigned)c >= (unsigned)nc) continue;
        const int kd = kdim[c];
        for (int k = 0; k < kd; ++k) {
            const double w = weight(Xr, f, kd, k);
#pragma unroll
            for (int d = 0; d < 3; ++d) atomicAdd(g_c + 3 * (int64_t)(base[c] + k) + d, w * g[3 * f + d]);
        }
    }
}

__device__ __forceinline__ bool inv3(const double *A, double *R)
{
    const double c00 = A[4] * A[8] - A[5] * A[7];
    const double c01 = A[5] * A[6] - A[3] * A[8];
    const double c02 = A[3] * A[7] - A[4] * A[6];
    const double det = A[0] * c00 + A[1] * c01 + A[2] * c02;
    if (!(fabs(det) > 0.0) || !isfinite(det)) return false;
    const double id = 1.0 / det;
    R[0] = c00 * id;
    R[1] = (A[2] * A[7] - A[1] * A[8]) * id;
    R[2] = (A[1] * A[5] - A[2] * A[4]) * id;
    R[3] = c01 * id;
    R[4] = (A[0] * A[8] - A[2] * A[6]) * id;
    R[5] = (A[2] * A[3] - A[0] * A[5]) * id;
    R[6] = c02 * id;
    R[7] = (A[1] * A[6] - A[0] * A[7]) * id;
    R[8] = (A[0] * A[4] - A[1] * A[3]) * id;
    return true;
}

// 3x3 block-Jacobi inverses of the expanded diagonal blocks (symmetrised)
__global__ void dinv_kernel(const int32_t *__restrict__ n_rows_dev, const int32_t *__restrict__ rp,
                            const int32_t *__restrict__ col, int64_t cap, const double *__restrict__ val,
                            double *__restrict__ dinv, uint32_t *status)
{
    const int32_t nr = *n_rows_dev;
    for (int64_t a = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; a < nr; a += (int64_t)gridDim.x * blockDim.x) {
        const int64_t q = find_in_row(rp, col, cap, (int32_t)a, (int32_t)a);
        double R[9];
        bool ok = q >= 0;
        if (ok) {
            double D[9];
#pragma unroll
            for (int e = 0; e < 9; ++e) D[e] = val[9 * q + e];
            D[3] = D[1] = 0.5 * (D[1] + D[3]);
            D[6] = D[2] = 0.5 * (D[2] + D[6]);
            D[7] = D[5] = 0.5 * (D[5] + D[7]);
            ok = inv3(D, R);
        }
        if (!ok) {
            set_status(status, ST_NONFINITE);
#pragma unroll
            for (int e = 0; e < 9; ++e) R[e] = 0.0;
        }
#pragma unroll
        for (int e = 0; e < 9; ++e) dinv[9 * a + e] = R[e];
    }
}

__global__ void prolongate_kernel(int32_t n, const int32_t *__restrict__ labels, const int32_t *__restrict__ n_c_dev,
                                  const double *__restrict__ Xr, const int32_t *__restrict__ base,
                                  const int32_t *__restrict__ kdim, const double *__restrict__ y,
                                  double *__restrict__ dx, uint32_t *status)
{
    const int32_t nc = *n_c_dev;
    for (int64_t f = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; f < n; f += (int64_t)gridDim.x * blockDim.x) {
        const int32_t c = labels[f];
        if ((unsigned)c >= (unsigned)nc || base[c] < 0 || base[c] + kdim[c] > n) {
            set_status(status, ST_BAD_INDEX);
            dx[3 * f] = dx[3 * f + 1] = dx[3 * f + 2] = 0.0;
            continue;
        }
        const int kd = kdim[c] == 4 ? 4 : 1;
        double o[3] = {0.0, 0.0, 0.0};
        for (int k = 0; k < kd; ++k) {
            const double w = weight(Xr, f, kd, k);
#pragma unroll
            for (int d = 0; d < 3; ++d) o[d] = fma(w, y[3 * (int64_t)(base[c] + k) + d], o[d]);
        }
        dx[3 * f] = o[0];
        dx[3 * f + 1] = o[1];
        dx[3 * f + 2] = o[2];
    }
}

unsigned grid_for(const agipc_ctx *ctx, int64_t work, int tb)
{
    return (unsigned)max64(1, min64(div_up(work, tb), (int64_t)ctx->num_sms * 32));
}

}  // namespace

extern "C" int agipc_affine_plan(agipc_ctx *ctx, int32_t n_fine, const int32_t *labels, const int32_t *n_coarse_dev,
                                 int32_t threshold, int32_t *coarse_base, int32_t *coarse_k, int32_t *n_rows_dev)
{
    if (!ctx || n_fine <= 0 || n_fine > ctx->max_n || !labels || !n_coarse_dev || threshold < 3 || !coarse_base ||
        !coarse_k || !n_rows_dev)
        return AGIPC_ERR_INVALID_ARG;
    cudaStream_t st = ctx->stream;
    const int tb = 256;
    int32_t *cnt = ctx->parent;    // [max_n]: fine nodes per coarse node
    int32_t *a = ctx->rank;        // [max_n + 1]: 3-DoF ranks, total at [n_fine]
    int32_t *b = ctx->long_rows;   // [max_n + 1]: 12-DoF ranks, total at [n_fine]
    if (cudaMemsetAsync(cnt, 0, sizeof(int32_t) * (size_t)n_fine, st) != cudaSuccess) return AGIPC_ERR_CUDA;
    count_kernel<<<grid_for(ctx, n_fine, tb), tb, 0, st>>>(n_fine, labels, n_coarse_dev, cnt, ctx->status);
    classify_kernel<<<grid_for(ctx, n_fine, tb), tb, 0, st>>>(n_fine, n_coarse_dev, cnt, threshold, a, b);
    if (!scan_exclusive_i32(a, a, n_fine, nullptr, ctx->scan_part, st) ||
        !scan_exclusive_i32(b, b, n_fine, nullptr, ctx->scan_part, st))
        return AGIPC_ERR_CAPACITY;
    base_kernel<<<grid_for(ctx, n_fine, tb), tb, 0, st>>>(n_fine, n_coarse_dev, a, b, cnt, threshold, coarse_base,
                                                          coarse_k, n_rows_dev);
    return cudaPeekAtLastError() == cudaSuccess ? AGIPC_OK : AGIPC_ERR_CUDA;
}

extern "C" int agipc_assemble_affine(agipc_ctx *ctx, int32_t n_fine, const int32_t *labels,
                                     const int32_t *n_coarse_dev, const double *X_rest, const int32_t *coarse_base,
                                     const int32_t *coarse_k, const int32_t *n_rows_dev, const int32_t *label_row_ptr,
                                     const int32_t *label_col, const int32_t *fine_row_ptr, const int32_t *fine_col,
                                     const double *fine_val, int64_t fine_nnzb, int64_t n_pairs,
                                     const int32_t *pair_idx, const double *pair_blk, const double *g,
                                     int32_t *row_ptr, int32_t *col, double *val, int64_t cap_nnzb,
                                     int32_t *nnzb_dev, double *g_c, double *dinv)
{
    if (!ctx || n_fine <= 0 || n_fine > ctx->max_n || !labels || !n_coarse_dev || !X_rest || !coarse_base ||
        !coarse_k || !n_rows_dev || !label_row_ptr || !label_col || !fine_row_ptr || !fine_col || !fine_val ||
        fine_nnzb < 0 || n_pairs < 0 || (n_pairs > 0 && (!pair_idx || !pair_blk)) || !g || !row_ptr || !col ||
        !val || cap_nnzb <= 0 || !nnzb_dev || !g_c || !dinv)
        return AGIPC_ERR_INVALID_ARG;
    cudaStream_t st = ctx->stream;
    const int tb = 256;
    int32_t *lens = ctx->row_cnt;  // [max_n + 1]; n_rows <= n_fine when threshold >= 3
    if (cudaMemsetAsync(lens, 0, sizeof(int32_t) * ((size_t)n_fine + 1), st) != cudaSuccess) return AGIPC_ERR_CUDA;
    rowlen_kernel<<<grid_for(ctx, n_fine, tb), tb, 0, st>>>(n_coarse_dev, label_row_ptr, label_col, coarse_base,
                                                            coarse_k, lens, ctx->status);
    // rows past n_rows have length 0, so the scan of n_fine rows ends at the total
    if (!scan_exclusive_i32(lens, row_ptr, n_fine, nnzb_dev, ctx->scan_part, st)) return AGIPC_ERR_CAPACITY;
    fill_cols_kernel<<<grid_for(ctx, n_fine, tb), tb, 0, st>>>(n_coarse_dev, label_row_ptr, label_col, coarse_base,
                                                               coarse_k, row_ptr, cap_nnzb, col, ctx->status);
    zero_kernel<<<(unsigned)ctx->num_sms * 8, tb, 0, st>>>(n_rows_dev, row_ptr, cap_nnzb, val, g_c);
    Expand X{labels, X_rest, coarse_base, coarse_k, row_ptr, col, cap_nnzb, val, ctx->status};
    numeric_fine_kernel<<<grid_for(ctx, n_fine, tb), tb, 0, st>>>(X, n_fine, fine_row_ptr, fine_col, fine_val,
                                                                  fine_nnzb, n_coarse_dev);
    if (n_pairs > 0)
        numeric_pair_kernel<<<grid_for(ctx, 10 * n_pairs, tb), tb, 0, st>>>(X, n_fine, n_pairs, pair_idx, pair_blk,
                                                                            n_coarse_dev);
    gradient_kernel<<<grid_for(ctx, n_fine, tb), tb, 0, st>>>(n_fine, labels, n_coarse_dev, X_rest, coarse_base,
                                                              coarse_k, g, g_c);
    dinv_kernel<<<grid_for(ctx, n_fine, tb), tb, 0, st>>>(n_rows_dev, row_ptr, col, cap_nnzb, val, dinv,
                                                          ctx->status);
    return cudaPeekAtLastError() == cudaSuccess ? AGIPC_OK : AGIPC_ERR_CUDA;
}

extern "C" int agipc_prolongate_affine(agipc_ctx *ctx, int32_t n_fine, const int32_t *labels,
                                       const int32_t *n_coarse_dev, const double *X_rest, const int32_t *coarse_base,
                                       const int32_t *coarse_k, const double *y, double *dx)
{
    if (!ctx || n_fine <= 0 || n_fine > ctx->max_n || !labels || !n_coarse_dev || !X_rest || !coarse_base ||
        !coarse_k || !y || !dx)
        return AGIPC_ERR_INVALID_ARG;
    const int tb = 256;
    prolongate_kernel<<<grid_for(ctx, n_fine, tb), tb, 0, ctx->stream>>>(n_fine, labels, n_coarse_dev, X_rest,
                                                                          coarse_base, coarse_k, y, dx, ctx->status);
    return cudaPeekAtLastError() == cudaSuccess ? AGIPC_OK : AGIPC_ERR_CUDA;
}
