// Block-Jacobi PCG on a full-storage 3x3 BSR matrix (Algorithm 1's coarse
// solve d_c = -H_c^-1 g_c; Sec. 5 stops on the relative residual norm and
// Sec. 5.1 names the 3x3 block-Jacobi preconditioner).
//
// The whole solve is one persistent cooperative kernel with device-side
// convergence.  The recurrence is the Chronopoulos-Gear form of PCG, which
// is algebraically the textbook method but needs a single reduction per
// iteration (gamma = r.u, rho = r.r and delta = u.Au together):
//     u = M^-1 r,  w = A u,  gamma = (r,u),  delta = (w,u)
//     beta = gamma/gamma_old,  alpha = gamma/(delta - beta*gamma/alpha_old)
//     p = u + beta p,  s = w + beta s,  x += alpha p,  r -= alpha s
// Per iteration the kernel runs two phases separated by grid barriers:
//   S: w = A u (nnz-balanced: every warp owns an equal, 32-aligned slice of
//      the blocks; the warp stages its 32 blocks (2304 B) in shared memory
//      with coalesced 16-byte loads, multiplies, and reduces rows with a
//      segmented shuffle scan; rows cut by a slice boundary are added with
//      atomics) and the partial delta = sum over blocks of u_row^T B u_col;
//   P: the row-local updates above, the preconditioner and the partial
//      gamma/rho of the next iteration.
// Partial sums go to a per-CTA slot and every CTA reduces all slots in the
// same order, so the scalars are bitwise identical in every CTA and from run
// to run.  Barrier waits are bounded (ST_TIMEOUT).
#include <algorithm>

#include "agipc_common.cuh"

namespace {

constexpr int kPcgBlock = 512;
constexpr int kPcgWarps = kPcgBlock / 32;

struct PcgArgs {
    const int32_t *n_dev;
    const int32_t *rp;
    const int32_t *col;
    const double *val;
    const double *dinv;
    const double *b;
    double *x;
    double sign;
    double tol;
    int32_t max_iter;
    int32_t max_rows;
    int64_t max_nnzb;
    int32_t *iters_dev;
    double *relres_dev;
    PcgScratch S;
    uint32_t *status;
};

// Sum two values over the CTA; thread 0 receives the totals (fixed order).
__device__ __forceinline__ void block_sum2(double &a, double &b, double (*s_red)[4])
{
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    a = warp_sum(a);
    b = warp_sum(b);
    if (lane == 0) { s_red[wid][0] = a; s_red[wid][1] = b; }
    __syncthreads();
    if (wid == 0) {
        a = lane < kPcgWarps ? s_red[lane][0] : 0.0;
        b = lane < kPcgWarps ? s_red[lane][1] : 0.0;
        a = warp_sum(a);
        b = warp_sum(b);
    }
    __syncthreads();
}

__device__ __forceinline__ void emit_row(double *w, const uint8_t *rowflag, int row, double y0, double y1, double y2)
{
    double *dst = w + 3 * (int64_t)row;
    if (rowflag[row] & 1) {
        atomicAdd(dst, y0);
        atomicAdd(dst + 1, y1);
        atomicAdd(dst + 2, y2);
    } else {
        dst[0] = y0;
        dst[1] = y1;
        dst[2] = y2;
    }
}

__global__ void __launch_bounds__(kPcgBlock) pcg_kernel(PcgArgs A)
{
    __shared__ __align__(16) double s_stage[kPcgWarps][9 * 32];
    __shared__ double s_red[kPcgWarps][4];
    __shared__ double s_scal[4];

    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const unsigned nblocks = gridDim.x;
    const int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t nthreads = (int64_t)nblocks * blockDim.x;
    const int64_t gwarp = (int64_t)blockIdx.x * kPcgWarps + wib;
    const int64_t nwarps = (int64_t)nblocks * kPcgWarps;

    const int32_t n = *A.n_dev;
    if (n < 0 || n > A.max_rows) {
        if (tid == 0) set_status(A.status, ST_BAD_INDEX);
        return;
    }
    const int64_t nnz = A.rp[n];
    if (nnz < 0 || nnz > A.max_nnzb) {
        if (tid == 0) set_status(A.status, nnz < 0 ? ST_BAD_INDEX : ST_CAPACITY);
        return;
    }
    const int64_t chunk = max64(32, div_up(div_up(nnz, nwarps), 32) * 32);

    double *__restrict__ r = A.S.r;
    double *u = A.S.u;
    double *w = A.S.w;
    double *__restrict__ p = A.S.p;
    double *__restrict__ s = A.S.s;
    double *__restrict__ x = A.x;
    int32_t *brow = A.S.brow;
    uint8_t *rowflag = A.S.rowflag;
    double *partials = A.S.partials;
    const int pstride = A.S.max_grid * 4;

    // ---- setup: block rows, split flags, x = 0, r = b, u = M^-1 r, p = s = w = 0
    double gpart = 0.0, rpart = 0.0;
    for (int64_t i = tid; i < n; i += nthreads) {
        const int32_t k0 = A.rp[i], k1 = A.rp[i + 1];
        bool bad = k0 < 0 || k1 < k0 || k1 > nnz;
        for (int32_t k = k0; !bad && k < k1; ++k) {
            brow[k] = (int32_t)i;
            bad = (unsigned)A.col[k] >= (unsigned)n;
        }
        if (bad) atomicOr(A.S.bar + 2, 1u);
        uint8_t f = 0;
        if (k1 == k0) f = 2;
        else if (k0 / chunk != (k1 - 1) / chunk) f = 1;
        rowflag[i] = f;
        double rr[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            rr[c] = A.sign * A.b[3 * i + c];
            x[3 * i + c] = 0.0;
            p[3 * i + c] = 0.0;
            s[3 * i + c] = 0.0;
            w[3 * i + c] = 0.0;
            r[3 * i + c] = rr[c];
        }
        const double *D = A.dinv + 9 * i;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const double uc = D[3 * c] * rr[0] + D[3 * c + 1] * rr[1] + D[3 * c + 2] * rr[2];
            u[3 * i + c] = uc;
            gpart += rr[c] * uc;
            rpart += rr[c] * rr[c];
        }
    }
    block_sum2(gpart, rpart, s_red);
    if (threadIdx.x == 0) {
        partials[blockIdx.x * 4 + 0] = gpart;
        partials[blockIdx.x * 4 + 1] = rpart;
    }
    bool ok = grid_barrier(A.S.bar, nblocks, A.status);
    if (ok && ld_acquire_u32(A.S.bar + 2) != 0u) {
        // a row pointer or column index out of range: nothing gathers through it
        if (tid == 0) set_status(A.status, ST_BAD_INDEX);
        ok = false;
    }

    double alpha_old = 1.0, gamma_old = 1.0, bnorm = 0.0, rnorm = 0.0;
    int32_t it = 0;
    bool converged = false;
    while (ok) {
        const int par = it & 1;
        double *part = partials + par * pstride;
        // ---- S phase: w = A u, partial delta
        double dpart = 0.0;
        {
            double *stage = s_stage[wib];
            const int64_t kb = gwarp * chunk;
            const int64_t ke = min64(kb + chunk, nnz);
            int carry_row = -1;
            double c0 = 0.0, c1 = 0.0, c2 = 0.0;
            for (int64_t base = kb; base < ke; base += 32) {
                const int cnt = (int)min64(32, ke - base);
                const int nd = 9 * cnt;
                const double2 *src = reinterpret_cast<const double2 *>(A.val + 9 * base);
                double2 *dst2 = reinterpret_cast<double2 *>(stage);
                for (int q = lane; q < (nd >> 1); q += 32) dst2[q] = __ldg(src + q);
                if ((nd & 1) && lane == 0) stage[nd - 1] = __ldg(A.val + 9 * base + nd - 1);
                __syncwarp();
                int row = -1;
                double y0 = 0.0, y1 = 0.0, y2 = 0.0;
                if (lane < cnt) {
                    const int64_t k = base + lane;
                    row = __ldcg(brow + k);
                    const int32_t cj = __ldg(A.col + k);
                    const double *B = stage + 9 * lane;
                    const double x0 = __ldcg(u + 3 * (int64_t)cj), x1 = __ldcg(u + 3 * (int64_t)cj + 1),
                                 x2 = __ldcg(u + 3 * (int64_t)cj + 2);
                    y0 = B[0] * x0 + B[1] * x1 + B[2] * x2;
                    y1 = B[3] * x0 + B[4] * x1 + B[5] * x2;
                    y2 = B[6] * x0 + B[7] * x1 + B[8] * x2;
                    dpart += __ldcg(u + 3 * (int64_t)row) * y0 + __ldcg(u + 3 * (int64_t)row + 1) * y1 +
                             __ldcg(u + 3 * (int64_t)row + 2) * y2;
                }
                __syncwarp();
                // segmented suffix sums: rows are non-decreasing across lanes
#pragma unroll
                for (int off = 1; off < 32; off <<= 1) {
                    const double n0 = __shfl_down_sync(kFull, y0, off);
                    const double n1 = __shfl_down_sync(kFull, y1, off);
                    const double n2 = __shfl_down_sync(kFull, y2, off);
                    const int nr = __shfl_down_sync(kFull, row, off);
                    if (lane + off < 32 && nr == row) { y0 += n0; y1 += n1; y2 += n2; }
                }
                const int prev = __shfl_up_sync(kFull, row, 1);
                const bool head = row >= 0 && (lane == 0 || prev != row);
                if (lane == 0) {
                    if (carry_row >= 0 && carry_row == row) { y0 += c0; y1 += c1; y2 += c2; }
                    else if (carry_row >= 0) emit_row(w, rowflag, carry_row, c0, c1, c2);
                }
                const unsigned heads = __ballot_sync(kFull, head);
                const int last = 31 - __clz(heads);
                if (head && lane != last) emit_row(w, rowflag, row, y0, y1, y2);
                carry_row = __shfl_sync(kFull, row, last);
                c0 = __shfl_sync(kFull, y0, last);
                c1 = __shfl_sync(kFull, y1, last);
                c2 = __shfl_sync(kFull, y2, last);
            }
            if (lane == 0 && carry_row >= 0) emit_row(w, rowflag, carry_row, c0, c1, c2);
        }
        {
            double dummy = 0.0;
            block_sum2(dpart, dummy, s_red);
            if (threadIdx.x == 0) part[blockIdx.x * 4 + 2] = dpart;
        }
        if (!grid_barrier(A.S.bar, nblocks, A.status)) { ok = false; break; }

        // ---- global scalars, reduced identically in every CTA
        if (wib == 0) {
            double g = 0.0, rh = 0.0, dl = 0.0;
            for (unsigned k = lane; k < nblocks; k += 32) {
                g += __ldcg(part + k * 4 + 0);
                rh += __ldcg(part + k * 4 + 1);
                dl += __ldcg(part + k * 4 + 2);
            }
            g = warp_sum(g);
            rh = warp_sum(rh);
            dl = warp_sum(dl);
            if (lane == 0) { s_scal[0] = g; s_scal[1] = rh; s_scal[2] = dl; }
        }
        __syncthreads();
        const double gamma = s_scal[0], rho = s_scal[1], delta = s_scal[2];
        __syncthreads();
        rnorm = sqrt(rho);
        if (it == 0) bnorm = rnorm;
        if (!isfinite(rho) || !isfinite(gamma) || !isfinite(delta)) {
            if (tid == 0) set_status(A.status, ST_NONFINITE);
            break;
        }
        if (bnorm == 0.0 || rnorm <= A.tol * bnorm) { converged = true; break; }
        if (it >= A.max_iter) break;
        const double beta = it == 0 ? 0.0 : gamma / gamma_old;
        const double alpha = it == 0 ? gamma / delta : gamma / (delta - beta * gamma / alpha_old);
        if (!isfinite(alpha) || !isfinite(beta)) {
            if (tid == 0) set_status(A.status, ST_NONFINITE);
            break;
        }

        // ---- P phase: row-local updates, preconditioner, next partials
        double *npart = partials + (par ^ 1) * pstride;
        gpart = 0.0;
        rpart = 0.0;
        for (int64_t i = tid; i < n; i += nthreads) {
            double uu[3], ww[3], pp[3], ss[3], rr[3];
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                uu[c] = __ldcg(u + 3 * i + c);
                ww[c] = __ldcg(w + 3 * i + c);
                pp[c] = p[3 * i + c];
                ss[c] = s[3 * i + c];
                rr[c] = r[3 * i + c];
            }
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                pp[c] = uu[c] + beta * pp[c];
                ss[c] = ww[c] + beta * ss[c];
                x[3 * i + c] += alpha * pp[c];
                rr[c] -= alpha * ss[c];
                p[3 * i + c] = pp[c];
                s[3 * i + c] = ss[c];
                r[3 * i + c] = rr[c];
            }
            const double *D = A.dinv + 9 * i;
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                const double uc = D[3 * c] * rr[0] + D[3 * c + 1] * rr[1] + D[3 * c + 2] * rr[2];
                u[3 * i + c] = uc;
                gpart += rr[c] * uc;
                rpart += rr[c] * rr[c];
            }
            if (rowflag[i]) {
                w[3 * i] = 0.0;
                w[3 * i + 1] = 0.0;
                w[3 * i + 2] = 0.0;
            }
        }
        block_sum2(gpart, rpart, s_red);
        if (threadIdx.x == 0) {
            npart[blockIdx.x * 4 + 0] = gpart;
            npart[blockIdx.x * 4 + 1] = rpart;
        }
        gamma_old = gamma;
        alpha_old = alpha;
        ++it;
        if (!grid_barrier(A.S.bar, nblocks, A.status)) { ok = false; break; }
    }
    if (tid == 0 && (ok || it > 0)) {
        *A.iters_dev = it;
        *A.relres_dev = bnorm > 0.0 ? rnorm / bnorm : 0.0;
        if (ok && !converged) set_status(A.status, ST_NOT_CONVERGED);
    }
}

}  // namespace

int pcg_block_size() { return kPcgBlock; }

const void *pcg_kernel_ptr() { return reinterpret_cast<const void *>(&pcg_kernel); }

extern "C" int agipc_pcg(agipc_ctx *ctx, int32_t max_rows, const int32_t *n_rows_dev, const int32_t *row_ptr,
                         const int32_t *col, const double *val, const double *dinv, const double *b, double *x,
                         const agipc_pcg_options *opt, int32_t *iters_dev, double *relres_dev)
{
    if (!ctx || !opt || max_rows < 0 || max_rows > ctx->max_n || !n_rows_dev || !row_ptr || !dinv || !b || !x ||
        !iters_dev || !relres_dev)
        return AGIPC_ERR_INVALID_ARG;
    if (!(opt->tol >= 0.0) || opt->max_iter < 0 || (opt->rhs_sign != 1 && opt->rhs_sign != -1))
        return AGIPC_ERR_INVALID_ARG;
    if (((uintptr_t)val & 15u) != 0 || ((uintptr_t)dinv & 7u) != 0 || ((uintptr_t)b & 7u) != 0 ||
        ((uintptr_t)x & 7u) != 0)
        return AGIPC_ERR_INVALID_ARG;
    PcgArgs A;
    A.n_dev = n_rows_dev;
    A.rp = row_ptr;
    A.col = col;
    A.val = val;
    A.dinv = dinv;
    A.b = b;
    A.x = x;
    A.sign = (double)opt->rhs_sign;
    A.tol = opt->tol;
    A.max_iter = opt->max_iter;
    A.max_rows = max_rows;
    A.max_nnzb = ctx->max_nnzb;
    A.iters_dev = iters_dev;
    A.relres_dev = relres_dev;
    A.S = ctx->pcg;
    A.status = ctx->status;
    if (cudaMemsetAsync(ctx->pcg.bar, 0, 4 * sizeof(unsigned), ctx->stream) != cudaSuccess) return AGIPC_ERR_CUDA;
    void *args[] = {&A};
    cudaError_t e = cudaLaunchCooperativeKernel((const void *)pcg_kernel, dim3((unsigned)ctx->pcg_grid),
                                                dim3(kPcgBlock), args, 0, ctx->stream);
    return e == cudaSuccess ? AGIPC_OK : AGIPC_ERR_CUDA;
}
