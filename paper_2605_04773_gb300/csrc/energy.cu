// The incremental potential of the StVK problem and the two vector
// reductions the Newton loop's line search needs (the inner loop of
// Algorithm 1: E(x_prev + alpha d) < E_prev, and the stopping test on
// ||d||_inf / dt).
//
// With the fine system of agipc_fine_assemble_stvk (Eq. 1 divided by dt^2,
// no barrier or friction terms), the energy whose gradient that routine sums
// is
//   E(x) = sum_i (m_i / h^2) / 2 |x_i - x_hat_i|^2 + sum_e Psi_e(x) + g_extra . x
// with x_hat_i = X_rest_i + shift and Psi_e = V_e (mu |G|_F^2 + lam/2 tr(G)^2),
// G = (F^T F - I) / 2, F = Ds Dm^-1, V_e = |det Dm| / 6.
//
// The sum is deterministic: every CTA reduces its grid-stride share in a
// fixed order and stores one partial; the last CTA to arrive adds the
// partials in CTA order.  No CTA waits on another.
#include <math.h>

#include <algorithm>

#include "agipc_common.cuh"

namespace {

constexpr int kEnergyThreads = 256;

struct Shift {
    double v[3];
};

// x0 + alpha d with the product and the sum rounded separately (no
// contraction), so the trial point is the one a plain FP64 evaluation of
// x0 + alpha * d gives.
__device__ __forceinline__ double trial(const double *x0, const double *d, double alpha, int64_t k)
{
    return d ? __dadd_rn(x0[k], __dmul_rn(alpha, d[k])) : x0[k];
}

__device__ __forceinline__ double tet_psi(const double X[4][3], const double x[4][3], double mu, double lam)
{
    double Dm[3][3], Ds[3][3];
#pragma unroll
    for (int c = 0; c < 3; ++c)
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            Dm[c][k] = X[k + 1][c] - X[0][c];
            Ds[c][k] = x[k + 1][c] - x[0][c];
        }
    // Dm^-1 = adj(Dm) / det(Dm)
    double A[3][3];
    A[0][0] = Dm[1][1] * Dm[2][2] - Dm[1][2] * Dm[2][1];
    A[0][1] = Dm[0][2] * Dm[2][1] - Dm[0][1] * Dm[2][2];
    A[0][2] = Dm[0][1] * Dm[1][2] - Dm[0][2] * Dm[1][1];
    A[1][0] = Dm[1][2] * Dm[2][0] - Dm[1][0] * Dm[2][2];
    A[1][1] = Dm[0][0] * Dm[2][2] - Dm[0][2] * Dm[2][0];
    A[1][2] = Dm[0][2] * Dm[1][0] - Dm[0][0] * Dm[1][2];
    A[2][0] = Dm[1][0] * Dm[2][1] - Dm[1][1] * Dm[2][0];
    A[2][1] = Dm[0][1] * Dm[2][0] - Dm[0][0] * Dm[2][1];
    A[2][2] = Dm[0][0] * Dm[1][1] - Dm[0][1] * Dm[1][0];
    const double det = Dm[0][0] * A[0][0] + Dm[0][1] * A[1][0] + Dm[0][2] * A[2][0];
    const double id = 1.0 / det;
    double F[3][3];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) F[i][j] = (Ds[i][0] * A[0][j] + Ds[i][1] * A[1][j] + Ds[i][2] * A[2][j]) * id;
    double g2 = 0.0, tr = 0.0;
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            const double c = F[0][i] * F[0][j] + F[1][i] * F[1][j] + F[2][i] * F[2][j];
            const double G = 0.5 * (i == j ? c - 1.0 : c);
            g2 += G * G;
            if (i == j) tr += G;
        }
    return fabs(det) * (1.0 / 6.0) * (mu * g2 + 0.5 * lam * tr * tr);
}

// Block sum in a fixed order: warp trees, then warp 0 over the warp sums.
__device__ __forceinline__ double block_sum(double v)
{
    __shared__ double s_w[kEnergyThreads / kWarp];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(kFull, v, o);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) s_w[wid] = v;
    __syncthreads();
    double t = 0.0;
    if (wid == 0) {
        t = lane < kEnergyThreads / kWarp ? s_w[lane] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(kFull, t, o);
    }
    return t;   // valid in thread 0
}

__global__ void __launch_bounds__(kEnergyThreads) energy_kernel(
    int32_t n, int64_t nt, const int32_t *__restrict__ tets, const double *__restrict__ Xr,
    const double *__restrict__ x0, const double *__restrict__ d, double alpha, Shift shift,
    const double *__restrict__ E, double nu, const double *__restrict__ mass_h2, const double *__restrict__ g_extra,
    double *__restrict__ x_out, double *part, unsigned *ticket, double *energy, uint32_t *status)
{
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    double acc = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += stride) {
        double in = 0.0, lin = 0.0;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const double xi = trial(x0, d, alpha, 3 * i + c);
            if (x_out) x_out[3 * i + c] = xi;
            const double r = xi - (Xr[3 * i + c] + shift.v[c]);
            in += r * r;
            if (g_extra) lin += g_extra[3 * i + c] * xi;
        }
        acc += 0.5 * mass_h2[i] * in + lin;
    }
    const double mu_per_E = 1.0 / (2.0 * (1.0 + nu));
    const double lam_per_E = nu / ((1.0 + nu) * (1.0 - 2.0 * nu));
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nt; e += stride) {
        int vid[4];
        bool ok = true;
#pragma unroll
        for (int a = 0; a < 4; ++a) {
            vid[a] = tets[4 * e + a];
            ok = ok && (unsigned)vid[a] < (unsigned)n;
        }
        if (!ok) {
            set_status(status, ST_BAD_INDEX);
            continue;
        }
        double X[4][3], x[4][3];
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                X[a][c] = Xr[3 * (int64_t)vid[a] + c];
                x[a][c] = trial(x0, d, alpha, 3 * (int64_t)vid[a] + c);
            }
        const double Ee = E[e];
        acc += tet_psi(X, x, Ee * mu_per_E, Ee * lam_per_E);
    }
    const double bsum = block_sum(acc);
    __shared__ bool s_last;
    if (threadIdx.x == 0) {
        part[blockIdx.x] = bsum;
        __threadfence();
        s_last = atomicAdd(ticket, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!s_last || threadIdx.x >= kWarp) return;
    __threadfence();
    // the last CTA: partials in CTA order, lane-strided then a fixed tree
    double t = 0.0;
    for (unsigned b = threadIdx.x; b < gridDim.x; b += kWarp) t += __ldcg(part + b);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(kFull, t, o);
    if (threadIdx.x == 0) {
        *energy = t;
        *ticket = 0u;
    }
}

__global__ void max_abs_kernel(int64_t m, const double *__restrict__ v, unsigned long long *out)
{
    double mx = 0.0;
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < m; k += (int64_t)gridDim.x * blockDim.x)
        mx = fmax(mx, fabs(v[k]));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_down_sync(kFull, mx, o));
    // non-negative doubles order like their bit patterns
    if ((threadIdx.x & 31) == 0) atomicMax(out, (unsigned long long)__double_as_longlong(mx));
}

}  // namespace

extern "C" int agipc_stvk_energy(agipc_ctx *ctx, int32_t n_fine, int64_t n_tets, const int32_t *tets,
                                 const double *X_rest, const double *x0, const double *d, double alpha,
                                 const double *xhat_shift, const double *E, double nu, const double *mass_h2,
                                 const double *g_extra, double *x_out, double *energy_dev)
{
    if (!ctx || n_fine <= 0 || n_fine > ctx->max_n || n_tets < 0 || n_tets > INT32_MAX || !X_rest || !x0 ||
        !xhat_shift || !mass_h2 || !energy_dev || (n_tets > 0 && (!tets || !E)) || !(nu > -1.0 && nu < 0.5) ||
        !isfinite(alpha) || (x_out && (x_out == x0 || x_out == d)))
        return AGIPC_ERR_INVALID_ARG;
    const Shift shift{{xhat_shift[0], xhat_shift[1], xhat_shift[2]}};
    const int64_t work = std::max<int64_t>(n_fine, n_tets);
    const int grid = (int)min64(min64(div_up(work, kEnergyThreads), (int64_t)ctx->num_sms * 4), kRedMaxCtas);
    energy_kernel<<<grid, kEnergyThreads, 0, ctx->stream>>>(n_fine, n_tets, tets, X_rest, x0, d, alpha, shift, E, nu,
                                                            mass_h2, g_extra, x_out, ctx->red_part, ctx->red_ticket,
                                                            energy_dev, ctx->status);
    return cudaPeekAtLastError() == cudaSuccess ? AGIPC_OK : AGIPC_ERR_CUDA;
}

extern "C" int agipc_max_abs(agipc_ctx *ctx, int64_t n, const double *v, double *out_dev)
{
    if (!ctx || n < 0 || (n > 0 && !v) || !out_dev) return AGIPC_ERR_INVALID_ARG;
    if (cudaMemsetAsync(out_dev, 0, sizeof(double), ctx->stream) != cudaSuccess) return AGIPC_ERR_CUDA;
    if (n > 0) {
        const int tb = 256;
        max_abs_kernel<<<(unsigned)min64(div_up(n, tb), (int64_t)ctx->num_sms * 8), tb, 0, ctx->stream>>>(
            n, v, reinterpret_cast<unsigned long long *>(out_dev));
    }
    return cudaPeekAtLastError() == cudaSuccess ? AGIPC_OK : AGIPC_ERR_CUDA;
}
