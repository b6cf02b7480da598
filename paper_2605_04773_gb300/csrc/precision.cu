// Input split of the precision form: the fine Hessian blocks and the barrier
// stencils are rounded to FP32, except the stencils whose gap is below a
// limit, which stay in FP64 (the precision form keeps barrier terms at small
// gap distances in FP64; the paper itself is all FP64, Sec. 5).  The stencil
// lists keep the input order (a stable compaction), so the coarse assembly
// that follows sums the same terms in the same order on every run.
#include <algorithm>

#include "agipc_common.cuh"

namespace {

__global__ void round_blocks_kernel(int64_t n, const double *__restrict__ v, float *__restrict__ v32)
{
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += stride) v32[k] = (float)v[k];
}

// flag[p] = 1 when stencil p keeps FP64 (its gap is below the limit)
__global__ void gap_flags_kernel(int64_t n_pairs, const double *__restrict__ gap, double limit, int32_t *flag)
{
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n_pairs; p += stride)
        flag[p] = gap[p] < limit ? 1 : 0;
}

// pos[p] = number of FP64 stencils before p (exclusive scan of the flags,
// pos[n_pairs] = their total): stencil p goes to slot pos[p] of the FP64 list
// or slot p - pos[p] of the FP32 list.  One thread per (stencil, value).
__global__ void scatter_pairs_kernel(int64_t n_pairs, const int32_t *__restrict__ pos,
                                     const int32_t *__restrict__ idx, const double *__restrict__ blk,
                                     int32_t *__restrict__ idx32, float *__restrict__ blk32,
                                     int32_t *__restrict__ idx64, double *__restrict__ blk64, int32_t *counts)
{
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t total = 90 * n_pairs;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += stride) {
        const int64_t p = e / 90;
        const int j = (int)(e - 90 * p);
        const int64_t q64 = pos[p];
        const bool keep64 = pos[p + 1] != q64;
        if (keep64) {
            blk64[90 * q64 + j] = blk[e];
            if (j < 4) idx64[4 * q64 + j] = idx[4 * p + j];
        } else {
            const int64_t q32 = p - q64;
            blk32[90 * q32 + j] = (float)blk[e];
            if (j < 4) idx32[4 * q32 + j] = idx[4 * p + j];
        }
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        counts[1] = pos[n_pairs];
        counts[0] = (int32_t)(n_pairs - pos[n_pairs]);
    }
}

}  // namespace

extern "C" int agipc_precision_split(agipc_ctx *ctx, int64_t fine_nnzb, const double *val, float *val32,
                                     int64_t n_pairs, const int32_t *pair_idx, const double *pair_blk,
                                     const double *pair_gap, double gap_limit, int32_t *pair_idx32,
                                     float *pair_blk32, int32_t *pair_idx64, double *pair_blk64, int32_t *counts_dev)
{
    if (!ctx || fine_nnzb < 0 || fine_nnzb > ctx->max_fine_nnzb || n_pairs < 0 || n_pairs > ctx->max_pairs ||
        !counts_dev)
        return AGIPC_ERR_INVALID_ARG;
    if ((fine_nnzb > 0 && (!val || !val32)) ||
        (n_pairs > 0 && (!pair_idx || !pair_blk || !pair_gap || !pair_idx32 || !pair_blk32 || !pair_idx64 ||
                         !pair_blk64)))
        return AGIPC_ERR_INVALID_ARG;
    if (!(gap_limit == gap_limit)) return AGIPC_ERR_INVALID_ARG;   // NaN limit
    // the scan needs n_pairs + 1 int32 words; the assembly's key set (at least
    // 1.25 x (fine blocks + 10 x pairs) 64-bit slots) is free before assembly
    if ((n_pairs + 1) > 2 * ctx->hcap) return AGIPC_ERR_INVALID_ARG;
    cudaStream_t st = ctx->stream;
    const int tb = 256;
    const int64_t cap_grid = (int64_t)ctx->num_sms * 16;
    if (fine_nnzb > 0) {
        const unsigned g = (unsigned)std::min<int64_t>(div_up(9 * fine_nnzb, tb), cap_grid);
        round_blocks_kernel<<<g, tb, 0, st>>>(9 * fine_nnzb, val, val32);
    }
    int32_t *pos = reinterpret_cast<int32_t *>(ctx->hkeys);
    if (n_pairs == 0) {
        if (cudaMemsetAsync(counts_dev, 0, 2 * sizeof(int32_t), st) != cudaSuccess) return AGIPC_ERR_CUDA;
        return cudaPeekAtLastError() == cudaSuccess ? AGIPC_OK : AGIPC_ERR_CUDA;
    }
    const unsigned gf = (unsigned)std::min<int64_t>(div_up(n_pairs, tb), cap_grid);
    gap_flags_kernel<<<gf, tb, 0, st>>>(n_pairs, pair_gap, gap_limit, pos);
    if (!scan_exclusive_i32(pos, pos, n_pairs, nullptr, ctx->scan_part, st)) return AGIPC_ERR_INVALID_ARG;
    const unsigned gs = (unsigned)std::min<int64_t>(div_up(90 * n_pairs, tb), cap_grid);
    scatter_pairs_kernel<<<gs, tb, 0, st>>>(n_pairs, pos, pair_idx, pair_blk, pair_idx32, pair_blk32, pair_idx64,
                                            pair_blk64, counts_dev);
    return cudaPeekAtLastError() == cudaSuccess ? AGIPC_OK : AGIPC_ERR_CUDA;
}
