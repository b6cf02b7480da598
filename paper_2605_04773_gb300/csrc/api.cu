// Context management, status reporting and the prolongation dx = U^T y
// (Sec. 4.3) of the GB300 coarsening library.
#include <algorithm>
#include <cstdlib>
#include <new>

#include "agipc_common.cuh"

int pcg_block_size();
int pcg_smem_bytes();
const void *pcg_kernel_ptr();
const void *pcg_mixed_kernel_ptr();
bool pcg_mixed_wide_configure();
bool pcg_wide_configure();
int assemble_long_row_ctas();
bool batched_configure(agipc_ctx *c);

namespace {

struct Carve {
    char *base;
    size_t off;
    template <class T>
    T *take(size_t count)
    {
        off = (off + 255) & ~size_t(255);
        T *p = base ? reinterpret_cast<T *>(base + off) : nullptr;
        off += sizeof(T) * (count > 0 ? count : 1);
        return p;
    }
};

void carve_all(agipc_ctx *c, char *base, size_t *total)
{
    Carve cv{base, 0};
    const size_t n = (size_t)c->max_n;
    c->status = cv.take<uint32_t>(1);
    c->parent = cv.take<int32_t>(n);
    c->ghash = cv.take<uint32_t>(n);
    c->rank = cv.take<int32_t>(n + 1);
    c->scan_part = cv.take<int32_t>(kScanMaxParts);
    c->hkeys = cv.take<unsigned long long>((size_t)c->hcap);
    c->row_cnt = cv.take<int32_t>(n + 1);
    c->row_cur = cv.take<int32_t>(n);
    c->fine_brow = cv.take<int32_t>((size_t)c->max_fine_nnzb);
    c->long_rows = cv.take<int32_t>(n + 1);
    c->bitmap = cv.take<uint32_t>((size_t)assemble_long_row_ctas() * (size_t)c->bitmap_words);
    c->dinv64 = cv.take<double>(9 * n);
    c->pcg.r = cv.take<double>(3 * n);
    c->pcg.u = cv.take<double>(3 * n);
    c->pcg.w = cv.take<double>(3 * n);
    c->pcg.p = cv.take<double>(3 * n);
    c->pcg.s = cv.take<double>(3 * n);
    c->pcg.brow = cv.take<int32_t>((size_t)c->max_nnzb);
    c->pcg.rowflag = cv.take<uint8_t>(n);
    c->pcg.partials = cv.take<double>(2 * (size_t)c->pcg.max_grid * 4);
    c->pcg.bar = cv.take<unsigned>(64);
    c->batch_acc = cv.take<double>(6 * (size_t)kBatchMaxInst);
    c->red_part = cv.take<double>(kRedMaxCtas);
    c->red_ticket = cv.take<unsigned>(32);
    *total = cv.off;
}

__global__ void prolongate_kernel(int32_t n, const int32_t *__restrict__ labels, const double *__restrict__ y,
                                  const double *__restrict__ base, double *__restrict__ dx, uint32_t *status)
{
    const int64_t m = 3 * (int64_t)n;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < m; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t f = e / 3;
        const int c = (int)(e - 3 * f);
        const int32_t lab = labels[f];
        if ((unsigned)lab >= (unsigned)n) {
            if (c == 0) set_status(status, ST_BAD_INDEX);
            dx[e] = 0.0;
            continue;
        }
        const double v = y[3 * (int64_t)lab + c];
        dx[e] = base ? base[e] + v : v;
    }
}

}  // namespace

extern "C" int agipc_create(agipc_ctx **out, void *cuda_stream, int32_t max_fine_nodes, int64_t max_edges,
                            int64_t max_fine_nnzb, int64_t max_pairs)
{
    if (!out) return AGIPC_ERR_INVALID_ARG;
    *out = nullptr;
    if (max_fine_nodes < 0 || max_edges < 0 || max_fine_nnzb < 0 || max_pairs < 0) return AGIPC_ERR_INVALID_ARG;
    const int64_t max_nnzb = 2 * max_fine_nnzb + 16 * max_pairs;
    if (max_nnzb > INT32_MAX || max_fine_nnzb + 10 * max_pairs > (1ll << 40)) return AGIPC_ERR_INVALID_ARG;
    agipc_ctx *c = new (std::nothrow) agipc_ctx();
    if (!c) return AGIPC_ERR_CUDA;
    c->stream = (cudaStream_t)cuda_stream;
    if (cudaGetDevice(&c->device) != cudaSuccess ||
        cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, c->device) != cudaSuccess) {
        delete c;
        return AGIPC_ERR_CUDA;
    }
    c->max_n = max_fine_nodes;
    c->max_edges = max_edges;
    c->max_fine_nnzb = max_fine_nnzb;
    c->max_pairs = max_pairs;
    c->max_nnzb = max_nnzb;
    const int64_t terms = max_fine_nnzb + 10 * max_pairs;
    c->hbits = 10;
    while ((1ll << c->hbits) < terms + terms / 4) ++c->hbits;
    c->hcap = 1ll << c->hbits;
    c->bitmap_words = div_up(std::max<int64_t>(max_fine_nodes, 1), 32);

    // Persistent PCG: as many co-resident CTAs as the occupancy allows, capped
    // at two per SM (the grid barrier's cost grows with the CTA count).
    int per_sm = 0;
    int per_sm_mixed = 0;
    if (cudaFuncSetAttribute(pcg_mixed_kernel_ptr(), cudaFuncAttributeMaxDynamicSharedMemorySize, pcg_smem_bytes()) !=
            cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm_mixed, pcg_mixed_kernel_ptr(), pcg_block_size(),
                                                      pcg_smem_bytes()) != cudaSuccess ||
        per_sm_mixed < 1) {
        delete c;
        return AGIPC_ERR_CUDA;
    }
    if (cudaFuncSetAttribute(pcg_kernel_ptr(), cudaFuncAttributeMaxDynamicSharedMemorySize, pcg_smem_bytes()) !=
            cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, pcg_kernel_ptr(), pcg_block_size(), pcg_smem_bytes()) !=
            cudaSuccess ||
        per_sm < 1) {
        delete c;
        return AGIPC_ERR_CUDA;
    }
    int cap_per_sm = 2;
    if (const char *env = std::getenv("AGIPC_PCG_CTAS_PER_SM")) cap_per_sm = std::max(1, std::atoi(env));
    c->pcg_block = pcg_block_size();
    c->asm_run = 32;
    c->pcg_grid = std::min(std::min(per_sm, per_sm_mixed), cap_per_sm) * c->num_sms;
    c->pcg.max_grid = c->pcg_grid;
    if (c->num_sms > c->pcg.max_grid || !pcg_wide_configure() || !pcg_mixed_wide_configure() ||
        !batched_configure(c)) {
        delete c;
        return AGIPC_ERR_CUDA;
    }

    size_t bytes = 0;
    carve_all(c, nullptr, &bytes);
    if (cudaMalloc(&c->arena, bytes) != cudaSuccess) {
        delete c;
        return AGIPC_ERR_CUDA;
    }
    c->arena_bytes = bytes;
    carve_all(c, static_cast<char *>(c->arena), &bytes);
    if (cudaMemsetAsync(c->arena, 0, bytes, c->stream) != cudaSuccess || cudaStreamSynchronize(c->stream) != cudaSuccess) {
        cudaFree(c->arena);
        delete c;
        return AGIPC_ERR_CUDA;
    }
    *out = c;
    return AGIPC_OK;
}

extern "C" int agipc_destroy(agipc_ctx *ctx)
{
    if (!ctx) return AGIPC_ERR_INVALID_ARG;
    int rc = AGIPC_OK;
    if (cudaStreamSynchronize(ctx->stream) != cudaSuccess) rc = AGIPC_ERR_CUDA;
    if (cudaFree(ctx->arena) != cudaSuccess) rc = AGIPC_ERR_CUDA;
    delete ctx;
    return rc;
}

extern "C" int agipc_set_stream(agipc_ctx *ctx, void *cuda_stream)
{
    if (!ctx) return AGIPC_ERR_INVALID_ARG;
    ctx->stream = (cudaStream_t)cuda_stream;
    return AGIPC_OK;
}

extern "C" int agipc_set_assembly_run(agipc_ctx *ctx, int32_t terms_per_lane)
{
    if (!ctx || (terms_per_lane != 4 && terms_per_lane != 8 && terms_per_lane != 16 && terms_per_lane != 32)) return AGIPC_ERR_INVALID_ARG;
    ctx->asm_run = terms_per_lane;
    return AGIPC_OK;
}

extern "C" int agipc_status(agipc_ctx *ctx)
{
    if (!ctx) return AGIPC_ERR_INVALID_ARG;
    uint32_t bits = 0;
    if (cudaMemcpyAsync(&bits, ctx->status, sizeof(bits), cudaMemcpyDeviceToHost, ctx->stream) != cudaSuccess ||
        cudaMemsetAsync(ctx->status, 0, sizeof(uint32_t), ctx->stream) != cudaSuccess ||
        cudaStreamSynchronize(ctx->stream) != cudaSuccess)
        return AGIPC_ERR_CUDA;
    if (bits & ST_TIMEOUT) return AGIPC_ERR_TIMEOUT;
    if (bits & ST_BAD_INDEX) return AGIPC_ERR_BAD_INDEX;
    if (bits & ST_CAPACITY) return AGIPC_ERR_CAPACITY;
    if (bits & ST_NONFINITE) return AGIPC_ERR_NONFINITE;
    if (bits & ST_NOT_CONVERGED) return AGIPC_ERR_NOT_CONVERGED;
    return AGIPC_OK;
}

extern "C" const char *agipc_status_string(int status)
{
    switch (status) {
    case AGIPC_OK: return "ok";
    case AGIPC_ERR_INVALID_ARG: return "invalid argument";
    case AGIPC_ERR_CUDA: return "CUDA runtime error";
    case AGIPC_ERR_CAPACITY: return "output capacity exceeded";
    case AGIPC_ERR_NONFINITE: return "non-finite value or singular diagonal block";
    case AGIPC_ERR_NOT_CONVERGED: return "PCG did not converge within max_iter";
    case AGIPC_ERR_TIMEOUT: return "bounded device wait timed out";
    case AGIPC_ERR_BAD_INDEX: return "index out of range";
    default: return "unknown status";
    }
}

extern "C" int agipc_prolongate(agipc_ctx *ctx, int32_t n_fine, const int32_t *labels, const double *y, double *dx)
{
    if (!ctx || n_fine < 0 || n_fine > ctx->max_n || (n_fine > 0 && (!labels || !y || !dx))) return AGIPC_ERR_INVALID_ARG;
    if (n_fine == 0) return AGIPC_OK;
    const int tb = 256;
    const int64_t m = 3 * (int64_t)n_fine;
    const unsigned grid = (unsigned)std::min<int64_t>(div_up(m, tb), (int64_t)ctx->num_sms * 32);
    prolongate_kernel<<<grid, tb, 0, ctx->stream>>>(n_fine, labels, y, nullptr, dx, ctx->status);
    return cudaPeekAtLastError() == cudaSuccess ? AGIPC_OK : AGIPC_ERR_CUDA;
}

extern "C" int agipc_prolongate_add(agipc_ctx *ctx, int32_t n_fine, const int32_t *labels, const double *y,
                                    const double *base, double *out)
{
    if (!ctx || n_fine < 0 || n_fine > ctx->max_n || (n_fine > 0 && (!labels || !y || !base || !out)))
        return AGIPC_ERR_INVALID_ARG;
    if (n_fine == 0) return AGIPC_OK;
    const int tb = 256;
    const int64_t m = 3 * (int64_t)n_fine;
    const unsigned grid = (unsigned)std::min<int64_t>(div_up(m, tb), (int64_t)ctx->num_sms * 32);
    prolongate_kernel<<<grid, tb, 0, ctx->stream>>>(n_fine, labels, y, base, out, ctx->status);
    return cudaPeekAtLastError() == cudaSuccess ? AGIPC_OK : AGIPC_ERR_CUDA;
}
