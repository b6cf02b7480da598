// Device-wide exclusive prefix sum of int32 values: tile reduce, scan of the
// tile totals in one CTA, then a tile-local scan plus the tile's offset.
#include "agipc_common.cuh"

namespace {

__device__ __forceinline__ int block_excl_scan(int v, int *s_warp, int *s_total)
{
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int nw = blockDim.x >> 5;
    int incl = warp_incl_scan(v);
    if (lane == 31) s_warp[wid] = incl;
    __syncthreads();
    if (wid == 0) {
        int t = lane < nw ? s_warp[lane] : 0;
        int ti = warp_incl_scan(t);
        if (lane < nw) s_warp[lane] = ti - t;
        if (lane == nw - 1) *s_total = ti;
    }
    __syncthreads();
    return incl - v + s_warp[wid];
}

__global__ void __launch_bounds__(kScanBlock) scan_reduce_kernel(const int32_t *__restrict__ in, int64_t n,
                                                                 int32_t *__restrict__ parts)
{
    __shared__ int s_warp[kScanBlock / 32];
    __shared__ int s_total;
    const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
    int sum = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k)
        if (base + k < n) sum += in[base + k];
    block_excl_scan(sum, s_warp, &s_total);
    if (threadIdx.x == 0) parts[blockIdx.x] = s_total;
}

__global__ void __launch_bounds__(1024) scan_parts_kernel(int32_t *__restrict__ parts, int nparts,
                                                          int32_t *__restrict__ out, int64_t n,
                                                          int32_t *__restrict__ total_out)
{
    __shared__ int s_warp[32];
    __shared__ int s_total;
    constexpr int kItems = kScanMaxParts / 1024;
    int v[kItems];
    int sum = 0;
#pragma unroll
    for (int k = 0; k < kItems; ++k) {
        int idx = threadIdx.x * kItems + k;
        v[k] = idx < nparts ? parts[idx] : 0;
        sum += v[k];
    }
    int run = block_excl_scan(sum, s_warp, &s_total);
#pragma unroll
    for (int k = 0; k < kItems; ++k) {
        int idx = threadIdx.x * kItems + k;
        if (idx < nparts) parts[idx] = run;
        run += v[k];
    }
    if (threadIdx.x == 0) {
        out[n] = s_total;
        if (total_out) *total_out = s_total;
    }
}

__global__ void __launch_bounds__(kScanBlock) scan_down_kernel(const int32_t *in, int64_t n,
                                                               const int32_t *__restrict__ parts, int32_t *out)
{
    __shared__ int s_warp[kScanBlock / 32];
    __shared__ int s_total;
    const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
    int v[kScanItems];
    int sum = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        v[k] = base + k < n ? in[base + k] : 0;
        sum += v[k];
    }
    int run = block_excl_scan(sum, s_warp, &s_total) + parts[blockIdx.x];
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        if (base + k < n) out[base + k] = run;
        run += v[k];
    }
}

}  // namespace

bool scan_exclusive_i32(const int32_t *in, int32_t *out, int64_t n, int32_t *total_out, int32_t *parts,
                        cudaStream_t stream)
{
    int64_t nparts = div_up(n > 0 ? n : 1, kScanTile);
    if (nparts > kScanMaxParts) return false;
    scan_reduce_kernel<<<(unsigned)nparts, kScanBlock, 0, stream>>>(in, n, parts);
    scan_parts_kernel<<<1, 1024, 0, stream>>>(parts, (int)nparts, out, n, total_out);
    scan_down_kernel<<<(unsigned)nparts, kScanBlock, 0, stream>>>(in, n, parts, out);
    return true;
}
