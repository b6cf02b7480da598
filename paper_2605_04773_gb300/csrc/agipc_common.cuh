// Shared device helpers of the GB300 coarsening library: context layout,
// device status bits, memory-order primitives, the bounded grid barrier used
// by the persistent PCG kernel, and a device-wide exclusive scan.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "agipc.h"

// Device status bits, OR-ed by kernels into ctx->status and mapped to the
// public AGIPC_ERR_* codes by agipc_status().
enum : uint32_t {
    ST_BAD_INDEX = 1u,
    ST_CAPACITY = 2u,
    ST_NONFINITE = 4u,
    ST_NOT_CONVERGED = 8u,
    ST_TIMEOUT = 16u,
};

constexpr int kWarp = 32;
constexpr unsigned kFull = 0xffffffffu;
constexpr unsigned long long kEmptyKey = ~0ull;

// Spin budget of every device-side wait: ~seconds on a GB300, far above any
// legitimate wait, far below a hang.
constexpr long long kSpinLimit = 1ll << 22;

struct PcgScratch {
    double *r, *u, *w, *p, *s;  // [3 * max_rows] each
    int32_t *brow;              // [max_nnzb] row of every block
    uint8_t *rowflag;           // [max_rows] bit0: row split across warps, bit1: empty row
    double *partials;           // [2][max_grid][4]
    unsigned *bar;              // [64]: [0] barrier arrivals, [32] bad-input flag (separate lines)
    int max_grid;
};

constexpr int kBatchMaxInst = 512;    // instances of one batched PCG launch
constexpr int kBatchVariants = 4;     // slice widths of the batched PCG (4, 5, 6, 8 blocks per lane)

struct agipc_ctx {
    cudaStream_t stream;
    int device;
    int num_sms;
    int32_t max_n;
    int64_t max_edges, max_fine_nnzb, max_pairs, max_nnzb;

    void *arena;          // one cudaMalloc holding every scratch array below
    size_t arena_bytes;
    uint32_t *status;     // device status word

    // aggregation
    int32_t *parent;      // [max_n]
    uint32_t *ghash;      // [max_n]
    int32_t *rank;        // [max_n + 1]

    // scan
    int32_t *scan_part;   // [kScanMaxParts]

    // assembly
    unsigned long long *hkeys;  // [hcap]
    int64_t hcap;
    int hbits;
    int32_t *row_cnt;     // [max_n + 1]
    int32_t *row_cur;     // [max_n]
    int32_t *fine_brow;   // [max_fine_nnzb]
    int32_t *long_rows;   // [max_n + 1]; [max_n] holds the count
    uint32_t *bitmap;     // [kLongRowCtas][bitmap_words]
    int64_t bitmap_words;
    double *dinv64;       // [max_n][9] FP64 inverses before rounding (precision form)

    PcgScratch pcg;
    int pcg_block;
    int pcg_grid;

    // coarse assembly: terms each lane of the numeric phase folds (4, 8, 16, 32)
    int asm_run;

    // batched PCG
    double *batch_acc;                // [6 * kBatchMaxInst] per-instance sums
    int batch_grid[kBatchVariants];   // cooperative grid of each slice-width variant

    // deterministic reductions (energy): one partial per CTA, then the last
    // CTA to arrive sums them in CTA order
    double *red_part;                 // [kRedMaxCtas]
    unsigned *red_ticket;             // [32]: [0] arrivals (reset by the last CTA)
};

constexpr int kRedMaxCtas = 1024;

// --------------------------------------------------------------------------
// memory-order helpers (gpu scope)
// --------------------------------------------------------------------------
__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned *p)
{
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void set_status(uint32_t *status, uint32_t bit) { atomicOr(status, bit); }

// --------------------------------------------------------------------------
// Grid barrier for a cooperative (co-resident) launch, on a per-launch
// monotone arrival counter (zeroed before the launch): the k-th barrier of a
// CTA waits until k * nblocks CTAs have arrived.  Release = fence.acq_rel +
// relaxed add, acquire = polling load.  The wait is bounded: after
// kSpinLimit polls the CTA records ST_TIMEOUT and the call returns false,
// so the kernel winds down instead of hanging.
// --------------------------------------------------------------------------
__device__ __forceinline__ bool grid_sync(unsigned *count, unsigned nblocks, unsigned &epoch, uint32_t *status)
{
    __shared__ int s_ok;
    __syncthreads();
    ++epoch;
    if (threadIdx.x == 0) {
        asm volatile("fence.acq_rel.gpu;" ::: "memory");
        asm volatile("red.relaxed.gpu.global.add.u32 [%0], %1;" ::"l"(count), "r"(1u) : "memory");
        const unsigned target = epoch * nblocks;
        int ok = 1;
        long long spins = 0;
        while ((int)(ld_acquire_u32(count) - target) < 0) {
            if (++spins > kSpinLimit) {
                set_status(status, ST_TIMEOUT);
                ok = 0;
                break;
            }
        }
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

// --------------------------------------------------------------------------
// warp / block reductions
// --------------------------------------------------------------------------
__device__ __forceinline__ double warp_sum(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
    return v;
}

__device__ __forceinline__ int warp_incl_scan(int v)
{
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int t = __shfl_up_sync(kFull, v, o);
        if (lane >= o) v += t;
    }
    return v;
}

// --------------------------------------------------------------------------
// Device-wide exclusive scan of int32 (three passes; sizes up to
// kScanTile * kScanMaxParts elements).
// --------------------------------------------------------------------------
constexpr int kScanBlock = 512;
constexpr int kScanItems = 8;
constexpr int kScanTile = kScanBlock * kScanItems;  // 4096
constexpr int kScanMaxParts = 8192;                 // 33.5M elements

// Enqueue out[i] = sum_{k<i} in[k] for i in [0, n]; out[n] = total.  `in`
// and `out` may alias.  If total_out is non-null the total is copied there.
// Returns false when n exceeds the supported size.
bool scan_exclusive_i32(const int32_t *in, int32_t *out, int64_t n, int32_t *total_out, int32_t *parts,
                        cudaStream_t stream);

// Rounded-up integer division and 64-bit min/max, for host and device code.
__host__ __device__ __forceinline__ int64_t div_up(int64_t a, int64_t b) { return (a + b - 1) / b; }
__host__ __device__ __forceinline__ int64_t min64(int64_t a, int64_t b) { return a < b ? a : b; }
__host__ __device__ __forceinline__ int64_t max64(int64_t a, int64_t b) { return a > b ? a : b; }
