// Super-node labeller (Sec. 4.1; supplement Sec. 1, Algorithms 1-2).
//
// Result: labels[f] = rank of the smallest fine index in f's connected
// component of the collapsible-edge graph.  This is the fixed point that the
// paper's recursive group hashing reaches when it is repeated until no merge
// is left (supplement Sec. 1.2-1.3), numbered in the supplement's order of
// coarse indices (first set bit of the hash, prefix sum over groups).
//
// GB300 design (the paper's per-level recursion is replaced by one global
// pass, so a super-node that spans many groups costs no extra levels):
//   1. group hashes: every node of a 32-node group starts with its own lane
//      bit; each collapsible edge inside a group ORs the other endpoint's bit
//      into both endpoints (Algorithm 1).
//   2. one warp per group closes the hashes transitively with shuffles
//      (Algorithm 2's OR-propagation) and elects the first set bit of the
//      shared hash as the local root (__match_any_sync groups the lanes that
//      hold identical hashes).  parent[v] = that local root <= v.
//   3. cross-group collapsible edges are merged by a lock-free union-find that
//      always hooks the larger root under the smaller one, so every
//      component's final root is its minimum index whatever the order.
//   4. full path compression, root flags, exclusive scan, relabel.
#include "agipc_common.cuh"

namespace {

__global__ void agg_init_kernel(int32_t n, uint32_t *__restrict__ ghash)
{
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x)
        ghash[v] = 1u << (v & 31);
}

// Algorithm 1: direct-neighbour bits of collapsible edges inside a group.
__global__ void agg_group_edges_kernel(int32_t n, int64_t n_edges, const int32_t *__restrict__ edges,
                                       const uint8_t *__restrict__ tags, uint32_t *__restrict__ ghash,
                                       uint32_t *status)
{
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n_edges;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int2 uv = reinterpret_cast<const int2 *>(edges)[e];
        const int u = uv.x, v = uv.y;
        if ((unsigned)u >= (unsigned)n || (unsigned)v >= (unsigned)n) {
            set_status(status, ST_BAD_INDEX);
            continue;
        }
        if (!tags[e] || u == v || (u >> 5) != (v >> 5)) continue;
        atomicOr(&ghash[u], 1u << (v & 31));
        atomicOr(&ghash[v], 1u << (u & 31));
    }
}

// Algorithm 2: transitive closure of the group hashes and leader election.
__global__ void agg_group_close_kernel(int32_t n, const uint32_t *__restrict__ ghash, int32_t *__restrict__ parent)
{
    const int lane = threadIdx.x & 31;
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t grp = warp; grp * 32 < n; grp += nwarps) {
        const int64_t v = grp * 32 + lane;
        const bool valid = v < n;
        uint32_t h = valid ? ghash[v] : 0u;
        // OR in the hash of every member already known; each round doubles
        // the path length covered, so 5 rounds close any 32-node group.
        for (int round = 0; round < 5; ++round) {
            uint32_t acc = h;
#pragma unroll
            for (int j = 0; j < 32; ++j) {
                uint32_t hj = __shfl_sync(kFull, h, j);
                if ((h >> j) & 1u) acc |= hj;
            }
            bool changed = acc != h;
            h = acc;
            if (!__any_sync(kFull, changed)) break;
        }
        // Lanes of one component now hold the same hash; its first set bit is
        // the component's smallest member inside the group.
        // __match_any_sync gathers the lanes holding the same final hash
        // (one coarse node each); the lowest of them is the local root.
        const uint32_t same = __match_any_sync(kFull, h);
        const int leader = __ffs(same) - 1;
        if (valid) parent[v] = (int32_t)(grp * 32 + leader);
    }
}

__device__ __forceinline__ int32_t uf_root(int32_t *parent, int32_t v)
{
    int32_t p = __ldcg(parent + v);
    while (p != v) {
        int32_t gp = __ldcg(parent + p);
        if (gp != p) __stcg(parent + v, gp);  // path halving; v is not a root
        v = p;
        p = gp;
    }
    return v;
}

// Cross-group collapsible edges: lock-free hooking of the larger root under
// the smaller one.  A failed CAS means another thread hooked that root, so
// the retries are bounded by the number of hooks; the explicit cap only
// guards against a corrupted parent array.
__global__ void agg_union_kernel(int32_t n, int64_t n_edges, const int32_t *__restrict__ edges,
                                 const uint8_t *__restrict__ tags, int32_t *parent, uint32_t *status)
{
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n_edges;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int2 uv = reinterpret_cast<const int2 *>(edges)[e];
        int u = uv.x, v = uv.y;
        if ((unsigned)u >= (unsigned)n || (unsigned)v >= (unsigned)n) continue;
        if (!tags[e] || (u >> 5) == (v >> 5)) continue;
        bool done = false;
        for (long long it = 0; it < kSpinLimit; ++it) {
            u = uf_root(parent, u);
            v = uf_root(parent, v);
            if (u == v) { done = true; break; }
            const int hi = u > v ? u : v, lo = u > v ? v : u;
            if (atomicCAS(parent + hi, hi, lo) == hi) { done = true; break; }
        }
        if (!done) set_status(status, ST_TIMEOUT);
    }
}

__global__ void agg_compress_kernel(int32_t n, int32_t *parent, int32_t *__restrict__ flag)
{
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
        int32_t r = uf_root(parent, (int32_t)v);
        __stcg(parent + v, r);
        flag[v] = (r == v) ? 1 : 0;
    }
}

__global__ void agg_relabel_kernel(int32_t n, const int32_t *parent, const int32_t *__restrict__ rank,
                                   int32_t *__restrict__ labels)
{
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
        int32_t r = v;
        // after compression every node points at its root directly; follow
        // defensively in case a halving write landed after the compression
        int32_t p = parent[r];
        while (p != r) { r = p; p = parent[r]; }
        labels[v] = rank[r];
    }
}

}  // namespace

extern "C" int agipc_aggregate(agipc_ctx *ctx, int32_t n_fine, int64_t n_edges, const int32_t *edges,
                               const uint8_t *tags, int32_t *labels, int32_t *n_coarse_dev)
{
    if (!ctx || n_fine < 0 || n_edges < 0 || n_fine > ctx->max_n || n_edges > ctx->max_edges) return AGIPC_ERR_INVALID_ARG;
    if ((n_fine > 0 && !labels) || !n_coarse_dev || (n_edges > 0 && (!edges || !tags))) return AGIPC_ERR_INVALID_ARG;
    if (((uintptr_t)edges & 7u) != 0) return AGIPC_ERR_INVALID_ARG;
    cudaStream_t st = ctx->stream;
    if (n_fine == 0) {
        if (cudaMemsetAsync(n_coarse_dev, 0, sizeof(int32_t), st) != cudaSuccess) return AGIPC_ERR_CUDA;
        return AGIPC_OK;
    }
    const int tb = 256;
    const unsigned gn = (unsigned)div_up(n_fine, tb);
    const unsigned ge = (unsigned)(n_edges > 0 ? div_up(n_edges, tb) : 1);
    const unsigned gg = (unsigned)div_up(div_up(n_fine, 32) * 32, tb);
    agg_init_kernel<<<gn, tb, 0, st>>>(n_fine, ctx->ghash);
    if (n_edges > 0) agg_group_edges_kernel<<<ge, tb, 0, st>>>(n_fine, n_edges, edges, tags, ctx->ghash, ctx->status);
    agg_group_close_kernel<<<gg, tb, 0, st>>>(n_fine, ctx->ghash, ctx->parent);
    if (n_edges > 0) agg_union_kernel<<<ge, tb, 0, st>>>(n_fine, n_edges, edges, tags, ctx->parent, ctx->status);
    agg_compress_kernel<<<gn, tb, 0, st>>>(n_fine, ctx->parent, ctx->rank);
    if (!scan_exclusive_i32(ctx->rank, ctx->rank, n_fine, n_coarse_dev, ctx->scan_part, st)) return AGIPC_ERR_INVALID_ARG;
    agg_relabel_kernel<<<gn, tb, 0, st>>>(n_fine, ctx->parent, ctx->rank, labels);
    return cudaPeekAtLastError() == cudaSuccess ? AGIPC_OK : AGIPC_ERR_CUDA;
}

// ---------------------------------------------------------------------------
// agipc_aggregate_static: the labeller for callers that cannot allocate GPU
// memory.  Its scratch lives in a fixed array in the library's device image
// instead of an agipc_ctx arena (whose creation calls cudaMalloc).
// ---------------------------------------------------------------------------
#include <mutex>

namespace {

constexpr int64_t kStaticAggNodes = AGIPC_AGGREGATE_STATIC_MAX_NODES;
// parent [N] + group hashes [N] + ranks [N + 1] + scan partials, in 32-bit words
constexpr int64_t kStaticAggWords = 3 * kStaticAggNodes + 1 + kScanMaxParts;

// Every GPU that loads the library holds this array (about 12 MiB) until the
// process exits.  Host code must not take its address directly: on the host
// the name is only a stand-in, so the device address comes from
// cudaGetSymbolAddress.
static __device__ __align__(256) int32_t g_static_agg_scratch[kStaticAggWords];

std::mutex g_static_agg_mutex;
int32_t *g_static_agg_ptr[256];  // device address of the array, per device

}  // namespace

extern "C" int agipc_aggregate_static(void *cuda_stream, int32_t n_fine, int64_t n_edges, const int32_t *edges,
                                      const uint8_t *tags, int32_t *labels, int32_t *n_coarse_dev,
                                      uint32_t *status_dev)
{
    if (n_fine < 0 || n_edges < 0 || n_fine > kStaticAggNodes) return AGIPC_ERR_INVALID_ARG;
    if ((n_fine > 0 && !labels) || !n_coarse_dev || !status_dev || (n_edges > 0 && (!edges || !tags)))
        return AGIPC_ERR_INVALID_ARG;
    if (((uintptr_t)edges & 7u) != 0) return AGIPC_ERR_INVALID_ARG;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 256) return AGIPC_ERR_CUDA;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    cudaStreamCaptureStatus capture = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st, &capture) != cudaSuccess) return AGIPC_ERR_CUDA;
    int32_t *scratch = nullptr;
    {
        // Outside capture the address is looked up afresh (a device reset
        // reloads the array elsewhere); under capture the last one is reused,
        // since the lookup may load the module, which capture forbids.
        std::lock_guard<std::mutex> lock(g_static_agg_mutex);
        if (capture == cudaStreamCaptureStatusNone || !g_static_agg_ptr[dev]) {
            if (capture != cudaStreamCaptureStatusNone) return AGIPC_ERR_CUDA;
            void *p = nullptr;
            if (cudaGetSymbolAddress(&p, g_static_agg_scratch) != cudaSuccess || !p) return AGIPC_ERR_CUDA;
            g_static_agg_ptr[dev] = static_cast<int32_t *>(p);
        }
        scratch = g_static_agg_ptr[dev];
    }
    int32_t *parent = scratch;
    uint32_t *ghash = reinterpret_cast<uint32_t *>(scratch + kStaticAggNodes);
    int32_t *rank = scratch + 2 * kStaticAggNodes;
    int32_t *parts = scratch + 3 * kStaticAggNodes + 1;
    // The array keeps the previous call's contents; every word this call
    // reads is written by this call first, and the status starts at zero.
    if (cudaMemsetAsync(status_dev, 0, sizeof(uint32_t), st) != cudaSuccess) return AGIPC_ERR_CUDA;
    if (n_fine == 0) {
        if (cudaMemsetAsync(n_coarse_dev, 0, sizeof(int32_t), st) != cudaSuccess) return AGIPC_ERR_CUDA;
        return AGIPC_OK;
    }
    const int tb = 256;
    const unsigned gn = (unsigned)div_up(n_fine, tb);
    const unsigned ge = (unsigned)(n_edges > 0 ? div_up(n_edges, tb) : 1);
    const unsigned gg = (unsigned)div_up(div_up(n_fine, 32) * 32, tb);
    agg_init_kernel<<<gn, tb, 0, st>>>(n_fine, ghash);
    if (n_edges > 0) agg_group_edges_kernel<<<ge, tb, 0, st>>>(n_fine, n_edges, edges, tags, ghash, status_dev);
    agg_group_close_kernel<<<gg, tb, 0, st>>>(n_fine, ghash, parent);
    if (n_edges > 0) agg_union_kernel<<<ge, tb, 0, st>>>(n_fine, n_edges, edges, tags, parent, status_dev);
    agg_compress_kernel<<<gn, tb, 0, st>>>(n_fine, parent, rank);
    if (!scan_exclusive_i32(rank, rank, n_fine, n_coarse_dev, parts, st)) return AGIPC_ERR_INVALID_ARG;
    agg_relabel_kernel<<<gn, tb, 0, st>>>(n_fine, parent, rank, labels);
    return cudaPeekAtLastError() == cudaSuccess ? AGIPC_OK : AGIPC_ERR_CUDA;
}
