// Coarse system assembly (Sec. 4.1; supplement Sec. 2): g_c = U g and
// H_c = U H U^T for the aggregation operator U of the labels.
//
// Every fine term - a stored upper block (i, j) of H or one of the 10 upper
// blocks of a barrier stencil - lands in the coarse upper block
// (min(a, b), max(a, b)) with (a, b) = (map i, map j):
//     a <  b : B,        a > b : B^T,
//     a == b : B + B^T for an off-diagonal source (i != j), B for a diagonal one,
// because a fine upper block (i, j), i != j, also stands for B^T at (j, i).
// The lower triangle of H_c is the transpose of the upper one, so the output
// is exactly symmetric.
//
// GB300 design (a sorted-key segmented reduction without a global sort):
//   1. symbolic: the distinct coarse keys go into an open-addressing hash set
//      (64-bit key (lo << 32) | hi, linear probing, CAS insert).  A warp first
//      merges equal keys with __match_any_sync so each key is inserted once
//      per warp; a fresh insert bumps the row counts of both coarse rows.
//   2. exclusive scan of the row counts -> coarse row_ptr.
//   3. the set's keys are scattered into their rows and every row is sorted
//      (warp bitonic sort for rows <= 32 blocks, shared-memory bitonic sort
//      up to 8192, a column bitmap beyond).
//   4. numeric: lanes fold runs of consecutive terms with the same coarse key
//      (the interior of a super-node) in registers and add each run to its
//      upper position (binary search in the sorted row) with FP64 atomics,
//      which execute in the L2; warps whose lanes all end on one key reduce
//      it with shuffles first.  FP64 is slow on the SM of this part, so the
//      SM only adds where a key repeats.
//   5. the lower triangle is written as transposes; the diagonal blocks are
//      symmetrised and inverted (thread per row) for the block-Jacobi
//      preconditioner.
//   6. g_c by atomics with the same warp merge.
#include <algorithm>

#include "agipc_common.cuh"

namespace {

constexpr int kTb = 256;
constexpr int kLongSmem = 8192;  // entries sorted in shared memory per long row
constexpr int kLongRowCtas = 64;

__constant__ int8_t c_stencil_s[10] = {0, 0, 0, 0, 1, 1, 1, 2, 2, 3};
__constant__ int8_t c_stencil_t[10] = {0, 1, 2, 3, 1, 2, 3, 2, 3, 3};

__device__ __forceinline__ unsigned long long pack_key(int32_t lo, int32_t hi)
{
    return ((unsigned long long)(uint32_t)lo << 32) | (uint32_t)hi;
}

__device__ __forceinline__ int64_t slot_of(unsigned long long key, int bits)
{
    return (int64_t)((key * 0x9E3779B97F4A7C15ull) >> (64 - bits));
}

// Sources of terms: fine upper blocks (FP64 or FP32), barrier stencils
// (FP64 or FP32) and, for the precision form, a second list of stencils kept
// in FP64 (small gaps).  Term t indexes them in that order.
struct TermArgs {
    int32_t n;
    const int32_t *labels;
    const int32_t *n_c_dev;
    const int32_t *fine_brow;
    const int32_t *fine_col;
    const double *fine_val;
    const float *fine_val32;  // used when fine_val is null
    int64_t fine_nnzb;
    const int32_t *pair_idx;
    const double *pair_blk;
    const float *pair_blk32;  // used when pair_blk is null
    int64_t n_pairs;
    const int32_t *pair_idx2;
    const double *pair_blk2;
    int64_t n_pairs2;
    int64_t n_terms;
};

// Coarse (row label, column label) of term t and whether its source block is
// off-diagonal; false when an index is out of range.  `src` is the offset of
// the term's 9 values in its array and `kind` which array: 0 fine FP64,
// 1 fine FP32, 2 stencil FP64, 3 stencil FP32, 4 second stencil list (FP64).
__device__ __forceinline__ bool term_labels(const TermArgs &A, int64_t t, int32_t nc, int32_t &a, int32_t &b,
                                            bool &offdiag, int64_t &src, int &kind)
{
    int32_t vi, vj;
    if (t < A.fine_nnzb) {
        vi = A.fine_brow[t];
        vj = A.fine_col[t];
        offdiag = vi != vj;
        src = 9 * t;
        kind = A.fine_val ? 0 : 1;
        if ((unsigned)vi >= (unsigned)A.n || (unsigned)vj >= (unsigned)A.n || vj < vi) return false;
    } else {
        int64_t u = t - A.fine_nnzb;
        const int32_t *idx;
        if (u < 10 * A.n_pairs) {
            idx = A.pair_idx;
            kind = A.pair_blk ? 2 : 3;
        } else {
            u -= 10 * A.n_pairs;
            idx = A.pair_idx2;
            kind = 4;
        }
        const int64_t p = u / 10;
        const int q = (int)(u - 10 * p);
        vi = idx[4 * p + c_stencil_s[q]];
        vj = idx[4 * p + c_stencil_t[q]];
        offdiag = c_stencil_s[q] != c_stencil_t[q];
        src = 90 * p + 9 * q;
        if ((unsigned)vi >= (unsigned)A.n || (unsigned)vj >= (unsigned)A.n) return false;
    }
    a = A.labels[vi];
    b = A.labels[vj];
    return (unsigned)a < (unsigned)nc && (unsigned)b < (unsigned)nc;
}

__device__ __forceinline__ void load_term(const TermArgs &A, int64_t src, int kind, double B[9])
{
    switch (kind) {
    case 0:
#pragma unroll
        for (int e = 0; e < 9; ++e) B[e] = __ldg(A.fine_val + src + e);
        break;
    case 1:
#pragma unroll
        for (int e = 0; e < 9; ++e) B[e] = (double)__ldg(A.fine_val32 + src + e);
        break;
    case 2:
#pragma unroll
        for (int e = 0; e < 9; ++e) B[e] = __ldg(A.pair_blk + src + e);
        break;
    case 3:
#pragma unroll
        for (int e = 0; e < 9; ++e) B[e] = (double)__ldg(A.pair_blk32 + src + e);
        break;
    default:
#pragma unroll
        for (int e = 0; e < 9; ++e) B[e] = __ldg(A.pair_blk2 + src + e);
        break;
    }
}

__global__ void fine_rows_kernel(int32_t n, const int32_t *__restrict__ rp, int64_t nnzb, int32_t *__restrict__ brow,
                                 uint32_t *status)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int32_t k0 = rp[i], k1 = rp[i + 1];
        if (k0 < 0 || k1 < k0 || k1 > nnzb || (i == 0 && k0 != 0) || (i == n - 1 && k1 != nnzb)) {
            set_status(status, ST_BAD_INDEX);
            continue;
        }
        for (int32_t k = k0; k < k1; ++k) brow[k] = (int32_t)i;
    }
}

// Insert key; true when this call created it.
__device__ __forceinline__ bool hash_insert(unsigned long long *keys, int bits, unsigned long long key, uint32_t *status)
{
    const int64_t mask = (1ll << bits) - 1;
    int64_t h = slot_of(key, bits);
    for (int64_t probe = 0; probe <= mask; ++probe) {
        unsigned long long cur = __ldcg(keys + h);
        if (cur == key) return false;
        if (cur == kEmptyKey) {
            unsigned long long old = atomicCAS(keys + h, kEmptyKey, key);
            if (old == kEmptyKey) return true;
            if (old == key) return false;
        }
        h = (h + 1) & mask;
    }
    set_status(status, ST_CAPACITY);
    return false;
}

__global__ void symbolic_kernel(TermArgs A, unsigned long long *keys, int bits, int32_t *row_cnt, uint32_t *status)
{
    const int lane = threadIdx.x & 31;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int32_t nc = *A.n_c_dev;
    for (int64_t t0 = ((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5) * 32; t0 < A.n_terms; t0 += nwarps * 32) {
        const int64_t t = t0 + lane;
        unsigned long long key = kEmptyKey;
        int32_t a = 0, b = 0;
        if (t < A.n_terms) {
            bool off;
            int64_t src;
            int kind;
            if (term_labels(A, t, nc, a, b, off, src, kind))
                key = pack_key(min(a, b), max(a, b));
            else
                set_status(status, ST_BAD_INDEX);
        }
        const unsigned same = __match_any_sync(kFull, key);
        if (key != kEmptyKey && __ffs(same) - 1 == lane) {
            if (hash_insert(keys, bits, key, status)) {
                const int32_t lo = min(a, b), hi = max(a, b);
                atomicAdd(row_cnt + lo, 1);
                if (lo != hi) atomicAdd(row_cnt + hi, 1);
            }
        }
    }
}

__global__ void scatter_cols_kernel(const unsigned long long *__restrict__ keys, int64_t nslots,
                                    const int32_t *__restrict__ row_ptr, int32_t *row_cur, int32_t *col, int64_t cap,
                                    uint32_t *status)
{
    for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < nslots; s += (int64_t)gridDim.x * blockDim.x) {
        const unsigned long long key = keys[s];
        if (key == kEmptyKey) continue;
        const int32_t lo = (int32_t)(key >> 32), hi = (int32_t)(key & 0xffffffffu);
        int64_t pos = (int64_t)row_ptr[lo] + atomicAdd(row_cur + lo, 1);
        if (pos < cap) col[pos] = hi; else set_status(status, ST_CAPACITY);
        if (lo != hi) {
            pos = (int64_t)row_ptr[hi] + atomicAdd(row_cur + hi, 1);
            if (pos < cap) col[pos] = lo; else set_status(status, ST_CAPACITY);
        }
    }
}

__device__ __forceinline__ int32_t warp_bitonic_sort(int32_t v)
{
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int k = 2; k <= 32; k <<= 1) {
#pragma unroll
        for (int j = k >> 1; j > 0; j >>= 1) {
            const int32_t o = __shfl_xor_sync(kFull, v, j);
            const bool up = (lane & k) == 0;
            const bool low = (lane & j) == 0;
            v = (low == up) ? min(v, o) : max(v, o);
        }
    }
    return v;
}

__global__ void sort_rows_short_kernel(const int32_t *__restrict__ n_c_dev, const int32_t *__restrict__ row_ptr,
                                       int32_t *col, int64_t cap, int32_t *long_rows, int32_t *long_count)
{
    const int lane = threadIdx.x & 31;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int32_t nc = *n_c_dev;
    for (int64_t a = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; a < nc; a += nwarps) {
        const int32_t k0 = row_ptr[a], k1 = row_ptr[a + 1];
        if (k1 > cap) continue;
        const int32_t len = k1 - k0;
        if (len <= 32) {
            int32_t v = lane < len ? col[k0 + lane] : INT32_MAX;
            v = warp_bitonic_sort(v);
            if (lane < len) col[k0 + lane] = v;
        } else if (lane == 0) {
            long_rows[atomicAdd(long_count, 1)] = (int32_t)a;
        }
    }
}

__device__ __forceinline__ int block_excl_scan_i32(int v, int *s_warp, int *s_total)
{
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
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
    int r = incl - v + s_warp[wid];
    __syncthreads();
    return r;
}

__global__ void __launch_bounds__(kTb) sort_rows_long_kernel(const int32_t *__restrict__ long_rows,
                                                             const int32_t *__restrict__ long_count,
                                                             const int32_t *__restrict__ n_c_dev,
                                                             const int32_t *__restrict__ row_ptr, int32_t *col,
                                                             int64_t cap, uint32_t *bitmap_base, int64_t bitmap_words)
{
    __shared__ int32_t sbuf[kLongSmem];
    __shared__ int s_warp[kTb / 32];
    __shared__ int s_total;
    const int count = *long_count;
    const int32_t nc = *n_c_dev;
    uint32_t *bitmap = bitmap_base + blockIdx.x * bitmap_words;
    for (int idx = blockIdx.x; idx < count; idx += gridDim.x) {
        const int32_t a = long_rows[idx];
        const int32_t k0 = row_ptr[a], k1 = row_ptr[a + 1];
        if (k1 > cap) continue;
        const int32_t len = k1 - k0;
        if (len <= kLongSmem) {
            int n2 = 64;
            while (n2 < len) n2 <<= 1;
            for (int t = threadIdx.x; t < n2; t += blockDim.x) sbuf[t] = t < len ? col[k0 + t] : INT32_MAX;
            __syncthreads();
            for (int k = 2; k <= n2; k <<= 1)
                for (int j = k >> 1; j > 0; j >>= 1) {
                    for (int t = threadIdx.x; t < n2; t += blockDim.x) {
                        const int o = t ^ j;
                        if (o > t) {
                            const bool up = (t & k) == 0;
                            const int32_t x = sbuf[t], y = sbuf[o];
                            if ((x > y) == up) { sbuf[t] = y; sbuf[o] = x; }
                        }
                    }
                    __syncthreads();
                }
            for (int t = threadIdx.x; t < len; t += blockDim.x) col[k0 + t] = sbuf[t];
            __syncthreads();
        } else {
            // columns are distinct: set one bit per column, read them back in order
            for (int32_t k = k0 + threadIdx.x; k < k1; k += blockDim.x) {
                const int32_t c = col[k];
                atomicOr(bitmap + (c >> 5), 1u << (c & 31));
            }
            __syncthreads();
            const int64_t nwords = div_up(nc, 32) < bitmap_words ? div_up(nc, 32) : bitmap_words;
            int32_t running = 0;
            for (int64_t w0 = 0; w0 < nwords; w0 += blockDim.x) {
                const int64_t w = w0 + threadIdx.x;
                uint32_t bits = w < nwords ? bitmap[w] : 0u;
                const int excl = block_excl_scan_i32(__popc(bits), s_warp, &s_total);
                int32_t pos = k0 + running + excl;
                if (w < nwords) bitmap[w] = 0u;
                while (bits) {
                    const int bpos = __ffs(bits) - 1;
                    col[pos++] = (int32_t)(w * 32 + bpos);
                    bits &= bits - 1;
                }
                running += s_total;
            }
            __syncthreads();
        }
    }
}

__global__ void zero_outputs_kernel(const int32_t *__restrict__ n_c_dev, const int32_t *__restrict__ nnz_dev, int64_t cap,
                                    double *__restrict__ val, double *__restrict__ g_c)
{
    const int64_t nnz = min((int64_t)*nnz_dev, cap);
    const int64_t nc = *n_c_dev;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < 9 * nnz; k += stride) val[k] = 0.0;
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < 3 * nc; k += stride) g_c[k] = 0.0;
}

// Position of column c in the sorted coarse row `row`; -1 when absent, -2
// when the row does not fit in the caller's capacity.
__device__ __forceinline__ int64_t find_col(const int32_t *__restrict__ row_ptr, const int32_t *__restrict__ col,
                                            int32_t row, int32_t c, int64_t cap)
{
    int32_t lo = row_ptr[row], hi = row_ptr[row + 1];
    if (hi > cap) return -2;
    while (lo < hi) {
        const int32_t mid = (lo + hi) >> 1;
        if (col[mid] < c) lo = mid + 1; else hi = mid;
    }
    return (lo < row_ptr[row + 1] && col[lo] == c) ? lo : -1;
}

// Upper coarse block (lo, hi) = (min(a, b), max(a, b)) of term t and its
// 3x3 value oriented for row lo (see the rules at the top of this file).
__device__ __forceinline__ bool term_value(const TermArgs &A, int64_t t, int32_t nc, int32_t &lo, int32_t &hi,
                                           double V[9])
{
    int32_t a, b;
    bool off;
    int64_t src;
    int kind;
    if (!term_labels(A, t, nc, a, b, off, src, kind)) return false;
    double B[9];
    load_term(A, src, kind, B);
    if (a == b) {
#pragma unroll
        for (int r = 0; r < 3; ++r)
#pragma unroll
            for (int c = 0; c < 3; ++c) V[3 * r + c] = off ? B[3 * r + c] + B[3 * c + r] : B[3 * r + c];
    } else if (a < b) {
#pragma unroll
        for (int e = 0; e < 9; ++e) V[e] = B[e];
    } else {
#pragma unroll
        for (int r = 0; r < 3; ++r)
#pragma unroll
            for (int c = 0; c < 3; ++c) V[3 * r + c] = B[3 * c + r];
    }
    lo = min(a, b);
    hi = max(a, b);
    return true;
}

// Add a folded run to its coarse block with L2 atomics (the adds run in the
// L2, not in the SM's FP64 unit).
__device__ __forceinline__ void flush_run(unsigned long long key, const double acc[9], const int32_t *row_ptr,
                                          const int32_t *col, int64_t cap, double *val, uint32_t *status)
{
    const int32_t lo = (int32_t)(key >> 32), hi = (int32_t)(key & 0xffffffffu);
    const int64_t pos = find_col(row_ptr, col, lo, hi, cap);
    if (pos < 0) {
        set_status(status, pos == -2 ? ST_CAPACITY : ST_BAD_INDEX);
        return;
    }
    double *dst = val + 9 * pos;
#pragma unroll
    for (int e = 0; e < 9; ++e) atomicAdd(dst + e, acc[e]);
}

// Numeric phase.  A warp takes 32 x kRun consecutive terms; each lane folds
// its kRun terms left to right, adding a term to the running block while the
// coarse key repeats (the interior of a super-node) and flushing the run
// with atomics when it changes.  If all 32 lanes end on the same key the warp
// reduces it with shuffles first, so a large super-node's diagonal block
// receives one atomic set per 32 x kRun terms instead of one per term.
// kRun (4, 8, 16 or 32) is the context's launch shape (agipc_set_assembly_run).
template <int kRun>
__global__ void __launch_bounds__(kTb) numeric_kernel(TermArgs A, const int32_t *__restrict__ row_ptr,
                                                      const int32_t *__restrict__ col, int64_t cap, double *val,
                                                      uint32_t *status)
{
    const int lane = threadIdx.x & 31;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int32_t nc = *A.n_c_dev;
    const int64_t span = 32 * kRun;
    for (int64_t t0 = ((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5) * span; t0 < A.n_terms;
         t0 += nwarps * span) {
        unsigned long long key = kEmptyKey;
        double acc[9];
#pragma unroll
        for (int e = 0; e < 9; ++e) acc[e] = 0.0;
        for (int j = 0; j < kRun; ++j) {
            const int64_t t = t0 + (int64_t)lane * kRun + j;
            if (t >= A.n_terms) break;
            int32_t lo, hi;
            double V[9];
            if (!term_value(A, t, nc, lo, hi, V)) {
                set_status(status, ST_BAD_INDEX);
                continue;
            }
            const unsigned long long k = pack_key(lo, hi);
            if (k == key) {
#pragma unroll
                for (int e = 0; e < 9; ++e) acc[e] += V[e];
            } else {
                if (key != kEmptyKey) flush_run(key, acc, row_ptr, col, cap, val, status);
                key = k;
#pragma unroll
                for (int e = 0; e < 9; ++e) acc[e] = V[e];
            }
        }
        const unsigned same = __match_any_sync(kFull, key);
        if (same == kFull && key != kEmptyKey) {
#pragma unroll
            for (int e = 0; e < 9; ++e) acc[e] = warp_sum(acc[e]);
            if (lane == 0) flush_run(key, acc, row_ptr, col, cap, val, status);
        } else if (key != kEmptyKey) {
            flush_run(key, acc, row_ptr, col, cap, val, status);
        }
    }
}

__device__ __forceinline__ bool inverse3(const double *A, double *R)
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

// Lower triangle = transpose of the upper one (warp per coarse row; pure
// data movement).
__global__ void mirror_kernel(const int32_t *__restrict__ n_c_dev, const int32_t *__restrict__ row_ptr,
                              const int32_t *__restrict__ col, int64_t cap, double *val, uint32_t *status)
{
    const int lane = threadIdx.x & 31;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int32_t nc = *n_c_dev;
    for (int64_t a = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; a < nc; a += nwarps) {
        const int32_t k0 = row_ptr[a], k1 = row_ptr[a + 1];
        if (k1 > cap) continue;
        for (int32_t k = k0 + lane; k < k1; k += 32) {
            const int32_t b = col[k];
            if (b >= a) break;  // columns ascend: the rest is the diagonal and the upper part
            const int64_t q = find_col(row_ptr, col, b, (int32_t)a, cap);
            if (q < 0) { set_status(status, q == -2 ? ST_CAPACITY : ST_BAD_INDEX); continue; }
            const double *src = val + 9 * q;
            double *dst = val + 9 * (int64_t)k;
            double T[9];
#pragma unroll
            for (int r = 0; r < 3; ++r)
#pragma unroll
                for (int c = 0; c < 3; ++c) T[3 * r + c] = src[3 * c + r];
#pragma unroll
            for (int e = 0; e < 9; ++e) dst[e] = T[e];
        }
    }
}

// Diagonal blocks: symmetrise (lower from upper) and invert for the
// block-Jacobi preconditioner; one thread per coarse row, so every FP64
// instruction runs with a full warp.
__global__ void dinv_kernel(const int32_t *__restrict__ n_c_dev, const int32_t *__restrict__ row_ptr,
                            const int32_t *__restrict__ col, int64_t cap, double *val, double *__restrict__ dinv,
                            uint32_t *status)
{
    const int32_t nc = *n_c_dev;
    for (int64_t a = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; a < nc; a += (int64_t)gridDim.x * blockDim.x) {
        const int64_t q = find_col(row_ptr, col, (int32_t)a, (int32_t)a, cap);
        double R[9];
        bool ok = q >= 0;
        if (ok) {
            double *d = val + 9 * q;
            double D[9];
#pragma unroll
            for (int e = 0; e < 9; ++e) D[e] = d[e];
            D[3] = D[1];
            D[6] = D[2];
            D[7] = D[5];
            d[3] = D[3];
            d[6] = D[6];
            d[7] = D[7];
            ok = inverse3(D, R);
#pragma unroll
            for (int e = 0; e < 9; ++e) ok = ok && isfinite(R[e]);
        } else if (q == -2) {
            set_status(status, ST_CAPACITY);
        }
        if (!ok) {
            if (q != -2) set_status(status, ST_NONFINITE);
#pragma unroll
            for (int e = 0; e < 9; ++e) R[e] = 0.0;
        }
#pragma unroll
        for (int e = 0; e < 9; ++e) dinv[9 * a + e] = R[e];
    }
}

__global__ void gradient_kernel(int32_t n, const int32_t *__restrict__ labels, const int32_t *__restrict__ n_c_dev,
                                const double *__restrict__ g, double *g_c, uint32_t *status)
{
    const int lane = threadIdx.x & 31;
    const int32_t nc = *n_c_dev;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t f0 = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) & ~31ll; f0 < n; f0 += stride) {
        const int64_t f = f0 + lane;
        int32_t c = -1;
        double v0 = 0.0, v1 = 0.0, v2 = 0.0;
        if (f < n) {
            c = labels[f];
            if ((unsigned)c >= (unsigned)nc) { set_status(status, ST_BAD_INDEX); c = -1; }
            else { v0 = g[3 * f]; v1 = g[3 * f + 1]; v2 = g[3 * f + 2]; }
        }
        const unsigned same = __match_any_sync(kFull, c);
        if (same == kFull && c >= 0) {
            v0 = warp_sum(v0); v1 = warp_sum(v1); v2 = warp_sum(v2);
            if (lane == 0) {
                atomicAdd(g_c + 3 * c, v0);
                atomicAdd(g_c + 3 * c + 1, v1);
                atomicAdd(g_c + 3 * c + 2, v2);
            }
        } else if (c >= 0) {
            atomicAdd(g_c + 3 * c, v0);
            atomicAdd(g_c + 3 * c + 1, v1);
            atomicAdd(g_c + 3 * c + 2, v2);
        }
    }
}

__global__ void to_fp32_kernel(const int32_t *__restrict__ n_c_dev, const int32_t *__restrict__ nnz_dev, int64_t cap,
                               const double *__restrict__ val, float *__restrict__ val32,
                               const double *__restrict__ dinv, float *__restrict__ dinv32)
{
    const int64_t nnz = min64((int64_t)*nnz_dev, cap);
    const int64_t nc = *n_c_dev;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < 9 * nnz; k += stride) val32[k] = (float)val[k];
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < 9 * nc; k += stride) dinv32[k] = (float)dinv[k];
}

}  // namespace

static int assemble_impl(agipc_ctx *ctx, int32_t n_fine, const int32_t *fine_row_ptr, TermArgs &A,
                         const double *g, int32_t *coarse_row_ptr, int32_t *coarse_col, double *coarse_val,
                         int64_t coarse_cap_nnzb, int32_t *coarse_nnzb_dev, double *g_c, double *dinv)
{
    cudaStream_t st = ctx->stream;
    const int64_t n_terms = A.n_terms;
    const int32_t *n_coarse_dev = A.n_c_dev;
    int bits = 10;
    while ((1ll << bits) < n_terms + n_terms / 4 && bits < ctx->hbits) ++bits;
    const int64_t nslots = 1ll << bits;

    if (cudaMemsetAsync(ctx->hkeys, 0xff, sizeof(unsigned long long) * nslots, st) != cudaSuccess ||
        cudaMemsetAsync(ctx->row_cnt, 0, sizeof(int32_t) * ((size_t)n_fine + 1), st) != cudaSuccess ||
        cudaMemsetAsync(ctx->row_cur, 0, sizeof(int32_t) * (size_t)n_fine, st) != cudaSuccess ||
        cudaMemsetAsync(ctx->long_rows + ctx->max_n, 0, sizeof(int32_t), st) != cudaSuccess)
        return AGIPC_ERR_CUDA;

    const unsigned grid_sm = (unsigned)ctx->num_sms * 8;
    fine_rows_kernel<<<(unsigned)div_up(n_fine, kTb), kTb, 0, st>>>(n_fine, fine_row_ptr, A.fine_nnzb, ctx->fine_brow,
                                                                    ctx->status);
    const unsigned gt = (unsigned)std::min<int64_t>(div_up(n_terms > 0 ? n_terms : 1, kTb), (int64_t)grid_sm * 4);
    symbolic_kernel<<<gt, kTb, 0, st>>>(A, ctx->hkeys, bits, ctx->row_cnt, ctx->status);
    if (!scan_exclusive_i32(ctx->row_cnt, coarse_row_ptr, n_fine, coarse_nnzb_dev, ctx->scan_part, st))
        return AGIPC_ERR_INVALID_ARG;
    scatter_cols_kernel<<<(unsigned)std::min<int64_t>(div_up(nslots, kTb), (int64_t)grid_sm * 4), kTb, 0, st>>>(
        ctx->hkeys, nslots, coarse_row_ptr, ctx->row_cur, coarse_col, coarse_cap_nnzb, ctx->status);
    const unsigned gw = (unsigned)std::min<int64_t>(div_up((int64_t)n_fine * 32, kTb), (int64_t)grid_sm * 4);
    sort_rows_short_kernel<<<gw, kTb, 0, st>>>(n_coarse_dev, coarse_row_ptr, coarse_col, coarse_cap_nnzb, ctx->long_rows,
                                               ctx->long_rows + ctx->max_n);
    sort_rows_long_kernel<<<kLongRowCtas, kTb, 0, st>>>(ctx->long_rows, ctx->long_rows + ctx->max_n, n_coarse_dev,
                                                       coarse_row_ptr, coarse_col, coarse_cap_nnzb, ctx->bitmap,
                                                       ctx->bitmap_words);
    zero_outputs_kernel<<<grid_sm, kTb, 0, st>>>(n_coarse_dev, coarse_nnzb_dev, coarse_cap_nnzb, coarse_val, g_c);
    const int run = ctx->asm_run == 4 || ctx->asm_run == 8 || ctx->asm_run == 16 ? ctx->asm_run : 32;
    const unsigned gnum = (unsigned)std::min<int64_t>(div_up(n_terms > 0 ? n_terms : 1, (int64_t)kTb * run),
                                                      (int64_t)grid_sm * 4);
    if (run == 4)
        numeric_kernel<4><<<gnum, kTb, 0, st>>>(A, coarse_row_ptr, coarse_col, coarse_cap_nnzb, coarse_val, ctx->status);
    else if (run == 8)
        numeric_kernel<8><<<gnum, kTb, 0, st>>>(A, coarse_row_ptr, coarse_col, coarse_cap_nnzb, coarse_val, ctx->status);
    else if (run == 16)
        numeric_kernel<16><<<gnum, kTb, 0, st>>>(A, coarse_row_ptr, coarse_col, coarse_cap_nnzb, coarse_val,
                                                 ctx->status);
    else
        numeric_kernel<32><<<gnum, kTb, 0, st>>>(A, coarse_row_ptr, coarse_col, coarse_cap_nnzb, coarse_val,
                                                 ctx->status);
    mirror_kernel<<<gw, kTb, 0, st>>>(n_coarse_dev, coarse_row_ptr, coarse_col, coarse_cap_nnzb, coarse_val,
                                      ctx->status);
    dinv_kernel<<<(unsigned)std::min<int64_t>(div_up(n_fine, kTb), (int64_t)grid_sm * 4), kTb, 0, st>>>(
        n_coarse_dev, coarse_row_ptr, coarse_col, coarse_cap_nnzb, coarse_val, dinv, ctx->status);
    gradient_kernel<<<(unsigned)std::min<int64_t>(div_up(n_fine, kTb), (int64_t)grid_sm * 4), kTb, 0, st>>>(
        n_fine, A.labels, n_coarse_dev, g, g_c, ctx->status);
    return cudaPeekAtLastError() == cudaSuccess ? AGIPC_OK : AGIPC_ERR_CUDA;
}

extern "C" int agipc_assemble_coarse(agipc_ctx *ctx, int32_t n_fine, const int32_t *labels, const int32_t *n_coarse_dev,
                                     const int32_t *fine_row_ptr, const int32_t *fine_col, const double *fine_val,
                                     int64_t fine_nnzb, int64_t n_pairs, const int32_t *pair_idx,
                                     const double *pair_blk, const double *g, int32_t *coarse_row_ptr,
                                     int32_t *coarse_col, double *coarse_val, int64_t coarse_cap_nnzb,
                                     int32_t *coarse_nnzb_dev, double *g_c, double *dinv)
{
    if (!ctx || n_fine <= 0 || n_fine > ctx->max_n || fine_nnzb < 0 || fine_nnzb > ctx->max_fine_nnzb || n_pairs < 0 ||
        n_pairs > ctx->max_pairs || coarse_cap_nnzb < 0)
        return AGIPC_ERR_INVALID_ARG;
    if (!labels || !n_coarse_dev || !fine_row_ptr || (fine_nnzb > 0 && (!fine_col || !fine_val)) ||
        (n_pairs > 0 && (!pair_idx || !pair_blk)) || !g || !coarse_row_ptr || !coarse_nnzb_dev || !g_c || !dinv ||
        (coarse_cap_nnzb > 0 && (!coarse_col || !coarse_val)))
        return AGIPC_ERR_INVALID_ARG;
    if (coarse_cap_nnzb > INT32_MAX) return AGIPC_ERR_INVALID_ARG;
    TermArgs A = {};
    A.n = n_fine;
    A.labels = labels;
    A.n_c_dev = n_coarse_dev;
    A.fine_brow = ctx->fine_brow;
    A.fine_col = fine_col;
    A.fine_val = fine_val;
    A.fine_nnzb = fine_nnzb;
    A.pair_idx = pair_idx;
    A.pair_blk = pair_blk;
    A.n_pairs = n_pairs;
    A.n_terms = fine_nnzb + 10 * n_pairs;
    return assemble_impl(ctx, n_fine, fine_row_ptr, A, g, coarse_row_ptr, coarse_col, coarse_val, coarse_cap_nnzb,
                         coarse_nnzb_dev, g_c, dinv);
}

extern "C" int agipc_assemble_coarse_mixed(agipc_ctx *ctx, int32_t n_fine, const int32_t *labels,
                                           const int32_t *n_coarse_dev, const int32_t *fine_row_ptr,
                                           const int32_t *fine_col, const float *fine_val32, int64_t fine_nnzb,
                                           int64_t n_pairs32, const int32_t *pair_idx32, const float *pair_blk32,
                                           int64_t n_pairs64, const int32_t *pair_idx64, const double *pair_blk64,
                                           const double *g, int32_t *coarse_row_ptr, int32_t *coarse_col,
                                           double *coarse_val, float *coarse_val32, int64_t coarse_cap_nnzb,
                                           int32_t *coarse_nnzb_dev, double *g_c, float *dinv32)
{
    if (!ctx || n_fine <= 0 || n_fine > ctx->max_n || fine_nnzb < 0 || fine_nnzb > ctx->max_fine_nnzb ||
        n_pairs32 < 0 || n_pairs64 < 0 || n_pairs32 + n_pairs64 > ctx->max_pairs || coarse_cap_nnzb < 0)
        return AGIPC_ERR_INVALID_ARG;
    if (!labels || !n_coarse_dev || !fine_row_ptr || (fine_nnzb > 0 && (!fine_col || !fine_val32)) ||
        (n_pairs32 > 0 && (!pair_idx32 || !pair_blk32)) || (n_pairs64 > 0 && (!pair_idx64 || !pair_blk64)) || !g ||
        !coarse_row_ptr || !coarse_nnzb_dev || !g_c || !dinv32 ||
        (coarse_cap_nnzb > 0 && (!coarse_col || !coarse_val || !coarse_val32)))
        return AGIPC_ERR_INVALID_ARG;
    if (coarse_cap_nnzb > INT32_MAX) return AGIPC_ERR_INVALID_ARG;
    TermArgs A = {};
    A.n = n_fine;
    A.labels = labels;
    A.n_c_dev = n_coarse_dev;
    A.fine_brow = ctx->fine_brow;
    A.fine_col = fine_col;
    A.fine_val32 = fine_val32;
    A.fine_nnzb = fine_nnzb;
    A.pair_idx = pair_idx32;
    A.pair_blk32 = pair_blk32;
    A.n_pairs = n_pairs32;
    A.pair_idx2 = pair_idx64;
    A.pair_blk2 = pair_blk64;
    A.n_pairs2 = n_pairs64;
    A.n_terms = fine_nnzb + 10 * (n_pairs32 + n_pairs64);
    int rc = assemble_impl(ctx, n_fine, fine_row_ptr, A, g, coarse_row_ptr, coarse_col, coarse_val, coarse_cap_nnzb,
                           coarse_nnzb_dev, g_c, ctx->dinv64);
    if (rc != AGIPC_OK) return rc;
    const unsigned grid = (unsigned)ctx->num_sms * 8;
    to_fp32_kernel<<<grid, kTb, 0, ctx->stream>>>(n_coarse_dev, coarse_nnzb_dev, coarse_cap_nnzb, coarse_val,
                                                   coarse_val32, ctx->dinv64, dinv32);
    return cudaPeekAtLastError() == cudaSuccess ? AGIPC_OK : AGIPC_ERR_CUDA;
}

// Scratch sizes of this file (used by agipc_create).
int assemble_long_row_ctas() { return kLongRowCtas; }
