// Slice machinery shared by the persistent PCG kernels: constants of the
// warp slices, slice staging (cp.async, and TMA bulk copies completing on
// mbarriers), CTA sums, and the slice SpMV w = A u over 128 consecutive 3x3
// blocks (32 lanes x 4 blocks) in two steps (gather, then multiply),
// templated on the type of the matrix values, the vectors and the
// accumulation.
#pragma once

#include "agipc_common.cuh"

namespace pcgs {

constexpr int kPcgBlock = 256;
constexpr int kPcgWarps = kPcgBlock / 32;
constexpr int kK = 4;                          // consecutive blocks per lane
// (4 rather than 5: 128-block slices spread the coarse matrix more evenly over
// the SM sub-partitions; 6.5 % less time per coarse iteration on GB300)
constexpr int kSlice = 32 * kK;                // blocks per warp slice
constexpr int kValBytes = kSlice * 9 * 8;      // 9216
constexpr int kIdxBytes = kSlice * 4;          // 512 per index array
constexpr int kBufBytes = kValBytes + 2 * kIdxBytes;
// A slice buffer holds the values (9 per block, of type T), then the column
// and the row of every block.  FP32 slices take 5632 bytes, so three of them
// fit where two FP64 slices go.
template <class T>
struct SliceLayout {
    static constexpr int kVal = kSlice * 9 * (int)sizeof(T);
    static constexpr int kBuf = kVal + 2 * kIdxBytes;
};
constexpr int kJoinBytes = 32 * (3 * 8 + 3 * 4);
constexpr int kWarpSmem = 2 * kBufBytes + kJoinBytes;
constexpr int kPartBytes = kPcgBlock * 3 * 8;
constexpr int kPcgSmem = kPcgWarps * kWarpSmem + kPartBytes;
constexpr int kMaxGridLanes = 8;               // the grid reduction handles up to 256 CTAs
constexpr int kWalkMax = 2;                    // longer chains of whole-lane rows take the scan join


__device__ __forceinline__ void cp_async16(void *smem_dst, const void *gmem_src, int src_bytes)
{
    const unsigned d = (unsigned)__cvta_generic_to_shared(smem_dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(d), "l"(gmem_src), "r"(src_bytes) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

// ---- TMA bulk copies of whole slices, completing on a shared-memory
// mbarrier (one per ring slot).  A full slice is three 16-byte-aligned runs
// (values, columns, rows) whose lengths are multiples of 16 bytes; one lane
// issues them.  Waits poll mbarrier.test_wait (which returns at once) and
// give up after kSpinLimit polls.
__device__ __forceinline__ unsigned smem_u32(const void *p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t *bar)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(bar)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

template <class T>
__device__ __forceinline__ void issue_slice_bulk(unsigned char *buf, int64_t sl, const T *val, const int32_t *col,
                                                 const int32_t *brow, uint64_t *bar, int lane)
{
    if (lane != 0) return;
    constexpr unsigned kV = SliceLayout<T>::kVal, kI = kIdxBytes;
    const unsigned b = smem_u32(bar), d = smem_u32(buf);
    // the warp's earlier reads of this buffer (generic proxy) come before
    // the copy's writes (async proxy)
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(b), "r"(kV + 2 * kI) : "memory");
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(d),
                 "l"(val + 9 * sl * kSlice), "r"(kV), "r"(b)
                 : "memory");
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     d + kV),
                 "l"(col + sl * kSlice), "r"(kI), "r"(b)
                 : "memory");
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     d + kV + kI),
                 "l"(brow + sl * kSlice), "r"(kI), "r"(b)
                 : "memory");
}

// Waits (every lane) for the phase of parity `parity` of `bar` to complete;
// false after kSpinLimit polls.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, unsigned parity)
{
    const unsigned b = smem_u32(bar);
    for (long long spins = 0; spins < kSpinLimit; ++spins) {
        unsigned done;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
            : "=r"(done)
            : "r"(b), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}

// Copy slice `sl` (values, columns, rows) into a warp buffer; zero-fills
// past the last block so no byte beyond the arrays is read.
template <class T>
__device__ __forceinline__ void issue_slice(unsigned char *buf, int64_t sl, int64_t nnz, const T *val,
                                            const int32_t *col, const int32_t *brow, int lane)
{
    const int64_t base = sl * kSlice;
    const int cnt = (int)min64(kSlice, nnz - base);
    const int vbytes = 9 * (int)sizeof(T) * cnt, ibytes = 4 * cnt;
    const unsigned char *vs = reinterpret_cast<const unsigned char *>(val + 9 * base);
    const unsigned char *cs = reinterpret_cast<const unsigned char *>(col + base);
    const unsigned char *rs = reinterpret_cast<const unsigned char *>(brow + base);
    for (int q = lane; 16 * q < vbytes; q += 32) cp_async16(buf + 16 * q, vs + 16 * q, min(16, vbytes - 16 * q));
    for (int q = lane; 16 * q < ibytes; q += 32) {
        cp_async16(buf + SliceLayout<T>::kVal + 16 * q, cs + 16 * q, min(16, ibytes - 16 * q));
        cp_async16(buf + SliceLayout<T>::kVal + kIdxBytes + 16 * q, rs + 16 * q, min(16, ibytes - 16 * q));
    }
}

// Sum of N values per thread over a CTA of kW warps: threads park their
// values in shared memory, warp k adds value k (each warp sits on its own SM
// sub-partition, whose FP64 pipe is the bottleneck) with a tree over the kW
// warps' slots, then 5 shuffle levels.  Totals land in v for every thread.
template <int N, int kW = kPcgWarps>
__device__ __forceinline__ void cta_sum(double (&v)[N], double *s_part, double *s_out)
{
    static_assert(N <= kW, "one warp per value");
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < N; ++k) s_part[N * threadIdx.x + k] = v[k];
    __syncthreads();
    if (wid < N) {
        double t[kW];
#pragma unroll
        for (int q = 0; q < kW; ++q) t[q] = s_part[N * (lane + 32 * q) + wid];
#pragma unroll
        for (int h = kW / 2; h > 0; h >>= 1)
#pragma unroll
            for (int q = 0; q < h; ++q) t[q] += t[q + h];
        const double tot = warp_sum(t[0]);
        if (lane == 0) s_out[wid] = tot;
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < N; ++k) v[k] = s_out[k];
}

template <class T>
__device__ __forceinline__ void store_row(T *w, int row, bool split, const T y[3])
{
    T *dst = w + 3 * (int64_t)row;
    if (split) {
        atomicAdd(dst, y[0]);
        atomicAdd(dst + 1, y[1]);
        atomicAdd(dst + 2, y[2]);
    } else {
        dst[0] = y[0];
        dst[1] = y[1];
        dst[2] = y[2];
    }
}

// Selects on the bit pattern: integer moves, no floating-point instruction.
__device__ __forceinline__ double dsel(bool c, double a, double b)
{
    return __longlong_as_double(c ? __double_as_longlong(a) : __double_as_longlong(b));
}
__device__ __forceinline__ float dsel(bool c, float a, float b)
{
    return __int_as_float(c ? __float_as_int(a) : __float_as_int(b));
}

// Stores the rows that cross lanes of a warp slice.  Each lane passes its
// first segment (row fr, partial fa; the lane's only one when lr < 0) and its
// last segment (row lr, partial la).  A lane's tail row may continue into the
// next lanes, whose head rows then carry on.  Short chains are joined by the
// lane where the row starts, walking forward through shared memory; when
// more than kWalkMax lanes lie wholly inside one row (the rows of large
// aggregates), a segmented inclusive scan over the lanes (5 shuffle steps)
// replaces the walk and the lane where a row's run of lanes ends stores it.
// kScanOnly always takes the scan (no shared memory; `join` unused).
template <class T, bool kScanOnly = false>
__device__ __forceinline__ void join_rows(int lane, int fr, T (&fa)[3], bool f_split, int lr, T (&la)[3], bool l_split,
                                          T *w, unsigned char *join)
{
    const bool single = lr < 0;
    const int tr = single ? fr : lr;
    // every lane takes part in the shuffles and the ballot (full mask)
    const int tr_prev = __shfl_up_sync(kFull, tr, 1);
    const bool cont = lane > 0 && fr >= 0 && fr == tr_prev;
    const unsigned chain = __ballot_sync(kFull, single && cont);
    if (kScanOnly || __popc(chain) > kWalkMax) {
        T v[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) v[c] = single ? fa[c] : la[c];
        int st = (single && cont) ? 0 : 1;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            T o[3];
#pragma unroll
            for (int c = 0; c < 3; ++c) o[c] = __shfl_up_sync(kFull, v[c], d);
            const int ost = __shfl_up_sync(kFull, st, d);
            if (lane >= d && !st) {
#pragma unroll
                for (int c = 0; c < 3; ++c) v[c] += o[c];
                st = ost;
            }
        }
        T ci[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const T prev = __shfl_up_sync(kFull, v[c], 1);
            ci[c] = cont ? prev : T(0);
        }
        const int cont_next = __shfl_down_sync(kFull, cont ? 1 : 0, 1);
        const bool next_cont = lane < 31 && cont_next != 0;
        if (!single && fr >= 0) {
            T y[3];
#pragma unroll
            for (int c = 0; c < 3; ++c) y[c] = ci[c] + fa[c];
            store_row(w, fr, f_split, y);
        }
        if (tr >= 0 && !next_cont) store_row(w, tr, single ? f_split : l_split, v);
        __syncwarp();
        return;
    }
    T *s_fa = reinterpret_cast<T *>(join);
    int32_t *s_fr = reinterpret_cast<int32_t *>(join + 32 * 24);
    int32_t *s_single = s_fr + 32;
    int32_t *s_last = s_fr + 64;
    s_fr[lane] = fr;
    s_single[lane] = single ? 1 : 0;
    s_last[lane] = tr;
    s_fa[3 * lane] = fa[0];
    s_fa[3 * lane + 1] = fa[1];
    s_fa[3 * lane + 2] = fa[2];
    __syncwarp();
    if (!single) {
        for (int q = lane + 1; q < 32 && s_fr[q] == lr; ++q) {
            la[0] += s_fa[3 * q]; la[1] += s_fa[3 * q + 1]; la[2] += s_fa[3 * q + 2];
            if (!s_single[q]) break;
        }
        store_row(w, lr, l_split, la);
    }
    if (fr >= 0 && (lane == 0 || s_last[lane - 1] != fr)) {
        if (single) {
            for (int q = lane + 1; q < 32 && s_fr[q] == fr; ++q) {
                fa[0] += s_fa[3 * q]; fa[1] += s_fa[3 * q + 1]; fa[2] += s_fa[3 * q + 2];
                if (!s_single[q]) break;
            }
        }
        store_row(w, fr, f_split, fa);
    }
    __syncwarp();
}

// A lane's kK blocks take 9 kK sizeof(T) bytes (144 in FP32, 288 in FP64)
// and every slice buffer starts on a 16-byte boundary, so each 144-byte
// chunk of a lane (4 FP32 or 2 FP64 blocks) is read with nine 16-byte
// shared loads: conflict-free at this lane stride, where scalar loads met
// 4-way bank conflicts.
__device__ __forceinline__ void load_chunk(const float *src, float (&v)[36])
{
    const float4 *s4 = reinterpret_cast<const float4 *>(src);
#pragma unroll
    for (int m = 0; m < 9; ++m) {
        const float4 t = s4[m];
        v[4 * m] = t.x;
        v[4 * m + 1] = t.y;
        v[4 * m + 2] = t.z;
        v[4 * m + 3] = t.w;
    }
}
__device__ __forceinline__ void load_chunk(const double *src, double (&v)[18])
{
    const double2 *s2 = reinterpret_cast<const double2 *>(src);
#pragma unroll
    for (int m = 0; m < 9; ++m) {
        const double2 t = s2[m];
        v[2 * m] = t.x;
        v[2 * m + 1] = t.y;
    }
}

// What a lane gathers from global memory for its kK blocks of a slice: the
// rows, u at the columns, u at the row of each segment's first block and the
// row's flag word (bit 0: the row is split).  Issued by slice_gather,
// consumed by slice_compute, so a streamed loop can gather slice k + 1 while
// it multiplies slice k: the gather step only issues loads and never uses a
// loaded value (the flag's bit is tested in slice_compute).
//
// The gathers are plain (L1-cacheable) loads: the rows of a slice share most
// of their neighbour columns, and routed past L1 every component became its
// own L2 sector request, which bounded the streamed SpMV.  u and the flags
// are written only in other phases, each followed by a grid barrier whose
// acquire orders those writes before these loads (PTX memory model), so no
// L1 line read here can predate them.
//
// kLazy keeps u of the segment rows only for the lane's first block (which
// always starts a segment); slice_compute loads it for later segment starts
// when it meets them.  That saves 9 registers of T per lane, which the
// 16-warp FP64 kernel (at most 128 registers) would otherwise spill.
template <class T, bool kLazy = false>
struct SliceGather {
    int rows_[kK];
    T xv[kK][3];
    T ur[kLazy ? 1 : kK][3];
    int flags[kK];
};

template <class T, bool kLazy = false>
__device__ __forceinline__ void slice_gather(const unsigned char *buf, int cnt, const T *u, const uint8_t *rowflag,
                                             int lane, SliceGather<T, kLazy> &G)
{
    const int32_t *s_col = reinterpret_cast<const int32_t *>(buf + SliceLayout<T>::kVal);
    const int32_t *s_row = reinterpret_cast<const int32_t *>(buf + SliceLayout<T>::kVal + kIdxBytes);
#pragma unroll
    for (int j = 0; j < kK; ++j) {
        const int q = lane * kK + j;
        G.rows_[j] = -1;
        G.flags[j] = 0;
        G.xv[j][0] = G.xv[j][1] = G.xv[j][2] = T(0);
        if (!kLazy || j == 0) G.ur[kLazy ? 0 : j][0] = G.ur[kLazy ? 0 : j][1] = G.ur[kLazy ? 0 : j][2] = T(0);
        if (q < cnt) {
            const int rj = s_row[q];
            G.rows_[j] = rj;
            const T *uc = u + 3 * (int64_t)s_col[q];
            G.xv[j][0] = uc[0];
            G.xv[j][1] = uc[1];
            G.xv[j][2] = uc[2];
            if (j == 0 || rj != s_row[q - 1]) {  // first block of a row segment
                if (!kLazy || j == 0) {
                    const T *up = u + 3 * (int64_t)rj;
                    G.ur[kLazy ? 0 : j][0] = up[0];
                    G.ur[kLazy ? 0 : j][1] = up[1];
                    G.ur[kLazy ? 0 : j][2] = up[2];
                }
                G.flags[j] = rowflag[rj];
            }
        }
    }
}

// The same gathers from a packed FP32 vector: row i at u4[i] = (u_0, u_1,
// u_2, the row's flag bits), so a column costs one 16-byte load and the
// split flag rides with u of the segment's row.
__device__ __forceinline__ void slice_gather_packed(const unsigned char *buf, int cnt, const float4 *u4, int lane,
                                                    SliceGather<float> &G)
{
    const int32_t *s_col = reinterpret_cast<const int32_t *>(buf + SliceLayout<float>::kVal);
    const int32_t *s_row = reinterpret_cast<const int32_t *>(buf + SliceLayout<float>::kVal + kIdxBytes);
#pragma unroll
    for (int j = 0; j < kK; ++j) {
        const int q = lane * kK + j;
        G.rows_[j] = -1;
        G.flags[j] = 0;
        G.xv[j][0] = G.xv[j][1] = G.xv[j][2] = 0.0f;
        G.ur[j][0] = G.ur[j][1] = G.ur[j][2] = 0.0f;
        if (q < cnt) {
            const int rj = s_row[q];
            G.rows_[j] = rj;
            const float4 c4 = u4[s_col[q]];
            G.xv[j][0] = c4.x;
            G.xv[j][1] = c4.y;
            G.xv[j][2] = c4.z;
            if (j == 0 || rj != s_row[q - 1]) {  // first block of a row segment
                const float4 r4 = u4[rj];
                G.ur[j][0] = r4.x;
                G.ur[j][1] = r4.y;
                G.ur[j][2] = r4.z;
                G.flags[j] = __float_as_int(r4.w);
            }
        }
    }
}

// w = A u over one slice held in `buf` (rows inside the slice) or += (rows
// cut by its ends), with the lane's gathers in G; with kDelta, adds this
// lane's share of delta = u . A u (accumulated in T over the lane's row
// segments) to dpart.  T is the type of the matrix values, of u and w and
// of the accumulation.
//
// Per lane the kK blocks are folded left to right into one running row
// accumulator (reset at a row change by a select, so the FP64 work is
// exactly 9 FMAs per block with no divergence); a row segment's total is the
// accumulator at the segment's last block.  delta is linear in w, so each
// lane adds u_row . (its own part of the row) once per segment: for its
// first and last segments after the fold (6 FMAs), for the rare rows wholly
// inside the lane where they are stored.  Segments that cross lanes are
// joined by the lane where the row starts, which walks forward over the
// lanes that continue it.
template <class T, bool kDelta, bool kLazy = false>
__device__ __forceinline__ void slice_compute(const unsigned char *buf, const SliceGather<T, kLazy> &G, T *w,
                                              unsigned char *join, int lane, double &dpart, const T *u = nullptr)
{
    const T *s_val = reinterpret_cast<const T *>(buf);
    const int(&rows_)[kK] = G.rows_;
    const T(&xv)[kK][3] = G.xv;
    bool split[kK];
#pragma unroll
    for (int j = 0; j < kK; ++j) split[j] = (G.flags[j] & 1) != 0;
    // running accumulator; segment bookkeeping by selects
    T acc[3] = {T(0), T(0), T(0)};
    T fa[3] = {T(0), T(0), T(0)}, la[3] = {T(0), T(0), T(0)};
    T fu[3] = {T(0), T(0), T(0)}, lu[3] = {T(0), T(0), T(0)};
    T dloc = T(0);
    int fr = -1, lr = -1;
    bool f_split = false, l_split = false, s_cur = false, first_open = true;
    T cu[3] = {T(0), T(0), T(0)};
    constexpr int kBpc = 16 / (int)sizeof(T);   // blocks per 144-byte chunk
    static_assert(kK % kBpc == 0, "a lane's blocks are whole chunks");
    T ch[9 * kBpc];
#pragma unroll
    for (int j = 0; j < kK; ++j) {
        const bool valid = rows_[j] >= 0;
        const bool start = valid && (j == 0 || rows_[j] != rows_[j - 1]);
        const bool end = valid && (j == kK - 1 || rows_[j + 1] != rows_[j]);
        // blocks past the slice's end read stale shared memory, which may
        // hold NaN bit patterns: select zeros for them (NaN * 0 is NaN)
        if (j % kBpc == 0) load_chunk(s_val + 9 * (lane * kK + j), ch);
        T B[9];
#pragma unroll
        for (int e = 0; e < 9; ++e) B[e] = dsel(valid, ch[9 * (j % kBpc) + e], T(0));
        if (kDelta && kLazy && j > 0 && start) {   // a later segment start: u of its row now
            const T *up = u + 3 * (int64_t)rows_[j];
            cu[0] = up[0];
            cu[1] = up[1];
            cu[2] = up[2];
        }
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            if (!kLazy) cu[c] = dsel(start, G.ur[j][c], cu[c]);
            else if (j == 0) cu[c] = dsel(start, G.ur[0][c], cu[c]);
            acc[c] = dsel(start, T(0), acc[c]);
            acc[c] = fma(B[3 * c + 2], xv[j][2], fma(B[3 * c + 1], xv[j][1], fma(B[3 * c], xv[j][0], acc[c])));
        }
        s_cur = start ? split[j] : s_cur;
        if (end) {
            const bool last = j == kK - 1 || rows_[j + 1] < 0;
            if (first_open) {                       // the lane's first segment: joined below
                fr = rows_[j]; f_split = s_cur;
                fa[0] = acc[0]; fa[1] = acc[1]; fa[2] = acc[2];
                fu[0] = cu[0]; fu[1] = cu[1]; fu[2] = cu[2];
                first_open = false;
            } else if (last) {                      // the lane's last segment: joined below
                lr = rows_[j]; l_split = s_cur;
                la[0] = acc[0]; la[1] = acc[1]; la[2] = acc[2];
                lu[0] = cu[0]; lu[1] = cu[1]; lu[2] = cu[2];
            } else {                                // a row wholly inside this lane
                if (kDelta) dloc = fma(cu[0], acc[0], fma(cu[1], acc[1], fma(cu[2], acc[2], dloc)));
                store_row(w, rows_[j], s_cur, acc);
            }
        }
    }
    if (kDelta) {
        // this lane's parts of its first and last rows (zeros when absent)
        dloc = fma(fu[0], fa[0], fma(fu[1], fa[1], fma(fu[2], fa[2], dloc)));
        dloc = fma(lu[0], la[0], fma(lu[1], la[1], fma(lu[2], la[2], dloc)));
        dpart += (double)dloc;
    }
    join_rows(lane, fr, fa, f_split, lr, la, l_split, w, join);
}

// Gather, then multiply: one slice with nothing overlapped.
template <class T, bool kDelta, bool kLazy = false>
__device__ __forceinline__ void slice_spmv(const unsigned char *buf, int cnt, const T *u, T *w,
                                           const uint8_t *rowflag, unsigned char *join, int lane, double &dpart)
{
    SliceGather<T, kLazy> G;
    slice_gather<T, kLazy>(buf, cnt, u, rowflag, lane, G);
    slice_compute<T, kDelta, kLazy>(buf, G, w, join, lane, dpart, u);
}

}  // namespace pcgs
