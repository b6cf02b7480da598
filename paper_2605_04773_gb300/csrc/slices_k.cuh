// Warp slices with a compile-time width and instance-aligned placement, for
// the batched PCG.  A slice covers up to 32*K consecutive 3x3 blocks; lane L
// folds blocks L*K .. L*K+K-1 of the slice.  A slice is staged from a block
// index that is a multiple of 4 (so every cp.async source is 16-byte
// aligned in FP32 and FP64) and only its positions [qlo, cnt) are valid: the
// positions before qlo belong to the previous instance and are ignored.
#pragma once

#include "pcg_slices.cuh"

namespace bsl {

using pcgs::cp_async16;
using pcgs::dsel;
using pcgs::store_row;

template <class T, int K>
struct Geom {
    static constexpr int kSlice = 32 * K;
    static constexpr int kValBytes = kSlice * 9 * (int)sizeof(T);
    static constexpr int kIdxBytes = kSlice * 4;
    static constexpr int kBufBytes = kValBytes + 2 * kIdxBytes;
};
constexpr int kJoinBytes = 32 * (3 * 8 + 3 * 4);

// Stage blocks [abase, abase + cnt) (values, columns, block rows); abase is a
// multiple of 4.  Bytes past cnt are zero-filled; nothing past the arrays is
// read.
template <class T, int K>
__device__ __forceinline__ void stage(unsigned char *buf, int64_t abase, int cnt, const T *val, const int32_t *col,
                                      const int32_t *brow, int lane)
{
    using G = Geom<T, K>;
    const int vbytes = 9 * (int)sizeof(T) * cnt, ibytes = 4 * cnt;
    const unsigned char *vs = reinterpret_cast<const unsigned char *>(val + 9 * abase);
    const unsigned char *cs = reinterpret_cast<const unsigned char *>(col + abase);
    const unsigned char *rs = reinterpret_cast<const unsigned char *>(brow + abase);
    for (int q = lane; 16 * q < vbytes; q += 32) cp_async16(buf + 16 * q, vs + 16 * q, min(16, vbytes - 16 * q));
    for (int q = lane; 16 * q < ibytes; q += 32) {
        cp_async16(buf + G::kValBytes + 16 * q, cs + 16 * q, min(16, ibytes - 16 * q));
        cp_async16(buf + G::kValBytes + G::kIdxBytes + 16 * q, rs + 16 * q, min(16, ibytes - 16 * q));
    }
}

// w = A u over the valid positions of one staged slice (rows inside the
// slice stored, rows cut by its ends added atomically); with kDelta returns
// this lane's share of u . A u (accumulated in T, once per row segment).
// Same folding as pcgs::slice_spmv: one running accumulator per lane reset
// by selects at row starts, 9 FMAs per block, segments that cross lanes
// joined by pcgs::join_rows with the shuffle scan only (no shared memory,
// so the warp's buffers can take a further pipeline stage; `join` unused).
template <class T, bool kDelta, int K>
__device__ __forceinline__ double spmv(const unsigned char *buf, int qlo, int cnt, const T *u, T *w,
                                       const uint8_t *rowflag, unsigned char *join, int lane)
{
    using G = Geom<T, K>;
    const T *s_val = reinterpret_cast<const T *>(buf);
    const int32_t *s_col = reinterpret_cast<const int32_t *>(buf + G::kValBytes);
    const int32_t *s_row = reinterpret_cast<const int32_t *>(buf + G::kValBytes + G::kIdxBytes);
    // The gathers are plain (L1-cacheable) loads: u and the flags are written
    // only in other phases, each followed by a grid barrier whose acquire
    // orders those writes before these loads.  The flag byte is kept as
    // loaded and tested where it is used.
    int rows_[K];
    T xv[K][3];
    T ur[K][3];
    int flags[K];
#pragma unroll
    for (int j = 0; j < K; ++j) {
        const int q = lane * K + j;
        rows_[j] = -1;
        flags[j] = 0;
        xv[j][0] = xv[j][1] = xv[j][2] = T(0);
        ur[j][0] = ur[j][1] = ur[j][2] = T(0);
        if (q >= qlo && q < cnt) {
            const int rj = s_row[q];
            rows_[j] = rj;
            const T *uc = u + 3 * (int64_t)s_col[q];
            xv[j][0] = uc[0];
            xv[j][1] = uc[1];
            xv[j][2] = uc[2];
            if (j == 0 || q == qlo || rj != s_row[q - 1]) {  // first block of a row segment
                const T *up = u + 3 * (int64_t)rj;
                ur[j][0] = up[0];
                ur[j][1] = up[1];
                ur[j][2] = up[2];
                flags[j] = rowflag[rj];
            }
        }
    }
    // Values: when the lane's K blocks start on a 16-byte boundary (9 K
    // sizeof(T) a multiple of 16: K = 4, 8 in FP32, even K in FP64) they are
    // read chunk by chunk with pcgs::load_chunk (144-byte chunks of 4 FP32 or
    // 2 FP64 blocks, 16-byte loads, no bank conflicts at that stride); other
    // widths read scalars.
    constexpr int kBpc = 16 / (int)sizeof(T);
    constexpr bool kChunked = (9 * K * (int)sizeof(T)) % 16 == 0 && K % kBpc == 0;
    T ch[9 * kBpc];
    T acc[3] = {T(0), T(0), T(0)};
    T fa[3] = {T(0), T(0), T(0)}, la[3] = {T(0), T(0), T(0)};
    T fu[3] = {T(0), T(0), T(0)}, lu[3] = {T(0), T(0), T(0)};
    T dloc = T(0);
    int fr = -1, lr = -1;
    bool f_split = false, l_split = false, s_cur = false, first_open = true;
    T cu[3] = {T(0), T(0), T(0)};
#pragma unroll
    for (int j = 0; j < K; ++j) {
        const bool valid = rows_[j] >= 0;
        const bool start = valid && (j == 0 || rows_[j] != rows_[j - 1]);
        const bool end = valid && (j == K - 1 || rows_[j + 1] != rows_[j]);
        // positions outside [qlo, cnt) read stale or foreign shared memory:
        // select zeros for them
        T B[9];
        if constexpr (kChunked) {
            if (j % kBpc == 0) pcgs::load_chunk(s_val + 9 * (lane * K + j), ch);
#pragma unroll
            for (int e = 0; e < 9; ++e) B[e] = dsel(valid, ch[9 * (j % kBpc) + e], T(0));
        } else {
            const T *Bs = s_val + 9 * (lane * K + j);
#pragma unroll
            for (int e = 0; e < 9; ++e) B[e] = dsel(valid, Bs[e], T(0));
        }
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            cu[c] = dsel(start, ur[j][c], cu[c]);
            acc[c] = dsel(start, T(0), acc[c]);
            acc[c] = fma(B[3 * c + 2], xv[j][2], fma(B[3 * c + 1], xv[j][1], fma(B[3 * c], xv[j][0], acc[c])));
        }
        s_cur = start ? (flags[j] & 1) != 0 : s_cur;
        if (end) {
            const bool last = j == K - 1 || rows_[j + 1] < 0;
            if (first_open) {
                fr = rows_[j];
                f_split = s_cur;
                fa[0] = acc[0];
                fa[1] = acc[1];
                fa[2] = acc[2];
                fu[0] = cu[0];
                fu[1] = cu[1];
                fu[2] = cu[2];
                first_open = false;
            } else if (last) {
                lr = rows_[j];
                l_split = s_cur;
                la[0] = acc[0];
                la[1] = acc[1];
                la[2] = acc[2];
                lu[0] = cu[0];
                lu[1] = cu[1];
                lu[2] = cu[2];
            } else {
                if (kDelta) dloc = fma(cu[0], acc[0], fma(cu[1], acc[1], fma(cu[2], acc[2], dloc)));
                store_row(w, rows_[j], s_cur, acc);
            }
        }
    }
    if (kDelta) {
        // delta is linear in w: this lane's parts of its first and last rows
        dloc = fma(fu[0], fa[0], fma(fu[1], fa[1], fma(fu[2], fa[2], dloc)));
        dloc = fma(lu[0], la[0], fma(lu[1], la[1], fma(lu[2], la[2], dloc)));
    }
    pcgs::join_rows<T, true>(lane, fr, fa, f_split, lr, la, l_split, w, join);
    return (double)dloc;
}

}  // namespace bsl
