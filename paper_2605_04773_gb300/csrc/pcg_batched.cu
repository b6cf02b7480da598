// Batched precision-form PCG: many independent coarse systems, stored one
// after another in a block-diagonal BSR matrix, solved in one persistent
// cooperative launch with per-instance scalars and per-instance convergence.
//
// Each instance runs the method of pcg_mixed.cu (Chronopoulos-Gear PCG with
// FP32 blocks, SpMV and block-Jacobi preconditioner, FP64 dot products, x
// and r in FP64, FP64 residual replacement every refine_every iterations and
// a true-residual check before it stops).  The whole GPU works on all
// instances at once, so a large instance never waits on one SM:
//   S phase   the slices of the still-active instances, numbered in
//             instance order, are cut into equal contiguous chunks, one per
//             warp; each slice lies inside one instance (its start is
//             rounded down to a multiple of 4 blocks for 16-byte cp.async
//             and the positions before the instance's first block are
//             ignored), so delta = u . A u is summed per warp run of one
//             instance and added to the instance's accumulator;
//   scalars   every CTA computes every instance's alpha, beta and decision
//             from the accumulators (one owner thread per instance; the
//             recurrence state lives in that thread's registers), so the
//             values agree bitwise across CTAs;
//   P phase   each CTA updates a fixed contiguous range of rows; gamma and
//             rho are reduced per warp and per CTA before one atomic per
//             instance and CTA.
// Instances that have stopped cost nothing in later iterations.  The number
// of blocks a lane folds (K = 4, 5, 6 or 8, the slice width 32 K) is a template
// parameter chosen by the caller (the Python autotuner picks it by timing).
// The per-instance sums are added with atomics, so alpha and beta may differ
// in the last bits from run to run.
#include <algorithm>

#include "agipc_common.cuh"
#include "slices_k.cuh"

using namespace pcgs;

namespace {

constexpr int kInstPerThread = kBatchMaxInst / kPcgBlock;
constexpr int kLocalTab = 64;  // per-CTA table of instance sums

struct BatchArgs {
    int32_t n_inst;
    const int32_t *inst_row;  // [n_inst + 1]
    int32_t max_rows;
    int64_t max_nnzb;
    const int32_t *rp;
    const int32_t *col;
    const double *val64;
    const float *val32;
    const float *dinv32;
    const double *b;
    double *x;
    double sign, tol;
    int32_t max_iter, refine_every;
    int32_t *iters_out;
    double *relres_out;
    PcgScratch S;
    double *acc;  // [2][kBatchMaxInst][2] gamma, rho, then [2][kBatchMaxInst] delta
    uint32_t *status;
};

constexpr int cmax(int a, int b) { return a > b ? a : b; }

// cp.async stages of the S phase's FP32 slices: three for the narrow tiles,
// two for the wide ones.  More stages fit, but shared memory then crowds out
// the L1 that the u gathers hit (4 stages at 4 blocks a lane and 3 at 6 were
// 9 % and 17 % slower on the 256-instance batch).
template <int K>
__host__ __device__ constexpr int s_stages() { return K <= 5 ? 3 : 2; }

template <int K>
struct Layout {
    static constexpr int kWarp =
        (cmax(s_stages<K>() * bsl::Geom<float, K>::kBufBytes, bsl::Geom<double, K>::kBufBytes) + 15) & ~15;
    static constexpr int kWarps = kPcgWarps * kWarp;
    static constexpr int kInt = 3 * (kBatchMaxInst + 1) * 4 + 4;           // irow, b0, sptr (+pad to 8)
    static constexpr int kDbl = 2 * kBatchMaxInst * 8 + kLocalTab * 2 * 8;  // alpha, beta, local table
    static constexpr int kScan = (kBatchMaxInst + 1) * 4 * 4;               // active/refine slice and row prefixes
    static constexpr int kByte = 2 * kBatchMaxInst;                         // dec, ref
    static constexpr int kTotal = kWarps + kInt + kDbl + kScan + kByte;
};

__device__ __forceinline__ void precond32(const float *D, const double r[3], float u[3])
{
    const float r0 = (float)r[0], r1 = (float)r[1], r2 = (float)r[2];
#pragma unroll
    for (int c = 0; c < 3; ++c) u[c] = fmaf(D[3 * c + 2], r2, fmaf(D[3 * c + 1], r1, D[3 * c] * r0));
}

// Block-wide exclusive scan of cnt(i), i in [0, n], n <= kBatchMaxInst, into
// out[0..n]; out[n] is the total.  Every thread returns the total.
template <class F>
__device__ int block_scan(int n, F cnt, int32_t *out, int32_t *s_warp)
{
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int v[kInstPerThread];
    int sum = 0;
#pragma unroll
    for (int q = 0; q < kInstPerThread; ++q) {
        const int i = threadIdx.x * kInstPerThread + q;
        v[q] = i < n ? cnt(i) : 0;
        sum += v[q];
    }
    const int incl = warp_incl_scan(sum);
    if (lane == 31) s_warp[wid] = incl;
    __syncthreads();
    if (wid == 0) {
        const int t = lane < kPcgWarps ? s_warp[lane] : 0;
        const int ti = warp_incl_scan(t);
        if (lane < kPcgWarps) s_warp[lane] = ti - t;
        if (lane == kPcgWarps - 1) s_warp[kPcgWarps] = ti;
    }
    __syncthreads();
    int run = s_warp[wid] + incl - sum;
#pragma unroll
    for (int q = 0; q < kInstPerThread; ++q) {
        const int i = threadIdx.x * kInstPerThread + q;
        if (i < n) out[i] = run;
        run += v[q];
    }
    const int total = s_warp[kPcgWarps];
    if (threadIdx.x == 0) out[n] = total;
    __syncthreads();
    return total;
}

// Instance of element k of a monotone prefix p[0..n] (p[i] <= k < p[i+1]).
__device__ __forceinline__ int find_seg(const int32_t *p, int n, int64_t k)
{
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (p[mid] <= k) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// Per-CTA sums of (gamma, rho) per instance over the rows of a P pass.
// Rows are visited by warps in groups of 32 consecutive rows; each warp
// keeps one running instance, and sums reach global memory through a
// shared table (instances [ilo, ilo + kLocalTab)) or directly.
struct RowSums {
    double *tab;     // shared [kLocalTab][2]
    double *gacc;    // global [kBatchMaxInst][2] of the target slot
    int ilo;
    __device__ __forceinline__ void add(int inst, double g, double r) const
    {
        const int o = inst - ilo;
        if (o >= 0 && o < kLocalTab) {
            atomicAdd(tab + 2 * o, g);
            atomicAdd(tab + 2 * o + 1, r);
        } else {
            atomicAdd(gacc + 2 * inst, g);
            atomicAdd(gacc + 2 * inst + 1, r);
        }
    }
};

template <int K>
__global__ void __launch_bounds__(kPcgBlock, 1) pcg_batched_kernel(BatchArgs A)
{
    using L = Layout<K>;
    constexpr int S = 32 * K;
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int32_t s_warp[kPcgWarps + 1];
    __shared__ int s_n_active;

    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const unsigned nblocks = gridDim.x;
    const int64_t nwarps = (int64_t)nblocks * kPcgWarps;
    const int64_t gwarp = (int64_t)blockIdx.x * kPcgWarps + wib;  // contiguous per CTA
    const int64_t gtid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;

    unsigned char *wbuf = smem + (size_t)wib * L::kWarp;
    unsigned char *join = nullptr;   // the batched slices join rows by shuffles only
    int32_t *s_irow = reinterpret_cast<int32_t *>(smem + L::kWarps);
    int32_t *s_b0 = s_irow + (kBatchMaxInst + 1);
    int32_t *s_sptr = s_b0 + (kBatchMaxInst + 1);
    double *s_alpha = reinterpret_cast<double *>(smem + L::kWarps + L::kInt);
    double *s_beta = s_alpha + kBatchMaxInst;
    double *s_tab = s_beta + kBatchMaxInst;
    int32_t *s_aptr = reinterpret_cast<int32_t *>(smem + L::kWarps + L::kInt + L::kDbl);
    int32_t *s_rptr = s_aptr + (kBatchMaxInst + 1);
    int32_t *s_arow = s_rptr + (kBatchMaxInst + 1);
    int32_t *s_rrow = s_arow + (kBatchMaxInst + 1);
    int8_t *s_dec = reinterpret_cast<int8_t *>(smem + L::kWarps + L::kInt + L::kDbl + L::kScan);
    int8_t *s_ref = s_dec + kBatchMaxInst;

    const int ni = A.n_inst;
    bool ok = ni > 0 && ni <= kBatchMaxInst && nblocks <= 32 * kMaxGridLanes;
    // ---- instance tables (every CTA holds its own copy)
    if (ok) {
        for (int i = threadIdx.x; i <= ni; i += blockDim.x) s_irow[i] = A.inst_row[i];
    }
    __syncthreads();
    if (ok && threadIdx.x == 0) {
        bool good = s_irow[0] == 0 && s_irow[ni] <= A.max_rows;
        for (int i = 0; good && i < ni; ++i) good = s_irow[i] <= s_irow[i + 1];
        s_n_active = good ? 1 : 0;
    }
    __syncthreads();
    ok = ok && s_n_active != 0;
    if (!ok) {
        if (gtid == 0) set_status(A.status, ST_BAD_INDEX);
        return;
    }
    const int32_t n = s_irow[ni];
    for (int i = threadIdx.x; i <= ni; i += blockDim.x) s_b0[i] = A.rp[s_irow[i]];
    __syncthreads();
    const int64_t nnz = s_b0[ni];
    if (nnz < 0 || nnz > A.max_nnzb) {
        if (gtid == 0) set_status(A.status, nnz < 0 ? ST_BAD_INDEX : ST_CAPACITY);
        return;
    }
    // slices per instance, from the instance's first block rounded down to 4
    auto nsl = [&](int i) -> int {
        const int32_t b0 = s_b0[i], b1 = s_b0[i + 1];
        return b1 > b0 ? (int)div_up(b1 - (b0 & ~3), S) : 0;
    };
    block_scan(ni, nsl, s_sptr, s_warp);

    const int64_t rows_per_cta = div_up(n, nblocks);
    const int64_t row0 = min64((int64_t)blockIdx.x * rows_per_cta, n);
    const int64_t row1 = min64(row0 + rows_per_cta, n);
    const int ilo = row0 < row1 ? find_seg(s_irow, ni, row0) : 0;

    double *__restrict__ r = A.S.r;
    double *ax = A.S.u;
    float *w = reinterpret_cast<float *>(A.S.w);
    float *u = w + 3 * (int64_t)A.max_rows;
    float *__restrict__ p = reinterpret_cast<float *>(A.S.p);
    float *__restrict__ s = reinterpret_cast<float *>(A.S.s);
    double *__restrict__ x = A.x;
    int32_t *brow = A.S.brow;
    uint8_t *rowflag = A.S.rowflag;
    unsigned *count = A.S.bar;
    unsigned epoch = 0;
    double *acc_gr = A.acc;                              // [2][kBatchMaxInst][2]
    double *acc_d = A.acc + 4 * kBatchMaxInst;           // [2][kBatchMaxInst]

    // P-pass row walk: warps take groups of 32 consecutive rows of the CTA's
    // range; f(row, inst, sums) is called for each row (lane-parallel).
    auto row_pass = [&](double *gacc, auto f) {
        for (int k = threadIdx.x; k < kLocalTab * 2; k += blockDim.x) s_tab[k] = 0.0;
        __syncthreads();
        RowSums rs{s_tab, gacc, ilo};
        int cur = ilo;
        double gsum = 0.0, rsum = 0.0;
        for (int64_t g0 = row0 + 32 * wib; g0 < row1; g0 += 32 * kPcgWarps) {
            const int64_t i = g0 + lane;
            const int64_t glast = min64(g0 + 31, row1 - 1);
            const bool uniform = glast < s_irow[cur + 1];
            int inst = cur;
            if (!uniform) {
                // flush the running sums, then take this group row by row
                const double gs = warp_sum(gsum), rsm = warp_sum(rsum);
                if (lane == 0 && (gs != 0.0 || rsm != 0.0)) rs.add(cur, gs, rsm);
                gsum = rsum = 0.0;
                if (i < row1) inst = find_seg(s_irow, ni, i);
            }
            double gi = 0.0, ri = 0.0;
            if (i < row1) f(i, inst, gi, ri);
            if (uniform) {
                gsum += gi;
                rsum += ri;
            } else {
                if (i < row1 && (gi != 0.0 || ri != 0.0)) rs.add(inst, gi, ri);
                cur = find_seg(s_irow, ni, glast);
            }
        }
        {
            const double gs = warp_sum(gsum), rsm = warp_sum(rsum);
            if (lane == 0 && (gs != 0.0 || rsm != 0.0)) rs.add(cur, gs, rsm);
        }
        __syncthreads();
        for (int k = threadIdx.x; k < kLocalTab; k += blockDim.x) {
            const double gv = s_tab[2 * k], rv = s_tab[2 * k + 1];
            if ((gv != 0.0 || rv != 0.0) && ilo + k < ni) {
                atomicAdd(gacc + 2 * (ilo + k), gv);
                atomicAdd(gacc + 2 * (ilo + k) + 1, rv);
            }
        }
    };

    // Pass over the rows of the instances counted in the prefix `pre` (rows
    // numbered instance by instance): every warp takes an equal contiguous
    // chunk and visits it 64 rows at a time, lane l taking rows l and l + 32
    // so that two rows' loads are in flight together.  f(rowA, instA, okA,
    // rowB, instB, okB, gA, rA, gB, rB) updates both rows and returns their
    // gamma and rho shares, which are summed per run of one instance and
    // added to gacc with one atomic per run.
    auto act_pass = [&](const int32_t *pre, double *gacc, auto f) {
        const int64_t tot = pre[ni];
        const int64_t per = div_up(div_up(tot, nwarps), 64) * 64;
        const int64_t a0 = min64(gwarp * per, tot), a1 = min64(a0 + per, tot);
        int cur = a0 < a1 ? find_seg(pre, ni, a0) : 0;
        double gsum = 0.0, rsum = 0.0;
        for (int64_t g0 = a0; g0 < a1; g0 += 64) {
            const int64_t glast = min64(g0 + 63, a1 - 1);
            const bool uniform = glast < pre[cur + 1];
            if (!uniform) {
                const double gs = warp_sum(gsum), rsm = warp_sum(rsum);
                if (lane == 0 && (gs != 0.0 || rsm != 0.0)) {
                    atomicAdd(gacc + 2 * cur, gs);
                    atomicAdd(gacc + 2 * cur + 1, rsm);
                }
                gsum = rsum = 0.0;
            }
            const int64_t aA = g0 + lane, aB = g0 + 32 + lane;
            const bool okA = aA < a1, okB = aB < a1;
            int iA = cur, iB = cur;
            if (!uniform) {
                if (okA)
                    while (aA >= pre[iA + 1]) ++iA;
                iB = iA;
                if (okB)
                    while (aB >= pre[iB + 1]) ++iB;
            }
            const int64_t rowA = okA ? s_irow[iA] + (aA - pre[iA]) : 0;
            const int64_t rowB = okB ? s_irow[iB] + (aB - pre[iB]) : 0;
            double gA = 0.0, rA = 0.0, gB = 0.0, rB = 0.0;
            f(rowA, iA, okA, rowB, iB, okB, gA, rA, gB, rB);
            if (uniform) {
                gsum += gA + gB;
                rsum += rA + rB;
            } else {
                if (okA && (gA != 0.0 || rA != 0.0)) {
                    atomicAdd(gacc + 2 * iA, gA);
                    atomicAdd(gacc + 2 * iA + 1, rA);
                }
                if (okB && (gB != 0.0 || rB != 0.0)) {
                    atomicAdd(gacc + 2 * iB, gB);
                    atomicAdd(gacc + 2 * iB + 1, rB);
                }
                while (glast >= pre[cur + 1]) ++cur;  // warp-uniform: from the old run
            }
        }
        const double gs = warp_sum(gsum), rsm = warp_sum(rsum);
        if (lane == 0 && (gs != 0.0 || rsm != 0.0)) {
            atomicAdd(gacc + 2 * cur, gs);
            atomicAdd(gacc + 2 * cur + 1, rsm);
        }
    };

    // ---- setup: block rows, split flags, r = sign b, u = D r, gamma, rho
    for (int k = threadIdx.x; k < kBatchMaxInst; k += blockDim.x) {
        s_dec[k] = 0;
        s_ref[k] = 0;
    }
    row_pass(acc_gr, [&](int64_t i, int inst, double &gi, double &ri) {
        const int32_t k0 = A.rp[i], k1 = A.rp[i + 1];
        const int32_t c0 = s_irow[inst], c1 = s_irow[inst + 1];
        bool bad = k0 < 0 || k1 < k0 || k1 > nnz;
        for (int32_t k = k0; !bad && k < k1; ++k) {
            brow[k] = (int32_t)i;
            const int32_t cj = A.col[k];
            bad = cj < c0 || cj >= c1;  // block-diagonal: columns stay in the instance
        }
        if (bad) atomicOr(A.S.bar + 32, 1u);
        const int32_t ab = s_b0[inst] & ~3;
        uint8_t fl = 0;
        if (k1 == k0) fl = 2;
        else if ((k0 - ab) / S != (k1 - 1 - ab) / S) fl = 1;
        rowflag[i] = fl;
        double rr[3];
        float uu[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            rr[c] = A.sign * A.b[3 * i + c];
            x[3 * i + c] = 0.0;
            p[3 * i + c] = 0.0f;
            s[3 * i + c] = 0.0f;
            w[3 * i + c] = 0.0f;
            r[3 * i + c] = rr[c];
        }
        precond32(A.dinv32 + 9 * i, rr, uu);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            u[3 * i + c] = uu[c];
            gi = fma(rr[c], (double)uu[c], gi);
            ri = fma(rr[c], rr[c], ri);
        }
    });
    ok = grid_sync(count, nblocks, epoch, A.status);
    if (ok && ld_acquire_u32(A.S.bar + 32) != 0u) {
        if (gtid == 0) set_status(A.status, ST_BAD_INDEX);
        ok = false;
    }

    // ---- per-instance recurrence state, in the owner thread's registers
    double alpha_old[kInstPerThread], gamma_old[kInstPerThread], bnorm2[kInstPerThread], rnorm2[kInstPerThread];
    int32_t it[kInstPerThread];
    uint8_t fresh[kInstPerThread], tight[kInstPerThread], last_verify[kInstPerThread], restart[kInstPerThread],
        done[kInstPerThread];
#pragma unroll
    for (int q = 0; q < kInstPerThread; ++q) {
        alpha_old[q] = gamma_old[q] = 1.0;
        bnorm2[q] = rnorm2[q] = 0.0;
        it[q] = 0;
        fresh[q] = 1;
        tight[q] = last_verify[q] = restart[q] = 0;
        done[q] = 0;
    }
    const double tol2 = A.tol * A.tol;
    // slices of the active instances for the next S phase (all at first)
    block_scan(ni, nsl, s_aptr, s_warp);

    for (int64_t kk = 0; ok; ++kk) {
        const int par = (int)(kk & 1);
        double *gr_cur = acc_gr + par * 2 * kBatchMaxInst;
        double *gr_next = acc_gr + (par ^ 1) * 2 * kBatchMaxInst;
        double *d_cur = acc_d + par * kBatchMaxInst;
        double *d_next = acc_d + (par ^ 1) * kBatchMaxInst;
        // gr_next was last read in the scalar step of kk - 1
        if (blockIdx.x == 0)
            for (int k = threadIdx.x; k < 2 * ni; k += blockDim.x) gr_next[k] = 0.0;

        // ---- S phase: w = A32 u over the active slices, delta per instance
        {
            const int64_t nact = s_aptr[ni];
            const int64_t per = div_up(nact, nwarps);
            const int64_t a0 = min64(gwarp * per, nact), a1 = min64(a0 + per, nact);
            int inst = a0 < a1 ? find_seg(s_aptr, ni, a0) : 0;
            double dsum = 0.0;
            auto slice_of = [&](int64_t a, int &si, int64_t &abase, int &qlo, int &cnt) {
                while (a >= s_aptr[si + 1]) ++si;
                const int64_t j = a - s_aptr[si];
                const int64_t ab = (int64_t)(s_b0[si] & ~3) + j * S;
                abase = ab;
                qlo = (int)max64(0, s_b0[si] - ab);
                cnt = (int)min64(S, s_b0[si + 1] - ab);
            };
            // NS-stage pipeline: slice a + NS - 1 streams in while slice a is used
            constexpr int NS = s_stages<K>();
            constexpr int kFB = bsl::Geom<float, K>::kBufBytes;
            int sp = inst;   // instance cursor of the prefetch, monotone like a
#pragma unroll
            for (int q = 0; q < NS - 1; ++q) {
                if (a0 + q < a1) {
                    int64_t ab;
                    int ql, cn;
                    slice_of(a0 + q, sp, ab, ql, cn);
                    bsl::stage<float, K>(wbuf + q * kFB, ab, cn, A.val32, A.col, brow, lane);
                }
                cp_async_commit();
            }
            int cur = 0;     // buffer of slice a
            for (int64_t a = a0; a < a1; ++a) {
                int64_t ab;
                int ql, cn;
                int sj = inst;
                slice_of(a, sj, ab, ql, cn);
                if (a + NS - 1 < a1) {
                    int64_t ab2;
                    int ql2, cn2;
                    slice_of(a + NS - 1, sp, ab2, ql2, cn2);
                    const int nbuf = cur + NS - 1 >= NS ? cur - 1 : cur + NS - 1;
                    bsl::stage<float, K>(wbuf + nbuf * kFB, ab2, cn2, A.val32, A.col, brow, lane);
                }
                cp_async_commit();
                cp_async_wait<NS - 1>();
                __syncwarp();
                if (sj != inst) {
                    const double t = warp_sum(dsum);
                    if (lane == 0 && t != 0.0) atomicAdd(d_cur + inst, t);
                    dsum = 0.0;
                    inst = sj;
                }
                dsum += bsl::spmv<float, true, K>(wbuf + cur * kFB, ql, cn, u, w, rowflag, join, lane);
                cur = cur + 1 == NS ? 0 : cur + 1;
            }
            cp_async_wait<0>();
            const double t = warp_sum(dsum);
            if (lane == 0 && a0 < a1 && t != 0.0) atomicAdd(d_cur + inst, t);
        }
        if (!grid_sync(count, nblocks, epoch, A.status)) { ok = false; break; }

        // ---- scalars: one owner thread per instance, in every CTA
#pragma unroll
        for (int q = 0; q < kInstPerThread; ++q) {
            const int i = threadIdx.x + q * kPcgBlock;
            if (i >= ni) continue;
            if (done[q]) {
                s_dec[i] = 5;
                s_ref[i] = 0;
                continue;
            }
            const double g = __ldcg(gr_cur + 2 * i), rh = __ldcg(gr_cur + 2 * i + 1), dl = __ldcg(d_cur + i);
            int decision = 0;
            double alpha = 0.0, beta = 0.0;
            rnorm2[q] = rh;
            if (it[q] == 0) bnorm2[q] = rh;
            if (!isfinite(rh) || !isfinite(g) || !isfinite(dl)) decision = 3;
            else if (bnorm2[q] == 0.0 || rh <= tol2 * bnorm2[q]) decision = (fresh[q] || A.refine_every == 0) ? 1 : 4;
            else if (it[q] >= A.max_iter) decision = 2;
            if (last_verify[q] && decision != 1 && !tight[q]) {
                tight[q] = 1;
                restart[q] = 1;
            }
            bool ref = false;
            if (decision == 0 || decision == 4) {
                ref = decision == 4 || tight[q] || (A.refine_every > 0 && ((it[q] + 1) % A.refine_every) == 0);
                fresh[q] = ref;
                last_verify[q] = decision == 4;
            }
            if (decision == 0) {
                if (it[q] == 0 || restart[q]) {
                    alpha = g / dl;
                    restart[q] = 0;
                } else {
                    const double t = gamma_old[q] * alpha_old[q];
                    beta = g / gamma_old[q];
                    alpha = (g * t) / fma(dl, t, -g * g);
                }
                if (!isfinite(alpha) || !isfinite(beta)) decision = 3;
                gamma_old[q] = g;
                alpha_old[q] = alpha;
            }
            if (decision == 1 || decision == 2 || decision == 3) {
                done[q] = 1;
                ref = false;
                if (blockIdx.x == 0) {
                    A.iters_out[i] = it[q];
                    A.relres_out[i] = bnorm2[q] > 0.0 ? sqrt(rnorm2[q] / bnorm2[q]) : 0.0;
                    if (decision == 2) set_status(A.status, ST_NOT_CONVERGED);
                    if (decision == 3) set_status(A.status, ST_NONFINITE);
                }
            } else if (decision == 0) {
                ++it[q];
            }
            s_alpha[i] = alpha;
            s_beta[i] = beta;
            s_dec[i] = (int8_t)decision;
            s_ref[i] = ref ? 1 : 0;
        }
        __syncthreads();
        // active slices for the next S phase, refining slices for this P phase
        const int n_act_slices =
            block_scan(ni, [&](int i) { return (s_dec[i] == 0 || s_dec[i] == 4) ? nsl(i) : 0; }, s_aptr, s_warp);
        const int n_ref_slices = block_scan(ni, [&](int i) { return s_ref[i] ? nsl(i) : 0; }, s_rptr, s_warp);
        block_scan(ni, [&](int i) { return (s_dec[i] == 0 || s_dec[i] == 4) ? s_irow[i + 1] - s_irow[i] : 0; },
                   s_arow, s_warp);
        block_scan(ni, [&](int i) { return s_ref[i] ? s_irow[i + 1] - s_irow[i] : 0; }, s_rrow, s_warp);
        if (n_act_slices == 0) break;  // every instance has stopped (same in every CTA)

        // delta slot of kk + 1 was last read in the scalar step of kk - 1
        if (blockIdx.x == 0)
            for (int k = threadIdx.x; k < ni; k += blockDim.x) d_next[k] = 0.0;

        // ---- P phase over the rows of the instances that step or verify
        act_pass(s_arow, gr_next, [&](int64_t iA, int instA, bool okA, int64_t iB, int instB, bool okB, double &gA,
                                      double &rA, double &gB, double &rB) {
            const int64_t rw[2] = {iA, iB};
            const int in_[2] = {instA, instB};
            const bool ok2[2] = {okA, okB};
            float uu[2][3], ww[2][3], pp[2][3], ss[2][3], D[2][9];
            double xx[2][3], rr[2][3];
            bool fl[2] = {false, false};
            // every load of both rows first (the flag byte and the
            // preconditioner too: after a store the compiler may not move
            // them up, a byte or float load could alias it)
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                if (!ok2[h]) continue;
                const int64_t i = rw[h];
                fl[h] = rowflag[i] != 0;
                if (s_dec[in_[h]] != 0) continue;
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    uu[h][c] = __ldcg(u + 3 * i + c);
                    ww[h][c] = __ldcg(w + 3 * i + c);
                    pp[h][c] = p[3 * i + c];
                    ss[h][c] = s[3 * i + c];
                    xx[h][c] = x[3 * i + c];
                    rr[h][c] = r[3 * i + c];
                }
                if (!s_ref[in_[h]]) {
#pragma unroll
                    for (int e = 0; e < 9; ++e) D[h][e] = A.dinv32[9 * i + e];
                }
            }
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                if (!ok2[h]) continue;
                const int64_t i = rw[h];
                const int inst = in_[h];
                const int dec = s_dec[inst];
                const bool flagged = fl[h];
                if (dec == 4) {
                    // verify: no Krylov step; only clear what receives atomics
                    if (flagged) {
#pragma unroll
                        for (int c = 0; c < 3; ++c) {
                            w[3 * i + c] = 0.0f;
                            ax[3 * i + c] = 0.0;
                        }
                    }
                    continue;
                }
                if (dec != 0) continue;
                const bool ref = s_ref[inst] != 0;
                const double alpha = s_alpha[inst];
                const float beta32 = (float)s_beta[inst];
                double rn[3];
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    const float pn = fmaf(beta32, pp[h][c], uu[h][c]);
                    const float sn = fmaf(beta32, ss[h][c], ww[h][c]);
                    p[3 * i + c] = pn;
                    s[3 * i + c] = sn;
                    x[3 * i + c] = fma(alpha, (double)pn, xx[h][c]);
                    rn[c] = fma(-alpha, (double)sn, rr[h][c]);
                    r[3 * i + c] = rn[c];
                }
                if (flagged) {
#pragma unroll
                    for (int c = 0; c < 3; ++c) {
                        w[3 * i + c] = 0.0f;
                        if (ref) ax[3 * i + c] = 0.0;
                    }
                }
                if (!ref) {
                    float un[3];
                    precond32(D[h], rn, un);
                    double gi = 0.0, ri = 0.0;
#pragma unroll
                    for (int c = 0; c < 3; ++c) {
                        u[3 * i + c] = un[c];
                        gi = fma(rn[c], (double)un[c], gi);
                        ri = fma(rn[c], rn[c], ri);
                    }
                    if (h == 0) { gA = gi; rA = ri; } else { gB = gi; rB = ri; }
                }
            }
        });
        if (n_ref_slices > 0) {
            // ---- residual replacement for the refining instances: r = b - A64 x
            if (!grid_sync(count, nblocks, epoch, A.status)) { ok = false; break; }
            const int64_t per = div_up(n_ref_slices, nwarps);
            const int64_t a0 = min64(gwarp * per, (int64_t)n_ref_slices);
            const int64_t a1 = min64(a0 + per, (int64_t)n_ref_slices);
            int si = a0 < a1 ? find_seg(s_rptr, ni, a0) : 0;
            for (int64_t a = a0; a < a1; ++a) {
                while (a >= s_rptr[si + 1]) ++si;
                const int64_t ab = (int64_t)(s_b0[si] & ~3) + (a - s_rptr[si]) * S;
                const int ql = (int)max64(0, s_b0[si] - ab);
                const int cn = (int)min64(S, s_b0[si + 1] - ab);
                bsl::stage<double, K>(wbuf, ab, cn, A.val64, A.col, brow, lane);
                cp_async_commit();
                cp_async_wait<0>();
                __syncwarp();
                bsl::spmv<double, false, K>(wbuf, ql, cn, x, ax, rowflag, join, lane);
            }
            if (!grid_sync(count, nblocks, epoch, A.status)) { ok = false; break; }
            act_pass(s_rrow, gr_next, [&](int64_t iA, int instA, bool okA, int64_t iB, int instB, bool okB,
                                          double &gA, double &rA, double &gB, double &rB) {
                const int64_t rw[2] = {iA, iB};
                const bool ok2[2] = {okA, okB};
                double axv[2][3], bv[2][3];
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    if (!ok2[h]) continue;
#pragma unroll
                    for (int c = 0; c < 3; ++c) {
                        axv[h][c] = __ldcg(ax + 3 * rw[h] + c);
                        bv[h][c] = A.b[3 * rw[h] + c];
                    }
                }
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    if (!ok2[h]) continue;
                    const int64_t i = rw[h];
                    double rn[3];
                    float un[3];
#pragma unroll
                    for (int c = 0; c < 3; ++c) {
                        rn[c] = fma(A.sign, bv[h][c], -axv[h][c]);
                        r[3 * i + c] = rn[c];
                    }
                    precond32(A.dinv32 + 9 * i, rn, un);
                    double gi = 0.0, ri = 0.0;
#pragma unroll
                    for (int c = 0; c < 3; ++c) {
                        u[3 * i + c] = un[c];
                        gi = fma(rn[c], (double)un[c], gi);
                        ri = fma(rn[c], rn[c], ri);
                    }
                    if (h == 0) { gA = gi; rA = ri; } else { gB = gi; rB = ri; }
                }
                (void)instA;
                (void)instB;
            });
        }
        if (!grid_sync(count, nblocks, epoch, A.status)) { ok = false; break; }
    }
    cp_async_wait<0>();
    // instances still running when a barrier timed out report what they have
    if (blockIdx.x == 0) {
#pragma unroll
        for (int q = 0; q < kInstPerThread; ++q) {
            const int i = threadIdx.x + q * kPcgBlock;
            if (i < ni && !done[q]) {
                A.iters_out[i] = it[q];
                A.relres_out[i] = bnorm2[q] > 0.0 ? sqrt(rnorm2[q] / bnorm2[q]) : 0.0;
                if (ok) set_status(A.status, ST_NOT_CONVERGED);
            }
        }
    }
}

__global__ void coarse_offsets_kernel(int32_t n_inst, int32_t n_fine, const int32_t *__restrict__ vert_ptr,
                                      const int32_t *__restrict__ labels, const int32_t *__restrict__ n_c_dev,
                                      int32_t *__restrict__ inst_row, uint32_t *status)
{
    const int32_t nc = *n_c_dev;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i <= n_inst; i += gridDim.x * blockDim.x) {
        const int32_t v = vert_ptr[i];
        if (v < 0 || v > n_fine) {
            set_status(status, ST_BAD_INDEX);
            inst_row[i] = 0;
            continue;
        }
        inst_row[i] = (i == n_inst || v == n_fine) ? nc : labels[v];
    }
}

template <int K>
const void *kernel_ptr()
{
    return reinterpret_cast<const void *>(&pcg_batched_kernel<K>);
}

const int kVariants[kBatchVariants] = {4, 5, 6, 8};

const void *variant_ptr(int v)
{
    switch (v) {
    case 0: return kernel_ptr<4>();
    case 1: return kernel_ptr<5>();
    case 2: return kernel_ptr<6>();
    default: return kernel_ptr<8>();
    }
}

int variant_smem(int v)
{
    switch (v) {
    case 0: return Layout<4>::kTotal;
    case 1: return Layout<5>::kTotal;
    case 2: return Layout<6>::kTotal;
    default: return Layout<8>::kTotal;
    }
}

}  // namespace

// Called by agipc_create: opt each variant into its shared memory and size
// its cooperative grid.  Returns false on a CUDA error.
bool batched_configure(agipc_ctx *c)
{
    for (int v = 0; v < kBatchVariants; ++v) {
        int per_sm = 0;
        if (cudaFuncSetAttribute(variant_ptr(v), cudaFuncAttributeMaxDynamicSharedMemorySize, variant_smem(v)) !=
                cudaSuccess ||
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, variant_ptr(v), kPcgBlock, variant_smem(v)) !=
                cudaSuccess)
            return false;
        c->batch_grid[v] = std::min(std::max(per_sm, 0), kMaxGridLanes * 32 / std::max(c->num_sms, 1)) * c->num_sms;
    }
    return true;
}

extern "C" int agipc_batch_coarse_offsets(agipc_ctx *ctx, int32_t n_inst, int32_t n_fine, const int32_t *vert_ptr,
                                          const int32_t *labels, const int32_t *n_coarse_dev, int32_t *inst_row)
{
    if (!ctx || n_inst <= 0 || n_inst > kBatchMaxInst || n_fine <= 0 || n_fine > ctx->max_n || !vert_ptr ||
        !labels || !n_coarse_dev || !inst_row)
        return AGIPC_ERR_INVALID_ARG;
    coarse_offsets_kernel<<<(unsigned)div_up(n_inst + 1, 256), 256, 0, ctx->stream>>>(n_inst, n_fine, vert_ptr, labels,
                                                                                  n_coarse_dev, inst_row, ctx->status);
    return cudaPeekAtLastError() == cudaSuccess ? AGIPC_OK : AGIPC_ERR_CUDA;
}

extern "C" int agipc_pcg_batched(agipc_ctx *ctx, int32_t n_inst, const int32_t *inst_row, int32_t max_rows,
                                 const int32_t *row_ptr, const int32_t *col, const double *val, const float *val32,
                                 const float *dinv32, const double *b, double *x, const agipc_pcg_options *opt,
                                 int32_t refine_every, int32_t blocks_per_lane, int32_t *iters_dev,
                                 double *relres_dev)
{
    if (!ctx || !opt || n_inst <= 0 || n_inst > kBatchMaxInst || max_rows < 0 || max_rows > ctx->max_n ||
        !inst_row || !row_ptr || !col || !val || !val32 || !dinv32 || !b || !x || !iters_dev || !relres_dev ||
        refine_every < 0)
        return AGIPC_ERR_INVALID_ARG;
    if (!(opt->tol >= 0.0) || opt->max_iter < 0 || (opt->rhs_sign != 1 && opt->rhs_sign != -1) || opt->use_x0)
        return AGIPC_ERR_INVALID_ARG;
    if (((uintptr_t)val & 15u) != 0 || ((uintptr_t)val32 & 15u) != 0 || ((uintptr_t)col & 15u) != 0 ||
        ((uintptr_t)dinv32 & 3u) != 0 || ((uintptr_t)b & 7u) != 0 || ((uintptr_t)x & 7u) != 0)
        return AGIPC_ERR_INVALID_ARG;
    int v = -1;
    for (int k = 0; k < kBatchVariants; ++k)
        if (kVariants[k] == (blocks_per_lane == 0 ? 5 : blocks_per_lane)) v = k;
    if (v < 0 || ctx->batch_grid[v] <= 0) return AGIPC_ERR_INVALID_ARG;
    BatchArgs A;
    A.n_inst = n_inst;
    A.inst_row = inst_row;
    A.max_rows = max_rows;
    A.max_nnzb = ctx->max_nnzb;
    A.rp = row_ptr;
    A.col = col;
    A.val64 = val;
    A.val32 = val32;
    A.dinv32 = dinv32;
    A.b = b;
    A.x = x;
    A.sign = (double)opt->rhs_sign;
    A.tol = opt->tol;
    A.max_iter = opt->max_iter;
    A.refine_every = refine_every;
    A.iters_out = iters_dev;
    A.relres_out = relres_dev;
    A.S = ctx->pcg;
    A.acc = ctx->batch_acc;
    A.status = ctx->status;
    if (cudaMemsetAsync(ctx->pcg.bar, 0, 64 * sizeof(unsigned), ctx->stream) != cudaSuccess ||
        cudaMemsetAsync(ctx->batch_acc, 0, 6 * kBatchMaxInst * sizeof(double), ctx->stream) != cudaSuccess)
        return AGIPC_ERR_CUDA;
    void *args[] = {&A};
    const cudaError_t e = cudaLaunchCooperativeKernel(variant_ptr(v), dim3((unsigned)ctx->batch_grid[v]),
                                                      dim3(kPcgBlock), args, (size_t)variant_smem(v), ctx->stream);
    return e == cudaSuccess ? AGIPC_OK : AGIPC_ERR_CUDA;
}
