// Block-Jacobi PCG on a full-storage 3x3 BSR matrix (Algorithm 1's coarse
// solve d_c = -H_c^-1 g_c; Sec. 5 stops on the relative residual norm and
// Sec. 5.1 names the 3x3 block-Jacobi preconditioner).
//
// The whole solve is one persistent cooperative kernel with device-side
// convergence.  The recurrence is the Chronopoulos-Gear form of PCG, which
// is algebraically the textbook method but needs a single reduction per
// iteration (gamma = r.u, rho = r.r and delta = u.Au together):
//     u = M^-1 r,  w = A u,  gamma = (r,u),  delta = (w,u)
//     beta = gamma/gamma_old,  alpha = gamma/(delta - beta*gamma/alpha_old)
//     p = u + beta p,  s = w + beta s,  x += alpha p,  r -= alpha s
//
// GB300 design.  The SM's FP64 unit retires about 1.7 FMA lanes per clock
// (one warp instruction per ~19 SM cycles), and one warp issues at most one
// FP64 instruction per ~64 cycles whether its instructions depend on each
// other or not, whatever the active mask; so the kernel counts FP64 warp
// instructions: a 3x3 block costs 9 FMAs and everything else per block, per
// row and per reduction is kept small next to that.
//   S phase (w = A u): the blocks are cut into slices of 128 (32 lanes x 4
//     consecutive blocks); slices go round-robin to warps spread over all
//     CTAs.  Two layouts (template kW):
//     - 8 warps per SM: each warp owns two shared-memory slice buffers.
//       When the matrix fits (at most one slice per warp) the slice is
//       loaded once by cp.async and stays resident for the whole solve;
//       otherwise the next slice (also the first slice of the next
//       iteration) streams in by TMA bulk copy, completing on the buffer's
//       mbarrier, while the current one is multiplied.
//     - 16 warps per SM (agipc_pcg_options.streamed): one buffer per warp,
//       the matrix always streamed by cp.async; twice the warps keep the
//       FP64 pipe busy while some wait for their slices.
//     Each lane reads its blocks with 16-byte shared loads and accumulates
//     them in registers, one accumulator per row segment; segments that
//     cross lanes are joined by the lane where the row starts.  Column
//     gathers of u, u of the lane's rows (for delta) and the rows' split
//     flags are plain L1-cacheable loads, all issued together before any is
//     used.  A row inside one slice is stored; a row cut by a slice boundary
//     is added with FP64 atomics (w of such rows is zeroed in the P phase).
//   P phase: rows are split evenly over the CTAs; each thread does the
//     row-local updates, the 3x3 preconditioner and its share of gamma, rho;
//     the CTA's sums of those shares are formed during the next S phase by
//     the CTA's last warp (the one with the fewest slices).
//   CTA sums go through shared memory, one warp per summed value; CTA
//     partials go to per-CTA slots and every CTA reduces all slots in the
//     same order (again one warp per value), so the scalars are bitwise
//     identical in every CTA and from run to run; one thread does the
//     divisions.
//   Each phase ends in a grid barrier (monotone arrival counter, bounded
//     spin).
#include <algorithm>

#include "agipc_common.cuh"
#include "pcg_slices.cuh"

using namespace pcgs;

namespace {

struct PcgArgs {
    const int32_t *n_dev;
    const int32_t *rp;
    const int32_t *col;
    const double *val;
    const double *dinv;
    const double *b;
    double *x;
    double sign;
    double tol;
    int32_t max_iter;
    int32_t use_x0;
    int32_t max_rows;
    int64_t max_nnzb;
    int32_t *iters_dev;
    double *relres_dev;
    PcgScratch S;
    uint32_t *status;
};

// FP64 class test on the bit pattern (integer instructions only).
__device__ __forceinline__ bool finite_bits(double v)
{
    return ((__double_as_longlong(v) >> 52) & 0x7ff) != 0x7ff;
}

// Row-local update of one row i: p = u + beta p, s = w + beta s,
// x += alpha p, r -= alpha s, u = M^-1 r; returns gamma, rho shares.
__device__ __forceinline__ void row_update(int64_t i, const double uu[3], const double ww[3], double pp[3], double ss[3],
                                           double rr[3], const double xx[3], const double D[9], double alpha, double beta,
                                           double *p, double *s, double *r, double *x, double *u, double *w,
                                           bool zero_w, double &gpart, double &rpart)
{
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        pp[c] = fma(beta, pp[c], uu[c]);
        ss[c] = fma(beta, ss[c], ww[c]);
        x[3 * i + c] = fma(alpha, pp[c], xx[c]);
        rr[c] = fma(-alpha, ss[c], rr[c]);
        p[3 * i + c] = pp[c];
        s[3 * i + c] = ss[c];
        r[3 * i + c] = rr[c];
    }
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const double uc = fma(D[3 * c + 2], rr[2], fma(D[3 * c + 1], rr[1], D[3 * c] * rr[0]));
        u[3 * i + c] = uc;
        gpart = fma(rr[c], uc, gpart);
        rpart = fma(rr[c], rr[c], rpart);
    }
    if (zero_w) {
        w[3 * i] = 0.0;
        w[3 * i + 1] = 0.0;
        w[3 * i + 2] = 0.0;
    }
}

// Shared-memory layout of the two variants.  kW = 8 warps (up to 255
// registers): each warp owns two slice buffers; a matrix whose slices fit one
// per warp is held there for the whole solve (resident mode), a larger one
// streams through both buffers.  kW = 16 warps (at most 128 registers): twice
// the warps keep the FP64 pipe fed while others wait for their slices; each
// warp's region holds one slice and the matrix always streams.
template <int kW>
struct PcgGeom {
    static constexpr bool kWide = kW > kPcgWarps;
    static constexpr int kBufArea = kWide ? kBufBytes : 2 * kBufBytes;   // slice buffers of one warp
    static constexpr int kRegion = kBufArea + kJoinBytes;
    static constexpr int kSmem = kW * kRegion + 32 * kW * 3 * 8;          // + the CTA-sum slots
    static_assert(kRegion % 16 == 0, "16-byte aligned slice buffers");
};

template <int kW>
__global__ void __launch_bounds__(32 * kW, 1) pcg_kernel(PcgArgs A)
{
    using Geo = PcgGeom<kW>;
    constexpr bool kWide = Geo::kWide;
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ double s_scal[2];
    __shared__ double s_tot[4];
    __shared__ double s_grid[4];
    __shared__ double s_gr[2 * 32 * kW];   // the P phase's per-thread gamma, rho shares
    __shared__ int s_dec;
    __shared__ int s_abort;
    __shared__ __align__(8) uint64_t s_mbar[2 * kW];   // one per slice buffer of each warp

    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const unsigned nblocks = gridDim.x;
    const int64_t nwarps = (int64_t)nblocks * kW;
    const int64_t gwarp = (int64_t)wib * nblocks + blockIdx.x;  // slices interleave over CTAs
    const int64_t gtid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;

    const int32_t n = *A.n_dev;
    if (n < 0 || n > A.max_rows || nblocks > 32 * kMaxGridLanes) {
        if (gtid == 0) set_status(A.status, ST_BAD_INDEX);
        return;
    }
    const int64_t nnz = A.rp[n];
    if (nnz < 0 || nnz > A.max_nnzb) {
        if (gtid == 0) set_status(A.status, nnz < 0 ? ST_BAD_INDEX : ST_CAPACITY);
        return;
    }
    const int64_t nslices = div_up(nnz, kSlice);
    // every warp keeps at most one slice in shared memory
    const bool resident = !kWide && nslices <= nwarps;
    // rows owned by this CTA in the row-local phases
    const int64_t rows_per_cta = div_up(n, nblocks);
    const int64_t row0 = min64((int64_t)blockIdx.x * rows_per_cta, n);
    const int64_t row1 = min64(row0 + rows_per_cta, n);
    // row state can be fetched ahead of the barrier (the 8-warp variant)
    const bool one_row = !kWide && rows_per_cta <= kPcgBlock;

    double *__restrict__ r = A.S.r;
    double *u = A.S.u;
    double *w = A.S.w;
    double *__restrict__ p = A.S.p;
    double *__restrict__ s = A.S.s;
    double *__restrict__ x = A.x;
    int32_t *brow = A.S.brow;
    uint8_t *rowflag = A.S.rowflag;
    double *partials = A.S.partials;
    unsigned *count = A.S.bar;
    // partial sums: scalar s of CTA k at [s * mg + k] (scalar-major, so a
    // warp reducing one scalar reads consecutive words)
    const int mg = A.S.max_grid;
    const int pstride = mg * 4;
    unsigned epoch = 0;
    unsigned char *wbuf = smem + (size_t)wib * Geo::kRegion;
    unsigned char *join = wbuf + Geo::kBufArea;
    double *s_part = reinterpret_cast<double *>(smem + (size_t)kW * Geo::kRegion);

    // ---- setup: block rows, split flags, x = 0 (or the given x0), r = b - A x0,
    // u = M^-1 r, p = s = w = 0; with x0 the residual needs A x0, so it is
    // formed after a first slice pass
    const bool x0 = A.use_x0 != 0;
    double gpart = 0.0, rpart = 0.0, bpart = 0.0;
    for (int64_t i = row0 + threadIdx.x; i < row1; i += blockDim.x) {
        const int32_t k0 = A.rp[i], k1 = A.rp[i + 1];
        bool bad = k0 < 0 || k1 < k0 || k1 > nnz;
        for (int32_t k = k0; !bad && k < k1; ++k) {
            brow[k] = (int32_t)i;
            bad = (unsigned)A.col[k] >= (unsigned)n;
        }
        if (bad) atomicOr(A.S.bar + 32, 1u);
        uint8_t f = 0;
        if (k1 == k0) f = 2;
        else if (k0 / kSlice != (k1 - 1) / kSlice) f = 1;
        rowflag[i] = f;
        double rr[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            rr[c] = A.sign * A.b[3 * i + c];
            bpart += rr[c] * rr[c];
            if (!x0) x[3 * i + c] = 0.0;
            p[3 * i + c] = 0.0;
            s[3 * i + c] = 0.0;
            w[3 * i + c] = 0.0;
            r[3 * i + c] = rr[c];
        }
        if (x0) continue;
        const double *D = A.dinv + 9 * i;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const double uc = D[3 * c] * rr[0] + D[3 * c + 1] * rr[1] + D[3 * c + 2] * rr[2];
            u[3 * i + c] = uc;
            gpart += rr[c] * uc;
            rpart += rr[c] * rr[c];
        }
    }
    bool ok = true;
    if (x0) {
        if (!grid_sync(count, nblocks, epoch, A.status)) ok = false;
        if (ok && ld_acquire_u32(A.S.bar + 32) != 0u) {
            if (gtid == 0) set_status(A.status, ST_BAD_INDEX);
            ok = false;
        }
        // w = A x0, one slice at a time
        double unused = 0.0;
        for (int64_t sl = gwarp; ok && sl < nslices; sl += nwarps) {
            issue_slice(wbuf, sl, nnz, A.val, A.col, brow, lane);
            cp_async_commit();
            cp_async_wait<0>();
            __syncwarp();
            const int cnt = (int)min64(kSlice, nnz - sl * kSlice);
            slice_spmv<double, false>(wbuf, cnt, x, w, rowflag, join, lane, unused);
        }
        if (ok && !grid_sync(count, nblocks, epoch, A.status)) ok = false;
        for (int64_t i = row0 + threadIdx.x; ok && i < row1; i += blockDim.x) {
            double rr[3];
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                rr[c] = fma(A.sign, A.b[3 * i + c], -__ldcg(w + 3 * i + c));
                r[3 * i + c] = rr[c];
                w[3 * i + c] = 0.0;
            }
            const double *D = A.dinv + 9 * i;
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                const double uc = D[3 * c] * rr[0] + D[3 * c + 1] * rr[1] + D[3 * c + 2] * rr[2];
                u[3 * i + c] = uc;
                gpart += rr[c] * uc;
                rpart += rr[c] * rr[c];
            }
        }
    }
    {
        double v[3] = {gpart, rpart, bpart};
        cta_sum<3, kW>(v, s_part, s_tot);
        if (threadIdx.x == 0) {
            partials[0 * mg + blockIdx.x] = v[0];
            partials[1 * mg + blockIdx.x] = v[1];
            partials[3 * mg + blockIdx.x] = v[2];
        }
    }
    ok = grid_sync(count, nblocks, epoch, A.status) && ok;
    if (ok && ld_acquire_u32(A.S.bar + 32) != 0u) {
        // a row pointer or column index out of range: nothing gathers through it
        if (gtid == 0) set_status(A.status, ST_BAD_INDEX);
        ok = false;
    }
    // Streamed slices of the 8-warp layout: a full slice goes by TMA bulk
    // copy and completes on its buffer's mbarrier; the ragged last slice of
    // the matrix goes by the zero-filling cp.async path (a bulk copy would
    // need lengths rounded up to 16 bytes, past the caller's arrays).  `ph`
    // holds each buffer's next parity, `pend` the buffers with a bulk copy in
    // flight (drained before the kernel ends).  A resident slice is loaded
    // once by cp.async.  The 16-warp layout keeps cp.async for every slice:
    // at its 128 registers the bulk path's state spills, and it measured
    // slower (100.3 against 96.1 us per iteration on the 2.28M-block fine
    // system).
    constexpr bool kBulk = !kWide;
    uint64_t *mbar = s_mbar + 2 * wib;
    unsigned ph = 0, pend = 0;
    if (threadIdx.x == 0) s_abort = 0;
    if (lane == 0) {
        mbar_init(mbar);
        mbar_init(mbar + 1);
    }
    __syncthreads();
    auto slice_issue = [&](int k, int64_t sl) {
        if (kBulk && !resident && (sl + 1) * kSlice <= nnz) {
            issue_slice_bulk<double>(wbuf + k * kBufBytes, sl, A.val, A.col, brow, mbar + k, lane);
            pend |= 1u << k;
        } else {
            issue_slice(wbuf + k * kBufBytes, sl, nnz, A.val, A.col, brow, lane);
            cp_async_commit();
        }
    };
    auto slice_wait = [&](int k, int64_t sl) {
        if (kBulk && !resident && (sl + 1) * kSlice <= nnz) {
            if (!mbar_wait(mbar + k, (ph >> k) & 1u)) {
                set_status(A.status, ST_TIMEOUT);
                s_abort = 1;
            }
            ph ^= 1u << k;
            pend &= ~(1u << k);
        } else {
            cp_async_wait<0>();
        }
        __syncwarp();
    };
    // The warp's first slice goes to buffer 0 (brow is complete after the
    // barrier).  Invariant: each iteration's first slice sits in buffer nb.
    int nb = 0;
    if (ok && gwarp < nslices) slice_issue(0, gwarp);

    double gamma_old = 1.0, bnorm2 = 0.0, rnorm2 = 0.0, tolb = 0.0;
    double tt = 1.0, ttg = 1.0;   // gamma_old alpha_old and its product with gamma_old
    const double tol2 = A.tol * A.tol;
    int32_t it = 0;
    bool converged = false;
    while (ok) {
        const int par = it & 1;
        double *part = partials + par * pstride;
        // ---- S phase: w = A u, partial delta
        double dpart = 0.0;
        if constexpr (kWide) {
            // one buffer: the warp's first slice was issued at the end of the
            // previous iteration (it loads during the grid barrier), each later
            // one after the warp has multiplied with the one before; the other
            // warps keep the FP64 pipe busy meanwhile
            for (int64_t sl = gwarp; sl < nslices; sl += nwarps) {
                if (sl != gwarp) slice_issue(0, sl);
                slice_wait(0, sl);
                const int cnt = (int)min64(kSlice, nnz - sl * kSlice);
                slice_spmv<double, true, true>(wbuf, cnt, u, w, rowflag, join, lane, dpart);
            }
        } else {
            for (int64_t sl = gwarp; sl < nslices; sl += nwarps) {
                if (!resident) {
                    // stream the next slice of this iteration, or the first slice
                    // of the next one, into the other buffer while this one is used
                    const int64_t next = sl + nwarps < nslices ? sl + nwarps : gwarp;
                    slice_issue(nb ^ 1, next);
                    slice_wait(nb, sl);
                } else {
                    cp_async_wait<0>();
                    __syncwarp();
                }
                const int cnt = (int)min64(kSlice, nnz - sl * kSlice);
                slice_spmv<double, true>(wbuf + nb * kBufBytes, cnt, u, w, rowflag, join, lane, dpart);
                if (!resident) nb ^= 1;
            }
        }
        if (it > 0 && wib == kW - 1) {
            // the previous P phase's gamma and rho shares, summed over the CTA
            // (fixed order) by the last warp, which holds the fewest slices, so
            // the sum overlaps the other warps' SpMV instead of delaying the
            // barrier after the P phase
            // (eight warps' slots at a time: a tree of three levels each, the
            // groups added in order; with one group a0 = 0 + tree is the tree)
            double a0 = 0.0, a1 = 0.0;
#pragma unroll
            for (int g = 0; g < kW; g += 8) {
                double t0[8], t1[8];
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    t0[q] = s_gr[2 * (lane + 32 * (g + q))];
                    t1[q] = s_gr[2 * (lane + 32 * (g + q)) + 1];
                }
#pragma unroll
                for (int h = 4; h > 0; h >>= 1)
#pragma unroll
                    for (int q = 0; q < h; ++q) {
                        t0[q] += t0[q + h];
                        t1[q] += t1[q + h];
                    }
                a0 += t0[0];
                a1 += t1[0];
            }
            const double g0 = warp_sum(a0), g1 = warp_sum(a1);
            if (lane == 0) {
                part[0 * mg + blockIdx.x] = g0;
                part[1 * mg + blockIdx.x] = g1;
            }
        }
        // one row per thread: fetch the row's own state now, so that only w
        // (written by other CTAs) is read after the barrier
        const int64_t my_row = row0 + threadIdx.x;
        const bool has_row = one_row && my_row < row1;
        double ru[3], rp_[3], rs[3], rr_[3], rx[3], rD[9], rw[3];
        if (has_row) {
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                ru[c] = __ldcg(u + 3 * my_row + c);
                rp_[c] = p[3 * my_row + c];
                rs[c] = s[3 * my_row + c];
                rr_[c] = r[3 * my_row + c];
                rx[c] = x[3 * my_row + c];
            }
#pragma unroll
            for (int e = 0; e < 9; ++e) rD[e] = A.dinv[9 * my_row + e];
        }
        {
            double v[1] = {dpart};
            cta_sum<1, kW>(v, s_part, s_tot);
            if (threadIdx.x == 0) part[2 * mg + blockIdx.x] = v[0];
        }
        if (s_abort) { ok = false; break; }   // a slice never arrived (ST_TIMEOUT is set)
        if (!grid_sync(count, nblocks, epoch, A.status)) { ok = false; break; }
        if (has_row) {
#pragma unroll
            for (int c = 0; c < 3; ++c) rw[c] = __ldcg(w + 3 * my_row + c);
        }

        // ---- global scalars: every CTA reduces all slots in the same order;
        // thread 0 alone does the FP64 divisions and square root.
        if (wib < 4) {
            // warp k reduces scalar k of all CTAs (fixed order); slot 3 holds
            // ||b||^2 in the first iteration
            double pv[kMaxGridLanes];
#pragma unroll
            for (int q = 0; q < kMaxGridLanes; ++q) {
                const unsigned k = lane + 32 * q;
                pv[q] = k < nblocks ? __ldcg(part + wib * mg + k) : 0.0;
            }
#pragma unroll
            for (int h = kMaxGridLanes / 2; h > 0; h >>= 1)
#pragma unroll
                for (int q = 0; q < h; ++q) pv[q] += pv[q + h];
            const double tot = warp_sum(pv[0]);
            if (lane == 0) s_grid[wib] = tot;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            const double g = s_grid[0], rh = s_grid[1], dl = s_grid[2], bb = s_grid[3];
            // 0 iterate, 1 converged, 2 iteration cap, 3 non-finite.  The test
            // ||r|| <= tol ||b|| is done on squares; alpha needs one division:
            // g / (dl - beta g / alpha_old) with beta = g / gamma_old equals
            // g t / (dl t - g^2), t = gamma_old alpha_old.
            // The class tests and the range test read the exponent bits
            // (integer instructions): on this part every FP64 instruction,
            // compares included, is a long step of the dependent chain.
            int decision = 0;
            double alpha = 0.0, beta = 0.0;
            rnorm2 = rh;
            if (it == 0) {
                bnorm2 = bb;
                tolb = tol2 * bnorm2;
            }
            if (!finite_bits(rh) || !finite_bits(g) || !finite_bits(dl)) decision = 3;
            else if (bnorm2 == 0.0 || rh <= tolb) decision = 1;
            else if (it >= A.max_iter) decision = 2;
            else {
                if (it == 0) {
                    alpha = g / dl;
                } else {
                    // beta = g / gamma_old and alpha = g t / den (t carried as
                    // tt, t gamma_old as ttg) share one division by gamma_old
                    // den (an FP64 division is a long dependent chain here);
                    // the two quotients are used when that product leaves the
                    // normal range
                    const double den = fma(dl, tt, -g * g);
                    const double q = gamma_old * den;
                    const int eq = (int)((__double_as_longlong(q) >> 52) & 0x7ff);
                    if (eq >= 1 && eq <= 2019) {
                        const double gi = g * (1.0 / q);
                        beta = gi * den;
                        alpha = gi * ttg;
                    } else {
                        beta = g / gamma_old;
                        alpha = (g * tt) / den;
                    }
                }
                if (!finite_bits(alpha) || !finite_bits(beta)) decision = 3;
            }
            s_scal[0] = alpha;
            s_scal[1] = beta;
            s_dec = decision;
            if (decision == 0) {   // after publishing: the next iteration's products
                gamma_old = g;
                tt = g * alpha;
                ttg = tt * g;
            }
        }
        __syncthreads();
        const double alpha = s_scal[0], beta = s_scal[1];
        const int decision = s_dec;
        __syncthreads();
        if (decision == 3) {
            if (gtid == 0) set_status(A.status, ST_NONFINITE);
            break;
        }
        if (decision == 1) { converged = true; break; }
        if (decision == 2) break;

        // ---- P phase: row-local updates, preconditioner, gamma and rho shares
        // (summed over the CTA during the next S phase)
        gpart = 0.0;
        rpart = 0.0;
        if (one_row) {
            if (has_row) row_update(my_row, ru, rw, rp_, rs, rr_, rx, rD, alpha, beta, p, s, r, x, u, w,
                                    rowflag[my_row] != 0, gpart, rpart);
        } else {
            // kRows rows per thread per pass: every load of the pass is
            // issued before the first store, so their latencies overlap
            constexpr int kRows = kWide ? 1 : 2;
            for (int64_t i0 = row0 + threadIdx.x; i0 < row1; i0 += kRows * (int64_t)blockDim.x) {
                double uu[kRows][3], ww[kRows][3], pp[kRows][3], ss[kRows][3], rr[kRows][3], xx[kRows][3];
                double D[kRows][9];
                bool fl[kRows];
#pragma unroll
                for (int j = 0; j < kRows; ++j) {
                    const int64_t i = i0 + j * (int64_t)blockDim.x;
                    const int64_t k = i < row1 ? i : i0;   // a row of this pass that exists
                    fl[j] = rowflag[k] != 0;
#pragma unroll
                    for (int c = 0; c < 3; ++c) {
                        uu[j][c] = __ldcg(u + 3 * k + c);
                        ww[j][c] = __ldcg(w + 3 * k + c);
                        pp[j][c] = p[3 * k + c];
                        ss[j][c] = s[3 * k + c];
                        rr[j][c] = r[3 * k + c];
                        xx[j][c] = x[3 * k + c];
                    }
#pragma unroll
                    for (int e = 0; e < 9; ++e) D[j][e] = A.dinv[9 * k + e];
                }
#pragma unroll
                for (int j = 0; j < kRows; ++j) {
                    const int64_t i = i0 + j * (int64_t)blockDim.x;
                    if (i >= row1) break;
                    row_update(i, uu[j], ww[j], pp[j], ss[j], rr[j], xx[j], D[j], alpha, beta, p, s, r, x, u, w,
                               fl[j], gpart, rpart);
                }
            }
        }
        s_gr[2 * threadIdx.x] = gpart;
        s_gr[2 * threadIdx.x + 1] = rpart;
        ++it;
        if constexpr (kWide) {
            // the next S phase's first slice loads during the barrier
            if (gwarp < nslices) slice_issue(0, gwarp);
        }
        if (!grid_sync(count, nblocks, epoch, A.status)) { ok = false; break; }
    }
    // no copy into this CTA's shared memory may outlive it
    for (int k = 0; k < 2; ++k)
        if ((pend >> k) & 1u) mbar_wait(mbar + k, (ph >> k) & 1u);
    cp_async_wait<0>();
    if (gtid == 0 && (ok || it > 0)) {
        *A.iters_dev = it;
        *A.relres_dev = bnorm2 > 0.0 ? sqrt(rnorm2 / bnorm2) : 0.0;
        if (ok && !converged) set_status(A.status, ST_NOT_CONVERGED);
    }
    // b = 0: the solution is 0 whatever the initial guess
    if (ok && converged && bnorm2 == 0.0 && x0)
        for (int64_t i = row0 + threadIdx.x; i < row1; i += blockDim.x) {
            x[3 * i] = 0.0;
            x[3 * i + 1] = 0.0;
            x[3 * i + 2] = 0.0;
        }
}

}  // namespace

int pcg_block_size() { return kPcgBlock; }
int pcg_smem_bytes() { return kPcgSmem; }

const void *pcg_kernel_ptr() { return reinterpret_cast<const void *>(&pcg_kernel<kPcgWarps>); }

// The 16-warp streaming variant runs one CTA per SM; false if the SM cannot
// hold it (its shared memory or registers).
bool pcg_wide_configure()
{
    constexpr int kW = 2 * kPcgWarps;
    const void *k = reinterpret_cast<const void *>(&pcg_kernel<kW>);
    int per_sm = 0;
    return cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, PcgGeom<kW>::kSmem) ==
               cudaSuccess &&
           cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, 32 * kW, PcgGeom<kW>::kSmem) == cudaSuccess &&
           per_sm >= 1;
}

extern "C" int agipc_pcg(agipc_ctx *ctx, int32_t max_rows, const int32_t *n_rows_dev, const int32_t *row_ptr,
                         const int32_t *col, const double *val, const double *dinv, const double *b, double *x,
                         const agipc_pcg_options *opt, int32_t *iters_dev, double *relres_dev)
{
    if (!ctx || !opt || max_rows < 0 || max_rows > ctx->max_n || !n_rows_dev || !row_ptr || !dinv || !b || !x ||
        !iters_dev || !relres_dev)
        return AGIPC_ERR_INVALID_ARG;
    if (!(opt->tol >= 0.0) || opt->max_iter < 0 || (opt->rhs_sign != 1 && opt->rhs_sign != -1))
        return AGIPC_ERR_INVALID_ARG;
    if (((uintptr_t)val & 15u) != 0 || ((uintptr_t)col & 15u) != 0 || ((uintptr_t)dinv & 7u) != 0 ||
        ((uintptr_t)b & 7u) != 0 || ((uintptr_t)x & 7u) != 0)
        return AGIPC_ERR_INVALID_ARG;
    PcgArgs A;
    A.n_dev = n_rows_dev;
    A.rp = row_ptr;
    A.col = col;
    A.val = val;
    A.dinv = dinv;
    A.b = b;
    A.x = x;
    A.sign = (double)opt->rhs_sign;
    A.tol = opt->tol;
    A.max_iter = opt->max_iter;
    A.use_x0 = opt->use_x0 != 0;
    A.max_rows = max_rows;
    A.max_nnzb = ctx->max_nnzb;
    A.iters_dev = iters_dev;
    A.relres_dev = relres_dev;
    A.S = ctx->pcg;
    A.status = ctx->status;
    if (cudaMemsetAsync(ctx->pcg.bar, 0, 64 * sizeof(unsigned), ctx->stream) != cudaSuccess) return AGIPC_ERR_CUDA;
    void *args[] = {&A};
    static_assert(PcgGeom<kPcgWarps>::kSmem == kPcgSmem, "the 8-warp layout is the shared PCG layout");
    cudaError_t e;
    if (opt->streamed) {
        constexpr int kW = 2 * kPcgWarps;
        e = cudaLaunchCooperativeKernel(reinterpret_cast<const void *>(&pcg_kernel<kW>), dim3((unsigned)ctx->num_sms),
                                        dim3(32 * kW), args, PcgGeom<kW>::kSmem, ctx->stream);
    } else {
        e = cudaLaunchCooperativeKernel(reinterpret_cast<const void *>(&pcg_kernel<kPcgWarps>),
                                        dim3((unsigned)ctx->pcg_grid), dim3(kPcgBlock), args, kPcgSmem, ctx->stream);
    }
    return e == cudaSuccess ? AGIPC_OK : AGIPC_ERR_CUDA;
}
