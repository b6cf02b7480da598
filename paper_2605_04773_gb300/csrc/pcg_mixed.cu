// Mixed-precision block-Jacobi PCG: the precision form of the coarse solve.
//
// The 3x3 blocks, the SpMV and the block-Jacobi preconditioner run in FP32;
// the dot products (gamma = r.u, rho = r.r, delta = u.Au) are accumulated in
// FP64; x and r are kept in FP64, and every `refine_every` iterations r is
// replaced by the true residual b - A x computed with the FP64 master matrix
// (residual replacement), so the iteration converges to the FP64 system's
// solution while nearly all of its arithmetic runs on the FP32 units, which
// on GB300 are ~56x faster than the FP64 ones.
//
// Same structure as the FP64 kernel (pcg.cu): one persistent cooperative
// launch, Chronopoulos-Gear recurrence, FP32 slices of 128 blocks, in the
// same two layouts: 8 warps per SM (slices resident in shared memory when
// they fit, else streamed through a ring of three) or 16 warps per SM (a
// ring of two, always streamed).  Streamed full slices arrive by TMA bulk
// copy on per-slot mbarriers.  A refinement iteration adds an FP64 slice
// SpMV of x (staged in the warp's free buffer space) and one grid barrier.
#include <algorithm>

#include "agipc_common.cuh"
#include "pcg_slices.cuh"

using namespace pcgs;

namespace {

struct MixedArgs {
    const int32_t *n_dev;
    const int32_t *rp;
    const int32_t *col;
    const double *val64;
    const float *val32;
    const float *dinv32;
    const double *b;
    double *x;
    double sign;
    double tol;
    int32_t max_iter;
    int32_t refine_every;
    int32_t max_rows;
    int64_t max_nnzb;
    int32_t *iters_dev;
    double *relres_dev;
    PcgScratch S;
    uint32_t *status;
};

__device__ __forceinline__ void precond32(const float *D, const double r[3], float u[3])
{
    const float r0 = (float)r[0], r1 = (float)r[1], r2 = (float)r[2];
#pragma unroll
    for (int c = 0; c < 3; ++c) u[c] = fmaf(D[3 * c + 2], r2, fmaf(D[3 * c + 1], r1, D[3 * c] * r0));
}

// Shared-memory layout of the two variants.  kW = 8 warps (255 registers):
// each warp owns a region of two FP64 slice buffers; a matrix that fits is
// held there for the whole solve (resident mode), a larger one streams
// through a ring of three FP32 slices.  kW = 16 warps (at most 128
// registers): twice the warps to hide the latency of a streamed matrix; each
// warp's region holds a ring of two FP32 slices (or one FP64 slice of a
// residual replacement) and the matrix always streams.
template <int kW>
struct MixedGeom {
    static constexpr bool kWide = kW > kPcgWarps;
    static constexpr int kRing = kWide ? 2 : 3;
    static constexpr int kB32 = SliceLayout<float>::kBuf;
    static constexpr int kB64 = SliceLayout<double>::kBuf;
    static constexpr int kBufArea = kWide ? kRing * kB32 : 2 * kBufBytes;   // slice buffers of one warp
    static constexpr int kRegion = kBufArea + kJoinBytes;
    static constexpr int kSmem = kW * kRegion + 32 * kW * 3 * 8;            // + the CTA-sum slots
    static_assert(kRing * kB32 <= kBufArea && (kWide ? kB64 : 2 * kB64) <= kBufArea &&
                      (kWide || kB32 + kB64 <= kBufArea) && kB32 % 16 == 0 && kB64 % 16 == 0 &&
                      kRegion % 16 == 0,
                  "slice buffers overflow the warp's region");
};

template <int kW>
__global__ void __launch_bounds__(32 * kW, 1) pcg_mixed_kernel(MixedArgs A)
{
    using Geo = MixedGeom<kW>;
    constexpr bool kWide = Geo::kWide;
    constexpr int kRing = Geo::kRing;
    constexpr int kB32 = Geo::kB32;
    constexpr int kB64 = Geo::kB64;
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ double s_scal[2];
    __shared__ double s_tot[4];
    __shared__ double s_grid[3];
    __shared__ double s_gr[2 * 32 * kW];   // the P phase's per-thread gamma, rho shares
    __shared__ int s_dec;
    __shared__ bool s_ref;
    __shared__ int s_abort;
    __shared__ __align__(8) uint64_t s_mbar[kW * kRing];   // one per ring slot of each warp

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
    const bool resident = !kWide && nslices <= nwarps;
    const int64_t rows_per_cta = div_up(n, nblocks);
    const int64_t row0 = min64((int64_t)blockIdx.x * rows_per_cta, n);
    const int64_t row1 = min64(row0 + rows_per_cta, n);

    // vectors: r, ax in FP64; u, w, p, s in FP32.  u is packed 16 bytes per
    // row, (u_0, u_1, u_2, the row's flag bits), so a slice gathers a column
    // with one load; it fills 4 of the 6 FP32 words per row of an FP64-sized
    // scratch array, and w shares s's array (3 + 3 words per row).
    double *__restrict__ r = A.S.r;
    double *ax = A.S.u;
    float4 *u4 = reinterpret_cast<float4 *>(A.S.w);
    float *__restrict__ p = reinterpret_cast<float *>(A.S.p);
    float *__restrict__ s = reinterpret_cast<float *>(A.S.s);
    float *w = s + 3 * (int64_t)A.max_rows;
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

    // ---- setup
    double gpart = 0.0, rpart = 0.0;
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
        u4[i] = make_float4(uu[0], uu[1], uu[2], __int_as_float((int)f));
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            gpart = fma(rr[c], (double)uu[c], gpart);
            rpart = fma(rr[c], rr[c], rpart);
        }
    }
    {
        double v[2] = {gpart, rpart};
        cta_sum<2, kW>(v, s_part, s_tot);
        if (threadIdx.x == 0) {
            partials[0 * mg + blockIdx.x] = v[0];
            partials[1 * mg + blockIdx.x] = v[1];
        }
    }
    bool ok = grid_sync(count, nblocks, epoch, A.status);
    if (ok && ld_acquire_u32(A.S.bar + 32) != 0u) {
        if (gtid == 0) set_status(A.status, ST_BAD_INDEX);
        ok = false;
    }
    // Resident mode: the warp's one FP32 slice stays in buffer 0 and the FP64
    // slice of a residual replacement goes to the region after it.  Streamed
    // mode (the matrix does not fit in shared memory): the warp cycles its
    // slices through a ring of kRing FP32 buffers, kRing - 1 of them loading
    // while it multiplies with another; the first kRing - 1 slices of an S
    // phase are issued at the end of the previous iteration, so they load
    // during the grid barrier.  The FP64 slices of a residual replacement
    // go over the ring's region (double-buffered where two fit).
    // A full slice goes by TMA bulk copy and completes on its slot's
    // mbarrier; the ragged last slice of the matrix goes by the zero-filling
    // cp.async path (a bulk copy would need lengths rounded up to 16 bytes,
    // past the caller's arrays).  `ph` holds each slot's next parity, `pend`
    // the slots with a bulk copy in flight (drained before the kernel ends).
    uint64_t *mbar = s_mbar + kRing * wib;
    unsigned ph = 0, pend = 0;
    if (threadIdx.x == 0) s_abort = 0;
    if (lane == 0)
        for (int k = 0; k < kRing; ++k) mbar_init(mbar + k);
    __syncthreads();
    auto ring_issue = [&](int k, int64_t sl) {
        if ((sl + 1) * kSlice <= nnz) {
            issue_slice_bulk<float>(wbuf + k * kB32, sl, A.val32, A.col, brow, mbar + k, lane);
            pend |= 1u << k;
        } else {
            issue_slice(wbuf + k * kB32, sl, nnz, A.val32, A.col, brow, lane);
            cp_async_commit();
        }
    };
    auto ring_wait = [&](int k, int64_t sl) {
        if ((sl + 1) * kSlice <= nnz) {
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
    auto prefetch_ring = [&]() {
#pragma unroll
        for (int k = 0; k < kRing - 1; ++k) {
            const int64_t sl = gwarp + k * nwarps;
            if (sl < nslices) ring_issue(k, sl);
        }
    };
    if (ok) {
        if (!resident) {
            prefetch_ring();
        } else {
            if (gwarp < nslices) issue_slice(wbuf, gwarp, nnz, A.val32, A.col, brow, lane);
            cp_async_commit();
        }
    }

    double alpha_old = 1.0, gamma_old = 1.0, bnorm2 = 0.0, rnorm2 = 0.0;
    const double tol2 = A.tol * A.tol;
    bool fresh = true;  // the residual was just computed as b - A64 x (x = 0 at the start)
    bool tight = false, last_verify = false, restart = false;
    int32_t it = 0;
    bool converged = false;
    bool pending = false;   // gamma, rho shares of a P phase wait in s_gr
    while (ok) {
        const int par = it & 1;
        double *part = partials + par * pstride;
        // ---- S phase: w = A32 u (FP32), delta accumulated in FP64 per lane
        double dpart = 0.0;
        if (resident) {
            if (gwarp < nslices) {
                cp_async_wait<0>();
                __syncwarp();
                const int cnt = (int)min64(kSlice, nnz - gwarp * kSlice);
                SliceGather<float> G;
                slice_gather_packed(wbuf, cnt, u4, lane, G);
                slice_compute<float, true>(wbuf, G, w, join, lane, dpart);
            }
        } else {
          if constexpr (kRing == 3) {
            // The k-th slice of the warp sits in ring slot k mod kRing.  While
            // slice k is multiplied, the gathers of slice k + 1 (landed) are in
            // flight and slice k + 2 loads into the slot slice k - 1 used.
            // Two gather sets alternate (no copies between them, which would
            // wait for the loads in flight).
            SliceGather<float> G0, G1;
            int slot = 0;
            if (gwarp < nslices) {
                ring_wait(0, gwarp);          // the first prefetched slice
                slice_gather_packed(wbuf, (int)min64(kSlice, nnz - gwarp * kSlice), u4, lane, G0);
            }
            // one step: refill the slot slice k - 1 used with slice k + 2,
            // gather slice k + 1 into Gn, multiply slice k with Gc
            auto step = [&](int64_t sl, SliceGather<float> &Gc, SliceGather<float> &Gn) {
                const int64_t ahead = sl + (kRing - 1) * nwarps;
                if (ahead < nslices) ring_issue(slot == 0 ? kRing - 1 : slot - 1, ahead);
                const int nslot = slot == kRing - 1 ? 0 : slot + 1;
                const int64_t nx = sl + nwarps;
                if (nx < nslices) {
                    ring_wait(nslot, nx);     // slice k + 1 (slice k + 2 may still load)
                    slice_gather_packed(wbuf + nslot * kB32, (int)min64(kSlice, nnz - nx * kSlice), u4, lane, Gn);
                }
                slice_compute<float, true>(wbuf + slot * kB32, Gc, w, join, lane, dpart);
                slot = nslot;
            };
            for (int64_t sl = gwarp; sl < nslices; sl += 2 * nwarps) {
                step(sl, G0, G1);
                if (sl + nwarps < nslices) step(sl + nwarps, G1, G0);
            }
          } else {
            // Two slots: slice k + 1 loads into the slot slice k - 1 used while
            // slice k is gathered and multiplied (the other warps hide the
            // gathers' latency).
            int slot = 0;
            for (int64_t sl = gwarp; sl < nslices; sl += nwarps) {
                const int64_t nx = sl + nwarps;
                if (nx < nslices) ring_issue(slot ^ 1, nx);
                ring_wait(slot, sl);
                SliceGather<float> G;
                slice_gather_packed(wbuf + slot * kB32, (int)min64(kSlice, nnz - sl * kSlice), u4, lane, G);
                slice_compute<float, true>(wbuf + slot * kB32, G, w, join, lane, dpart);
                slot ^= 1;
            }
          }
        }
        if (pending && wib == kW - 1) {
            // the previous P phase's gamma and rho shares, summed over the CTA
            // (fixed order) by the last warp while the others multiply
            double t0[kW], t1[kW];
#pragma unroll
            for (int q = 0; q < kW; ++q) {
                t0[q] = s_gr[2 * (lane + 32 * q)];
                t1[q] = s_gr[2 * (lane + 32 * q) + 1];
            }
#pragma unroll
            for (int h = kW / 2; h > 0; h >>= 1)
#pragma unroll
                for (int q = 0; q < h; ++q) {
                    t0[q] += t0[q + h];
                    t1[q] += t1[q + h];
                }
            const double g0 = warp_sum(t0[0]), g1 = warp_sum(t1[0]);
            if (lane == 0) {
                part[0 * mg + blockIdx.x] = g0;
                part[1 * mg + blockIdx.x] = g1;
            }
        }
        {
            double v[1] = {dpart};
            cta_sum<1, kW>(v, s_part, s_tot);
            if (threadIdx.x == 0) part[2 * mg + blockIdx.x] = v[0];
        }
        if (s_abort) { ok = false; break; }   // a slice never arrived (ST_TIMEOUT is set)
        if (!grid_sync(count, nblocks, epoch, A.status)) { ok = false; break; }

        // ---- global scalars (as in the FP64 kernel)
        if (wib < 3) {
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
            const double g = s_grid[0], rh = s_grid[1], dl = s_grid[2];
            // 0 iterate, 1 converged, 2 iteration cap, 3 non-finite, 4 verify:
            // the recurrence residual met the tolerance but was not freshly
            // recomputed, so replace it by b - A64 x before stopping
            int decision = 0;
            double alpha = 0.0, beta = 0.0;
            rnorm2 = rh;
            if (it == 0) bnorm2 = rh;
            if (!isfinite(rh) || !isfinite(g) || !isfinite(dl)) decision = 3;
            else if (bnorm2 == 0.0 || rh <= tol2 * bnorm2) decision = (fresh || A.refine_every == 0) ? 1 : 4;
            else if (it >= A.max_iter) decision = 2;
            // A verify that did not confirm convergence: the FP32 recurrences
            // of r and s = A p have drifted.  Restart the recurrence once
            // (beta = 0: p = u, s = w = A u from the fresh residual) and from
            // then on replace the residual every iteration.
            if (last_verify && decision != 1 && !tight) {
                tight = true;
                restart = true;
            }
            if (decision == 0 || decision == 4) {
                s_ref = decision == 4 || tight ||
                        (A.refine_every > 0 && ((it + 1) % A.refine_every) == 0);
                fresh = s_ref;
                last_verify = decision == 4;
            }
            if (decision != 0) {
                // no Krylov step this time
            } else {
                if (it == 0 || restart) {
                    alpha = g / dl;
                    restart = false;
                } else {
                    // beta = g / gamma_old and alpha = g t / den share one
                    // division by gamma_old den (an FP64 division is a long
                    // dependent chain here); the two quotients are used when
                    // that product leaves the normal range
                    const double t = gamma_old * alpha_old;
                    const double den = fma(dl, t, -g * g);
                    const double q = gamma_old * den;
                    if (fabs(q) >= 2.2250738585072014e-308 && fabs(q) <= 1.0e300) {
                        const double inv = 1.0 / q;
                        beta = g * den * inv;
                        alpha = g * t * gamma_old * inv;
                    } else {
                        beta = g / gamma_old;
                        alpha = (g * t) / den;
                    }
                }
                if (!isfinite(alpha) || !isfinite(beta)) decision = 3;
                gamma_old = g;
                alpha_old = alpha;
            }
            s_scal[0] = alpha;
            s_scal[1] = beta;
            s_dec = decision;
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

        const bool verify = decision == 4;
        const bool refine = s_ref;
        const float beta32 = (float)beta;
        // ---- P phase.  The next reduction reads the slot of parity (it + 1);
        // a verify step does not advance it, so its partials go to slot `par`
        // (already read by every CTA two barriers ago).  The CTA's sums of
        // the gamma, rho shares are formed in the next S phase, which writes
        // them to that slot.
        gpart = 0.0;
        rpart = 0.0;
        if (verify) {
            // no Krylov step: only clear the rows that receive atomics
            for (int64_t i = row0 + threadIdx.x; i < row1; i += blockDim.x)
                if (rowflag[i]) {
                    w[3 * i] = 0.0f;
                    w[3 * i + 1] = 0.0f;
                    w[3 * i + 2] = 0.0f;
                    ax[3 * i] = 0.0;
                    ax[3 * i + 1] = 0.0;
                    ax[3 * i + 2] = 0.0;
                }
        } else {
            // kRows rows per thread per pass: every load of the pass is issued
            // before the first store, so their latencies overlap
            constexpr int kRows = kWide ? 1 : 2;
            for (int64_t i0 = row0 + threadIdx.x; i0 < row1; i0 += kRows * (int64_t)blockDim.x) {
                float uu[kRows][3], ww[kRows][3], pp[kRows][3], ss[kRows][3], D[kRows][9];
                double xx[kRows][3], rr[kRows][3];
                uint8_t fl[kRows];
#pragma unroll
                for (int j = 0; j < kRows; ++j) {
                    const int64_t i = i0 + j * (int64_t)blockDim.x;
                    const bool has = i < row1;
                    const int64_t k = has ? i : i0;   // a row of this pass that exists
                    fl[j] = has ? rowflag[k] : 0;
                    const float4 u_k = __ldcg(u4 + k);
                    uu[j][0] = u_k.x;
                    uu[j][1] = u_k.y;
                    uu[j][2] = u_k.z;
#pragma unroll
                    for (int c = 0; c < 3; ++c) {
                        ww[j][c] = __ldcg(w + 3 * k + c);
                        pp[j][c] = p[3 * k + c];
                        ss[j][c] = s[3 * k + c];
                        xx[j][c] = x[3 * k + c];
                        rr[j][c] = r[3 * k + c];
                    }
                    if (!refine) {
#pragma unroll
                        for (int e = 0; e < 9; ++e) D[j][e] = A.dinv32[9 * k + e];
                    }
                }
#pragma unroll
                for (int j = 0; j < kRows; ++j) {
                    const int64_t i = i0 + j * (int64_t)blockDim.x;
                    if (i >= row1) break;
#pragma unroll
                    for (int c = 0; c < 3; ++c) {
                        pp[j][c] = fmaf(beta32, pp[j][c], uu[j][c]);
                        ss[j][c] = fmaf(beta32, ss[j][c], ww[j][c]);
                        p[3 * i + c] = pp[j][c];
                        s[3 * i + c] = ss[j][c];
                        x[3 * i + c] = fma(alpha, (double)pp[j][c], xx[j][c]);
                        rr[j][c] = fma(-alpha, (double)ss[j][c], rr[j][c]);
                        r[3 * i + c] = rr[j][c];
                    }
                    if (fl[j]) {
                        w[3 * i] = 0.0f;
                        w[3 * i + 1] = 0.0f;
                        w[3 * i + 2] = 0.0f;
                        if (refine) {
                            ax[3 * i] = 0.0;
                            ax[3 * i + 1] = 0.0;
                            ax[3 * i + 2] = 0.0;
                        }
                    }
                    if (!refine) {
                        float un[3];
                        precond32(D[j], rr[j], un);
                        u4[i] = make_float4(un[0], un[1], un[2], __int_as_float((int)fl[j]));
#pragma unroll
                        for (int c = 0; c < 3; ++c) {
                            gpart = fma(rr[j][c], (double)un[c], gpart);
                            rpart = fma(rr[j][c], rr[j][c], rpart);
                        }
                    }
                }
            }
        }
        if (refine) {
            // ---- residual replacement: r = b - A64 x with the FP64 master matrix
            if (!grid_sync(count, nblocks, epoch, A.status)) { ok = false; break; }
            double dummy = 0.0;
            if (resident) {
                unsigned char *fb = wbuf + kB32;
                if (gwarp < nslices) {
                    issue_slice(fb, gwarp, nnz, A.val64, A.col, brow, lane);
                    cp_async_commit();
                    cp_async_wait<0>();
                    __syncwarp();
                    const int cnt = (int)min64(kSlice, nnz - gwarp * kSlice);
                    slice_spmv<double, false>(fb, cnt, x, ax, rowflag, join, lane, dummy);
                }
            } else if constexpr (kWide) {
                // one FP64 slice at a time over the (empty) ring's region
                for (int64_t sl = gwarp; sl < nslices; sl += nwarps) {
                    issue_slice(wbuf, sl, nnz, A.val64, A.col, brow, lane);
                    cp_async_commit();
                    cp_async_wait<0>();
                    __syncwarp();
                    const int cnt = (int)min64(kSlice, nnz - sl * kSlice);
                    slice_spmv<double, false>(wbuf, cnt, x, ax, rowflag, join, lane, dummy);
                }
            } else {
                // the ring is empty here (the next S phase's slices are issued
                // after this pass)
                int fbi = 0;
                if (gwarp < nslices) issue_slice(wbuf, gwarp, nnz, A.val64, A.col, brow, lane);
                cp_async_commit();
                for (int64_t sl = gwarp; sl < nslices; sl += nwarps) {
                    const int64_t next = sl + nwarps;
                    if (next < nslices) issue_slice(wbuf + (fbi ^ 1) * kB64, next, nnz, A.val64, A.col, brow, lane);
                    cp_async_commit();
                    cp_async_wait<1>();
                    __syncwarp();
                    const int cnt = (int)min64(kSlice, nnz - sl * kSlice);
                    slice_spmv<double, false>(wbuf + fbi * kB64, cnt, x, ax, rowflag, join, lane, dummy);
                    fbi ^= 1;
                }
            }
            if (!grid_sync(count, nblocks, epoch, A.status)) { ok = false; break; }
            for (int64_t i = row0 + threadIdx.x; i < row1; i += blockDim.x) {
                double rr[3];
                float uu[3];
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    rr[c] = fma(A.sign, A.b[3 * i + c], -__ldcg(ax + 3 * i + c));
                    r[3 * i + c] = rr[c];
                }
                precond32(A.dinv32 + 9 * i, rr, uu);
                u4[i] = make_float4(uu[0], uu[1], uu[2], __int_as_float((int)rowflag[i]));
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    gpart = fma(rr[c], (double)uu[c], gpart);
                    rpart = fma(rr[c], rr[c], rpart);
                }
            }
        }
        s_gr[2 * threadIdx.x] = gpart;
        s_gr[2 * threadIdx.x + 1] = rpart;
        pending = true;
        if (!verify) ++it;
        if (!resident) prefetch_ring();
        if (!grid_sync(count, nblocks, epoch, A.status)) { ok = false; break; }
    }
    // no copy into this CTA's shared memory may outlive it
    for (int k = 0; k < kRing; ++k)
        if ((pend >> k) & 1u) mbar_wait(mbar + k, (ph >> k) & 1u);
    cp_async_wait<0>();
    if (gtid == 0 && (ok || it > 0)) {
        *A.iters_dev = it;
        *A.relres_dev = bnorm2 > 0.0 ? sqrt(rnorm2 / bnorm2) : 0.0;
        if (ok && !converged) set_status(A.status, ST_NOT_CONVERGED);
    }
}

}  // namespace

const void *pcg_mixed_kernel_ptr() { return reinterpret_cast<const void *>(&pcg_mixed_kernel<kPcgWarps>); }

// The 16-warp streaming variant runs one CTA per SM; false if the SM cannot
// hold it (its shared memory or registers).
bool pcg_mixed_wide_configure()
{
    constexpr int kW = 2 * kPcgWarps;
    const void *k = reinterpret_cast<const void *>(&pcg_mixed_kernel<kW>);
    int per_sm = 0;
    return cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, MixedGeom<kW>::kSmem) ==
               cudaSuccess &&
           cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, 32 * kW, MixedGeom<kW>::kSmem) == cudaSuccess &&
           per_sm >= 1;
}

extern "C" int agipc_pcg_mixed(agipc_ctx *ctx, int32_t max_rows, const int32_t *n_rows_dev, const int32_t *row_ptr,
                               const int32_t *col, const double *val, const float *val32, const float *dinv32,
                               const double *b, double *x, const agipc_pcg_options *opt, int32_t refine_every,
                               int32_t *iters_dev, double *relres_dev)
{
    if (!ctx || !opt || max_rows < 0 || max_rows > ctx->max_n || !n_rows_dev || !row_ptr || !val || !val32 ||
        !dinv32 || !b || !x || !iters_dev || !relres_dev || refine_every < 0)
        return AGIPC_ERR_INVALID_ARG;
    if (!(opt->tol >= 0.0) || opt->max_iter < 0 || (opt->rhs_sign != 1 && opt->rhs_sign != -1) || opt->use_x0)
        return AGIPC_ERR_INVALID_ARG;
    if (((uintptr_t)val & 15u) != 0 || ((uintptr_t)val32 & 15u) != 0 || ((uintptr_t)col & 15u) != 0 ||
        ((uintptr_t)dinv32 & 3u) != 0 || ((uintptr_t)b & 7u) != 0 || ((uintptr_t)x & 7u) != 0)
        return AGIPC_ERR_INVALID_ARG;
    MixedArgs A;
    A.n_dev = n_rows_dev;
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
    A.max_rows = max_rows;
    A.max_nnzb = ctx->max_nnzb;
    A.iters_dev = iters_dev;
    A.relres_dev = relres_dev;
    A.S = ctx->pcg;
    A.status = ctx->status;
    if (cudaMemsetAsync(ctx->pcg.bar, 0, 64 * sizeof(unsigned), ctx->stream) != cudaSuccess) return AGIPC_ERR_CUDA;
    void *args[] = {&A};
    static_assert(MixedGeom<kPcgWarps>::kSmem == kPcgSmem, "the 8-warp layout is the shared PCG layout");
    cudaError_t e;
    if (opt->streamed) {
        constexpr int kW = 2 * kPcgWarps;
        e = cudaLaunchCooperativeKernel(reinterpret_cast<const void *>(&pcg_mixed_kernel<kW>),
                                        dim3((unsigned)ctx->num_sms), dim3(32 * kW), args, MixedGeom<kW>::kSmem,
                                        ctx->stream);
    } else {
        e = cudaLaunchCooperativeKernel(reinterpret_cast<const void *>(&pcg_mixed_kernel<kPcgWarps>),
                                        dim3((unsigned)ctx->pcg_grid), dim3(kPcgBlock), args, kPcgSmem, ctx->stream);
    }
    return e == cudaSuccess ? AGIPC_OK : AGIPC_ERR_CUDA;
}
