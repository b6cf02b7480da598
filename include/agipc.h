/*
 * agipc.h - C ABI of the GB300 in-solve algebraic coarsening step.
 *
 * One Newton iteration of the adaptive solver of arxiv 2605.04773 (Algorithm 1:
 * the mapping update, the mapping of H and grad E to the coarse level, the
 * coarse solve, and the prolongation of Sec. 4.3) as four calls:
 *
 *   agipc_aggregate        tags -> super-node labels            (Sec. 4.1; supplement Sec. 1)
 *   agipc_assemble_coarse  labels, H, g -> H_c = U H U^T, g_c = U g, block-Jacobi (Sec. 4.1; supplement Sec. 2)
 *   agipc_pcg              H_c y = -g_c by block-Jacobi PCG      (Algorithm 1; Sec. 5, Preconditioners)
 *   agipc_prolongate       dx = U^T y                            (Sec. 4.3)
 *
 * plus the precision form (agipc_precision_split, agipc_*_mixed), the differentiation form
 * (agipc_fine_assemble_stvk, agipc_restrict, agipc_stvk_vjp), the batched
 * form (agipc_batch_coarse_offsets, agipc_pcg_batched) and
 * agipc_prolongate_add, agipc_aggregate_static.
 *
 * Conventions for every call:
 *   - All array arguments are DEVICE pointers owned by the caller; the
 *     library never frees them.  Scratch memory belongs to the context and is
 *     allocated once by agipc_create.
 *   - Every call is asynchronous: it checks its host-side arguments, enqueues
 *     kernels on the context's CUDA stream and returns.  Errors that only the
 *     GPU can see (non-finite values, capacity overflow, PCG not converged,
 *     a bounded device wait that ran out) are OR-ed into a device status word;
 *     agipc_status() synchronizes the stream, returns the first of them as a
 *     status code and clears the word.
 *   - Sizes that only the GPU knows (n_c, nnz_c, PCG iterations) stay in
 *     caller-owned device scalars, so a whole step can be captured in a CUDA
 *     graph.  Nothing here synchronizes with the host except agipc_status and
 *     agipc_destroy.
 *   - 3x3 blocks are 9 contiguous FP64 values in row-major order; vectors of
 *     nodes are [n][3] FP64.  Index arrays are int32.
 *   - Return value: AGIPC_OK or a negative AGIPC_ERR_* code.
 */
#ifndef AGIPC_H
#define AGIPC_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
    AGIPC_OK = 0,
    AGIPC_ERR_INVALID_ARG = -1,   /* host-checked argument error; nothing was enqueued */
    AGIPC_ERR_CUDA = -2,          /* a CUDA runtime call failed */
    AGIPC_ERR_CAPACITY = -3,      /* an output would exceed its caller-given capacity */
    AGIPC_ERR_NONFINITE = -4,     /* NaN/Inf met, or a singular diagonal block */
    AGIPC_ERR_NOT_CONVERGED = -5, /* PCG hit max_iter; x holds the last iterate */
    AGIPC_ERR_TIMEOUT = -6,       /* a bounded device-side wait gave up */
    AGIPC_ERR_BAD_INDEX = -7      /* an index array held a value out of range */
};

typedef struct agipc_ctx agipc_ctx;

/*
 * Create a context bound to the current CUDA device and to `cuda_stream`
 * (a cudaStream_t; NULL = the legacy default stream).  Scratch memory is
 * sized for the largest problem the context will see:
 *   max_fine_nodes    n of any fine system
 *   max_edges         mesh edges passed to agipc_aggregate
 *   max_fine_nnzb     3x3 blocks of any fine upper-triangular BSR matrix
 *   max_pairs         barrier stencils passed to agipc_assemble_coarse
 * The largest matrix agipc_pcg will accept then has 2*max_fine_nnzb +
 * 16*max_pairs blocks and max_fine_nodes rows.  Returns INVALID_ARG on a
 * negative size and CUDA when device memory cannot be had.
 */
int agipc_create(agipc_ctx **ctx, void *cuda_stream, int32_t max_fine_nodes, int64_t max_edges,
                 int64_t max_fine_nnzb, int64_t max_pairs);

/* Synchronize the context's stream and release its scratch memory. */
int agipc_destroy(agipc_ctx *ctx);

/* Rebind the context to another stream (e.g. the caller's current stream). */
int agipc_set_stream(agipc_ctx *ctx, void *cuda_stream);

/*
 * Launch shape of the coarse assembly's reduction (the numeric phase of
 * agipc_assemble_coarse and agipc_assemble_coarse_mixed, supplement Sec. 2):
 * each lane folds terms_per_lane consecutive sorted terms into running 3x3
 * blocks before flushing them with atomics (a warp covers 32 x that many).
 * Longer runs mean fewer atomics inside large super-nodes but a longer
 * serial chain per lane.  4, 8, 16 or 32 (the default: the fastest on the
 * 64-box domino's coarse assembly on GB300); anything else returns
 * AGIPC_ERR_INVALID_ARG.  The results agree to rounding order (the atomics'
 * order changes).  Applies to later calls on the context.
 */
int agipc_set_assembly_run(agipc_ctx *ctx, int32_t terms_per_lane);

/*
 * Super-node labels (Sec. 4.1: nodes are coalesced only across paths of
 * collapsible edges; supplement Sec. 1, Algorithms 1-2 and the worked
 * examples of Sec. 1.2-1.3).
 *   n_fine            number of fine nodes
 *   n_edges           number of mesh edges
 *   edges   [E][2]    int32 endpoints, any order, 0 <= u, v < n_fine
 *   tags    [E]       uint8, nonzero = collapsible (tau_e = 1), 0 = protected
 *   labels  [n_fine]  out: int32 coarse index of every fine node
 *   n_coarse_dev      out: device int32, the number of super-nodes n_c
 * Labels are the connected components of the collapsible-edge graph, ranked
 * by each component's smallest fine index (the supplement's ordering: first
 * set bit of the group hash, then a prefix sum over groups), so they are
 * dense in [0, n_c) and identical whatever the GPU's scheduling.
 * Out-of-range endpoints set AGIPC_ERR_BAD_INDEX in the status word.
 */
int agipc_aggregate(agipc_ctx *ctx, int32_t n_fine, int64_t n_edges, const int32_t *edges, const uint8_t *tags,
                    int32_t *labels, int32_t *n_coarse_dev);

/*
 * Coarse system (Sec. 4.1: g_c = sum of the children's g_f; each fine 3x3
 * block (i, j) is summed into (map(i), map(j)), i.e. H_c = U H U^T;
 * supplement Sec. 2 for the reduction; contact Hessians join the fine
 * system before coarsening, Sec. 4.3).
 *   n_fine, labels, n_coarse_dev      as produced by agipc_aggregate
 *   fine_row_ptr [n_fine+1], fine_col [fine_nnzb], fine_val [fine_nnzb][9]
 *                   the fine Hessian's diagonal and upper triangle (col >= row)
 *                   as BSR; each diagonal block must be symmetric
 *   n_pairs, pair_idx [P][4], pair_blk [P][10][9]
 *                   barrier stencils: 4 vertices and the 10 upper 3x3 blocks in
 *                   the local order (0,0),(0,1),(0,2),(0,3),(1,1),(1,2),(1,3),
 *                   (2,2),(2,3),(3,3); a block (s,t), s<t, also stands for its
 *                   transpose at (t,s)
 *   g [n_fine][3]   fine gradient
 *   coarse_row_ptr [n_fine+1]   out: full-storage BSR of H_c (both triangles),
 *   coarse_col [cap], coarse_val [cap][9]   columns ascending in each row;
 *                   row_ptr entries past n_c repeat nnz_c
 *   coarse_cap_nnzb capacity of coarse_col/coarse_val; 2*fine_nnzb + 16*P
 *                   always suffices
 *   coarse_nnzb_dev out: device int32, nnz_c
 *   g_c [n_fine][3] out: coarse gradient (first n_c rows written)
 *   dinv [n_fine][9] out: inverses of the diagonal blocks of H_c (block-Jacobi)
 * With labels = 0..n-1 this is the fine system itself in full storage (the
 * no-coarsening arm).  Overflowing coarse_cap_nnzb sets AGIPC_ERR_CAPACITY
 * and leaves the outputs incomplete; a singular or non-finite diagonal block
 * sets AGIPC_ERR_NONFINITE.
 */
int agipc_assemble_coarse(agipc_ctx *ctx, int32_t n_fine, const int32_t *labels, const int32_t *n_coarse_dev,
                          const int32_t *fine_row_ptr, const int32_t *fine_col, const double *fine_val,
                          int64_t fine_nnzb, int64_t n_pairs, const int32_t *pair_idx, const double *pair_blk,
                          const double *g, int32_t *coarse_row_ptr, int32_t *coarse_col, double *coarse_val,
                          int64_t coarse_cap_nnzb, int32_t *coarse_nnzb_dev, double *g_c, double *dinv);

/* PCG options.  rhs_sign multiplies b (use -1 to solve A y = -g_c from g_c). */
typedef struct {
    double tol;          /* stop when ||b - A x||_2 <= tol * ||b||_2 (recurrence residual) */
    int32_t max_iter;    /* iteration cap; reaching it sets AGIPC_ERR_NOT_CONVERGED */
    int32_t rhs_sign;    /* +1 or -1 */
    int32_t use_x0;      /* agipc_pcg only: nonzero = x holds the initial guess on entry (else x0 = 0);
                            the stop test stays relative to ||b||; b = 0 gives x = 0 */
    int32_t streamed;    /* agipc_pcg and agipc_pcg_mixed (agipc_pcg_batched ignores it): kernel layout
                            (results are the same up to rounding order).  0: 8 warps per SM,
                            the matrix held in shared memory when its 128-block slices fit one per warp
                            (1216 slices on 152 SMs), streamed from HBM every iteration otherwise.
                            Nonzero: 16 warps per SM and the matrix always streamed; for systems larger
                            than shared memory, where twice the warps hide the latency of the stream.
                            Occupies the struct's former padding: its size stays 24 bytes. */
} agipc_pcg_options;

/*
 * Block-Jacobi preconditioned conjugate gradients, x0 = 0 (Algorithm 1,
 * d_c = -H_c^-1 g_c; Sec. 5 uses a relative residual-norm stop and Sec. 5.1
 * the 3x3 block-Jacobi diagonal preconditioner).
 *   max_rows        host bound on the number of rows (launch sizing)
 *   n_rows_dev      device int32: the actual number of rows n <= max_rows
 *   row_ptr [n+1], col, val [..][9]   full-storage SPD BSR matrix
 *   dinv [n][9]     inverse diagonal blocks
 *   b [n][3]        right-hand side (scaled by opt->rhs_sign)
 *   x [n][3]        out: solution
 *   iters_dev       out: device int32, iterations performed
 *   relres_dev      out: device double, ||r||_2/||b||_2 at exit
 * The whole solve runs in one persistent kernel with device-side
 * convergence, so the host never waits inside the loop.  The iteration is
 * the Chronopoulos-Gear form of PCG (one fused reduction per iteration);
 * mathematically it is the same method as the textbook recurrence.
 * opt->streamed picks the kernel layout (see agipc_pcg_options); both reach
 * the same solution up to rounding order.
 */
int agipc_pcg(agipc_ctx *ctx, int32_t max_rows, const int32_t *n_rows_dev, const int32_t *row_ptr,
              const int32_t *col, const double *val, const double *dinv, const double *b, double *x,
              const agipc_pcg_options *opt, int32_t *iters_dev, double *relres_dev);

/*
 * Precision form of the coarse assembly: as agipc_assemble_coarse, with the
 * fine blocks and most barrier stencils given in FP32 and the stencils of
 * small gaps (whose stiffness FP32 would round too coarsely) given in FP64
 * as a second list.  Every contribution is accumulated in FP64 into
 * coarse_val (the FP64 master, used for residual replacement); coarse_val32
 * and dinv32 receive its FP32 rounding and the FP32 rounding of the FP64
 * block-Jacobi inverses.  Capacities and statuses as agipc_assemble_coarse
 * (the pair count limit applies to n_pairs32 + n_pairs64).
 */
int agipc_assemble_coarse_mixed(agipc_ctx *ctx, int32_t n_fine, const int32_t *labels, const int32_t *n_coarse_dev,
                                const int32_t *fine_row_ptr, const int32_t *fine_col, const float *fine_val32,
                                int64_t fine_nnzb, int64_t n_pairs32, const int32_t *pair_idx32,
                                const float *pair_blk32, int64_t n_pairs64, const int32_t *pair_idx64,
                                const double *pair_blk64, const double *g, int32_t *coarse_row_ptr,
                                int32_t *coarse_col, double *coarse_val, float *coarse_val32, int64_t coarse_cap_nnzb,
                                int32_t *coarse_nnzb_dev, double *g_c, float *dinv32);

/*
 * Inputs of the precision form from the FP64 ones (the paper computes in
 * FP64, Sec. 5; the precision form keeps only the barrier terms at small gap
 * distances in FP64, whose stiffness grows like (dhat/d)^2):
 *   val [fine_nnzb][9] FP64       -> val32 [fine_nnzb][9]: FP32 rounding (nearest even)
 *   pair_idx [P][4], pair_blk [P][90] FP64, pair_gap [P] FP64 (the stencils' gaps d)
 *   gap_limit (host)              stencils with gap < gap_limit stay FP64
 *   pair_idx32 [P][4], pair_blk32 [P][90] FP32   out: the other stencils, rounded
 *   pair_idx64 [P][4], pair_blk64 [P][90] FP64   out: the small-gap stencils, copied
 *   counts_dev  out: device int32[2] = {stencils in the FP32 list, in the FP64 list}
 * Each output list must have room for all P stencils; both keep the input
 * order.  The two counts are the n_pairs32 and n_pairs64 that
 * agipc_assemble_coarse_mixed takes on the host: read them once (one copy)
 * after this call.  Uses the context's assembly scratch, which the next
 * assembly overwrites.  The decision gap < gap_limit is an FP64 comparison.
 */
int agipc_precision_split(agipc_ctx *ctx, int64_t fine_nnzb, const double *val, float *val32, int64_t n_pairs,
                          const int32_t *pair_idx, const double *pair_blk, const double *pair_gap, double gap_limit,
                          int32_t *pair_idx32, float *pair_blk32, int32_t *pair_idx64, double *pair_blk64,
                          int32_t *counts_dev);

/*
 * Precision form of the PCG: the 3x3 blocks (val32), the SpMV and the
 * block-Jacobi preconditioner (dinv32) run in FP32; the dot products are
 * accumulated in FP64; x and r stay in FP64 and every refine_every
 * iterations r is replaced by b - A x computed with the FP64 master matrix
 * `val` (same structure), so the answer is that of the FP64 system.
 * refine_every = 0 disables the replacement.  Other arguments, layouts and
 * statuses as agipc_pcg.  val and val32 must be 16-byte aligned.
 */
int agipc_pcg_mixed(agipc_ctx *ctx, int32_t max_rows, const int32_t *n_rows_dev, const int32_t *row_ptr,
                    const int32_t *col, const double *val, const float *val32, const float *dinv32, const double *b,
                    double *x, const agipc_pcg_options *opt, int32_t refine_every, int32_t *iters_dev,
                    double *relres_dev);

/*
 * Prolongation d_f = U^T d_c (Sec. 4.3): dx[f] = y[labels[f]].
 *   n_fine, labels [n_fine], y [n_c][3]  ->  dx [n_fine][3]
 */
int agipc_prolongate(agipc_ctx *ctx, int32_t n_fine, const int32_t *labels, const double *y, double *dx);

/*
 * Prolongation followed by the Newton update (Sec. 4.3 and Algorithm 1,
 * x <- x + d_f at unit step length): out[f] = base[f] + y[labels[f]].
 * base and out may alias.  Arguments and statuses as agipc_prolongate.
 */
int agipc_prolongate_add(agipc_ctx *ctx, int32_t n_fine, const int32_t *labels, const double *y,
                         const double *base, double *out);

/*
 * Differentiation form.  The coarsened step x_next = x + U^T y with
 * y = -(U H U^T)^-1 U g is a function of per-tet Young's moduli E and of the
 * rest positions X_rest through the elastic terms of the incremental
 * potential (Eq. 1 divided by dt^2); the labels are piecewise constant in
 * both, so they carry no derivative (Galerkin coarse operator, Sec. 4.1).
 * For a loss with v = dL/dx_next the adjoint is
 *     H_c lambda_c = U v   (agipc_restrict, then agipc_pcg with rhs_sign +1),
 *     lambda = U^T lambda_c (agipc_prolongate),
 *     dL/dtheta = -lambda^T (dg/dtheta + dH/dtheta dx)   (agipc_stvk_vjp).
 *
 * Elasticity is St. Venant-Kirchhoff: Psi_e = V_e (mu |G|_F^2 + lam/2 tr(G)^2),
 * G = (F^T F - I)/2, F = Ds Dm^-1, mu = E/(2(1+nu)), lam = E nu/((1+nu)(1-2nu)),
 * V_e = |det Dm|/6; each tet's 12x12 Hessian is made PSD by clamping its
 * eigenvalues at zero before it is summed.
 */

/*
 * Fine Newton system of StVK tets (Eq. 1 divided by dt^2):
 *   H = M/h^2 + sum_e H_e+,   g = M/h^2 (x - x_hat) + sum_e dPsi_e/dx + g_extra
 * with the inertial target x_hat = X_rest + xhat_shift (h^2 gravity for a
 * body starting at rest; a velocity term h v is constant in the parameters
 * and belongs in g_extra as -M/h v), written into the VALUES of a given
 * upper BSR structure.
 *   n_fine, n_tets, tets [n_tets][4]   vertices of each tet
 *   X_rest, x [n_fine][3]              rest positions, current positions
 *   xhat_shift                         HOST array of 3 doubles
 *   E [n_tets], nu                     Young's modulus per tet, Poisson ratio in (-1, 0.5)
 *   mass_h2 [n_fine]                   lumped mass / h^2
 *   g_extra [n_fine][3] or NULL        further gradient terms (e.g. contact), added as is
 *   fine_row_ptr [n_fine+1], fine_col  upper BSR structure (column >= row, sorted,
 *                                      diagonal first in each row) that holds every
 *                                      vertex pair of every tet
 *   fine_val [fine_nnzb][9]            out: H (upper blocks); g [n_fine][3] out
 *   workspace, workspace_bytes         caller-owned device scratch, 128-byte aligned,
 *                                      at least agipc_stvk_workspace_bytes(n_tets) bytes
 *                                      (the list of tets whose Hessian is not clearly
 *                                      positive definite); n_tets <= INT32_MAX
 * Blocks absent from the structure, or tet vertices out of range or repeated,
 * set AGIPC_ERR_BAD_INDEX; a non-finite element gradient sets
 * AGIPC_ERR_NONFINITE.  Summation uses atomics, so the last bits of the sums
 * depend on scheduling.  fine_nnzb is capped by the context's max_fine_nnzb.
 */
int agipc_fine_assemble_stvk(agipc_ctx *ctx, int32_t n_fine, int64_t n_tets, const int32_t *tets,
                             const double *X_rest, const double *x, const double *xhat_shift, const double *E, double nu,
                             const double *mass_h2, const double *g_extra, const int32_t *fine_row_ptr,
                             const int32_t *fine_col, int64_t fine_nnzb, double *fine_val, double *g, void *workspace,
                             int64_t workspace_bytes);

/*
 * Restriction v_c = U v (the map of Sec. 4.1 applied to a fine vector):
 * v_c[c] = sum over labels[f] == c of v[f].
 *   v [n_fine][3]; v_c [n_fine][3] out (rows past n_c are zeroed)
 * Labels outside [0, n_c) set AGIPC_ERR_BAD_INDEX.
 */
int agipc_restrict(agipc_ctx *ctx, int32_t n_fine, const int32_t *labels, const int32_t *n_coarse_dev,
                   const double *v, double *v_c);

/*
 * Per-element vector-Jacobian product of the step, given the prolongated
 * adjoint lambda and the step dx:
 *   dL_dE[e]      = -lambda_e^T (g_e + H_e+ dx_e) / E_e   (Psi_e is linear in
 *                   E_e and the clamp commutes with positive scaling)
 *   dL_dX_rest    = -d/dX_rest [lambda^T g + lambda^T H+ dx] + lambda M/h^2
 * The derivative of the clamp goes through the element's eigen-
 * decomposition H_e = V diag(l) V^T: lambda^T dH+ dx = <dH, V (F o a b^T) V^T>,
 * a = V^T lambda_e, b = V^T dx_e, F the divided differences of max(., 0)
 * over the eigenvalues.  The last term comes from the inertial target
 * x_hat = X_rest + xhat_shift of agipc_fine_assemble_stvk; pass
 * mass_h2 = NULL to leave it out.  Masses are constants; x is data, not a
 * parameter.
 *   lam, dx [n_fine][3]; dL_dE [n_tets] out; dL_dX_rest [n_fine][3] out
 * Other arguments (workspace included) as agipc_fine_assemble_stvk.  The
 * per-tet terms are summed with atomics.
 */
int agipc_stvk_vjp(agipc_ctx *ctx, int32_t n_fine, int64_t n_tets, const int32_t *tets, const double *X_rest,
                   const double *x, const double *E, double nu, const double *mass_h2, const double *lam,
                   const double *dx, double *dL_dE, double *dL_dX_rest, void *workspace, int64_t workspace_bytes);

/*
 * Batched form.  Many independent meshes are concatenated into one
 * block-diagonal problem: instance i owns fine vertices
 * [vert_ptr[i], vert_ptr[i+1]) and no edge, tet, stencil or matrix block
 * couples two instances.  agipc_aggregate, agipc_assemble_coarse_mixed and
 * agipc_prolongate run on the concatenation unchanged: super-nodes never
 * cross instances and canonical labels are ranked by the smallest fine
 * index, so the coarse rows of instance i are the contiguous range
 * [inst_row[i], inst_row[i+1]) and the coarse matrix is block diagonal too.
 */
#define AGIPC_BATCH_MAX_INSTANCES 512

/*
 * inst_row[i] = labels[vert_ptr[i]] (the first coarse row of instance i),
 * inst_row[n_inst] = n_c.
 *   vert_ptr [n_inst+1] device int32, non-decreasing, vert_ptr[n_inst] = n_fine
 *   labels [n_fine], n_coarse_dev   from agipc_aggregate
 *   inst_row [n_inst+1]             out (device)
 * 1 <= n_inst <= AGIPC_BATCH_MAX_INSTANCES.
 */
int agipc_batch_coarse_offsets(agipc_ctx *ctx, int32_t n_inst, int32_t n_fine, const int32_t *vert_ptr,
                               const int32_t *labels, const int32_t *n_coarse_dev, int32_t *inst_row);

/*
 * Batched precision-form PCG: solves H_i y_i = sign b_i for every instance i
 * of a block-diagonal coarse system in one persistent launch, each instance
 * with its own alpha, beta, stopping test and iteration count, by the method
 * of agipc_pcg_mixed (FP32 blocks, SpMV and block-Jacobi, FP64 dot products,
 * FP64 residual replacement every refine_every iterations, true-residual
 * check before stopping).  Instances that have stopped cost nothing in
 * later iterations.
 *   inst_row [n_inst+1]            device, from agipc_batch_coarse_offsets
 *   max_rows, row_ptr, col, val, val32, dinv32, b, x, opt, refine_every
 *                                  as agipc_pcg_mixed (the whole concatenation)
 *   blocks_per_lane                slice width: each warp lane folds this many
 *                                  consecutive blocks (4, 5, 6 or 8; 0 = 5),
 *                                  the tile the autotuner picks
 *   iters_dev [n_inst], relres_dev [n_inst]   out, per instance
 * A block whose column leaves its instance sets AGIPC_ERR_BAD_INDEX.  Any
 * instance reaching max_iter sets AGIPC_ERR_NOT_CONVERGED (the others are
 * still solved).  The per-instance sums use atomics, so results may differ
 * in the last bits between runs.
 */
int agipc_pcg_batched(agipc_ctx *ctx, int32_t n_inst, const int32_t *inst_row, int32_t max_rows,
                      const int32_t *row_ptr, const int32_t *col, const double *val, const float *val32,
                      const float *dinv32, const double *b, double *x, const agipc_pcg_options *opt,
                      int32_t refine_every, int32_t blocks_per_lane, int32_t *iters_dev, double *relres_dev);

/*
 * Green-strain-increment tags (Sec. 4.2, Eq. 3), the step before
 * agipc_aggregate: per tet F = Ds Dm^-1 and G = (F^T F - I)/2 at the previous
 * and the current iterate; a tet with ||G(x_cur) - G(x_prev)||_F > threshold
 * protects (tag 0) its 6 edges, every other edge is collapsible (tag 1).
 * The paper uses threshold 5e-5 (5e-4 for twisting scenes).
 *   tets [n_tets][4], X_rest, x_prev, x_cur [n_fine][3]
 *   fine_row_ptr, fine_col, fine_nnzb   the fine upper structure, which is
 *       the static edge-element adjacency: each row holds its diagonal block
 *       first, then one block per edge (u, v > u); edge k of the sorted edge
 *       list is the k-th off-diagonal block
 *   tags [n_edges] out
 * A tet edge missing from the structure sets AGIPC_ERR_BAD_INDEX.  The
 * decision is taken on ||.||_F^2 > threshold^2 in FP64.
 */
int agipc_strain_tags(agipc_ctx *ctx, int32_t n_fine, int64_t n_tets, const int32_t *tets, const double *X_rest,
                      const double *x_prev, const double *x_cur, double threshold, const int32_t *fine_row_ptr,
                      const int32_t *fine_col, int64_t fine_nnzb, int64_t n_edges, uint8_t *tags);

/*
 * Adaptive affine embedding (Sec. 4.2, Eq. 4; the supplement's affine
 * mapping).  A coarse node whose aggregate holds more than `threshold` fine
 * nodes (the paper uses 32) gets 12 DoF: fine node f of it moves by
 * dx_f = A_f^T y_c, A_f = Xbar_f (x) I3, Xbar_f = (X_rest_f, 1), so y_c is four
 * 3-vectors; smaller aggregates keep dx_f = y_c.  Coarse 3-rows: every 3-DoF
 * node first, then every 12-DoF node as 4 consecutive rows, each class in
 * label order.  The coarse system is the Galerkin product with that
 * prolongation (g_c = P^T g, H_c = P^T H P), stored as a full 3x3 BSR matrix
 * solvable by agipc_pcg; its block-Jacobi inverses are of the 3x3 diagonal
 * blocks.
 *
 * agipc_affine_plan: coarse_base [n_fine] and coarse_k [n_fine] (first 3-row
 *   and width, 1 or 4, of every coarse node c < n_c), n_rows_dev (number of
 *   coarse 3-rows).  threshold >= 3 (then n_rows <= n_fine).
 * agipc_assemble_affine: label_row_ptr, label_col are the label-level full
 *   coarse structure (from agipc_assemble_coarse on the same labels); the
 *   fine upper BSR, stencils and g as agipc_assemble_coarse.  Outputs:
 *   row_ptr [n_fine+1] (rows past n_rows are empty), col, val [cap][9],
 *   nnzb_dev, g_c [n_fine][3], dinv [n_fine][9].  Sums use FP64 atomics.
 * agipc_prolongate_affine: dx = P y.
 * Labels out of range or blocks missing from the structure set
 * AGIPC_ERR_BAD_INDEX; overflowing cap_nnzb sets AGIPC_ERR_CAPACITY.
 */
int agipc_affine_plan(agipc_ctx *ctx, int32_t n_fine, const int32_t *labels, const int32_t *n_coarse_dev,
                      int32_t threshold, int32_t *coarse_base, int32_t *coarse_k, int32_t *n_rows_dev);
int agipc_assemble_affine(agipc_ctx *ctx, int32_t n_fine, const int32_t *labels, const int32_t *n_coarse_dev,
                          const double *X_rest, const int32_t *coarse_base, const int32_t *coarse_k,
                          const int32_t *n_rows_dev, const int32_t *label_row_ptr, const int32_t *label_col,
                          const int32_t *fine_row_ptr, const int32_t *fine_col, const double *fine_val,
                          int64_t fine_nnzb, int64_t n_pairs, const int32_t *pair_idx, const double *pair_blk,
                          const double *g, int32_t *row_ptr, int32_t *col, double *val, int64_t cap_nnzb,
                          int32_t *nnzb_dev, double *g_c, double *dinv);
int agipc_prolongate_affine(agipc_ctx *ctx, int32_t n_fine, const int32_t *labels, const int32_t *n_coarse_dev,
                            const double *X_rest, const int32_t *coarse_base, const int32_t *coarse_k,
                            const double *y, double *dx);

/* Bytes of device workspace agipc_fine_assemble_stvk and agipc_stvk_vjp
 * need for n_tets tets (-1 for a negative count). */
int64_t agipc_stvk_workspace_bytes(int64_t n_tets);

/*
 * Labeller without allocation.  The paper has no counterpart: this is a
 * convenience of this library.  It computes exactly what agipc_aggregate
 * computes, for callers that cannot allocate GPU memory - code that has no
 * agipc_ctx because agipc_create must cudaMalloc its scratch arena, e.g. a
 * plugin that only receives device pointers from its host application, or a
 * simulation loop whose memory manager forbids cudaMalloc after start-up.
 *   cuda_stream        cudaStream_t to enqueue on (NULL = legacy default stream)
 *   n_fine, n_edges, edges, tags, labels, n_coarse_dev   as agipc_aggregate
 *   status_dev         out: caller-owned device uint32; set to 0 by the call,
 *                      then to a nonzero bit pattern if the GPU met an
 *                      out-of-range edge endpoint or a bounded wait ran out
 * Scratch is one fixed array of AGIPC_AGGREGATE_STATIC_MAX_NODES-sized
 * buffers (about 12 MiB) compiled into the library's device image, so every
 * GPU that loads the library holds it until the process exits.  n_fine above
 * that maximum is rejected with AGIPC_ERR_INVALID_ARG before anything is
 * enqueued.  Every call made outside stream capture looks the array's device
 * address up (cudaGetSymbolAddress) for the current device and remembers it;
 * a call made while cuda_stream is being captured reuses the remembered
 * address.  So the first call on a device must come before any stream
 * capture, and after cudaDeviceReset (which unloads the array) one call
 * outside capture must come before the next captured one.  The call never
 * calls cudaMalloc or cudaFree.  All calls
 * share the one array: calls that overlap on the GPU (different streams, no
 * ordering between them) race and corrupt each other's results; serialize
 * them.  The array keeps the previous call's contents, which no call reads.
 */
#define AGIPC_AGGREGATE_STATIC_MAX_NODES (1 << 20)
int agipc_aggregate_static(void *cuda_stream, int32_t n_fine, int64_t n_edges, const int32_t *edges,
                           const uint8_t *tags, int32_t *labels, int32_t *n_coarse_dev, uint32_t *status_dev);

/*
 * Incremental potential of the StVK problem at a trial point (Eq. 1 divided
 * by dt^2, without barrier or friction terms; the quantity the backtracking
 * line search of Algorithm 1 compares, E(x) < E_prev):
 *   x = x0 + alpha d   (product and sum each rounded once; d may be NULL: x = x0)
 *   E(x) = sum_i mass_h2[i] / 2 |x_i - X_rest_i - xhat_shift|^2
 *        + sum_e V_e (mu_e |G_e|_F^2 + lam_e / 2 tr(G_e)^2) + g_extra . x
 * with G_e = (F^T F - I) / 2, F = Ds Dm^-1, V_e = |det Dm| / 6 and the Lame
 * parameters of E[e] and nu, i.e. the energy whose gradient and Hessian
 * agipc_fine_assemble_stvk sums (same arguments, same meaning).
 *   tets [n_tets][4], X_rest, x0, d [n_fine][3], E [n_tets], mass_h2 [n_fine],
 *   xhat_shift [3] host, g_extra [n_fine][3] or NULL
 *   x_out [n_fine][3] or NULL: receives x; must not overlap x0 or d
 *   energy_dev (device double) out
 * The sum is deterministic (same inputs and device: same bits).  A tet
 * index out of range sets AGIPC_ERR_BAD_INDEX and the tet is skipped.
 * Calls on one context are serialized by its stream; the reduction scratch
 * lives in the context.
 */
int agipc_stvk_energy(agipc_ctx *ctx, int32_t n_fine, int64_t n_tets, const int32_t *tets, const double *X_rest,
                      const double *x0, const double *d, double alpha, const double *xhat_shift, const double *E,
                      double nu, const double *mass_h2, const double *g_extra, double *x_out, double *energy_dev);

/*
 * out_dev = max_k |v[k]| over n doubles (0 for n = 0): the Newton loop's
 * stopping test ||d||_inf / dt <= eps_d (Algorithm 1).  Exact (no rounding).
 */
int agipc_max_abs(agipc_ctx *ctx, int64_t n, const double *v, double *out_dev);

/* Synchronize the context's stream; return (and clear) the first device-side
 * error recorded since the last call, or AGIPC_OK. */
int agipc_status(agipc_ctx *ctx);

/* Static, human-readable name of a status code. */
const char *agipc_status_string(int status);

#ifdef __cplusplus
}
#endif

#endif /* AGIPC_H */
