// StVK tetrahedra on the GPU: the fine system of the differentiation form and
// its vector-Jacobian product.
//
//   agipc_fine_assemble_stvk : per-tet gradient and PSD-projected 12x12
//       Hessian (Eq. 1 divided by dt^2: H = M/h^2 + d2Psi/dx2,
//       g = M/h^2 (x - x_hat) + dPsi/dx + g_extra, x_hat = X_rest + shift),
//       summed straight into the values of the static fine upper BSR.
//   agipc_restrict : v_c = U v, the adjoint's right-hand side.
//   agipc_stvk_vjp : the adjoint's per-element contraction.  With the
//       coarse adjoint lambda_c = H_c^-1 U v (v = dL/dx_next) and
//       lambda = U^T lambda_c, the step's sensitivity to a parameter theta
//       is dL/dtheta = -lambda^T (dg/dtheta + dH/dtheta dx).  For the rest
//       positions X this is the derivative of
//       phi_e(X) = lambda_e^T g_e(X) + lambda_e^T H_e+(X) dx_e, where the
//       clamp H+ = U max(L,0) U^T is differentiated through the
//       eigendecomposition (Daleckii-Krein): lambda^T dH+ dx = <dH, Z>,
//       Z = U (D o (a b^T)) U^T, a = U^T lambda, b = U^T dx, D the divided
//       differences of max(.,0) over the eigenvalues.  phi_e is then
//       differentiated in reverse mode, by hand.  For the per-tet Young's
//       modulus (Psi_e is linear in E_e at fixed nu and the clamp commutes
//       with positive scaling) dL/dE_e = -phi_e / E_e.  The inertia term
//       M/h^2 (x - x_hat), x_hat = X_rest + shift, adds lambda M/h^2.
//
// Element formulas (independent of the input generator, same physics):
//   F = Ds Dm^-1, G = (F^T F - I)/2, S = 2 mu G + lam tr(G) I, P = F S,
//   g[a,c] = V (P w_a)_c with w_a the shape-function gradients (rows of
//   Dm^-1, w_0 = -sum), and
//   H[a,c][b,d] = V (delta_cd w_a.S w_b + mu Y_b[c] Y_a[d] + mu (F F^T)_cd
//                 w_a.w_b + lam Y_a[c] Y_b[d]),  Y_a = F w_a.
//
// Translations are an exact null space of H, so the spectrum lives in the
// 9-dimensional complement: with the Helmert basis Q4 (4x3, orthonormal
// columns orthogonal to (1,1,1,1)) and Q = Q4 (x) I3, H = Q M Q^T where M
// has the same formula with the three reduced gradients wh_k = sum_a
// Q4[a][k] w_a in place of the four w_a; H+ = Q M+ Q^T.
//
// The projection is computed in two passes.  Every tet's exact Hessian H
// is summed; a cyclic Jacobi eigendecomposition of M in FP32 (rotation
// angles by the Rutishauser formulas, Golub & Van Loan, Matrix
// Computations, Sec. 8.5) then flags the tets whose smallest eigenvalue is
// not clearly positive (below 1e-4 of the largest, far above FP32's error).
// Those alone get the FP64 correction -Q M_neg Q^T: the FP32 eigenvectors,
// re-orthonormalised in FP64, turn M into a nearly diagonal A = U^T M U,
// FP64 Jacobi sweeps over the pairs that touch the flagged eigenvalues
// decouple the non-positive block, and M_neg = sum_{A_ii < 0} A_ii u_i u_i^T.
// Positive-definite tets (about half of a deformed mesh) so skip every FP64
// eigen step.  The VJP reuses the split: all tets take the unprojected
// terms (D = 1), flagged tets add the correction of D - 1.
#include <math.h>

#include "agipc_common.cuh"

namespace {

constexpr double kR2 = 0.70710678118654752440;   // 1/sqrt(2)
constexpr double kR6 = 0.40824829046386301637;   // 1/sqrt(6)
constexpr double kR12 = 0.28867513459481288225;  // 1/sqrt(12)

// Helmert basis of the complement of (1,1,1,1) in R^4.
__host__ __device__ constexpr double hq(int a, int k)
{
    return k == 0 ? (a == 0 ? kR2 : a == 1 ? -kR2 : 0.0)
         : k == 1 ? (a <= 1 ? kR6 : a == 2 ? -2.0 * kR6 : 0.0)
                  : (a <= 2 ? kR12 : -3.0 * kR12);
}

constexpr float kPdRel = 1e-4f;      // "clearly positive" eigenvalue threshold (x largest |eigenvalue|)
constexpr int kSweeps32 = 10;        // FP32 Jacobi sweep cap
constexpr int kSweeps64 = 4;         // FP64 refinement sweep cap
constexpr int kRefineThreads = 32;   // one warp per block in the refinement kernels
constexpr int kRefineSlots = 126;    // FP64 words of shared memory per refinement thread (32,256 B a block)

struct Tet {
    double V;           // volume
    double W[3][3];     // Dm^-1; row k is the shape gradient of vertex k+1
    double w0[3];       // shape gradient of vertex 0
    double wh[3][3];    // reduced gradients wh[k] = sum_a hq(a,k) w_a
    double xh[3][3];    // reduced positions
    double F[3][3], S[3][3], FFt[3][3];
    double Y[3][3];     // Y[k] = F wh[k]
    double s[3][3];     // wh_k . S wh_l
    double om[3][3];    // wh_k . wh_l
};

__device__ __forceinline__ void lame(double E, double nu, double &mu, double &lam)
{
    mu = E / (2.0 * (1.0 + nu));
    lam = E * nu / ((1.0 + nu) * (1.0 - 2.0 * nu));
}

__device__ __forceinline__ bool load_tet(const int32_t *tets, int64_t e, int32_t n, const double *Xr, const double *xc,
                                         int vid[4], double X[4][3], double x[4][3])
{
    bool ok = true;
#pragma unroll
    for (int a = 0; a < 4; ++a) {
        vid[a] = tets[4 * e + a];
        if ((unsigned)vid[a] >= (unsigned)n) ok = false;
    }
    if (!ok) return false;
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            X[a][c] = Xr[3 * (int64_t)vid[a] + c];
            x[a][c] = xc[3 * (int64_t)vid[a] + c];
        }
    return true;
}

__device__ __forceinline__ void tet_eval(const double X[4][3], const double x[4][3], double mu, double lam, Tet &t)
{
    double Dm[3][3];
#pragma unroll
    for (int c = 0; c < 3; ++c)
#pragma unroll
        for (int k = 0; k < 3; ++k) Dm[c][k] = X[k + 1][c] - X[0][c];
    const double c00 = Dm[1][1] * Dm[2][2] - Dm[1][2] * Dm[2][1];
    const double c01 = Dm[1][2] * Dm[2][0] - Dm[1][0] * Dm[2][2];
    const double c02 = Dm[1][0] * Dm[2][1] - Dm[1][1] * Dm[2][0];
    const double det = Dm[0][0] * c00 + Dm[0][1] * c01 + Dm[0][2] * c02;
    const double id = 1.0 / det;
    t.W[0][0] = c00 * id;
    t.W[0][1] = (Dm[0][2] * Dm[2][1] - Dm[0][1] * Dm[2][2]) * id;
    t.W[0][2] = (Dm[0][1] * Dm[1][2] - Dm[0][2] * Dm[1][1]) * id;
    t.W[1][0] = c01 * id;
    t.W[1][1] = (Dm[0][0] * Dm[2][2] - Dm[0][2] * Dm[2][0]) * id;
    t.W[1][2] = (Dm[0][2] * Dm[1][0] - Dm[0][0] * Dm[1][2]) * id;
    t.W[2][0] = c02 * id;
    t.W[2][1] = (Dm[0][1] * Dm[2][0] - Dm[0][0] * Dm[2][1]) * id;
    t.W[2][2] = (Dm[0][0] * Dm[1][1] - Dm[0][1] * Dm[1][0]) * id;
    t.V = fabs(det) * (1.0 / 6.0);
#pragma unroll
    for (int j = 0; j < 3; ++j) t.w0[j] = -(t.W[0][j] + t.W[1][j] + t.W[2][j]);
#pragma unroll
    for (int k = 0; k < 3; ++k)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            double v = hq(0, k) * t.w0[j];
#pragma unroll
            for (int a = 1; a < 4; ++a) v += hq(a, k) * t.W[a - 1][j];
            t.wh[k][j] = v;
            double u = 0.0;
#pragma unroll
            for (int a = 0; a < 4; ++a) u += hq(a, k) * x[a][j];
            t.xh[k][j] = u;
        }
    // F = sum_a x_a w_a^T = sum_k xh_k wh_k^T
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j)
            t.F[i][j] = t.xh[0][i] * t.wh[0][j] + t.xh[1][i] * t.wh[1][j] + t.xh[2][i] * t.wh[2][j];
    double G[3][3];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            const double v = t.F[0][i] * t.F[0][j] + t.F[1][i] * t.F[1][j] + t.F[2][i] * t.F[2][j];
            G[i][j] = 0.5 * (i == j ? v - 1.0 : v);
        }
    const double trG = G[0][0] + G[1][1] + G[2][2];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            t.S[i][j] = 2.0 * mu * G[i][j] + (i == j ? lam * trG : 0.0);
            t.FFt[i][j] = t.F[i][0] * t.F[j][0] + t.F[i][1] * t.F[j][1] + t.F[i][2] * t.F[j][2];
        }
#pragma unroll
    for (int k = 0; k < 3; ++k)
#pragma unroll
        for (int c = 0; c < 3; ++c)
            t.Y[k][c] = t.F[c][0] * t.wh[k][0] + t.F[c][1] * t.wh[k][1] + t.F[c][2] * t.wh[k][2];
#pragma unroll
    for (int k = 0; k < 3; ++k)
#pragma unroll
        for (int l = 0; l < 3; ++l) {
            double sv = 0.0, ov = 0.0;
#pragma unroll
            for (int i = 0; i < 3; ++i) {
                const double Swl = t.S[i][0] * t.wh[l][0] + t.S[i][1] * t.wh[l][1] + t.S[i][2] * t.wh[l][2];
                sv += t.wh[k][i] * Swl;
                ov += t.wh[k][i] * t.wh[l][i];
            }
            t.s[k][l] = sv;
            t.om[k][l] = ov;
        }
}

// Shape gradient of vertex a.
__device__ __forceinline__ double wgrad(const Tet &t, int a, int j) { return a == 0 ? t.w0[j] : t.W[a - 1][j]; }

// Packed upper-triangle index of a symmetric 9x9 matrix.
__host__ __device__ constexpr int pk(int i, int j)
{
    return i <= j ? 9 * i - (i * (i - 1)) / 2 + (j - i) : 9 * j - (j * (j - 1)) / 2 + (i - j);
}

// Reduced Hessian M (9x9, index 3k+c), packed upper, formed in FP32 from
// the FP64 invariants (it only feeds the FP32 classification).
__device__ __forceinline__ void reduced_m32(const Tet &t, double mu, double lam, float A[45])
{
    float Y[3][3], FF[3][3], om[3][3], sv[3][3];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            Y[i][j] = (float)t.Y[i][j];
            FF[i][j] = (float)t.FFt[i][j];
            om[i][j] = (float)t.om[i][j];
            sv[i][j] = (float)(t.V * t.s[i][j]);
        }
    const float vm = (float)(t.V * mu), vl = (float)(t.V * lam);
#pragma unroll
    for (int r = 0; r < 9; ++r)
#pragma unroll
        for (int q = r; q < 9; ++q) {
            const int k = r / 3, c = r % 3, l = q / 3, d = q % 3;
            float v = vm * (Y[l][c] * Y[k][d] + FF[c][d] * om[k][l]) + vl * Y[k][c] * Y[l][d];
            if (c == d) v += sv[k][l];
            A[pk(r, q)] = v;
        }
}

// Reduced Hessian M (9x9, index 3k+c), FP64, packed upper.
__device__ __forceinline__ void reduced_m64(const Tet &t, double mu, double lam, double M[45])
{
#pragma unroll
    for (int r = 0; r < 9; ++r)
#pragma unroll
        for (int q = r; q < 9; ++q) {
            const int k = r / 3, c = r % 3, l = q / 3, d = q % 3;
            double v = mu * (t.Y[l][c] * t.Y[k][d] + t.FFt[c][d] * t.om[k][l]) + lam * t.Y[k][c] * t.Y[l][d];
            if (c == d) v += t.s[k][l];
            M[pk(r, q)] = t.V * v;
        }
}

// Cyclic Jacobi on a packed symmetric 9x9 FP32 matrix: A becomes (nearly)
// diagonal, U collects the eigenvectors as columns.  Branch-free rotations;
// the warp leaves the sweep loop when all its lanes have converged.
__device__ __forceinline__ void jacobi9f(float A[45], float U[9][9])
{
#pragma unroll
    for (int i = 0; i < 9; ++i)
#pragma unroll
        for (int j = 0; j < 9; ++j) U[i][j] = i == j ? 1.f : 0.f;
    float fro = 0.f;
#pragma unroll
    for (int r = 0; r < 9; ++r)
#pragma unroll
        for (int q = r; q < 9; ++q) fro += (r == q ? 1.f : 2.f) * A[pk(r, q)] * A[pk(r, q)];
    const float scale = sqrtf(fro);
    const float thr = 1e-9f * scale;
    for (int sweep = 0; sweep < kSweeps32; ++sweep) {
        float off = 0.f;
#pragma unroll
        for (int p = 0; p < 9; ++p)
#pragma unroll
            for (int q = p + 1; q < 9; ++q) off = fmaxf(off, fabsf(A[pk(p, q)]));
        if (__all_sync(__activemask(), !(off > 1e-6f * scale))) break;
#pragma unroll
        for (int p = 0; p < 8; ++p)
#pragma unroll
            for (int q = p + 1; q < 9; ++q) {
                const float apq = A[pk(p, q)];
                const bool rot = fabsf(apq) > thr;
                const float theta = (A[pk(q, q)] - A[pk(p, p)]) / (2.f * (rot ? apq : 1.f));
                float tt = copysignf(1.f, theta) / (fabsf(theta) + sqrtf(theta * theta + 1.f));
                tt = rot ? tt : 0.f;
                const float c = rsqrtf(tt * tt + 1.f);
                const float s = tt * c;
                const float tau = s / (1.f + c);
                A[pk(p, p)] -= tt * apq;
                A[pk(q, q)] += tt * apq;
                A[pk(p, q)] = rot ? 0.f : apq;
#pragma unroll
                for (int k = 0; k < 9; ++k) {
                    if (k != p && k != q) {
                        const float akp = A[pk(k, p)], akq = A[pk(k, q)];
                        A[pk(k, p)] = akp - s * (akq + tau * akp);
                        A[pk(k, q)] = akq + s * (akp - tau * akq);
                    }
                    const float ukp = U[k][p], ukq = U[k][q];
                    U[k][p] = ukp - s * (ukq + tau * ukp);
                    U[k][q] = ukq + s * (ukp - tau * ukq);
                }
            }
    }
}

// FP32 eigen-classification of a tet's reduced Hessian: the number of
// eigenvalues that are not clearly positive.
__device__ __forceinline__ int flagged_count(const float A[45])
{
    float big = 0.f;
#pragma unroll
    for (int i = 0; i < 9; ++i) big = fmaxf(big, fabsf(A[pk(i, i)]));
    int m = 0;
#pragma unroll
    for (int i = 0; i < 9; ++i) m += A[pk(i, i)] <= kPdRel * big ? 1 : 0;
    return m;
}

// Shared-memory slots of one refinement thread: U (81 words, column j at
// 9j), then A (45 words, packed upper).  Slot s of thread `lane` lives at
// sm[s * kRefineThreads + lane] so that a warp's accesses hit 32 banks.
struct Slots {
    double *base;
    int lane;
    __device__ __forceinline__ double &u(int row, int col) const { return base[(9 * col + row) * kRefineThreads + lane]; }
    __device__ __forceinline__ double &a(int i, int j) const { return base[(81 + pk(i, j)) * kRefineThreads + lane]; }
    __device__ __forceinline__ double &raw(int s) const { return base[s * kRefineThreads + lane]; }
};

// FP32 eigenpairs of a flagged tet's reduced Hessian, written by pass 1 and
// read by pass 2: one 368-byte record per tet (92 floats, 16-byte aligned):
// the 9 eigenvalues, then eigenvector i's rows at 9 + 9 i + r, then 2 pad.
// A flagged tet's record is written whole (full sectors, no read-fill).
constexpr int kEigRec = 92;

struct EigStore {
    float *base;
    int64_t nt;
    __device__ __forceinline__ const float &val(int64_t e, int i) const { return base[e * kEigRec + i]; }
    __device__ __forceinline__ const float &vec(int64_t e, int r, int i) const
    {
        return base[e * kEigRec + 9 + 9 * i + r];
    }
};

__device__ __forceinline__ void store_eig(const EigStore &es, int64_t e, const float A[45], const float U[9][9])
{
    float rec[kEigRec];
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        rec[i] = A[pk(i, i)];
#pragma unroll
        for (int r = 0; r < 9; ++r) rec[9 + 9 * i + r] = U[r][i];
    }
    rec[90] = rec[91] = 0.f;
    float4 *dst = reinterpret_cast<float4 *>(es.base + e * kEigRec);
#pragma unroll
    for (int q = 0; q < kEigRec / 4; ++q) dst[q] = make_float4(rec[4 * q], rec[4 * q + 1], rec[4 * q + 2], rec[4 * q + 3]);
}

// Pass 1 parks every tet's FP32 reduced Hessian (45 floats, padded to 48) in
// the tet's record slot for the classification kernel; NaN in the first word
// marks a tet pass 1 rejected (bad index or non-finite element).
__device__ __forceinline__ void store_m32(const EigStore &es, int64_t e, const float A[45], bool valid)
{
    float4 *dst = reinterpret_cast<float4 *>(es.base + e * kEigRec);
#pragma unroll
    for (int q = 0; q < 12; ++q) {
        float v[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) v[k] = 4 * q + k < 45 ? A[4 * q + k] : 0.f;
        if (q == 0 && !valid) v[0] = __int_as_float(0x7fc00000);
        dst[q] = make_float4(v[0], v[1], v[2], v[3]);
    }
}

// FP64 refinement of a tet's FP32 eigenbasis (the pairs pass 1 stored).
// Orders the flagged eigenvalues first, re-orthonormalises U in FP64
// (modified Gram-Schmidt), forms A = U^T M U and runs FP64 Jacobi sweeps
// over every pair (p, q) with p < m_warp (all pairs when all_pairs),
// m_warp the warp's largest flagged count (the worklist is ordered by
// flagged count, so a warp's tets mostly share it).  Returns m_warp.
__device__ int refine64(const Tet &t, double mu, double lam, const Slots &sl, bool all_pairs, const EigStore &es,
                        int64_t e)
{
    float big = 0.f;
#pragma unroll
    for (int i = 0; i < 9; ++i) big = fmaxf(big, fabsf(es.val(e, i)));
    // order: flagged eigenvalues first (stable in index), then the rest
    int nf = 0;
#pragma unroll
    for (int i = 0; i < 9; ++i) nf += es.val(e, i) <= kPdRel * big ? 1 : 0;
    int fi = 0, pi = nf;
#pragma unroll 1
    for (int i = 0; i < 9; ++i) {
        const bool f = es.val(e, i) <= kPdRel * big;
        const int slot = f ? fi : pi;
        fi += f ? 1 : 0;
        pi += f ? 0 : 1;
#pragma unroll
        for (int r = 0; r < 9; ++r) sl.u(r, slot) = (double)es.vec(e, r, i);
    }
    const unsigned mask = __activemask();
    const int m_warp = all_pairs ? 8 : __reduce_max_sync(mask, nf);
    // modified Gram-Schmidt in FP64
#pragma unroll 1
    for (int j = 0; j < 9; ++j) {
        for (int i = 0; i < j; ++i) {
            double d = 0.0;
#pragma unroll
            for (int r = 0; r < 9; ++r) d += sl.u(r, i) * sl.u(r, j);
#pragma unroll
            for (int r = 0; r < 9; ++r) sl.u(r, j) -= d * sl.u(r, i);
        }
        double nrm = 0.0;
#pragma unroll
        for (int r = 0; r < 9; ++r) nrm += sl.u(r, j) * sl.u(r, j);
        const double inv = 1.0 / sqrt(nrm);
#pragma unroll
        for (int r = 0; r < 9; ++r) sl.u(r, j) *= inv;
    }
    // A = U^T M U with M formed once (45 entries): M u_j is 81 FMAs
    double M[45];
    reduced_m64(t, mu, lam, M);
    double scale = 0.0;
#pragma unroll 1
    for (int j = 0; j < 9; ++j) {
        double v[9], mv[9];
#pragma unroll
        for (int r = 0; r < 9; ++r) v[r] = sl.u(r, j);
#pragma unroll
        for (int r = 0; r < 9; ++r) {
            double acc = 0.0;
#pragma unroll
            for (int q = 0; q < 9; ++q) acc = fma(M[pk(r, q)], v[q], acc);
            mv[r] = acc;
        }
        for (int i = 0; i <= j; ++i) {
            double d = 0.0;
#pragma unroll
            for (int r = 0; r < 9; ++r) d += sl.u(r, i) * mv[r];
            sl.a(i, j) = d;
            scale = fmax(scale, fabs(d));
        }
    }
    for (int sweep = 0; sweep < kSweeps64; ++sweep) {
        double off = 0.0;
        for (int p = 0; p < m_warp; ++p)
            for (int q = p + 1; q < 9; ++q) off = fmax(off, fabs(sl.a(p, q)));
        if (__all_sync(mask, !(off > 1e-15 * scale))) break;
        for (int p = 0; p < m_warp; ++p)
            for (int q = p + 1; q < 9; ++q) {
                // The angle only decides how much of a_pq is removed, so it is
                // taken in FP32; c = 1/sqrt(1 + t^2) and s = t c in FP64 keep
                // the rotation orthogonal to FP64 precision, and the update
                // is the exact similarity J^T A J with J = [c s; -s c].
                const double apq = sl.a(p, q), app = sl.a(p, p), aqq = sl.a(q, q);
                const float fpq = (float)apq;
                float tf = 0.f;
                if (fpq != 0.f) {
                    const float th = ((float)aqq - (float)app) / (2.f * fpq);
                    tf = copysignf(1.f, th) / (fabsf(th) + sqrtf(fmaf(th, th, 1.f)));
                    tf = isfinite(tf) ? tf : 0.f;
                }
                const double tt = (double)tf;
                const double c = rsqrt(fma(tt, tt, 1.0));
                const double s = tt * c;
                const double cc = c * c, ss = s * s, cs = c * s;
                sl.a(p, p) = fma(cc, app, fma(-2.0 * cs, apq, ss * aqq));
                sl.a(q, q) = fma(ss, app, fma(2.0 * cs, apq, cc * aqq));
                sl.a(p, q) = fma(cc - ss, apq, cs * (app - aqq));
                for (int k = 0; k < 9; ++k) {
                    if (k != p && k != q) {
                        const double akp = sl.a(k, p), akq = sl.a(k, q);
                        sl.a(k, p) = fma(c, akp, -s * akq);
                        sl.a(k, q) = fma(s, akp, c * akq);
                    }
                    const double ukp = sl.u(k, p), ukq = sl.u(k, q);
                    sl.u(k, p) = fma(c, ukp, -s * ukq);
                    sl.u(k, q) = fma(s, ukp, c * ukq);
                }
            }
    }
    return m_warp;
}

// Position of block (r, c), r <= c, in the sorted columns of row r; -1 if the
// structure lacks it.
__device__ __forceinline__ int64_t find_block(const int32_t *__restrict__ row_ptr, const int32_t *__restrict__ col,
                                              int64_t nnzb, int32_t r, int32_t c)
{
    int32_t lo = row_ptr[r], hi = row_ptr[r + 1] - 1;
    if (lo < 0 || hi >= nnzb) return -1;
    while (lo <= hi) {
        const int32_t mid = (lo + hi) >> 1;
        const int32_t v = col[mid];
        if (v == c) return mid;
        if (v < c) lo = mid + 1;
        else hi = mid - 1;
    }
    return -1;
}

// Local vertex pairs (s, t), s <= t, of the 10 upper 3x3 blocks of a tet.
__host__ __device__ constexpr int pair_s(int q) { return q < 4 ? 0 : q < 7 ? 1 : q < 9 ? 2 : 3; }
__host__ __device__ constexpr int pair_t(int q) { return q < 4 ? q : q < 7 ? q - 3 : q < 9 ? q - 5 : 3; }

// Adds blk(c, d) to the fine block of local vertex pair (sa, sb); reports a
// missing block.
template <class Blk>
__device__ __forceinline__ void scatter_block(const int32_t *row_ptr, const int32_t *col, int64_t nnzb,
                                              double *fine_val, const int vid[4], int sa, int sb, Blk blk,
                                              uint32_t *status)
{
    const int32_t va = vid[sa], vb = vid[sb];
    if (sa != sb && va == vb) {
        set_status(status, ST_BAD_INDEX);
        return;
    }
    const bool tr = va > vb;
    const int64_t pos = find_block(row_ptr, col, nnzb, tr ? vb : va, tr ? va : vb);
    if (pos < 0) {
        set_status(status, ST_BAD_INDEX);
        return;
    }
    double *dst = fine_val + 9 * pos;
#pragma unroll
    for (int c = 0; c < 3; ++c)
#pragma unroll
        for (int d = 0; d < 3; ++d) atomicAdd(dst + (tr ? 3 * d + c : 3 * c + d), blk(c, d));
}

// Worklist of flagged tets, ordered by flagged count so that the warps of
// pass 2 mostly share it.  Workspace words: hdr[1..9] tets per count,
// hdr[10..18] scatter cursors, then the list, then one count byte per tet.
constexpr int kHdr = 32;

// Warp-aggregated count of a tet's flagged count m (0 = not flagged).
__device__ __forceinline__ void count_flag(int32_t *hdr, int m)
{
    const unsigned mask = __activemask();
    const unsigned peers = __match_any_sync(mask, m);
    if ((int)(threadIdx.x & 31) == __ffs(peers) - 1 && m > 0) atomicAdd(hdr + m, __popc(peers));
}

// list[offset(m) + k] = e for every flagged tet, offset(m) = sum of the
// counts below m.
__global__ void bucket_scatter_kernel(int64_t nt, const uint8_t *__restrict__ mcode, int32_t *hdr, int32_t *list)
{
    __shared__ int32_t s_off[10];
    if (threadIdx.x == 0) {
        int32_t o = 0;
        for (int m = 1; m <= 9; ++m) {
            s_off[m] = o;
            o += hdr[m];
        }
    }
    __syncthreads();
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nt; e += (int64_t)gridDim.x * blockDim.x) {
        const int m = mcode[e];
        const unsigned mask = __activemask();
        const unsigned peers = __match_any_sync(mask, m);
        const int lane = threadIdx.x & 31, leader = __ffs(peers) - 1;
        int base = 0;
        if (lane == leader && m > 0) base = atomicAdd(hdr + 9 + m, __popc(peers));
        base = __shfl_sync(mask, base, leader);
        if (m > 0 && m <= 9) list[s_off[m] + base + __popc(peers & ((1u << lane) - 1u))] = (int32_t)e;
    }
}

__device__ __forceinline__ int64_t flagged_total(const int32_t *hdr)
{
    int64_t t = 0;
    for (int m = 1; m <= 9; ++m) t += hdr[m];
    return t;
}

// A load the compiler may not merge with an earlier one.
__device__ __forceinline__ double ld_fresh(const double *p)
{
    double v;
    asm volatile("ld.global.f64 %0, [%1];" : "=d"(v) : "l"(p));
    return v;
}

struct Shift3 {
    double v[3];
};

// One thread per fine row: zero the row's blocks, put M/h^2 on its diagonal
// block and set g = M/h^2 (x - x_hat) (+ g_extra), x_hat = X_rest + shift.
__global__ void fine_init_kernel(int32_t n, const int32_t *__restrict__ row_ptr, const int32_t *__restrict__ col,
                                 int64_t nnzb, const double *__restrict__ mass_h2, const double *__restrict__ x,
                                 const double *__restrict__ Xr, Shift3 shift, const double *__restrict__ g_extra,
                                 double *__restrict__ fine_val, double *__restrict__ g, uint32_t *status)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int32_t b0 = row_ptr[i], b1 = row_ptr[i + 1];
        if (b0 < 0 || b1 < b0 || b1 > nnzb || b0 == b1 || col[b0] != i) {
            set_status(status, ST_BAD_INDEX);
            continue;
        }
        for (int64_t k = 9 * (int64_t)b0; k < 9 * (int64_t)b1; ++k) fine_val[k] = 0.0;
        const double m = mass_h2[i];
        fine_val[9 * (int64_t)b0] = m;
        fine_val[9 * (int64_t)b0 + 4] = m;
        fine_val[9 * (int64_t)b0 + 8] = m;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            double v = m * (x[3 * i + c] - (Xr[3 * i + c] + shift.v[c]));
            if (g_extra) v += g_extra[3 * i + c];
            g[3 * i + c] = v;
        }
    }
}

// Pass 1 of the assembly, one thread per tet: gradient and exact Hessian
// blocks in FP64, FP32 eigen-classification, flagged tets to the list.
__global__ void __launch_bounds__(128) elem_pass1_kernel(int32_t n, int64_t nt, const int32_t *__restrict__ tets,
                                                         const int32_t *__restrict__ row_ptr,
                                                         const int32_t *__restrict__ col, int64_t nnzb,
                                                         const double *__restrict__ Xr, const double *__restrict__ xc,
                                                         const double *__restrict__ E, double nu, double *fine_val,
                                                         double *g, EigStore es, uint32_t *status)
{
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nt; e += (int64_t)gridDim.x * blockDim.x) {
        int vid[4];
        double X[4][3], x[4][3];
        bool parked = false;
        if (!load_tet(tets, e, n, Xr, xc, vid, X, x)) {
            set_status(status, ST_BAD_INDEX);
        } else {
            double mu, lam;
            lame(E[e], nu, mu, lam);
            Tet t;
            tet_eval(X, x, mu, lam, t);
            double P[3][3];
#pragma unroll
            for (int i = 0; i < 3; ++i)
#pragma unroll
                for (int j = 0; j < 3; ++j) P[i][j] = t.F[i][0] * t.S[0][j] + t.F[i][1] * t.S[1][j] + t.F[i][2] * t.S[2][j];
            bool finite = isfinite(t.V) && t.V > 0.0;
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    const double ga =
                        t.V * (P[c][0] * wgrad(t, a, 0) + P[c][1] * wgrad(t, a, 1) + P[c][2] * wgrad(t, a, 2));
                    finite = finite && isfinite(ga);
                    atomicAdd(g + 3 * (int64_t)vid[a] + c, ga);
                }
            if (!finite) {
                set_status(status, ST_NONFINITE);
            } else {
                double Yf[4][3], Sw[4][3];
#pragma unroll
                for (int a = 0; a < 4; ++a)
#pragma unroll
                    for (int c = 0; c < 3; ++c) {
                        Yf[a][c] = t.F[c][0] * wgrad(t, a, 0) + t.F[c][1] * wgrad(t, a, 1) + t.F[c][2] * wgrad(t, a, 2);
                        Sw[a][c] = t.S[c][0] * wgrad(t, a, 0) + t.S[c][1] * wgrad(t, a, 1) + t.S[c][2] * wgrad(t, a, 2);
                    }
#pragma unroll
                for (int q = 0; q < 10; ++q) {
                    const int sa = pair_s(q), sb = pair_t(q);
                    double wSw = 0.0, ww = 0.0;
#pragma unroll
                    for (int j = 0; j < 3; ++j) {
                        wSw += wgrad(t, sa, j) * Sw[sb][j];
                        ww += wgrad(t, sa, j) * wgrad(t, sb, j);
                    }
                    scatter_block(row_ptr, col, nnzb, fine_val, vid, sa, sb,
                                  [&](int c, int d) {
                                      double h = mu * Yf[sb][c] * Yf[sa][d] + mu * t.FFt[c][d] * ww +
                                                 lam * Yf[sa][c] * Yf[sb][d];
                                      if (c == d) h += wSw;
                                      return t.V * h;
                                  },
                                  status);
                }
                float A32[45];
                reduced_m32(t, mu, lam, A32);
                store_m32(es, e, A32, true);
                parked = true;
            }
        }
        if (!parked) {
            float z[45] = {};
            store_m32(es, e, z, false);
        }
    }
}

// FP32 eigen-classification of every tet's reduced Hessian parked by pass 1
// (cyclic Jacobi), flagged tets' eigenpair records written over the parked
// matrix, counts for the worklist.  Kept apart from the FP64 element work so
// that each kernel's instruction stream stays small.
__global__ void __launch_bounds__(128) classify_kernel(int64_t nt, EigStore es, int32_t *hdr, uint8_t *mcode)
{
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nt; e += (int64_t)gridDim.x * blockDim.x) {
        const float4 *src = reinterpret_cast<const float4 *>(es.base + e * kEigRec);
        float A[48];
#pragma unroll
        for (int q = 0; q < 12; ++q) {
            const float4 v = src[q];
            A[4 * q] = v.x;
            A[4 * q + 1] = v.y;
            A[4 * q + 2] = v.z;
            A[4 * q + 3] = v.w;
        }
        int flag = 0;
        if (!isnan(A[0])) {
            float U[9][9];
            jacobi9f(A, U);
            flag = flagged_count(A);
            if (flag > 0) store_eig(es, e, A, U);
        }
        mcode[e] = (uint8_t)flag;
        count_flag(hdr, flag);
    }
}

// Pass 2 of the assembly, flagged tets only: H+ = H - Q M_neg Q^T.
__global__ void __launch_bounds__(kRefineThreads) elem_pass2_kernel(
    int32_t n, const int32_t *__restrict__ tets, const int32_t *__restrict__ row_ptr, const int32_t *__restrict__ col,
    int64_t nnzb, const double *__restrict__ Xr, const double *__restrict__ xc, const double *__restrict__ E, double nu,
    double *fine_val, const int32_t *__restrict__ hdr, const int32_t *__restrict__ list, int64_t cap, EigStore es,
    uint32_t *status)
{
    __shared__ double sm[kRefineSlots * kRefineThreads];
    const Slots sl{sm, (int)threadIdx.x};
    const int64_t cnt = min64(flagged_total(hdr), cap);
    for (int64_t i = blockIdx.x * (int64_t)kRefineThreads + threadIdx.x; i < cnt;
         i += (int64_t)gridDim.x * kRefineThreads) {
        const int64_t e = list[i];
        int vid[4];
        double X[4][3], x[4][3];
        if (!load_tet(tets, e, n, Xr, xc, vid, X, x)) continue;   // reported by pass 1
        double mu, lam;
        lame(E[e], nu, mu, lam);
        Tet t;
        tet_eval(X, x, mu, lam, t);
        const int m_w = refine64(t, mu, lam, sl, false, es, e);
        // negative part of the flagged block; R_i = Q u_i (12 words) is
        // written downwards from the top slot once A has been read: R_i
        // occupies [114 - 12 i, 126 - 12 i), above every column j < m_w <= 6
        // of U that is still needed.  Wider warps expand on the fly.
        double d[9];
        for (int i2 = 0; i2 < 9; ++i2) {
            const double aii = i2 < m_w ? sl.a(i2, i2) : 0.0;
            d[i2] = aii < 0.0 ? aii : 0.0;
        }
        const bool stored = m_w <= 6;
        if (stored) {
            for (int i2 = 0; i2 < m_w; ++i2) {
                double u[9];
#pragma unroll
                for (int r = 0; r < 9; ++r) u[r] = sl.u(r, i2);
#pragma unroll
                for (int a = 0; a < 4; ++a)
#pragma unroll
                    for (int c = 0; c < 3; ++c)
                        sl.raw(114 - 12 * i2 + 3 * a + c) = hq(a, 0) * u[c] + hq(a, 1) * u[3 + c] + hq(a, 2) * u[6 + c];
            }
        }
        auto rq = [&](int i2, int a, int c) -> double {
            if (stored) return sl.raw(114 - 12 * i2 + 3 * a + c);
            return hq(a, 0) * sl.u(c, i2) + hq(a, 1) * sl.u(3 + c, i2) + hq(a, 2) * sl.u(6 + c, i2);
        };
#pragma unroll 1
        for (int q = 0; q < 10; ++q) {
            const int sa = pair_s(q), sb = pair_t(q);
            scatter_block(row_ptr, col, nnzb, fine_val, vid, sa, sb,
                          [&](int c, int dd) {
                              double acc = 0.0;
                              for (int i2 = 0; i2 < m_w; ++i2) acc += d[i2] * rq(i2, sa, c) * rq(i2, sb, dd);
                              return -acc;
                          },
                          status);
        }
    }
}

// The Z-dependent sums of the reverse pass, accumulated one rank-one term
// Z = p q^T at a time (p, q as 3x3, p[k][c] = p_{3k+c}):
//   psi35 = sum z (lam Y_k[c] Y_l[d] + mu Y_k[d] Y_l[c]) and its Y-adjoint,
//   zt_kl = sum_c z(kc, lc), R_cd = sum_kl om_kl z(kc, ld),
//   rho_kl = sum_cd FFt_cd z(kc, ld).
struct ZAcc {
    double psi;
    double Yb[3][3], zt[3][3], R[3][3], rho[3][3];
};

__device__ __forceinline__ void zacc_init(ZAcc &a)
{
    a.psi = 0.0;
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) a.Yb[i][j] = a.zt[i][j] = a.R[i][j] = a.rho[i][j] = 0.0;
}

// The element invariants the Z sums read: Y and the symmetric om and FFt,
// from the element's registers ...
struct ZGeomRegs {
    const Tet &t;
    __device__ __forceinline__ double Y(int k, int c) const { return t.Y[k][c]; }
    __device__ __forceinline__ double om(int k, int l) const { return t.om[k][l]; }
    __device__ __forceinline__ double FFt(int c, int d) const { return t.FFt[c][d]; }
};

// ... or with om and FFt parked in shared-memory slots (upper triangles at
// slot base + sym3(i, j) and base + 6 + sym3(i, j)), Y in registers.
__host__ __device__ constexpr int sym3(int i, int j) { return i <= j ? (i == 0 ? j : i == 1 ? 2 + j : 5) : sym3(j, i); }

struct ZGeomShared {
    double Yr[3][3];
    const Slots &sl;
    int base;
    __device__ __forceinline__ double Y(int k, int c) const { return Yr[k][c]; }
    __device__ __forceinline__ double om(int k, int l) const { return sl.raw(base + sym3(k, l)); }
    __device__ __forceinline__ double FFt(int c, int d) const { return sl.raw(base + 6 + sym3(c, d)); }
};

template <class ZG>
__device__ __forceinline__ void zacc_rank1(const ZG &t, double mu, double lam, const double P[3][3],
                                           const double Q[3][3], ZAcc &a)
{
    // phases ordered so that few temporaries are live at once
    double pa = 0.0, qb = 0.0;
#pragma unroll
    for (int k = 0; k < 3; ++k)
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            pa += P[k][c] * t.Y(k, c);
            qb += Q[k][c] * t.Y(k, c);
        }
    a.psi += lam * pa * qb;
#pragma unroll
    for (int k = 0; k < 3; ++k)
#pragma unroll
        for (int c = 0; c < 3; ++c) a.Yb[k][c] += lam * (qb * P[k][c] + pa * Q[k][c]);
    // gam_kl = p_k . Y_l and del_lk = q_l . Y_k: psi_mu = mu sum gam_kl del_lk,
    // Yb_k += mu sum_l gam_kl q_l, Yb_l += mu sum_k del_lk p_k
#pragma unroll
    for (int k = 0; k < 3; ++k)
#pragma unroll
        for (int l = 0; l < 3; ++l) {
            const double gam = P[k][0] * t.Y(l, 0) + P[k][1] * t.Y(l, 1) + P[k][2] * t.Y(l, 2);
            const double del = Q[l][0] * t.Y(k, 0) + Q[l][1] * t.Y(k, 1) + Q[l][2] * t.Y(k, 2);
            a.psi += mu * gam * del;
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                a.Yb[k][c] += mu * gam * Q[l][c];
                a.Yb[l][c] += mu * del * P[k][c];
            }
        }
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) a.zt[i][j] += P[i][0] * Q[j][0] + P[i][1] * Q[j][1] + P[i][2] * Q[j][2];
    // R_cd += sum_k p_k[c] (om Q)_k[d], one column d at a time
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        double oq[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) oq[k] = t.om(k, 0) * Q[0][d] + t.om(k, 1) * Q[1][d] + t.om(k, 2) * Q[2][d];
#pragma unroll
        for (int c = 0; c < 3; ++c) a.R[c][d] += P[0][c] * oq[0] + P[1][c] * oq[1] + P[2][c] * oq[2];
    }
    // rho_kl += p_k . (FFt q_l), one l at a time
#pragma unroll
    for (int l = 0; l < 3; ++l) {
        double fq[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) fq[c] = t.FFt(c, 0) * Q[l][0] + t.FFt(c, 1) * Q[l][1] + t.FFt(c, 2) * Q[l][2];
#pragma unroll
        for (int k = 0; k < 3; ++k) a.rho[k][l] += P[k][0] * fq[0] + P[k][1] * fq[1] + P[k][2] * fq[2];
    }
}

// Reverse-mode derivative of psi = <P, Lam> + <Z, Mhat> with respect to the
// rest positions (Mhat = M / V; Z enters through its accumulated sums).
// Returns psi and adds dphi/dX (phi = V psi) to Xb.
__device__ __forceinline__ double reverse_phi(const Tet &t, double mu, double lam, const double lh[3][3],
                                              bool with_lambda, const ZAcc &za, double Xb[4][3])
{
    double Fb[3][3], whb[3][3], Yb[3][3];
    double zt[3][3], R[3][3], rho[3][3];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            Fb[i][j] = whb[i][j] = 0.0;
            Yb[i][j] = za.Yb[i][j];
            zt[i][j] = za.zt[i][j];
            R[i][j] = za.R[i][j];
            rho[i][j] = za.rho[i][j];
        }
    double psi = za.psi;
    // psi2 = <S, T>, T = sum_kl zt_kl wh_k wh_l^T; psi4 = mu <FFt, R>
    double T[3][3];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            double v = 0.0;
#pragma unroll
            for (int k = 0; k < 3; ++k)
#pragma unroll
                for (int l = 0; l < 3; ++l) v += zt[k][l] * t.wh[k][i] * t.wh[l][j];
            T[i][j] = v;
        }
    const double trT = T[0][0] + T[1][1] + T[2][2];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) psi += t.S[i][j] * T[i][j] + mu * t.FFt[i][j] * R[i][j];
    // Fbar from psi2: F (2 mu sym(T) + lam tr(T) I); from psi4: mu (R + R^T) F
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            double v = 0.0;
#pragma unroll
            for (int m = 0; m < 3; ++m) {
                const double Tsym = mu * (T[m][j] + T[j][m]) + (m == j ? lam * trT : 0.0);
                v += t.F[i][m] * Tsym + mu * (R[i][m] + R[m][i]) * t.F[m][j];
            }
            Fb[i][j] += v;
        }
    // Fbar and whbar from psi35 through Y_k = F wh_k
#pragma unroll
    for (int k = 0; k < 3; ++k)
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
            for (int j = 0; j < 3; ++j) {
                Fb[i][j] += Yb[k][i] * t.wh[k][j];
                whb[k][j] += t.F[i][j] * Yb[k][i];
            }
    // whbar from psi2 (explicit wh) and psi4 (omega)
#pragma unroll
    for (int k = 0; k < 3; ++k)
#pragma unroll
        for (int l = 0; l < 3; ++l) {
            const double cz = zt[k][l] + zt[l][k];
            const double cr = mu * (rho[k][l] + rho[l][k]);
#pragma unroll
            for (int j = 0; j < 3; ++j) {
                const double Swl = t.S[j][0] * t.wh[l][0] + t.S[j][1] * t.wh[l][1] + t.S[j][2] * t.wh[l][2];
                whb[k][j] += cz * Swl + cr * t.wh[l][j];
            }
        }
    if (with_lambda) {
        // psi1 = <P, Lam>, Lam = sum_k lh_k wh_k^T
        double P[3][3], Lam[3][3];
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
            for (int j = 0; j < 3; ++j) {
                P[i][j] = t.F[i][0] * t.S[0][j] + t.F[i][1] * t.S[1][j] + t.F[i][2] * t.S[2][j];
                Lam[i][j] = lh[0][i] * t.wh[0][j] + lh[1][i] * t.wh[1][j] + lh[2][i] * t.wh[2][j];
            }
        double LF = 0.0;
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
            for (int j = 0; j < 3; ++j) {
                psi += P[i][j] * Lam[i][j];
                LF += Lam[i][j] * t.F[i][j];
            }
        // Fbar += Lam S + mu F Lam^T F + mu FFt Lam + lam <Lam, F> F
        double FLt[3][3];
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
            for (int j = 0; j < 3; ++j)
                FLt[i][j] = t.F[i][0] * Lam[j][0] + t.F[i][1] * Lam[j][1] + t.F[i][2] * Lam[j][2];
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
            for (int j = 0; j < 3; ++j) {
                double v = lam * LF * t.F[i][j];
#pragma unroll
                for (int m = 0; m < 3; ++m)
                    v += Lam[i][m] * t.S[m][j] + mu * FLt[i][m] * t.F[m][j] + mu * t.FFt[i][m] * Lam[m][j];
                Fb[i][j] += v;
            }
        // whbar_k += P^T lh_k
#pragma unroll
        for (int k = 0; k < 3; ++k)
#pragma unroll
            for (int j = 0; j < 3; ++j) whb[k][j] += P[0][j] * lh[k][0] + P[1][j] * lh[k][1] + P[2][j] * lh[k][2];
    }
    // F = sum_k xh_k wh_k^T: whbar_k += Fbar^T xh_k
#pragma unroll
    for (int k = 0; k < 3; ++k)
#pragma unroll
        for (int j = 0; j < 3; ++j) whb[k][j] += Fb[0][j] * t.xh[k][0] + Fb[1][j] * t.xh[k][1] + Fb[2][j] * t.xh[k][2];
    // phi = V psi: wbar_a = V sum_k hq(a,k) whbar_k; Wbar[a-1] = wbar_a - wbar_0
    double Wb[3][3];
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        const double wb0 = t.V * (hq(0, 0) * whb[0][j] + hq(0, 1) * whb[1][j] + hq(0, 2) * whb[2][j]);
#pragma unroll
        for (int a = 1; a < 4; ++a)
            Wb[a - 1][j] = t.V * (hq(a, 0) * whb[0][j] + hq(a, 1) * whb[1][j] + hq(a, 2) * whb[2][j]) - wb0;
    }
    // Dmbar = -W^T Wbar W^T + psi V W^T
    double WtWb[3][3];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) WtWb[i][j] = t.W[0][i] * Wb[0][j] + t.W[1][i] * Wb[1][j] + t.W[2][i] * Wb[2][j];
#pragma unroll
    for (int c = 0; c < 3; ++c)
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const double Dmb = -(WtWb[c][0] * t.W[k][0] + WtWb[c][1] * t.W[k][1] + WtWb[c][2] * t.W[k][2]) +
                               psi * t.V * t.W[k][c];
            Xb[k + 1][c] += Dmb;
            Xb[0][c] -= Dmb;
        }
    return psi;
}

__device__ __forceinline__ void reduce_vec(const double v[4][3], double vh[3][3])
{
#pragma unroll
    for (int k = 0; k < 3; ++k)
#pragma unroll
        for (int c = 0; c < 3; ++c)
            vh[k][c] = hq(0, k) * v[0][c] + hq(1, k) * v[1][c] + hq(2, k) * v[2][c] + hq(3, k) * v[3][c];
}

__device__ __forceinline__ void load_pair(const int vid[4], const double *lam_f, const double *dx, double lh[3][3],
                                          double dh[3][3])
{
    double lv[4][3], dv[4][3];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            lv[a][c] = lam_f[3 * (int64_t)vid[a] + c];
            dv[a][c] = dx[3 * (int64_t)vid[a] + c];
        }
    reduce_vec(lv, lh);
    reduce_vec(dv, dh);
}

// VJP pass 1, one thread per tet: the unprojected terms (D = 1, Z = lh dh^T),
// dL/dE written, dL/dX accumulated, flagged tets to the list.
__global__ void __launch_bounds__(128) vjp_pass1_kernel(int32_t n, int64_t nt, const int32_t *__restrict__ tets,
                                                        const double *__restrict__ Xr, const double *__restrict__ xc,
                                                        const double *__restrict__ E, double nu,
                                                        const double *__restrict__ lam_f, const double *__restrict__ dx,
                                                        double *__restrict__ dL_dE, double *dL_dX,
                                                        EigStore es, uint32_t *status)
{
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nt; e += (int64_t)gridDim.x * blockDim.x) {
        int vid[4];
        double X[4][3], x[4][3];
        bool parked = false;
        if (!load_tet(tets, e, n, Xr, xc, vid, X, x)) {
            set_status(status, ST_BAD_INDEX);
            dL_dE[e] = 0.0;
        } else {
            double lh[3][3], dh[3][3];
            load_pair(vid, lam_f, dx, lh, dh);
            const double Ee = E[e];
            double mu, lam;
            lame(Ee, nu, mu, lam);
            Tet t;
            tet_eval(X, x, mu, lam, t);
            double Xb[4][3] = {};
            ZAcc za;
            zacc_init(za);
            zacc_rank1(ZGeomRegs{t}, mu, lam, lh, dh, za);   // Z = lh dh^T (D = 1)
            const double psi = reverse_phi(t, mu, lam, lh, true, za, Xb);
            dL_dE[e] = -t.V * psi / Ee;
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
                for (int c = 0; c < 3; ++c) atomicAdd(dL_dX + 3 * (int64_t)vid[a] + c, -Xb[a][c]);
            float A32[45];
            reduced_m32(t, mu, lam, A32);
            store_m32(es, e, A32, true);
            parked = true;
        }
        if (!parked) {
            float z[45] = {};
            store_m32(es, e, z, false);
        }
    }
}

// (D - 1)_ij, D the divided differences of max(., 0): 0 when both
// eigenvalues are positive, -1 when neither is, and min/(max - min)
// otherwise.  Selects only (no divergent branches).
__device__ __forceinline__ double dd_minus_one(double li, double lj)
{
    const bool pi = li > 0.0, pj = lj > 0.0;
    const double lo = fmin(li, lj), hi = fmax(li, lj);
    const double mixed = lo / (hi - lo);
    return pi == pj ? (pi ? 0.0 : -1.0) : mixed;
}

// VJP pass 2, flagged tets only: the clamp's correction Z = U ((D - 1) o
// (a b^T)) U^T in the refined eigenbasis (every pair rotated).
__global__ void __launch_bounds__(kRefineThreads) vjp_pass2_kernel(
    int32_t n, const int32_t *__restrict__ tets, const double *__restrict__ Xr, const double *__restrict__ xc,
    const double *__restrict__ E, double nu, const double *__restrict__ lam_f, const double *__restrict__ dx,
    double *__restrict__ dL_dE, double *dL_dX, const int32_t *__restrict__ hdr,
    const int32_t *__restrict__ list, int64_t cap, EigStore es)
{
    __shared__ double sm[kRefineSlots * kRefineThreads];
    const Slots sl{sm, (int)threadIdx.x};
    const int64_t cnt = min64(flagged_total(hdr), cap);
    for (int64_t i = blockIdx.x * (int64_t)kRefineThreads + threadIdx.x; i < cnt;
         i += (int64_t)gridDim.x * kRefineThreads) {
        const int64_t e = list[i];
        int vid[4];
        double X[4][3], x[4][3];
        if (!load_tet(tets, e, n, Xr, xc, vid, X, x)) continue;
        double lh[3][3], dh[3][3];
        load_pair(vid, lam_f, dx, lh, dh);
        const double Ee = E[e];
        double mu, lam;
        lame(Ee, nu, mu, lam);
        // the eigen step and the Z sums keep only the invariants they read;
        // the reverse pass recomputes the element (fewer live registers)
        ZGeomShared zg{{}, sl, 108};
        double om6[6], ff6[6];
        {
            Tet t;
            tet_eval(X, x, mu, lam, t);
#pragma unroll
            for (int i = 0; i < 3; ++i)
#pragma unroll
                for (int j = 0; j < 3; ++j) {
                    zg.Yr[i][j] = t.Y[i][j];
                    if (i <= j) {
                        om6[sym3(i, j)] = t.om[i][j];
                        ff6[sym3(i, j)] = t.FFt[i][j];
                    }
                }
            refine64(t, mu, lam, sl, true, es, e);
        }
        // eigenvalues (A's diagonal), a = U^T lh and b = U^T dh, then into
        // slots 81..107 and om, FFt into 108..119 once every diagonal entry of
        // A has been read (A is not needed after that)
        {
            double L[9], av[9], bv[9];
#pragma unroll
            for (int j = 0; j < 9; ++j) {
                L[j] = sl.a(j, j);
                double sa = 0.0, sb = 0.0;
#pragma unroll
                for (int r = 0; r < 9; ++r) {
                    sa += sl.u(r, j) * lh[r / 3][r % 3];
                    sb += sl.u(r, j) * dh[r / 3][r % 3];
                }
                av[j] = sa;
                bv[j] = sb;
            }
#pragma unroll
            for (int j = 0; j < 9; ++j) {
                sl.raw(81 + j) = L[j];
                sl.raw(90 + j) = av[j];
                sl.raw(99 + j) = bv[j];
            }
#pragma unroll
            for (int k = 0; k < 6; ++k) {
                sl.raw(108 + k) = om6[k];
                sl.raw(114 + k) = ff6[k];
            }
        }
        // Z = U C U^T with C = (D - 1) o (a b^T), nonzero only in the rows
        // and columns of the eigenvalues <= 0 (set N): Z is the sum over
        // i in N of u_i v_i^T + w_i u_i^T, v_i = sum_j C_ij u_j and
        // w_i = sum_{k not in N} C_ki u_k
        ZAcc za;
        zacc_init(za);
#pragma unroll 1
        for (int i2 = 0; i2 < 9; ++i2) {
            const double li = sl.raw(81 + i2);
            if (li > 0.0) continue;
            const double ai = sl.raw(90 + i2), bi = sl.raw(99 + i2);
            double P[3][3], Q[3][3];
#pragma unroll
            for (int r = 0; r < 9; ++r) {
                P[r / 3][r % 3] = sl.u(r, i2);
                Q[r / 3][r % 3] = 0.0;
            }
#pragma unroll 1
            for (int j = 0; j < 9; ++j) {
                const double cj = ai * dd_minus_one(li, sl.raw(81 + j)) * sl.raw(99 + j);
#pragma unroll
                for (int r = 0; r < 9; ++r) Q[r / 3][r % 3] += cj * sl.u(r, j);
            }
            zacc_rank1(zg, mu, lam, P, Q, za);
            double W[3][3];
#pragma unroll
            for (int r = 0; r < 9; ++r) W[r / 3][r % 3] = 0.0;
#pragma unroll 1
            for (int k = 0; k < 9; ++k) {
                const double lk = sl.raw(81 + k);
                const double ck = lk > 0.0 ? dd_minus_one(lk, li) * sl.raw(90 + k) * bi : 0.0;
#pragma unroll
                for (int r = 0; r < 9; ++r) W[r / 3][r % 3] += ck * sl.u(r, k);
            }
            zacc_rank1(zg, mu, lam, W, P, za);
        }
        // the element again, from fresh loads (so that X and x need not stay
        // live through the Z sums)
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                X[a][c] = ld_fresh(Xr + 3 * (int64_t)vid[a] + c);
                x[a][c] = ld_fresh(xc + 3 * (int64_t)vid[a] + c);
            }
        Tet t;
        tet_eval(X, x, mu, lam, t);
        double Xb[4][3] = {};
        const double psi = reverse_phi(t, mu, lam, lh, false, za, Xb);
        dL_dE[e] -= t.V * psi / Ee;
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int c = 0; c < 3; ++c) atomicAdd(dL_dX + 3 * (int64_t)vid[a] + c, -Xb[a][c]);
    }
}

__global__ void vjp_init_kernel(int32_t n, const double *__restrict__ lam_f, const double *__restrict__ mass_h2,
                                double *__restrict__ dL_dX)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < 3 * (int64_t)n;
         i += (int64_t)gridDim.x * blockDim.x)
        dL_dX[i] = mass_h2 ? lam_f[i] * mass_h2[i / 3] : 0.0;
}

__global__ void restrict_kernel(int32_t n, const int32_t *__restrict__ labels, const int32_t *__restrict__ n_c_dev,
                                const double *__restrict__ v, double *v_c, uint32_t *status)
{
    const int32_t nc = *n_c_dev;
    if (nc < 0 || nc > n) {
        if (blockIdx.x == 0 && threadIdx.x == 0) set_status(status, ST_BAD_INDEX);
        return;
    }
    for (int64_t f = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; f < n; f += (int64_t)gridDim.x * blockDim.x) {
        const int32_t c = labels[f];
        if ((unsigned)c >= (unsigned)nc) {
            set_status(status, ST_BAD_INDEX);
            continue;
        }
        atomicAdd(v_c + 3 * (int64_t)c, v[3 * f]);
        atomicAdd(v_c + 3 * (int64_t)c + 1, v[3 * f + 1]);
        atomicAdd(v_c + 3 * (int64_t)c + 2, v[3 * f + 2]);
    }
}

// Green-strain-increment tagging (Sec. 4.2, Eq. 3): every edge starts
// collapsible; a tet whose ||G(x_cur) - G(x_prev)||_F exceeds the threshold
// protects its 6 edges.  Edge k is the k-th off-diagonal block of the fine
// upper structure (diagonal first in each row, edges sorted), so the index
// of edge (u, v), u < v, is its block position minus u + 1.
__global__ void tags_init_kernel(int64_t ne, uint8_t *__restrict__ tags)
{
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < ne; k += (int64_t)gridDim.x * blockDim.x)
        tags[k] = 1;
}

__device__ __forceinline__ void green(const double W[3][3], const double x[4][3], double G[3][3])
{
    double F[3][3];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            double v = 0.0;
#pragma unroll
            for (int k = 0; k < 3; ++k) v += (x[k + 1][i] - x[0][i]) * W[k][j];
            F[i][j] = v;
        }
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            const double v = F[0][i] * F[0][j] + F[1][i] * F[1][j] + F[2][i] * F[2][j];
            G[i][j] = 0.5 * (i == j ? v - 1.0 : v);
        }
}

__global__ void strain_tag_kernel(int32_t n, int64_t nt, const int32_t *__restrict__ tets,
                                  const int32_t *__restrict__ row_ptr, const int32_t *__restrict__ col, int64_t nnzb,
                                  int64_t n_edges, const double *__restrict__ Xr, const double *__restrict__ xp,
                                  const double *__restrict__ xc, double thr2, uint8_t *tags, uint32_t *status)
{
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nt; e += (int64_t)gridDim.x * blockDim.x) {
        int vid[4];
        double X[4][3], x1[4][3], x0[4][3];
        if (!load_tet(tets, e, n, Xr, xc, vid, X, x1)) {
            set_status(status, ST_BAD_INDEX);
            continue;
        }
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int c = 0; c < 3; ++c) x0[a][c] = xp[3 * (int64_t)vid[a] + c];
        // Dm^-1 by cofactors
        double Dm[3][3], W[3][3];
#pragma unroll
        for (int c = 0; c < 3; ++c)
#pragma unroll
            for (int k = 0; k < 3; ++k) Dm[c][k] = X[k + 1][c] - X[0][c];
        const double c00 = Dm[1][1] * Dm[2][2] - Dm[1][2] * Dm[2][1];
        const double c01 = Dm[1][2] * Dm[2][0] - Dm[1][0] * Dm[2][2];
        const double c02 = Dm[1][0] * Dm[2][1] - Dm[1][1] * Dm[2][0];
        const double id = 1.0 / (Dm[0][0] * c00 + Dm[0][1] * c01 + Dm[0][2] * c02);
        W[0][0] = c00 * id;
        W[0][1] = (Dm[0][2] * Dm[2][1] - Dm[0][1] * Dm[2][2]) * id;
        W[0][2] = (Dm[0][1] * Dm[1][2] - Dm[0][2] * Dm[1][1]) * id;
        W[1][0] = c01 * id;
        W[1][1] = (Dm[0][0] * Dm[2][2] - Dm[0][2] * Dm[2][0]) * id;
        W[1][2] = (Dm[0][2] * Dm[1][0] - Dm[0][0] * Dm[1][2]) * id;
        W[2][0] = c02 * id;
        W[2][1] = (Dm[0][1] * Dm[2][0] - Dm[0][0] * Dm[2][1]) * id;
        W[2][2] = (Dm[0][0] * Dm[1][1] - Dm[0][1] * Dm[1][0]) * id;
        double G1[3][3], G0[3][3];
        green(W, x1, G1);
        green(W, x0, G0);
        double d2 = 0.0;
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
            for (int j = 0; j < 3; ++j) {
                const double d = G1[i][j] - G0[i][j];
                d2 += d * d;
            }
        if (!(d2 > thr2)) continue;
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int b = a + 1; b < 4; ++b) {
                const int32_t lo = min(vid[a], vid[b]), hi = max(vid[a], vid[b]);
                const int64_t pos = lo == hi ? -1 : find_block(row_ptr, col, nnzb, lo, hi);
                const int64_t k = pos - (int64_t)lo - 1;
                if (pos < 0 || k < 0 || k >= n_edges) {
                    set_status(status, ST_BAD_INDEX);
                    continue;
                }
                tags[k] = 0;
            }
    }
}

// Workspace: kHdr header words, the list (n_tets words), the count bytes
// (n_tets bytes), then the eigenpair records (kEigRec floats per tet) from a
// 16-byte boundary.
int64_t eig_offset_words(int64_t n_tets) { return div_up(kHdr + n_tets + div_up(n_tets, 4), 4) * 4; }
int64_t workspace_words(int64_t n_tets) { return eig_offset_words(n_tets) + kEigRec * n_tets; }

}  // namespace

extern "C" int64_t agipc_stvk_workspace_bytes(int64_t n_tets)
{
    if (n_tets < 0) return -1;
    return 4 * workspace_words(n_tets);
}

extern "C" int agipc_fine_assemble_stvk(agipc_ctx *ctx, int32_t n_fine, int64_t n_tets, const int32_t *tets,
                                        const double *X_rest, const double *x, const double *xhat_shift,
                                        const double *E, double nu, const double *mass_h2, const double *g_extra,
                                        const int32_t *fine_row_ptr, const int32_t *fine_col, int64_t fine_nnzb,
                                        double *fine_val, double *g, void *workspace, int64_t workspace_bytes)
{
    if (!ctx || n_fine <= 0 || n_fine > ctx->max_n || n_tets < 0 || n_tets > INT32_MAX || fine_nnzb < n_fine ||
        fine_nnzb > ctx->max_fine_nnzb || !X_rest || !x || !xhat_shift || !mass_h2 || !fine_row_ptr || !fine_col ||
        !fine_val || !g || (n_tets > 0 && (!tets || !E)) || !(nu > -1.0 && nu < 0.5) || !workspace ||
        workspace_bytes < 4 * workspace_words(n_tets) || (reinterpret_cast<uintptr_t>(workspace) & 127))
        return AGIPC_ERR_INVALID_ARG;
    cudaStream_t st = ctx->stream;
    int32_t *ws = static_cast<int32_t *>(workspace);
    Shift3 shift{{xhat_shift[0], xhat_shift[1], xhat_shift[2]}};
    const int tb = 256;
    fine_init_kernel<<<(unsigned)div_up(n_fine, tb), tb, 0, st>>>(n_fine, fine_row_ptr, fine_col, fine_nnzb, mass_h2,
                                                                  x, X_rest, shift, g_extra, fine_val, g, ctx->status);
    if (n_tets > 0) {
        int32_t *list = ws + kHdr;
        uint8_t *mcode = reinterpret_cast<uint8_t *>(list + n_tets);
        if (cudaMemsetAsync(ws, 0, kHdr * sizeof(int32_t), st) != cudaSuccess) return AGIPC_ERR_CUDA;
        const EigStore es{reinterpret_cast<float *>(ws + eig_offset_words(n_tets)), n_tets};
        elem_pass1_kernel<<<(unsigned)min64(div_up(n_tets, 128), (int64_t)ctx->num_sms * 16), 128, 0, st>>>(
            n_fine, n_tets, tets, fine_row_ptr, fine_col, fine_nnzb, X_rest, x, E, nu, fine_val, g, es, ctx->status);
        classify_kernel<<<(unsigned)min64(div_up(n_tets, 128), (int64_t)ctx->num_sms * 16), 128, 0, st>>>(
            n_tets, es, ws, mcode);
        bucket_scatter_kernel<<<(unsigned)min64(div_up(n_tets, 256), (int64_t)ctx->num_sms * 8), 256, 0, st>>>(
            n_tets, mcode, ws, list);
        elem_pass2_kernel<<<(unsigned)min64(div_up(n_tets, kRefineThreads), (int64_t)ctx->num_sms * 7),
                            kRefineThreads, 0, st>>>(n_fine, tets, fine_row_ptr, fine_col, fine_nnzb, X_rest, x, E,
                                                     nu, fine_val, ws, list, n_tets, es, ctx->status);
    }
    return cudaPeekAtLastError() == cudaSuccess ? AGIPC_OK : AGIPC_ERR_CUDA;
}

extern "C" int agipc_stvk_vjp(agipc_ctx *ctx, int32_t n_fine, int64_t n_tets, const int32_t *tets,
                              const double *X_rest, const double *x, const double *E, double nu,
                              const double *mass_h2, const double *lam, const double *dx, double *dL_dE,
                              double *dL_dX_rest, void *workspace, int64_t workspace_bytes)
{
    if (!ctx || n_fine <= 0 || n_fine > ctx->max_n || n_tets < 0 || n_tets > INT32_MAX || !X_rest || !x || !lam ||
        !dx || !dL_dX_rest || (n_tets > 0 && (!tets || !E || !dL_dE)) || !(nu > -1.0 && nu < 0.5) || !workspace ||
        workspace_bytes < 4 * workspace_words(n_tets) || (reinterpret_cast<uintptr_t>(workspace) & 127))
        return AGIPC_ERR_INVALID_ARG;
    cudaStream_t st = ctx->stream;
    int32_t *ws = static_cast<int32_t *>(workspace);
    const int tb = 256;
    vjp_init_kernel<<<(unsigned)div_up(3 * (int64_t)n_fine, tb), tb, 0, st>>>(n_fine, lam, mass_h2, dL_dX_rest);
    if (n_tets > 0) {
        int32_t *list = ws + kHdr;
        uint8_t *mcode = reinterpret_cast<uint8_t *>(list + n_tets);
        if (cudaMemsetAsync(ws, 0, kHdr * sizeof(int32_t), st) != cudaSuccess) return AGIPC_ERR_CUDA;
        const EigStore es{reinterpret_cast<float *>(ws + eig_offset_words(n_tets)), n_tets};
        vjp_pass1_kernel<<<(unsigned)min64(div_up(n_tets, 128), (int64_t)ctx->num_sms * 16), 128, 0, st>>>(
            n_fine, n_tets, tets, X_rest, x, E, nu, lam, dx, dL_dE, dL_dX_rest, es, ctx->status);
        classify_kernel<<<(unsigned)min64(div_up(n_tets, 128), (int64_t)ctx->num_sms * 16), 128, 0, st>>>(
            n_tets, es, ws, mcode);
        bucket_scatter_kernel<<<(unsigned)min64(div_up(n_tets, 256), (int64_t)ctx->num_sms * 8), 256, 0, st>>>(
            n_tets, mcode, ws, list);
        vjp_pass2_kernel<<<(unsigned)min64(div_up(n_tets, kRefineThreads), (int64_t)ctx->num_sms * 7),
                           kRefineThreads, 0, st>>>(n_fine, tets, X_rest, x, E, nu, lam, dx, dL_dE, dL_dX_rest, ws,
                                                    list, n_tets, es);
    }
    return cudaPeekAtLastError() == cudaSuccess ? AGIPC_OK : AGIPC_ERR_CUDA;
}

extern "C" int agipc_restrict(agipc_ctx *ctx, int32_t n_fine, const int32_t *labels, const int32_t *n_coarse_dev,
                              const double *v, double *v_c)
{
    if (!ctx || n_fine <= 0 || n_fine > ctx->max_n || !labels || !n_coarse_dev || !v || !v_c)
        return AGIPC_ERR_INVALID_ARG;
    cudaStream_t st = ctx->stream;
    // v_c is sized for n_fine rows (n_c <= n_fine); the rows past n_c are
    // zeroed too, so the whole buffer is defined.
    if (cudaMemsetAsync(v_c, 0, 3 * sizeof(double) * (size_t)n_fine, st) != cudaSuccess) return AGIPC_ERR_CUDA;
    const int tb = 256;
    restrict_kernel<<<(unsigned)min64(div_up(n_fine, tb), (int64_t)ctx->num_sms * 32), tb, 0, st>>>(
        n_fine, labels, n_coarse_dev, v, v_c, ctx->status);
    return cudaPeekAtLastError() == cudaSuccess ? AGIPC_OK : AGIPC_ERR_CUDA;
}

extern "C" int agipc_strain_tags(agipc_ctx *ctx, int32_t n_fine, int64_t n_tets, const int32_t *tets,
                                 const double *X_rest, const double *x_prev, const double *x_cur, double threshold,
                                 const int32_t *fine_row_ptr, const int32_t *fine_col, int64_t fine_nnzb,
                                 int64_t n_edges, uint8_t *tags)
{
    if (!ctx || n_fine <= 0 || n_fine > ctx->max_n || n_tets < 0 || n_edges < 0 || fine_nnzb < n_fine ||
        !X_rest || !x_prev || !x_cur || !fine_row_ptr || !fine_col || (n_edges > 0 && !tags) ||
        (n_tets > 0 && !tets) || !(threshold >= 0.0))
        return AGIPC_ERR_INVALID_ARG;
    cudaStream_t st = ctx->stream;
    const int tb = 256;
    if (n_edges > 0)
        tags_init_kernel<<<(unsigned)min64(div_up(n_edges, tb), (int64_t)ctx->num_sms * 32), tb, 0, st>>>(n_edges,
                                                                                                     tags);
    if (n_tets > 0)
        strain_tag_kernel<<<(unsigned)min64(div_up(n_tets, tb), (int64_t)ctx->num_sms * 32), tb, 0, st>>>(
            n_fine, n_tets, tets, fine_row_ptr, fine_col, fine_nnzb, n_edges, X_rest, x_prev, x_cur,
            threshold * threshold, tags, ctx->status);
    return cudaPeekAtLastError() == cudaSuccess ? AGIPC_OK : AGIPC_ERR_CUDA;
}
