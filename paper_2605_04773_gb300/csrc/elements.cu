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
//       is dL/dtheta = -lambda^T (dg/dtheta + dH/dtheta dx).  For the
//       per-element Young's modulus E_e (Psi_e is linear in E_e at fixed nu
//       and the eigenvalue clamp commutes with positive scaling) this is
//       -lambda_e^T (g_e + H_e dx_e) / E_e.  For the rest positions it is the
//       derivative of phi_e(X) = lambda_e^T g_e(X) + lambda_e^T H_e+(X) dx_e,
//       where the clamp H+ = V max(L,0) V^T is differentiated through the
//       eigendecomposition: lambda^T dH+ dx = <dH, V (F o (a b^T)) V^T> with
//       a = V^T lambda, b = V^T dx and F the divided differences of
//       max(.,0) over the eigenvalues; dH and dg come from forward-mode dual
//       numbers, one pass per rest coordinate.  The inertia term M/h^2 (x -
//       x_hat), x_hat = X_rest + h^2 gravity, adds lambda M/h^2 per vertex.
//
// Element formulas (independent of the input generator, same physics):
//   F = Ds Dm^-1, G = (F^T F - I)/2, S = 2 mu G + lam tr(G) I, P = F S,
//   g[a,c] = V sum_j P[c][j] w[a][j], with w the shape-function gradients
//   (rows of Dm^-1, w_0 = -sum), and
//   H[a,c][b,d] = V (delta_cd w_a.S w_b + mu Y_b[c] Y_a[d] + mu (F F^T)_cd
//                 w_a.w_b + lam Y_a[c] Y_b[d]),  Y_a = F w_a.
// The 12x12 eigendecomposition is the cyclic Jacobi method (rotation
// angles by the Rutishauser formulas, Golub & Van Loan, Matrix
// Computations, Sec. 8.5), run in FP64 by one thread per tet.
#include <math.h>

#include "agipc_common.cuh"

namespace {

struct Dual {
    double v, d;
};
__device__ __forceinline__ Dual operator+(Dual a, Dual b) { return {a.v + b.v, a.d + b.d}; }
__device__ __forceinline__ Dual operator-(Dual a, Dual b) { return {a.v - b.v, a.d - b.d}; }
__device__ __forceinline__ Dual operator-(Dual a) { return {-a.v, -a.d}; }
__device__ __forceinline__ Dual operator*(Dual a, Dual b) { return {a.v * b.v, a.v * b.d + a.d * b.v}; }
__device__ __forceinline__ Dual operator*(double s, Dual a) { return {s * a.v, s * a.d}; }
__device__ __forceinline__ Dual operator*(Dual a, double s) { return {s * a.v, s * a.d}; }
__device__ __forceinline__ Dual operator-(Dual a, double s) { return {a.v - s, a.d}; }
__device__ __forceinline__ Dual operator/(Dual a, Dual b)
{
    const double q = a.v / b.v;
    return {q, (a.d - q * b.d) / b.v};
}
__device__ __forceinline__ double val(double a) { return a; }
__device__ __forceinline__ double val(Dual a) { return a.v; }
template <class S>
__device__ __forceinline__ S sabs(S a)
{
    return val(a) < 0.0 ? -a : a;
}

// StVK gradient g[12] and (unprojected, symmetric) Hessian H[12][12] of one
// tet, for rest positions X[4][3] (scalar type S) and positions x[4][3].
template <class S>
__device__ void stvk_tet(const S X[4][3], const double x[4][3], double mu, double lam, S g[12], S H[12][12])
{
    S Dm[3][3];
    double Ds[3][3];
#pragma unroll
    for (int c = 0; c < 3; ++c)
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            Dm[c][k] = X[k + 1][c] - X[0][c];
            Ds[c][k] = x[k + 1][c] - x[0][c];
        }
    const S c00 = Dm[1][1] * Dm[2][2] - Dm[1][2] * Dm[2][1];
    const S c01 = Dm[1][2] * Dm[2][0] - Dm[1][0] * Dm[2][2];
    const S c02 = Dm[1][0] * Dm[2][1] - Dm[1][1] * Dm[2][0];
    const S det = Dm[0][0] * c00 + Dm[0][1] * c01 + Dm[0][2] * c02;
    S inv[3][3];
    inv[0][0] = c00 / det;
    inv[0][1] = (Dm[0][2] * Dm[2][1] - Dm[0][1] * Dm[2][2]) / det;
    inv[0][2] = (Dm[0][1] * Dm[1][2] - Dm[0][2] * Dm[1][1]) / det;
    inv[1][0] = c01 / det;
    inv[1][1] = (Dm[0][0] * Dm[2][2] - Dm[0][2] * Dm[2][0]) / det;
    inv[1][2] = (Dm[0][2] * Dm[1][0] - Dm[0][0] * Dm[1][2]) / det;
    inv[2][0] = c02 / det;
    inv[2][1] = (Dm[0][1] * Dm[2][0] - Dm[0][0] * Dm[2][1]) / det;
    inv[2][2] = (Dm[0][0] * Dm[1][1] - Dm[0][1] * Dm[1][0]) / det;
    const S vol = sabs(det) * (1.0 / 6.0);
    S w[4][3];
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        w[1][j] = inv[0][j];
        w[2][j] = inv[1][j];
        w[3][j] = inv[2][j];
        w[0][j] = -(inv[0][j] + inv[1][j] + inv[2][j]);
    }
    S F[3][3];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) F[i][j] = Ds[i][0] * inv[0][j] + Ds[i][1] * inv[1][j] + Ds[i][2] * inv[2][j];
    S Gm[3][3];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            S t = F[0][i] * F[0][j] + F[1][i] * F[1][j] + F[2][i] * F[2][j];
            Gm[i][j] = 0.5 * (i == j ? t - 1.0 : t);
        }
    const S trG = Gm[0][0] + Gm[1][1] + Gm[2][2];
    S Sm[3][3];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) Sm[i][j] = (2.0 * mu) * Gm[i][j] + (i == j ? lam * trG : 0.0 * trG);
    S P[3][3];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) P[i][j] = F[i][0] * Sm[0][j] + F[i][1] * Sm[1][j] + F[i][2] * Sm[2][j];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int c = 0; c < 3; ++c) g[3 * a + c] = vol * (P[c][0] * w[a][0] + P[c][1] * w[a][1] + P[c][2] * w[a][2]);
    S FFt[3][3], Y[4][3], Sw[4][3];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int k = 0; k < 3; ++k) FFt[i][k] = F[i][0] * F[k][0] + F[i][1] * F[k][1] + F[i][2] * F[k][2];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            Y[a][c] = F[c][0] * w[a][0] + F[c][1] * w[a][1] + F[c][2] * w[a][2];
            Sw[a][c] = Sm[c][0] * w[a][0] + Sm[c][1] * w[a][1] + Sm[c][2] * w[a][2];
        }
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            const S wSw = w[a][0] * Sw[b][0] + w[a][1] * Sw[b][1] + w[a][2] * Sw[b][2];
            const S ww = w[a][0] * w[b][0] + w[a][1] * w[b][1] + w[a][2] * w[b][2];
#pragma unroll
            for (int c = 0; c < 3; ++c)
#pragma unroll
                for (int d = 0; d < 3; ++d) {
                    S h = mu * (Y[b][c] * Y[a][d]) + mu * (FFt[c][d] * ww) + lam * (Y[a][c] * Y[b][d]);
                    if (c == d) h = h + wSw;
                    H[3 * a + c][3 * b + d] = vol * h;
                }
        }
}

// Cyclic Jacobi eigendecomposition of a symmetric 12x12 matrix: A is
// overwritten (its diagonal ends up holding the eigenvalues), V collects the
// eigenvectors as columns.
__device__ void jacobi12(double A[12][12], double V[12][12])
{
    for (int i = 0; i < 12; ++i)
        for (int j = 0; j < 12; ++j) V[i][j] = i == j ? 1.0 : 0.0;
    double scale = 0.0;
    for (int i = 0; i < 12; ++i) scale = fmax(scale, fabs(A[i][i]));
    for (int sweep = 0; sweep < 20; ++sweep) {
        double off = 0.0;
        for (int p = 0; p < 12; ++p)
            for (int q = p + 1; q < 12; ++q) off = fmax(off, fabs(A[p][q]));
        if (off <= 1e-15 * scale || off == 0.0) break;
        for (int p = 0; p < 11; ++p)
            for (int q = p + 1; q < 12; ++q) {
                const double apq = A[p][q];
                if (fabs(apq) <= 1e-300) continue;
                const double theta = (A[q][q] - A[p][p]) / (2.0 * apq);
                const double t = (theta >= 0.0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
                const double c = 1.0 / sqrt(t * t + 1.0);
                const double s = t * c;
                const double tau = s / (1.0 + c);
                A[p][p] -= t * apq;
                A[q][q] += t * apq;
                A[p][q] = A[q][p] = 0.0;
                for (int k = 0; k < 12; ++k) {
                    if (k != p && k != q) {
                        const double akp = A[k][p], akq = A[k][q];
                        const double np = akp - s * (akq + tau * akp);
                        const double nq = akq + s * (akp - tau * akq);
                        A[k][p] = A[p][k] = np;
                        A[k][q] = A[q][k] = nq;
                    }
                    const double vkp = V[k][p], vkq = V[k][q];
                    V[k][p] = vkp - s * (vkq + tau * vkp);
                    V[k][q] = vkq + s * (vkp - tau * vkq);
                }
            }
    }
}

__device__ __forceinline__ void lame(double E, double nu, double &mu, double &lam)
{
    mu = E / (2.0 * (1.0 + nu));
    lam = E * nu / ((1.0 + nu) * (1.0 - 2.0 * nu));
}

__device__ __forceinline__ void load_tet(const int32_t *tets, int64_t e, int32_t n, const double *Xr, const double *xc,
                                         int vid[4], double X[4][3], double x[4][3], bool &ok)
{
    ok = true;
#pragma unroll
    for (int a = 0; a < 4; ++a) {
        vid[a] = tets[4 * e + a];
        if ((unsigned)vid[a] >= (unsigned)n) ok = false;
    }
    if (!ok) return;
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            X[a][c] = Xr[3 * (int64_t)vid[a] + c];
            x[a][c] = xc[3 * (int64_t)vid[a] + c];
        }
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

__constant__ int kPairS[10] = {0, 0, 0, 0, 1, 1, 1, 2, 2, 3};
__constant__ int kPairT[10] = {0, 1, 2, 3, 1, 2, 3, 2, 3, 3};

__global__ void __launch_bounds__(128) elem_assemble_kernel(int32_t n, int64_t nt, const int32_t *__restrict__ tets,
                                                            const int32_t *__restrict__ row_ptr,
                                                            const int32_t *__restrict__ col, int64_t nnzb,
                                                            const double *__restrict__ Xr, const double *__restrict__ xc,
                                                            const double *__restrict__ E, double nu, double *fine_val,
                                                            double *g, uint32_t *status)
{
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nt; e += (int64_t)gridDim.x * blockDim.x) {
        int vid[4];
        double X[4][3], x[4][3];
        bool ok;
        load_tet(tets, e, n, Xr, xc, vid, X, x, ok);
        if (!ok) {
            set_status(status, ST_BAD_INDEX);
            continue;
        }
        double mu, lam;
        lame(E[e], nu, mu, lam);
        double ge[12], H[12][12], V[12][12];
        stvk_tet<double>(X, x, mu, lam, ge, H);
        bool finite = true;
        for (int r = 0; r < 12; ++r) finite = finite && isfinite(ge[r]);
        if (!finite) {
            set_status(status, ST_NONFINITE);
            continue;
        }
        // PSD projection: H+ = V max(L, 0) V^T
        jacobi12(H, V);
        double L[12];
        for (int k = 0; k < 12; ++k) L[k] = fmax(H[k][k], 0.0);
        for (int q = 0; q < 10; ++q) {
            const int sa = kPairS[q], sb = kPairT[q];
            const int32_t va = vid[sa], vb = vid[sb];
            if (sa != sb && va == vb) {
                set_status(status, ST_BAD_INDEX);
                continue;
            }
            const bool transpose = va > vb;
            const int64_t pos = find_block(row_ptr, col, nnzb, transpose ? vb : va, transpose ? va : vb);
            if (pos < 0) {
                set_status(status, ST_BAD_INDEX);
                continue;
            }
            double *dst = fine_val + 9 * pos;
            for (int c = 0; c < 3; ++c)
                for (int d = 0; d < 3; ++d) {
                    const int r = 3 * sa + c, s = 3 * sb + d;
                    double h = 0.0;
                    for (int k = 0; k < 12; ++k) h += V[r][k] * L[k] * V[s][k];
                    atomicAdd(dst + (transpose ? 3 * d + c : 3 * c + d), h);
                }
        }
        for (int a = 0; a < 4; ++a)
            for (int c = 0; c < 3; ++c) atomicAdd(g + 3 * (int64_t)vid[a] + c, ge[3 * a + c]);
    }
}

__global__ void __launch_bounds__(128) vjp_kernel(int32_t n, int64_t nt, const int32_t *__restrict__ tets,
                                                  const double *__restrict__ Xr, const double *__restrict__ xc,
                                                  const double *__restrict__ E, double nu,
                                                  const double *__restrict__ lam_f, const double *__restrict__ dx,
                                                  double *__restrict__ dL_dE, double *dL_dX, uint32_t *status)
{
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nt; e += (int64_t)gridDim.x * blockDim.x) {
        int vid[4];
        double X[4][3], x[4][3];
        bool ok;
        load_tet(tets, e, n, Xr, xc, vid, X, x, ok);
        if (!ok) {
            set_status(status, ST_BAD_INDEX);
            dL_dE[e] = 0.0;
            continue;
        }
        double lv[12], dv[12];
        for (int a = 0; a < 4; ++a)
            for (int c = 0; c < 3; ++c) {
                lv[3 * a + c] = lam_f[3 * (int64_t)vid[a] + c];
                dv[3 * a + c] = dx[3 * (int64_t)vid[a] + c];
            }
        const double Ee = E[e];
        double mu, lam;
        lame(Ee, nu, mu, lam);
        double ge[12], H[12][12], V[12][12];
        stvk_tet<double>(X, x, mu, lam, ge, H);
        jacobi12(H, V);
        double Lm[12], a_[12], b_[12];
        for (int k = 0; k < 12; ++k) {
            Lm[k] = H[k][k];
            double sa = 0.0, sb = 0.0;
            for (int r = 0; r < 12; ++r) {
                sa += V[r][k] * lv[r];
                sb += V[r][k] * dv[r];
            }
            a_[k] = sa;
            b_[k] = sb;
        }
        // dL/dE_e = -(lambda^T g + lambda^T H+ dx) / E
        double s = 0.0;
        for (int r = 0; r < 12; ++r) s += lv[r] * ge[r];
        for (int k = 0; k < 12; ++k) s += a_[k] * fmax(Lm[k], 0.0) * b_[k];
        dL_dE[e] = -s / Ee;
        // M = V (F o (a b^T)) V^T, F the divided differences of max(., 0)
        double Wk[12][12];
        for (int i = 0; i < 12; ++i)
            for (int j = 0; j < 12; ++j) {
                const double li = Lm[i], lj = Lm[j];
                double f;
                if (li > 0.0 && lj > 0.0) f = 1.0;
                else if (li <= 0.0 && lj <= 0.0) f = 0.0;
                else f = (fmax(li, 0.0) - fmax(lj, 0.0)) / (li - lj);
                Wk[i][j] = f * a_[i] * b_[j];
            }
        double M[12][12];
        for (int r = 0; r < 12; ++r) {
            double t[12];
            for (int j = 0; j < 12; ++j) {
                double acc = 0.0;
                for (int i = 0; i < 12; ++i) acc += V[r][i] * Wk[i][j];
                t[j] = acc;
            }
            for (int c = 0; c < 12; ++c) {
                double acc = 0.0;
                for (int j = 0; j < 12; ++j) acc += t[j] * V[c][j];
                M[r][c] = acc;
            }
        }
        // d/dX of lambda^T g(X) + <H(X), M>, one forward-mode pass per coordinate
        for (int a = 0; a < 4; ++a)
            for (int c = 0; c < 3; ++c) {
                Dual Xd[4][3];
                for (int p = 0; p < 4; ++p)
                    for (int q = 0; q < 3; ++q) Xd[p][q] = {X[p][q], (p == a && q == c) ? 1.0 : 0.0};
                Dual gd[12], Hd[12][12];
                stvk_tet<Dual>(Xd, x, mu, lam, gd, Hd);
                double phi = 0.0;
                for (int r = 0; r < 12; ++r) {
                    phi += lv[r] * gd[r].d;
                    for (int k = 0; k < 12; ++k) phi += M[r][k] * Hd[r][k].d;
                }
                atomicAdd(dL_dX + 3 * (int64_t)vid[a] + c, -phi);
            }
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

}  // namespace

extern "C" int agipc_fine_assemble_stvk(agipc_ctx *ctx, int32_t n_fine, int64_t n_tets, const int32_t *tets,
                                        const double *X_rest, const double *x, const double *xhat_shift,
                                        const double *E, double nu, const double *mass_h2, const double *g_extra,
                                        const int32_t *fine_row_ptr, const int32_t *fine_col, int64_t fine_nnzb,
                                        double *fine_val, double *g)
{
    if (!ctx || n_fine <= 0 || n_fine > ctx->max_n || n_tets < 0 || fine_nnzb < n_fine ||
        fine_nnzb > ctx->max_fine_nnzb || !X_rest || !x || !xhat_shift || !mass_h2 || !fine_row_ptr || !fine_col ||
        !fine_val || !g || (n_tets > 0 && (!tets || !E)) || !(nu > -1.0 && nu < 0.5))
        return AGIPC_ERR_INVALID_ARG;
    cudaStream_t st = ctx->stream;
    Shift3 shift{{xhat_shift[0], xhat_shift[1], xhat_shift[2]}};
    const int tb = 256;
    fine_init_kernel<<<(unsigned)div_up(n_fine, tb), tb, 0, st>>>(n_fine, fine_row_ptr, fine_col, fine_nnzb, mass_h2,
                                                                  x, X_rest, shift, g_extra, fine_val, g, ctx->status);
    if (n_tets > 0)
        elem_assemble_kernel<<<(unsigned)min64(div_up(n_tets, 128), (int64_t)ctx->num_sms * 16), 128, 0, st>>>(
            n_fine, n_tets, tets, fine_row_ptr, fine_col, fine_nnzb, X_rest, x, E, nu, fine_val, g, ctx->status);
    return cudaPeekAtLastError() == cudaSuccess ? AGIPC_OK : AGIPC_ERR_CUDA;
}

extern "C" int agipc_stvk_vjp(agipc_ctx *ctx, int32_t n_fine, int64_t n_tets, const int32_t *tets,
                              const double *X_rest, const double *x, const double *E, double nu,
                              const double *mass_h2, const double *lam, const double *dx, double *dL_dE,
                              double *dL_dX_rest)
{
    if (!ctx || n_fine <= 0 || n_fine > ctx->max_n || n_tets < 0 || !X_rest || !x || !lam || !dx || !dL_dX_rest ||
        (n_tets > 0 && (!tets || !E || !dL_dE)) || !(nu > -1.0 && nu < 0.5))
        return AGIPC_ERR_INVALID_ARG;
    cudaStream_t st = ctx->stream;
    const int tb = 256;
    vjp_init_kernel<<<(unsigned)div_up(3 * (int64_t)n_fine, tb), tb, 0, st>>>(n_fine, lam, mass_h2, dL_dX_rest);
    if (n_tets > 0)
        vjp_kernel<<<(unsigned)min64(div_up(n_tets, 128), (int64_t)ctx->num_sms * 16), 128, 0, st>>>(
            n_fine, n_tets, tets, X_rest, x, E, nu, lam, dx, dL_dE, dL_dX_rest, ctx->status);
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
