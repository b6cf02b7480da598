"""CPU FP64 oracle of the differentiation form: one coarsened Newton step as a
function of the per-element Young's modulus E and the rest positions X_rest,
and its adjoint gradient.

TEST INFRASTRUCTURE: only the test suite, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference leg of ``bench.py`` may import this module.

The step (Eq. 1 divided by dt^2, with the coarse solve of Sec. 4.1 and the
prolongation of Sec. 4.3):
    H = M/h^2 + sum_e H_e+   (H_e+ = PSD projection of the StVK element Hessian)
    g = M/h^2 (x - x_hat) + sum_e g_e,   x_hat = X_rest + h^2 gravity
    y = -(U H U^T)^-1 U g,  dx = U^T y,  x_next = x + dx
(U is the aggregation operator of the labels; labels are piecewise constant in
the parameters, so they carry no derivative.)  For a loss L(x_next) with
v = dL/dx_next, the adjoint is lambda_c = H_c^-1 U v, lambda = U^T lambda_c and
    dL/dtheta = -lambda^T (dg/dtheta + dH/dtheta dx).
Masses M are constants; the current positions x are data, not parameters.

The element routine below is written from the StVK definition of the inputs:
Psi_e = V_e (mu |G|_F^2 + lam/2 tr(G)^2), G = (F^T F - I)/2, F = Ds Dm^-1,
mu = E/(2(1+nu)), lam = E nu/((1+nu)(1-2nu)), V_e = |det Dm| / 6.  Gradient
and Hessian go through the 9x12 matrix B = dvec(F)/dx_e: g = V B^T vec(P) and
H = V B^T (dP/dF) B, with P = F S and S = 2 mu G + lam tr(G) I.  The PSD
projection clamps the eigenvalues of the 12x12 Hessian (numpy eigh) at zero.

dL/dE_e is the closed form (Psi_e is linear in E_e at fixed nu and the clamp
commutes with positive scaling): -lambda_e^T (g_e + H_e+ dx_e) / E_e.
dL/dX_rest is taken by central differences of the element routine (step eps,
with lambda and dx held fixed), plus the inertia term lambda M/h^2 that
x_hat = X_rest + const contributes.
"""
from __future__ import annotations

import numpy as np

from . import block_jacobi, coarse_gradient, galerkin, labels, pcg, prolongate

GRAVITY = np.array([0.0, 0.0, -9.81])


def lame(E, nu):
    E = np.asarray(E, dtype=np.float64)
    return E / (2.0 * (1.0 + nu)), E * nu / ((1.0 + nu) * (1.0 - 2.0 * nu))


def _shape_matrix(Xe):
    """Dm^-1, V and the 9x12 matrix B with vec(F) = B vec(x_e) (row-major
    vec: F index 3i+j, vertex coordinate index 3a+c)."""
    Xe = np.asarray(Xe, dtype=np.float64)
    Dm = np.stack([Xe[..., 1, :] - Xe[..., 0, :], Xe[..., 2, :] - Xe[..., 0, :], Xe[..., 3, :] - Xe[..., 0, :]],
                  axis=-1)
    W = np.linalg.inv(Dm)                      # W[k, j] = d(shape a=k+1)/dX_j
    V = np.abs(np.linalg.det(Dm)) / 6.0
    dN = np.concatenate([-W.sum(axis=-2, keepdims=True), W], axis=-2)   # [.., 4, 3]
    B = np.zeros(Xe.shape[:-2] + (9, 12))
    for i in range(3):
        for j in range(3):
            for a in range(4):
                B[..., 3 * i + j, 3 * a + i] = dN[..., a, j]
    return V, B


def stvk_element(Xe, xe, E, nu):
    """Energy, gradient [.., 12] and unprojected Hessian [.., 12, 12] of StVK
    tets (vectorised over the leading axes)."""
    V, B = _shape_matrix(Xe)
    mu, lam = lame(E, nu)
    mu = np.broadcast_to(mu, V.shape)
    lam = np.broadcast_to(lam, V.shape)
    xf = np.asarray(xe, dtype=np.float64).reshape(xe.shape[:-2] + (12,))
    F = np.einsum("...pk,...k->...p", B, xf).reshape(V.shape + (3, 3))
    I = np.eye(3)
    G = 0.5 * (np.einsum("...ki,...kj->...ij", F, F) - I)
    trG = np.trace(G, axis1=-2, axis2=-1)
    S = 2.0 * mu[..., None, None] * G + (lam * trG)[..., None, None] * I
    P = F @ S
    psi = V * (mu * np.sum(G * G, axis=(-2, -1)) + 0.5 * lam * trG ** 2)
    g = V[..., None] * np.einsum("...pk,...p->...k", B, P.reshape(V.shape + (9,)))
    # dP_ij/dF_kl = d_ik S_lj + mu F_il F_kj + mu (F F^T)_ik d_jl + lam F_ij F_kl
    FFt = F @ np.swapaxes(F, -1, -2)
    A = np.zeros(V.shape + (3, 3, 3, 3))
    for i in range(3):
        for j in range(3):
            for k in range(3):
                for l in range(3):
                    t = (S[..., l, j] if i == k else 0.0) + mu * F[..., i, l] * F[..., k, j] \
                        + (mu * FFt[..., i, k] if j == l else 0.0) + lam * F[..., i, j] * F[..., k, l]
                    A[..., i, j, k, l] = t
    A = A.reshape(V.shape + (9, 9))
    H = V[..., None, None] * np.einsum("...pk,...pq,...ql->...kl", B, A, B)
    return psi, g, H


def psd_project(H):
    """Clamp the eigenvalues of symmetric matrices at zero."""
    Hs = 0.5 * (H + np.swapaxes(H, -1, -2))
    lam_, Q = np.linalg.eigh(Hs)
    return np.einsum("...ik,...k,...jk->...ij", Q, np.maximum(lam_, 0.0), Q)


def element_terms(X_rest, x, tets, E, nu, chunk: int = 32768):
    """Per-tet gradient [nt, 12] and projected Hessian [nt, 12, 12]."""
    nt = tets.shape[0]
    g = np.empty((nt, 12))
    H = np.empty((nt, 12, 12))
    E = np.broadcast_to(np.asarray(E, dtype=np.float64), (nt,))
    for s in range(0, nt, chunk):
        t = tets[s:s + chunk]
        _, ge, He = stvk_element(X_rest[t], x[t], E[s:s + chunk], nu)
        g[s:s + chunk] = ge
        H[s:s + chunk] = psd_project(He)
    return g, H


def fine_upper(n, tets, row_ptr, col, Hel, mass_h2):
    """Sum the element Hessians and M/h^2 into the given upper BSR structure
    (column >= row): block (a, b) of tet e lands at (min, max) of its vertex
    pair, transposed when the pair is reversed.  Returns val [nnzb, 3, 3]."""
    val = np.zeros((col.size, 3, 3))

    def pos(r, c):
        lo, hi = row_ptr[r], row_ptr[r + 1]
        k = lo + np.searchsorted(col[lo:hi], c)
        if k >= hi or col[k] != c:
            raise ValueError("block (%d, %d) missing from the fine structure" % (r, c))
        return k

    for i in range(n):
        val[pos(i, i)] += mass_h2[i] * np.eye(3)
    for e in range(tets.shape[0]):
        for a in range(4):
            for b in range(4):
                va, vb = int(tets[e, a]), int(tets[e, b])
                if va > vb or (va == vb and a > b):
                    continue
                val[pos(va, vb)] += Hel[e, 3 * a:3 * a + 3, 3 * b:3 * b + 3]
    return val


def fine_upper_fast(n, tets, row_ptr, col, Hel, mass_h2):
    """Same sum as :func:`fine_upper`, vectorised with np.add.at (for the
    full-size cases)."""
    val = np.zeros((col.size, 9))
    rows = np.repeat(np.arange(n), np.diff(row_ptr))
    key = rows.astype(np.int64) * n + col
    diag = np.searchsorted(key, np.arange(n, dtype=np.int64) * (n + 1))
    val[diag, 0] += mass_h2
    val[diag, 4] += mass_h2
    val[diag, 8] += mass_h2
    for a in range(4):
        for b in range(4):
            va, vb = tets[:, a].astype(np.int64), tets[:, b].astype(np.int64)
            keep = (va < vb) | ((va == vb) & (a <= b))
            lo, hi = np.minimum(va, vb), np.maximum(va, vb)
            k = np.searchsorted(key, lo * n + hi)
            if np.any(key[k[keep]] != (lo * n + hi)[keep]):
                raise ValueError("element block missing from the fine structure")
            blk = Hel[:, 3 * a:3 * a + 3, 3 * b:3 * b + 3]
            blk = np.where((va <= vb)[:, None, None], blk, np.swapaxes(blk, 1, 2))
            np.add.at(val, k[keep], blk[keep].reshape(-1, 9))
    return val.reshape(-1, 3, 3)


def _scatter(n, tets, ge):
    out = np.zeros((n, 3))
    np.add.at(out, tets.reshape(-1), ge.reshape(-1, 3))
    return out


def forward(problem, E, X_rest, tol: float, max_iter: int = 100000, fast: bool = True, with_terms=False):
    """The coarsened step x_next(E, X_rest).

    problem: dict with n, tets, edges, tags, row_ptr, col, x, mass_h2, h, nu
    and optionally pair_idx/pair_blk/g_pairs (constant contact terms)."""
    n, tets, nu = problem["n"], problem["tets"], problem["nu"]
    x, mass_h2, h = problem["x"], problem["mass_h2"], problem["h"]
    ge, He = element_terms(X_rest, x, tets, E, nu)
    x_hat = X_rest + h * h * GRAVITY
    g = mass_h2[:, None] * (x - x_hat) + _scatter(n, tets, ge)
    if problem.get("g_pairs") is not None:
        g = g + problem["g_pairs"]
    val = (fine_upper_fast if fast else fine_upper)(n, tets, problem["row_ptr"], problem["col"], He, mass_h2)
    lab, nc = labels(n, problem["edges"], problem["tags"])
    pidx = problem.get("pair_idx", np.zeros((0, 4), np.int32))
    pblk = problem.get("pair_blk", np.zeros((0, 10, 3, 3)))
    crp, cci, cval = galerkin(lab, nc, problem["row_ptr"], problem["col"], val, pidx, pblk)
    dinv = block_jacobi(crp, cci, cval)
    gc = coarse_gradient(lab, nc, g)
    y, it, rr, conv = pcg(crp, cci, cval, dinv, -gc, tol, max_iter)
    dx = prolongate(lab, y)
    out = dict(x_next=x + dx, dx=dx, y=y, labels=lab, n_c=nc, coarse=(crp, cci, cval), dinv=dinv, g=g,
               fine_val=val, iters=it, relres=rr, converged=conv)
    if with_terms:
        out.update(elem_grad=ge, elem_hess=He)
    return out


def _phi(Xe, xe, E, nu, lam_e, dx_e):
    """lambda_e^T (g_e + H_e+ dx_e) for the elastic part of each tet."""
    _, g, H = stvk_element(Xe, xe, E, nu)
    Hp = psd_project(H)
    return np.einsum("...k,...k->...", lam_e, g) + np.einsum("...k,...kl,...l->...", lam_e, Hp, dx_e)


def vjp(problem, E, X_rest, lam, dx, eps: float = 1e-6, vertices=None, elements=None, terms=None):
    """Per-element vector-Jacobian product at a given adjoint lambda and step dx.

    dL_dE[e] = -lambda_e^T (g_e + H_e+ dx_e) / E_e (closed form).
    dL_dX[v] = lambda_v M_v/h^2 - sum over tets e around v of the central
    difference (step eps) of lambda_e^T (g_e + H_e+ dx_e) in X_rest[v].
    ``elements`` restricts dL_dE (others NaN), ``vertices`` restricts dL_dX
    (others NaN); ``terms`` = (g_e, H_e+) of all tets, if already known."""
    n, tets, nu = problem["n"], problem["tets"], problem["nu"]
    x, mass_h2 = problem["x"], problem["mass_h2"]
    nt = tets.shape[0]
    E = np.broadcast_to(np.asarray(E, dtype=np.float64), (nt,))
    lam_e = lam[tets].reshape(-1, 12)
    dx_e = dx[tets].reshape(-1, 12)
    dL_dE = np.full(nt, np.nan)
    sel_e = np.arange(nt) if elements is None else np.asarray(elements)
    if terms is None:
        ge, He = element_terms(X_rest, x, tets[sel_e], E[sel_e], nu)
    else:
        ge, He = terms[0][sel_e], terms[1][sel_e]
    dL_dE[sel_e] = -(np.einsum("ek,ek->e", lam_e[sel_e], ge)
                     + np.einsum("ek,ekl,el->e", lam_e[sel_e], He, dx_e[sel_e])) / E[sel_e]
    dL_dX = lam * mass_h2[:, None]
    if vertices is None:
        sel_t = np.arange(nt)
        mask = None
    else:
        mask = np.zeros(n, bool)
        mask[np.asarray(vertices)] = True
        sel_t = np.nonzero(mask[tets].any(1))[0]
    Xe = X_rest[tets[sel_t]]
    xe = x[tets[sel_t]]
    for a in range(4):
        for c in range(3):
            Xp = Xe.copy()
            Xm = Xe.copy()
            Xp[:, a, c] += eps
            Xm[:, a, c] -= eps
            d = (_phi(Xp, xe, E[sel_t], nu, lam_e[sel_t], dx_e[sel_t])
                 - _phi(Xm, xe, E[sel_t], nu, lam_e[sel_t], dx_e[sel_t])) / (2.0 * eps)
            np.add.at(dL_dX[:, c], tets[sel_t, a], -d)
    if mask is not None:
        dL_dX[~mask] = np.nan
    return dL_dE, dL_dX


def adjoint(problem, E, X_rest, fwd, v, tol: float, max_iter: int = 100000, eps: float = 1e-6,
            vertices=None, elements=None):
    """Gradients of L with v = dL/dx_next, given the forward result fwd:
    lambda_c = H_c^-1 U v, lambda = U^T lambda_c, then :func:`vjp`."""
    lab, nc = fwd["labels"], fwd["n_c"]
    crp, cci, cval = fwd["coarse"]
    vc = coarse_gradient(lab, nc, v)
    lam_c, it, rr, conv = pcg(crp, cci, cval, fwd["dinv"], vc, tol, max_iter)
    lam = prolongate(lab, lam_c)
    terms = None
    if "elem_grad" in fwd:
        terms = (fwd["elem_grad"], fwd["elem_hess"])
    dL_dE, dL_dX = vjp(problem, E, X_rest, lam, fwd["dx"], eps=eps, vertices=vertices, elements=elements,
                       terms=terms)
    return dict(lam=lam, lam_c=lam_c, dL_dE=dL_dE, dL_dX=dL_dX, iters=it, relres=rr, converged=conv)
