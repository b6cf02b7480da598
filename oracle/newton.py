"""CPU FP64 oracle of the coarsened Newton loop with backtracking line search
(the inner loop of Algorithm 1, Eq. 1-2 of Sec. 3, the tagging of Eq. 3,
the coarse solve of Sec. 4.1 and the post-coarsening of Sec. 4.3) on the
StVK problem without contact.

TEST INFRASTRUCTURE: only the test suite, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference leg of ``bench.py`` may import this module.

Energy (Eq. 1 divided by dt^2; no barrier or friction):
    E(x) = 1/2 (x - x_hat)^T (M/h^2) (x - x_hat) + Psi(x) + g_extra^T x,
    x_hat = X_rest + h^2 gravity,  Psi = sum_e V_e (mu |G|_F^2 + lam/2 tr(G)^2).
g_extra is a constant linear term (a non-uniform x_hat enters through it).
Its gradient and PSD-projected Hessian are the ones ``adjoint.forward``
assembles.

One Newton iteration, in the order of Algorithm 1:
    E_prev = E(x), x_prev = x
    g, H at x
    tags: an edge is protected when a tet touching it has
          |G(x) - G(x_before)|_F > threshold (Eq. 3), x_before the previous
          Newton iterate (at the first iteration: the positions x_last of the
          previous time step)
    labels -> H_c, g_c -> d_c = -H_c^-1 g_c (block-Jacobi PCG to tol)
    d = U^T d_c, then at most post_iters block-Jacobi PCG iterations on the
          fine system H d = -g started from that d (post-coarsening)
    alpha = 1; repeat x = x_prev + alpha d; alpha = alpha / 2 until
          E(x) < E_prev (no contact, so the feasible step is 1)
until |d|_inf / h <= eps_d.

Readings where the paper leaves a choice: the first iteration's previous
iterate is the last time step's positions; the line search gives up after
max_halvings + 1 trials, x stays at x_prev and the loop ends, converged when
|d|_inf / h <= eps_d (a step at rounding level cannot lower E), else
`stalled`.
"""
from __future__ import annotations

import numpy as np

from . import block_jacobi, coarse_gradient, galerkin, labels, pcg, prolongate
from .adjoint import GRAVITY, element_terms, fine_upper_fast, lame
from .tagging import strain_tags


def stvk_energy(Xe, xe, E, nu):
    """Psi_e of each tet [nt] (vectorised): V (mu |G|^2 + lam/2 tr(G)^2)."""
    Xe = np.asarray(Xe, dtype=np.float64)
    xe = np.asarray(xe, dtype=np.float64)
    Dm = np.stack([Xe[:, k + 1, :] - Xe[:, 0, :] for k in range(3)], axis=-1)
    Ds = np.stack([xe[:, k + 1, :] - xe[:, 0, :] for k in range(3)], axis=-1)
    F = Ds @ np.linalg.inv(Dm)
    G = 0.5 * (np.swapaxes(F, 1, 2) @ F - np.eye(3))
    mu, lam = lame(E, nu)
    tr = np.trace(G, axis1=1, axis2=2)
    V = np.abs(np.linalg.det(Dm)) / 6.0
    return V * (mu * np.sum(G * G, axis=(1, 2)) + 0.5 * lam * tr * tr)


def energy(problem, E, X_rest, x):
    """E(x) of the problem at positions x [n, 3]."""
    tets, h = problem["tets"], problem["h"]
    x_hat = np.asarray(X_rest) + h * h * GRAVITY
    r = np.asarray(x) - x_hat
    inertia = 0.5 * np.sum(problem["mass_h2"] * np.sum(r * r, axis=1))
    E = np.broadcast_to(np.asarray(E, dtype=np.float64), (tets.shape[0],))
    psi = 0.0
    for s in range(0, tets.shape[0], 65536):
        t = tets[s:s + 65536]
        psi += np.sum(stvk_energy(X_rest[t], x[t], E[s:s + 65536], problem["nu"]))
    lin = 0.0 if problem.get("g_extra") is None else float(np.sum(problem["g_extra"] * x))
    return inertia + psi + lin


def gradient_and_hessian(problem, E, X_rest, x):
    """g [n, 3] and the fine upper values [nnzb, 3, 3] of the PSD-projected
    Hessian at x (the fine system agipc_fine_assemble_stvk sums)."""
    n, tets, h = problem["n"], problem["tets"], problem["h"]
    ge, He = element_terms(X_rest, x, tets, E, problem["nu"])
    g = problem["mass_h2"][:, None] * (x - (X_rest + h * h * GRAVITY))
    np.add.at(g, tets.reshape(-1), ge.reshape(-1, 3))
    if problem.get("g_extra") is not None:
        g = g + problem["g_extra"]
    val = fine_upper_fast(n, tets, problem["row_ptr"], problem["col"], He, problem["mass_h2"])
    return g, val


def backtrack(energy_at, e_prev: float, max_halvings: int):
    """The line search of Algorithm 1: alpha = 1, 1/2, 1/4, ... until
    energy_at(alpha) < e_prev.  Returns (alpha, energy, trials) or
    (None, None, trials) after max_halvings + 1 failed trials."""
    alpha = 1.0
    for k in range(max_halvings + 1):
        e = energy_at(alpha)
        if e < e_prev:
            return alpha, e, k + 1
        alpha *= 0.5
    return None, None, max_halvings + 1


def newton(problem, E, X_rest, x_last, threshold: float = 5e-5, tol: float = 1e-3, eps_d: float = None,
           max_newton: int = 50, post_iters: int = 10, max_halvings: int = 30, pcg_max_iter: int = 100000):
    """The Newton loop from x = problem["x"].  eps_d defaults to the paper's
    1e-3 l (l the bounding-box diagonal, m/s).  Returns dict(x, history,
    converged, stalled); history holds one dict per iteration (e_prev, n_c,
    coarse_iters, post_iters, dnorm, alpha, trials, e_new)."""
    n, tets, edges, h = problem["n"], problem["tets"], problem["edges"], problem["h"]
    rp, col = problem["row_ptr"], problem["col"]
    x = np.array(problem["x"], dtype=np.float64)
    X_rest = np.asarray(X_rest, dtype=np.float64)
    if eps_d is None:
        eps_d = 1e-3 * float(np.linalg.norm(X_rest.max(0) - X_rest.min(0)))
    x_before = np.asarray(x_last, dtype=np.float64)
    e_prev = energy(problem, E, X_rest, x)
    hist = []
    converged = stalled = False
    ident = np.arange(n, dtype=np.int32)
    empty_idx = np.zeros((0, 4), np.int32)
    empty_blk = np.zeros((0, 10, 3, 3))
    for _ in range(max_newton):
        x_prev = x
        g, val = gradient_and_hessian(problem, E, X_rest, x)
        tags, _ = strain_tags(X_rest, x_before, x, tets, edges, threshold)
        lab, nc = labels(n, edges, tags)
        crp, cci, cval = galerkin(lab, nc, rp, col, val, empty_idx, empty_blk)
        dinv = block_jacobi(crp, cci, cval)
        gc = coarse_gradient(lab, nc, g)
        y, cit, _, _ = pcg(crp, cci, cval, dinv, -gc, tol, pcg_max_iter)
        d = prolongate(lab, y)
        pit = 0
        if post_iters > 0:
            frp, fci, fval = galerkin(ident, n, rp, col, val, empty_idx, empty_blk)
            fdinv = block_jacobi(frp, fci, fval)
            d, pit, _, _ = pcg(frp, fci, fval, fdinv, -g, tol, post_iters, x0=d)
        dnorm = float(np.abs(d).max())
        alpha, e_new, trials = backtrack(lambda a: energy(problem, E, X_rest, x_prev + a * d), e_prev, max_halvings)
        hist.append(dict(e_prev=e_prev, n_c=nc, coarse_iters=cit, post_iters=pit, dnorm=dnorm, alpha=alpha,
                         trials=trials, e_new=e_new, labels=lab, d=d))
        if alpha is None:
            # no decrease found: converged if the step is below the tolerance
            # anyway (rounding-level steps cannot lower E), else stalled
            converged = dnorm / h <= eps_d
            stalled = not converged
            break
        x_before = x_prev
        x = x_prev + alpha * d
        e_prev = e_new
        if dnorm / h <= eps_d:
            converged = True
            break
    return dict(x=x, history=hist, converged=converged, stalled=stalled, eps_d=eps_d)
