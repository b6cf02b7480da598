"""Seeded synthetic inputs for one Newton iteration of the coarsened solve.

This module produces the *inputs* of the in-solve coarsening path: the static
fine mesh (Kuhn 6-tet split of hex grids), its edge list, per-edge collapse
tags, the fine Hessian as an upper-triangular 3x3-block BSR matrix, the
synthetic IPC-barrier stencils (4 vertices, 10 upper 3x3 blocks each) and the
fine gradient.  It holds none of the coarsening method's arithmetic: no
aggregation, no coarse assembly, no solve and no prolongation.  Both the CUDA
path and the CPU oracle consume these arrays, and nothing else is shared
between them.

Physical model of the inputs (the incremental potential of Sec. 3, Eq. 1,
divided by dt^2):
    H = M/h^2 + d2Psi/dx2 (PSD-projected per tet) + sum_pairs kappa b''(d) grad_d grad_d^T
    g = M/h^2 (x - x_hat) + dPsi/dx + sum_pairs kappa b'(d) grad_d
with StVK elasticity Psi_e = V_e (mu |G|_F^2 + lambda/2 tr(G)^2),
G = (F^T F - I)/2, a lumped mass rho V_e / 4 per tet vertex, x_hat = X_rest +
h^2 gravity (zero velocity) and the IPC log barrier b(d) = -(d - dhat)^2
ln(d / dhat).  The barrier stencils are synthetic stand-ins for geometric
contact: a random unit normal n and barycentric weights give the distance
gradient ([n, -b0 n, -b1 n, -b2 n] for point-triangle, [(1-a) n, a n,
-(1-b) n, -b n] for edge-edge) and the gap d is drawn uniformly.

Tags follow Sec. 4.1: tau_e = 1 marks a collapsible edge, 0 a protected one.
Here a smooth random activity field (8 Fourier modes per body) stands in for
the Green-strain-increment criterion of Eq. 3: an edge is collapsible when the
mean activity magnitude of its two endpoints is strictly below the per-body
quantile that gives the requested collapsible fraction.
"""
from __future__ import annotations

import dataclasses
import itertools
import os
from concurrent.futures import ThreadPoolExecutor

import numpy as np

GRAVITY = np.array([0.0, 0.0, -9.81])

# Local vertex pairs (s, t), s <= t, of the 10 upper 3x3 blocks of a 4-vertex
# stencil, in the packed order used for the barrier-pair block array.
STENCIL_UPPER_PAIRS = ((0, 0), (0, 1), (0, 2), (0, 3), (1, 1), (1, 2), (1, 3), (2, 2), (2, 3), (3, 3))


@dataclasses.dataclass
class Scene:
    """One fine Newton system and the metadata that produced it.

    Arrays that the solve path reads (all host numpy):
      edges     int32  [E, 2]   static mesh edges, u < v, sorted
      tags      uint8  [E]      1 = collapsible, 0 = protected
      row_ptr   int32  [n+1]    fine upper BSR (column >= row), sorted columns
      col       int32  [nnzb]
      val       f64    [nnzb, 3, 3] row-major 3x3 blocks
      pair_idx  int32  [P, 4]   barrier stencil vertices
      pair_blk  f64    [P, 10, 3, 3] packed upper stencil blocks (STENCIL_UPPER_PAIRS)
      g         f64    [n, 3]   fine gradient
    """

    name: str
    seed: int
    n: int
    edges: np.ndarray
    tags: np.ndarray
    row_ptr: np.ndarray
    col: np.ndarray
    val: np.ndarray
    pair_idx: np.ndarray
    pair_blk: np.ndarray
    g: np.ndarray
    meta: dict = dataclasses.field(default_factory=dict)

    @property
    def n_edges(self) -> int:
        return int(self.edges.shape[0])

    @property
    def nnzb(self) -> int:
        return int(self.col.shape[0])

    @property
    def n_pairs(self) -> int:
        return int(self.pair_idx.shape[0])


# ----------------------------------------------------------------------------
# Mesh
# ----------------------------------------------------------------------------

def kuhn_hex_grid(nx: int, ny: int, nz: int, cell: float, origin=(0.0, 0.0, 0.0)):
    """Vertices and tets of an nx*ny*nz hex grid, each hex split into the 6
    Kuhn tets around its (0,0,0)-(1,1,1) diagonal.  Vertex index
    ix + (nx+1)*(iy + (ny+1)*iz); every tet is positively oriented."""
    ix, iy, iz = np.meshgrid(np.arange(nx + 1), np.arange(ny + 1), np.arange(nz + 1), indexing="ij")
    vid = lambda a, b, c: a + (nx + 1) * (b + (ny + 1) * c)  # noqa: E731
    X = np.stack([ix, iy, iz], -1).transpose(2, 1, 0, 3).reshape(-1, 3).astype(np.float64) * cell
    X += np.asarray(origin, dtype=np.float64)
    cx, cy, cz = np.meshgrid(np.arange(nx), np.arange(ny), np.arange(nz), indexing="ij")
    cx, cy, cz = (a.transpose(2, 1, 0).ravel() for a in (cx, cy, cz))
    tets = []
    for perm in itertools.permutations(range(3)):
        corner = np.zeros(3, dtype=np.int64)
        path = [corner.copy()]
        for axis in perm:
            corner[axis] += 1
            path.append(corner.copy())
        tets.append(np.stack([vid(cx + p[0], cy + p[1], cz + p[2]) for p in path], -1))
    tets = np.concatenate(tets, 0).astype(np.int64)
    d = X[tets[:, 1:]] - X[tets[:, :1]]
    neg = np.linalg.det(d) < 0
    tets[neg, 1], tets[neg, 2] = tets[neg, 2].copy(), tets[neg, 1].copy()
    return X, tets


def mesh_edges(tets: np.ndarray) -> np.ndarray:
    """Unique undirected edges (u < v) of a tet mesh, lexicographically sorted."""
    pairs = np.concatenate([tets[:, [a, b]] for a, b in itertools.combinations(range(4), 2)], 0)
    pairs.sort(axis=1)
    n = int(tets.max()) + 1
    key = np.unique(pairs[:, 0].astype(np.int64) * n + pairs[:, 1])
    return np.stack([key // n, key % n], 1).astype(np.int32)


# ----------------------------------------------------------------------------
# StVK elasticity and the IPC barrier (input physics, not the coarsening method)
# ----------------------------------------------------------------------------

def lame(E, nu):
    mu = E / (2.0 * (1.0 + nu))
    lam = E * nu / ((1.0 + nu) * (1.0 - 2.0 * nu))
    return mu, lam


def stvk_elements(Xt: np.ndarray, xt: np.ndarray, E, nu: float, project: bool = True):
    """Per-tet StVK energy, gradient [nt,12] and Hessian [nt,12,12] with
    respect to the 12 vertex coordinates (index 3*a + c), for rest and current
    tet positions Xt, xt [nt,4,3].  With project=True each Hessian is made PSD
    by clamping its negative eigenvalues to zero."""
    nt = Xt.shape[0]
    E = np.broadcast_to(np.asarray(E, dtype=np.float64), (nt,))
    mu, lam = lame(E, nu)
    Dm = (Xt[:, 1:] - Xt[:, :1]).transpose(0, 2, 1)
    Ds = (xt[:, 1:] - xt[:, :1]).transpose(0, 2, 1)
    Dminv = np.linalg.inv(Dm)
    vol = np.abs(np.linalg.det(Dm)) / 6.0
    F = Ds @ Dminv
    w = np.empty((nt, 4, 3))
    w[:, 1:, :] = Dminv
    w[:, 0, :] = -Dminv.sum(1)
    I3 = np.eye(3)
    G = 0.5 * (np.einsum("nki,nkj->nij", F, F) - I3)
    trG = np.einsum("nii->n", G)
    S = 2.0 * mu[:, None, None] * G + (lam * trG)[:, None, None] * I3
    P = F @ S
    energy = vol * (mu * np.einsum("nij,nij->n", G, G) + 0.5 * lam * trG**2)
    grad = vol[:, None, None] * np.einsum("ncj,naj->nac", P, w)
    FFt = np.einsum("nik,njk->nij", F, F)
    # dP_ij / dF_kl for StVK.
    K = (np.einsum("ik,nlj->nijkl", I3, S)
         + mu[:, None, None, None, None] * np.einsum("nil,nkj->nijkl", F, F)
         + mu[:, None, None, None, None] * np.einsum("nik,jl->nijkl", FFt, I3)
         + lam[:, None, None, None, None] * np.einsum("nij,nkl->nijkl", F, F))
    H = np.einsum("naj,ncjdl,nbl->nacbd", w, K, w, optimize=True) * vol[:, None, None, None, None]
    H = H.reshape(nt, 12, 12)
    H = 0.5 * (H + H.transpose(0, 2, 1))
    if project:
        lam_e, V = np.linalg.eigh(H)
        H = np.einsum("nij,nj,nkj->nik", V, np.maximum(lam_e, 0.0), V)
        H = 0.5 * (H + H.transpose(0, 2, 1))
    return energy, grad.reshape(nt, 12), H


def barrier_derivs(d: np.ndarray, dhat: float):
    """b(d) = -(d - dhat)^2 ln(d/dhat) for 0 < d < dhat, with b' and b''."""
    t = d - dhat
    ln = np.log(d / dhat)
    b = -t * t * ln
    b1 = -2.0 * t * ln - t * t / d
    b2 = -2.0 * ln - 4.0 * t / d + t * t / (d * d)
    return b, b1, b2


def barrier_stencils(grad_d: np.ndarray, d: np.ndarray, dhat: float, kappa: float):
    """Gradient [P,12] and packed upper Hessian blocks [P,10,3,3] of
    kappa * b(d) under the Gauss-Newton (PSD) approximation kappa b'' gd gd^T."""
    _, b1, b2 = barrier_derivs(d, dhat)
    grad = kappa * b1[:, None] * grad_d
    gd = grad_d.reshape(-1, 4, 3)
    s_idx = [s for s, _ in STENCIL_UPPER_PAIRS]
    t_idx = [t for _, t in STENCIL_UPPER_PAIRS]
    blk = gd[:, s_idx, :, None] * gd[:, t_idx, None, :]
    blk *= (kappa * b2)[:, None, None, None]
    return grad, blk


# ----------------------------------------------------------------------------
# Tags
# ----------------------------------------------------------------------------

def activity_field(X: np.ndarray, rng: np.random.Generator, n_modes: int = 8) -> np.ndarray:
    """Smooth random 3-vector field on a body: n_modes cosine modes with
    integer wavevectors in [-2, 2]^3 over the body's bounding box."""
    lo, hi = X.min(0), X.max(0)
    ext = np.where(hi > lo, hi - lo, 1.0)
    k = rng.integers(-2, 3, size=(n_modes, 3))
    phase = rng.uniform(0.0, 2 * np.pi, size=n_modes)
    amp = rng.standard_normal((n_modes, 3))
    arg = 2 * np.pi * ((X - lo) / ext) @ k.T + phase
    return np.cos(arg) @ amp


def tags_from_field(edges: np.ndarray, field: np.ndarray, frac_collapsible: float) -> np.ndarray:
    """tau_e = 1 where the edge's mean endpoint |field| is strictly below the
    frac_collapsible quantile of all edge values of the body."""
    mag = np.linalg.norm(field, axis=1)
    v = 0.5 * (mag[edges[:, 0]] + mag[edges[:, 1]])
    thr = np.quantile(v, frac_collapsible)
    return (v < thr).astype(np.uint8)


# ----------------------------------------------------------------------------
# Fine system
# ----------------------------------------------------------------------------

def fine_upper_bsr(n: int, tets: np.ndarray, Hel: np.ndarray, diag_mass: np.ndarray):
    """Sum per-tet 12x12 Hessians and the inertia diagonal into an upper 3x3
    BSR matrix (column >= row, sorted columns).  A tet block (a, b) lands at
    (v_a, v_b) when v_a <= v_b and as its transpose at (v_b, v_a) otherwise."""
    rows, cols, blks = [], [], []
    H4 = Hel.reshape(-1, 4, 3, 4, 3).transpose(0, 1, 3, 2, 4)  # [nt, a, b, 3, 3]
    for a in range(4):
        for b in range(a, 4):
            va, vb = tets[:, a], tets[:, b]
            B = H4[:, a, b]
            swap = va > vb
            r = np.where(swap, vb, va)
            c = np.where(swap, va, vb)
            B = np.where(swap[:, None, None], B.transpose(0, 2, 1), B)
            rows.append(r)
            cols.append(c)
            blks.append(B)
    rows.append(np.arange(n))
    cols.append(np.arange(n))
    blks.append(diag_mass[:, None, None] * np.eye(3))
    rows = np.concatenate(rows).astype(np.int64)
    cols = np.concatenate(cols).astype(np.int64)
    blks = np.concatenate(blks, 0).reshape(-1, 9)
    key = rows * n + cols
    ukey, inv = np.unique(key, return_inverse=True)
    val = np.stack([np.bincount(inv, weights=blks[:, k], minlength=ukey.size) for k in range(9)], 1)
    urow = ukey // n
    ucol = ukey % n
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(np.bincount(urow, minlength=n), out=row_ptr[1:])
    return row_ptr.astype(np.int32), ucol.astype(np.int32), val.reshape(-1, 3, 3)


def _scatter_grad(n: int, idx: np.ndarray, grad: np.ndarray) -> np.ndarray:
    out = np.zeros((n, 3))
    flat = idx.reshape(-1)
    gr = grad.reshape(-1, 3)
    for c in range(3):
        out[:, c] = np.bincount(flat, weights=gr[:, c], minlength=n)
    return out


def _unit(v):
    return v / np.linalg.norm(v, axis=-1, keepdims=True)


def _random_pt_grad(rng, normals):
    beta = rng.dirichlet(np.ones(3), size=normals.shape[0])
    return np.concatenate([normals, -beta[:, 0:1] * normals, -beta[:, 1:2] * normals, -beta[:, 2:3] * normals], 1)


def _random_ee_grad(rng, normals):
    a = rng.uniform(0, 1, size=(normals.shape[0], 1))
    b = rng.uniform(0, 1, size=(normals.shape[0], 1))
    return np.concatenate([(1 - a) * normals, a * normals, -(1 - b) * normals, -b * normals], 1)


@dataclasses.dataclass
class Body:
    nx: int
    ny: int
    nz: int
    cell: float
    origin: tuple
    E: float
    frac_collapsible: float


def build_scene(name: str, seed: int, bodies: list, nu: float, rho: float, h: float, dhat: float,
                pair_fn, keep_elements: bool = False, E_elem=None, disp_sigma: float = 0.05,
                small_gap_frac: float = 0.0) -> Scene:
    """Assemble the fine Newton system of a set of disjoint Kuhn-grid bodies.

    pair_fn(rng, body_info) -> (idx [P,4], grad_d [P,12], d [P], kappa [P])
    draws the synthetic barrier stencils.  E_elem, when given, overrides the
    per-tet Young's modulus (a flat array over all tets)."""
    rng = np.random.default_rng(seed)
    Xs, tets_all, tags_all, edges_all, body_info = [], [], [], [], []
    E_list = []
    off = 0
    box_cache = {}
    for bi, bd in enumerate(bodies):
        key = (bd.nx, bd.ny, bd.nz, bd.cell)
        if key not in box_cache:
            X0, tets0 = kuhn_hex_grid(bd.nx, bd.ny, bd.nz, bd.cell)
            box_cache[key] = (X0, tets0, mesh_edges(tets0))
        X0, tets, edges = box_cache[key]
        X = X0 + np.asarray(bd.origin, dtype=np.float64)
        field = activity_field(X, rng)
        tags = tags_from_field(edges, field, bd.frac_collapsible)
        Xs.append(X)
        tets_all.append(tets + off)
        edges_all.append(edges + off)
        tags_all.append(tags)
        E_list.append(np.full(tets.shape[0], bd.E))
        body_info.append(dict(offset=off, nx=bd.nx, ny=bd.ny, nz=bd.nz, cell=bd.cell, E=bd.E, index=bi))
        off += X.shape[0]
    n = off
    X = np.concatenate(Xs, 0)
    tets = np.concatenate(tets_all, 0)
    edges = np.concatenate(edges_all, 0).astype(np.int32)
    tags = np.concatenate(tags_all, 0)
    E_t = np.concatenate(E_list) if E_elem is None else np.asarray(E_elem, dtype=np.float64)
    cell_v = np.concatenate([np.full(x.shape[0], bd.cell) for x, bd in zip(Xs, bodies)])
    x = X + disp_sigma * cell_v[:, None] * rng.standard_normal(X.shape)

    # Elasticity, in chunks to bound the temporary 12x12x(3x3x3x3) arrays.
    nt = tets.shape[0]
    e_grad = np.empty((nt, 12))
    e_hess = np.empty((nt, 12, 12))
    vol = np.empty(nt)
    chunk = 16384

    def work(s):
        t = tets[s:s + chunk]
        _, gr, H = stvk_elements(X[t], x[t], E_t[s:s + chunk], nu)
        e_grad[s:s + chunk] = gr
        e_hess[s:s + chunk] = H
        Dm = X[t[:, 1:]] - X[t[:, :1]]
        vol[s:s + chunk] = np.abs(np.linalg.det(Dm)) / 6.0

    with ThreadPoolExecutor(max(1, min(16, os.cpu_count() or 1))) as ex:
        list(ex.map(work, range(0, nt, chunk)))
    mass = np.bincount(tets.reshape(-1), weights=np.repeat(rho * vol / 4.0, 4), minlength=n)
    x_hat = X + h * h * GRAVITY
    g = (mass / (h * h))[:, None] * (x - x_hat) + _scatter_grad(n, tets, e_grad.reshape(-1, 4, 3))

    row_ptr, col, val = fine_upper_bsr(n, tets, e_hess, mass / (h * h))

    pidx, grad_d, d, kappa = pair_fn(rng, body_info)
    if small_gap_frac > 0 and d.size:
        k = max(1, int(round(small_gap_frac * d.size)))
        sel = rng.choice(d.size, size=k, replace=False)
        d = d.copy()
        d[sel] = rng.uniform(0.01, 0.05, size=k) * dhat
    g_pairs = np.zeros((n, 3))
    if pidx.shape[0]:
        pgrad, pblk = barrier_stencils(grad_d, d, dhat, kappa) if np.isscalar(kappa) else \
            _barrier_stencils_vec(grad_d, d, dhat, kappa)
        g_pairs = _scatter_grad(n, pidx, pgrad.reshape(-1, 4, 3))
        g += g_pairs
    else:
        pblk = np.zeros((0, 10, 3, 3))
    meta = dict(X_rest=X, x=x, x_hat=x_hat, tets=tets, E_elem=E_t, nu=nu, rho=rho, h=h, dhat=dhat,
                mass=mass, pair_d=d, bodies=body_info, vol=vol, g_pairs=g_pairs)
    if keep_elements:
        meta.update(elem_grad=e_grad, elem_hess=e_hess, pair_grad_d=grad_d, pair_kappa=kappa)
    return Scene(name=name, seed=seed, n=n, edges=edges, tags=tags, row_ptr=row_ptr, col=col,
                 val=np.ascontiguousarray(val), pair_idx=pidx.astype(np.int32),
                 pair_blk=np.ascontiguousarray(pblk), g=g, meta=meta)


def _barrier_stencils_vec(grad_d, d, dhat, kappa):
    grad, blk = barrier_stencils(grad_d, d, dhat, 1.0)
    kappa = np.asarray(kappa, dtype=np.float64)
    return grad * kappa[:, None], blk * kappa[:, None, None, None]


def _random_pairs_in_body(n_pairs: int, kind: str = "pt"):
    """pair_fn drawing n_pairs point-triangle stencils on 4 distinct random
    vertices of the whole vertex range (the unit-cube workload)."""
    def fn(rng, body_info):
        n = sum((b["nx"] + 1) * (b["ny"] + 1) * (b["nz"] + 1) for b in body_info)
        if n_pairs == 0:
            return np.zeros((0, 4), np.int32), np.zeros((0, 12)), np.zeros(0), 1.0
        idx = np.stack([rng.choice(n, size=4, replace=False) for _ in range(n_pairs)], 0)
        normals = _unit(rng.standard_normal((n_pairs, 3)))
        grad_d = _random_pt_grad(rng, normals)
        b0 = body_info[0]
        d = rng.uniform(0.1, 1.0, size=n_pairs) * fn.dhat
        kappa = b0["E"] * b0["cell"]
        return idx.astype(np.int32), grad_d, d, kappa
    fn.dhat = None
    return fn


def _facing_pairs(n_total: int, layout: dict, dhat: float):
    """pair_fn drawing point-triangle and edge-edge stencils between the facing
    surfaces of neighbouring cuboids of a 2-D layout of identical boxes."""
    def fn(rng, body_info):
        gx_n, gy_n = layout["gx"], layout["gy"]
        nb = len(body_info)
        nbrs = []
        for b in range(nb):
            gx, gy = b % gx_n, b // gx_n
            if gx + 1 < gx_n:
                nbrs.append((b, b + 1, 0))
            if gy + 1 < gy_n:
                nbrs.append((b, b + gx_n, 1))
        per = np.full(len(nbrs), n_total // len(nbrs))
        per[: n_total - per.sum()] += 1
        idx_all, gd_all, d_all, k_all = [], [], [], []
        for (a, b, axis), m in zip(nbrs, per):
            A, B = body_info[a], body_info[b]
            dims = (A["nx"], A["ny"], A["nz"])

            def vid(info, i, j, k):
                return info["offset"] + i + (info["nx"] + 1) * (j + (info["ny"] + 1) * k)

            # face coordinates (u, w) span the two axes other than `axis`
            ax_u, ax_w = [q for q in range(3) if q != axis]
            nu_, nw_ = dims[ax_u], dims[ax_w]

            def face_vid(info, side, u, w):
                c = [0, 0, 0]
                c[axis] = dims[axis] if side == 1 else 0
                c[ax_u], c[ax_w] = u, w
                return vid(info, *c)

            m_pt = m // 2
            m_ee = m - m_pt
            # point-triangle: point on one face, triangle of the facing cell
            u = rng.integers(0, nu_ + 1, size=m_pt)
            w = rng.integers(0, nw_ + 1, size=m_pt)
            cu = np.clip(u - rng.integers(0, 2, size=m_pt), 0, nu_ - 1)
            cw = np.clip(w - rng.integers(0, 2, size=m_pt), 0, nw_ - 1)
            flip = rng.integers(0, 2, size=m_pt).astype(bool)
            upper_tri = rng.integers(0, 2, size=m_pt).astype(bool)
            P = np.empty((m_pt, 4), np.int64)
            for q in range(m_pt):
                pb, tb, ps, ts = (A, B, 1, 0) if not flip[q] else (B, A, 0, 1)
                quad = [face_vid(tb, ts, cu[q], cw[q]), face_vid(tb, ts, cu[q] + 1, cw[q]),
                        face_vid(tb, ts, cu[q] + 1, cw[q] + 1), face_vid(tb, ts, cu[q], cw[q] + 1)]
                tri = quad[:3] if upper_tri[q] else [quad[0], quad[2], quad[3]]
                P[q] = [face_vid(pb, ps, u[q], w[q])] + tri
            n0 = np.zeros((m_pt, 3))
            n0[:, axis] = np.where(flip, 1.0, -1.0)
            gd_pt = _random_pt_grad(rng, _unit(n0 + 0.1 * rng.standard_normal((m_pt, 3))))
            # edge-edge: an edge of each facing face, near each other
            eu = rng.integers(0, nu_, size=m_ee)
            ew = rng.integers(0, nw_, size=m_ee)
            dirA = rng.integers(0, 2, size=m_ee)
            dirB = rng.integers(0, 2, size=m_ee)
            Q = np.empty((m_ee, 4), np.int64)
            for q in range(m_ee):
                a0 = face_vid(A, 1, eu[q], ew[q])
                a1 = face_vid(A, 1, eu[q] + (dirA[q] == 0), ew[q] + (dirA[q] == 1))
                b0 = face_vid(B, 0, eu[q], ew[q])
                b1 = face_vid(B, 0, eu[q] + (dirB[q] == 0), ew[q] + (dirB[q] == 1))
                Q[q] = [a0, a1, b0, b1]
            n1 = np.zeros((m_ee, 3))
            n1[:, axis] = -1.0
            gd_ee = _random_ee_grad(rng, _unit(n1 + 0.1 * rng.standard_normal((m_ee, 3))))
            idx_all += [P, Q]
            gd_all += [gd_pt, gd_ee]
            d_all.append(rng.uniform(0.1, 1.0, size=m) * dhat)
            k_all.append(np.full(m, A["E"] * A["cell"]))
        return (np.concatenate(idx_all, 0).astype(np.int32), np.concatenate(gd_all, 0),
                np.concatenate(d_all), np.concatenate(k_all))
    return fn


# ----------------------------------------------------------------------------
# Workloads
# ----------------------------------------------------------------------------

def unit_cube(seed: int = 1001, n_cells: int = 8, n_pairs: int = 64, frac: float = 0.7,
              keep_elements: bool = False) -> Scene:
    """Unit cube as an n^3 hex grid (8^3: 729 vertices, 3072 tets), StVK
    E = 1e5 Pa, nu = 0.4, h = 1/60 s, n_pairs point-triangle stencils with
    gap U(0.1, 1) dhat, dhat = 1e-3, 70 % of edges collapsible."""
    dhat = 1e-3
    fn = _random_pairs_in_body(n_pairs)
    fn.dhat = dhat
    body = Body(n_cells, n_cells, n_cells, 1.0 / n_cells, (0.0, 0.0, 0.0), 1e5, frac)
    sc = build_scene("unit_cube_%d" % n_cells, seed, [body], nu=0.4, rho=1000.0, h=1.0 / 60.0,
                     dhat=dhat, pair_fn=fn, keep_elements=keep_elements)
    return sc


def domino_grid(seed: int = 1002, gx: int = 8, gy: int = 8, dims=(6, 12, 24), n_pairs: int = 200_000,
                cell: float = 0.01, E: float = 3e5, frac_range=(0.4, 0.9), small_gap_frac: float = 0.0,
                keep_elements: bool = False) -> Scene:
    """gx*gy soft cuboids (default 64 boxes of 6x12x24 cells = 2275 vertices
    and 10368 tets each, 145,600 vertices and 663,552 tets in all) laid out on
    a 2-D grid like standing dominoes, StVK E = 3e5 Pa, ~200k point-triangle
    and edge-edge stencils between facing surfaces of neighbouring boxes, and
    a per-box collapsible fraction drawn from U(frac_range)."""
    dhat = 1e-3
    rng = np.random.default_rng(seed + 7919)
    nx, ny, nz = dims
    gap = 2 * cell
    bodies = []
    for b in range(gx * gy):
        ix, iy = b % gx, b // gx
        origin = (ix * (nx * cell + gap), iy * (ny * cell + gap), 0.0)
        bodies.append(Body(nx, ny, nz, cell, origin, E, float(rng.uniform(*frac_range))))
    fn = _facing_pairs(n_pairs, dict(gx=gx, gy=gy), dhat)
    return build_scene("domino_%dx%d" % (gx, gy), seed, bodies, nu=0.4, rho=1000.0, h=1.0 / 60.0,
                       dhat=dhat, pair_fn=fn, keep_elements=keep_elements, small_gap_frac=small_gap_frac)


def tiny_box(seed: int, nx: int = 1, ny: int = 1, nz: int = 1, n_pairs: int = 2, frac: float = 0.5,
             E: float = 1e5) -> Scene:
    """A small Kuhn box used by the dense-solve and brute-force checks."""
    dhat = 1e-3
    fn = _random_pairs_in_body(n_pairs)
    fn.dhat = dhat
    body = Body(nx, ny, nz, 0.1, (0.0, 0.0, 0.0), E, frac)
    return build_scene("tiny_%dx%dx%d" % (nx, ny, nz), seed, [body], nu=0.4, rho=1000.0, h=1.0 / 60.0,
                       dhat=dhat, pair_fn=fn, keep_elements=True)


def _no_pairs(rng, body_info):
    return np.zeros((0, 4), np.int32), np.zeros((0, 12)), np.zeros(0), 1.0


def diff_grid(seed: int = 1005, n_cells: int = 46, E_mean: float = 1e5, E_log_sigma: float = 0.5,
              frac: float = 0.7, target_sigma: float = 0.05, pairs: int = 0) -> Scene:
    """The differentiation workload: one n^3 hex grid of side 1 m (46^3:
    103,823 vertices, 584,016 tets), a per-tet Young's modulus drawn
    log-normal around E_mean (log-sd E_log_sigma), nu = 0.4, h = 1/60 s, 70 %
    of edges collapsible, no barrier pairs unless ``pairs`` > 0 (point-
    triangle stencils, constant in the parameters), and a target position
    field x_target = x + target_sigma * cell * N(0, 1) for the loss
    L = |x_next - x_target|^2."""
    rng = np.random.default_rng(seed + 104729)
    nt = 6 * n_cells ** 3
    E_t = E_mean * np.exp(E_log_sigma * rng.standard_normal(nt))
    dhat = 1e-3
    if pairs:
        fn = _random_pairs_in_body(pairs)
        fn.dhat = dhat
    else:
        fn = _no_pairs
    body = Body(n_cells, n_cells, n_cells, 1.0 / n_cells, (0.0, 0.0, 0.0), E_mean, frac)
    sc = build_scene("diff_grid_%d" % n_cells, seed, [body], nu=0.4, rho=1000.0, h=1.0 / 60.0, dhat=dhat,
                     pair_fn=fn, E_elem=E_t)
    cell = 1.0 / n_cells
    sc.meta["x_target"] = sc.meta["x"] + target_sigma * cell * rng.standard_normal(sc.meta["x"].shape)
    return sc


def diff_problem(sc: Scene) -> dict:
    """The inputs of the differentiation form from a scene: topology, the
    fine upper BSR structure, current positions, parameters (E per tet,
    X_rest), M/h^2, the constant contact terms and the loss target."""
    m = sc.meta
    h = m["h"]
    x_target = m.get("x_target")
    if x_target is None:
        rng = np.random.default_rng(sc.seed + 15485863)
        cell = min(b["cell"] for b in m["bodies"])
        x_target = m["x"] + 0.05 * cell * rng.standard_normal(m["x"].shape)
    return dict(n=sc.n, tets=np.ascontiguousarray(m["tets"], dtype=np.int32), edges=sc.edges, tags=sc.tags,
                row_ptr=sc.row_ptr, col=sc.col, x=m["x"], X_rest=m["X_rest"], E=np.asarray(m["E_elem"]),
                nu=m["nu"], h=h, mass_h2=m["mass"] / (h * h), pair_idx=sc.pair_idx, pair_blk=sc.pair_blk,
                g_pairs=m["g_pairs"], x_target=x_target)


def newton_problem(sc: Scene, v_drop: float = 1.0, bump_speed: float = 2.0, bump_radius: float = 0.15) -> dict:
    """The Newton-loop workload from a scene (normally ``diff_grid``): the body
    at its rest shape (x = X_rest) moving down at v_drop m/s, plus a
    compressive velocity bump of bump_speed m/s (Gaussian, radius
    bump_radius) at the top corner of the bounding box, as after an impact
    there.  x_hat = x + h v + h^2 gravity enters the solver as the constant
    linear term g_extra = -(M/h^2) h v (the fine system's inertia term uses
    X_rest + h^2 gravity); x_last = x - h v are the previous time step's
    positions, the reference of the first iteration's strain-increment
    tags."""
    pr = diff_problem(sc)
    X = np.asarray(pr["X_rest"], dtype=np.float64)
    h = pr["h"]
    corner = X.max(0)
    r2 = np.sum((X - corner) ** 2, axis=1)
    v = np.zeros_like(X)
    v[:, 2] = -v_drop - bump_speed * np.exp(-r2 / (2.0 * bump_radius ** 2))
    pr = dict(pr)
    pr["x"] = X.copy()
    pr["x_last"] = X - h * v
    pr["v"] = v
    pr["g_extra"] = -(pr["mass_h2"] * h)[:, None] * v
    pr["g_pairs"] = None
    return pr


# ----------------------------------------------------------------------------
# Batched form: many independent meshes of uneven sizes
# ----------------------------------------------------------------------------

# Upward edge vectors of the Kuhn split (all cube edges, the monotone face
# diagonals and the main diagonal), in the order of their index offsets.
KUHN_UP = ((1, 0, 0), (0, 1, 0), (1, 1, 0), (0, 0, 1), (1, 0, 1), (0, 1, 1), (1, 1, 1))


def kuhn_structure(nx: int, ny: int, nz: int):
    """Edges (u < v, lexicographic) and the upper BSR structure (row_ptr,
    col: the diagonal then the upward neighbours, sorted) of kuhn_hex_grid's
    mesh, written down directly: vertex (i, j, k) joins (i, j, k) + v for
    every v in KUHN_UP that stays in the grid."""
    ix, iy, iz = np.meshgrid(np.arange(nx + 1), np.arange(ny + 1), np.arange(nz + 1), indexing="ij")
    ix, iy, iz = (a.transpose(2, 1, 0).ravel() for a in (ix, iy, iz))
    n = ix.size
    sx, sy = 1, nx + 1
    sz = (nx + 1) * (ny + 1)
    v = np.arange(n, dtype=np.int64)
    cols = [v]
    valid = [np.ones(n, bool)]
    for dx, dy, dz in KUHN_UP:
        cols.append(v + dx * sx + dy * sy + dz * sz)
        valid.append((ix + dx <= nx) & (iy + dy <= ny) & (iz + dz <= nz))
    C = np.stack(cols, 1)
    Vm = np.stack(valid, 1)
    row_ptr = np.zeros(n + 1, np.int64)
    np.cumsum(Vm.sum(1), out=row_ptr[1:])
    col = C[Vm]
    rows = np.repeat(v, Vm[:, 1:].sum(1))
    edges = np.stack([rows, C[:, 1:][Vm[:, 1:]]], 1)
    return edges.astype(np.int32), row_ptr.astype(np.int32), col.astype(np.int32)


@dataclasses.dataclass
class Batch:
    """Independent instances concatenated into one block-diagonal problem.
    Instance i owns vertices [vert_ptr[i], vert_ptr[i+1]) and tets
    [tet_ptr[i], tet_ptr[i+1]); every index array is global."""
    n_inst: int
    vert_ptr: np.ndarray
    tet_ptr: np.ndarray
    dims: np.ndarray          # [n_inst, 3] cells per axis
    frac: np.ndarray          # collapsible fraction per instance
    edges: np.ndarray
    tags: np.ndarray
    row_ptr: np.ndarray
    col: np.ndarray
    tets: np.ndarray
    X_rest: np.ndarray
    x: np.ndarray
    E: np.ndarray
    nu: float
    h: float
    mass_h2: np.ndarray
    pair_idx: np.ndarray
    pair_blk: np.ndarray
    g_pairs: np.ndarray
    val: np.ndarray = None    # fine upper blocks (numpy-built batches only)
    g: np.ndarray = None

    @property
    def n(self) -> int:
        return int(self.vert_ptr[-1])

    def instance(self, i: int) -> Scene:
        """Instance i as a Scene (local indices); needs the numpy values."""
        v0, v1 = int(self.vert_ptr[i]), int(self.vert_ptr[i + 1])
        e_sel = (self.edges[:, 0] >= v0) & (self.edges[:, 0] < v1)
        p_sel = (self.pair_idx[:, 0] >= v0) & (self.pair_idx[:, 0] < v1) if self.pair_idx.size else np.zeros(0, bool)
        b0, b1 = int(self.row_ptr[v0]), int(self.row_ptr[v1])
        return Scene(name="batch_%d" % i, seed=-1, n=v1 - v0, edges=self.edges[e_sel] - v0, tags=self.tags[e_sel],
                     row_ptr=self.row_ptr[v0:v1 + 1] - b0, col=self.col[b0:b1] - v0, val=self.val[b0:b1],
                     pair_idx=self.pair_idx[p_sel] - v0, pair_blk=self.pair_blk[p_sel], g=self.g[v0:v1],
                     meta=dict(instance=i))


def _instance_dims(seed: int, i: int, v_range):
    """Hex-grid cells per axis of instance i (its stream's first draws) and
    the stream, positioned after them."""
    rng = np.random.default_rng([seed, i])
    nv = float(np.exp(rng.uniform(np.log(v_range[0]), np.log(v_range[1]))))
    rx, ry = np.exp(rng.uniform(-0.7, 0.7, size=2))
    t = (nv / (rx * ry)) ** (1.0 / 3.0)
    nx, ny, nz = (max(2, int(round(r * t)) - 1) for r in (rx, ry, 1.0))
    return (nx, ny, nz), rng


def instance_vertex_counts(seed: int = 1004, n_inst: int = 256, v_range=(2000, 60000), first: int = 0):
    """Vertex counts of instances first .. first + n_inst - 1 of the batched
    workload, without building their meshes."""
    out = []
    for i in range(first, first + n_inst):
        (nx, ny, nz), _ = _instance_dims(seed, i, v_range)
        out.append((nx + 1) * (ny + 1) * (nz + 1))
    return np.asarray(out, dtype=np.int64)


def batch_instances(seed: int = 1004, n_inst: int = 256, v_range=(2000, 60000), frac_range=(0.3, 0.9),
                    pair_frac_range=(0.0, 0.05), cell: float = 0.01, E: float = 1e5, nu: float = 0.4,
                    with_values=False, first: int = 0) -> Batch:
    """The batched workload: n_inst hex-grid bodies split into Kuhn tets,
    vertex counts log-uniform in v_range, random aspect ratios (each axis
    ratio e^U(-0.7, 0.7)), a collapsible fraction U(frac_range) per instance,
    U(pair_frac_range) of each instance's vertices in point-triangle barrier
    stencils (gap U(0.1, 1) dhat), StVK E, nu, rho = 1000, h = 1/60 s.
    with_values (True, or a collection of instance indices) also sums the
    fine system in numpy for those instances (val, g; NaN elsewhere): small
    batches, or the instances a check samples.  The rest get their values on
    the GPU from the same physics.  first > 0 builds instances first ..
    first + n_inst - 1 of the same workload (each instance has its own random
    stream), the contiguous range one rank takes when the batch is sharded.
    with_values indices are the instances' indices in the whole batch."""
    rho, h, dhat = 1000.0, 1.0 / 60.0, 1e-3
    vptr, tptr, dims, fracs = [0], [0], [], []
    parts = {k: [] for k in ("edges", "tags", "row_ptr", "col", "tets", "X", "x", "mass", "pidx", "pblk", "pgrad",
                             "val", "g")}
    nnz_off = 0
    for i in range(first, first + n_inst):
        (nx, ny, nz), rng = _instance_dims(seed, i, v_range)
        frac = float(rng.uniform(*frac_range))
        X, tets = kuhn_hex_grid(nx, ny, nz, cell)
        edges, row_ptr, col = kuhn_structure(nx, ny, nz)
        n = X.shape[0]
        x = X + 0.05 * cell * rng.standard_normal(X.shape)
        tags = tags_from_field(edges, activity_field(X, rng), frac)
        vol = np.abs(np.linalg.det(X[tets[:, 1:]] - X[tets[:, :1]])) / 6.0
        mass = np.bincount(tets.reshape(-1), weights=np.repeat(rho * vol / 4.0, 4), minlength=n)
        npair = int(rng.uniform(*pair_frac_range) * n) // 4
        if npair:
            pidx = np.stack([rng.choice(n, size=4, replace=False) for _ in range(npair)], 0)
            grad_d = _random_pt_grad(rng, _unit(rng.standard_normal((npair, 3))))
            d = rng.uniform(0.1, 1.0, size=npair) * dhat
            pgrad, pblk = barrier_stencils(grad_d, d, dhat, E * cell)
        else:
            pidx, pgrad, pblk = np.zeros((0, 4), np.int64), np.zeros((0, 12)), np.zeros((0, 10, 3, 3))
        g_pairs = _scatter_grad(n, pidx, pgrad.reshape(-1, 4, 3)) if npair else np.zeros((n, 3))
        off = vptr[-1]
        parts["edges"].append(edges + off)
        parts["tags"].append(tags)
        parts["row_ptr"].append(row_ptr[:-1] + nnz_off)
        parts["col"].append(col + off)
        parts["tets"].append(tets + off)
        parts["X"].append(X)
        parts["x"].append(x)
        parts["mass"].append(mass)
        parts["pidx"].append(pidx + off)
        parts["pblk"].append(pblk)
        parts["pgrad"].append(g_pairs)
        want = with_values is True or (with_values is not False and i in with_values)
        if not want and with_values is not False:
            parts["g"].append(np.full((n, 3), np.nan))
            parts["val"].append(np.full((int(row_ptr[-1]), 3, 3), np.nan))
        if want:
            _, e_grad, e_hess = stvk_elements(X[tets], x[tets], E, nu)
            x_hat = X + h * h * GRAVITY
            parts["g"].append((mass / (h * h))[:, None] * (x - x_hat) + _scatter_grad(n, tets, e_grad.reshape(-1, 4, 3))
                              + g_pairs)
            rp2, col2, val = fine_upper_bsr(n, tets, e_hess, mass / (h * h))
            assert np.array_equal(rp2, row_ptr) and np.array_equal(col2, col)
            parts["val"].append(val)
        nnz_off += int(row_ptr[-1])
        vptr.append(off + n)
        tptr.append(tptr[-1] + tets.shape[0])
        dims.append((nx, ny, nz))
        fracs.append(frac)
    cat = lambda k, dt: np.ascontiguousarray(np.concatenate(parts[k], 0).astype(dt))  # noqa: E731
    row_ptr = np.concatenate(parts["row_ptr"] + [np.array([nnz_off])]).astype(np.int32)
    n_total = vptr[-1]
    return Batch(n_inst=n_inst, vert_ptr=np.array(vptr, np.int64), tet_ptr=np.array(tptr, np.int64),
                 dims=np.array(dims, np.int32), frac=np.array(fracs), edges=cat("edges", np.int32),
                 tags=cat("tags", np.uint8), row_ptr=row_ptr, col=cat("col", np.int32), tets=cat("tets", np.int32),
                 X_rest=cat("X", np.float64), x=cat("x", np.float64),
                 E=np.full(int(tptr[-1]), E), nu=nu, h=h, mass_h2=cat("mass", np.float64) / (h * h),
                 pair_idx=cat("pidx", np.int32).reshape(-1, 4), pair_blk=cat("pblk", np.float64).reshape(-1, 10, 3, 3),
                 g_pairs=cat("pgrad", np.float64).reshape(n_total, 3),
                 val=cat("val", np.float64) if with_values is not False else None,
                 g=cat("g", np.float64) if with_values is not False else None)
