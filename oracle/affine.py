"""CPU oracle of the adaptive affine embedding (Sec. 4.2, Eq. 4, and the
supplement's affine mapping).

TEST INFRASTRUCTURE: only the test suite, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference leg of ``bench.py`` may import this module.

A coarse node whose aggregate holds more than `threshold` fine nodes gets 12
DoF: fine node f of it moves by dx_f = A_f^T y_c with A_f = Xbar_f (x) I3,
Xbar_f = (X_f, 1) its homogeneous rest position, i.e. y_c is four 3-vectors
and dx_f = sum_k Xbar_f[k] y_c[k].  Smaller aggregates keep 3 DoF (dx_f =
y_c).  Coarse rows are ordered with every 3-DoF node first (in label order),
then every 12-DoF node as 4 consecutive 3-rows (also in label order).  With
P the fine-from-coarse map (dx = P y), the coarse system is the Galerkin
product g_c = P^T g, H_c = P^T H P (Eq. 4 summed over fine nodes).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from . import fine_system_csr_blocks


def plan(labels, n_c: int, X_rest, threshold: int = 32):
    """Per coarse node: DoF (3 or 12) and first coarse 3-row; per fine node:
    its coarse first row, its weights (1 or Xbar_f) and the row count.
    Returns dict(dof, base, n3, n_rows, fine_base, fine_w [n, 4], fine_k)."""
    labels = np.asarray(labels)
    counts = np.bincount(labels, minlength=n_c)
    affine = counts > threshold
    # stable reorder: 3-DoF nodes first, each class in label order
    key = np.where(affine, np.arange(n_c) + n_c, np.arange(n_c))
    order = np.argsort(key, kind="stable")
    newpos = np.empty(n_c, np.int64)
    newpos[order] = np.arange(n_c)
    n3 = int((~affine).sum())
    base = np.where(affine, n3 + 4 * (newpos - n3), newpos)
    n_rows = n3 + 4 * int(affine.sum())
    n = labels.size
    fine_aff = affine[labels]
    fine_base = base[labels]
    fine_k = np.where(fine_aff, 4, 1)
    fine_w = np.zeros((n, 4))
    fine_w[~fine_aff, 0] = 1.0
    Xb = np.concatenate([np.asarray(X_rest, dtype=np.float64), np.ones((n, 1))], 1)
    fine_w[fine_aff] = Xb[fine_aff]
    return dict(dof=np.where(affine, 12, 3), base=base, n3=n3, n_rows=n_rows, fine_base=fine_base, fine_w=fine_w,
                fine_k=fine_k, affine=affine)


def prolongation(pl) -> sp.csr_matrix:
    """P (3n x 3 n_rows): dx = P y, as an explicit sparse matrix."""
    n = pl["fine_base"].size
    rows, cols, vals = [], [], []
    for f in range(n):
        for k in range(pl["fine_k"][f]):
            for c in range(3):
                rows.append(3 * f + c)
                cols.append(3 * (pl["fine_base"][f] + k) + c)
                vals.append(pl["fine_w"][f, k])
    return sp.csr_matrix((vals, (rows, cols)), shape=(3 * n, 3 * pl["n_rows"]))


def coarse_system(scene, labels, n_c: int, threshold: int = 32):
    """(plan, P, H_c, g_c) of the affine-embedded Galerkin system."""
    pl = plan(labels, n_c, scene.meta["X_rest"], threshold)
    P = prolongation(pl)
    H = fine_system_csr_blocks(scene)
    Hc = (P.T @ H @ P).tocsr()
    gc = P.T @ scene.g.reshape(-1)
    return pl, P, Hc, gc


def solve(scene, labels, n_c: int, threshold: int = 32):
    """y = -H_c^-1 g_c by a sparse direct solve and dx = P y."""
    from scipy.sparse.linalg import spsolve
    pl, P, Hc, gc = coarse_system(scene, labels, n_c, threshold)
    y = spsolve(Hc.tocsc(), -gc)
    return dict(plan=pl, P=P, Hc=Hc, gc=gc, y=y, dx=(P @ y).reshape(-1, 3))
