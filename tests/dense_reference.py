"""Dense reconstructions used to pin the oracle from outside it.

The fine Hessian is rebuilt here as a dense 3n x 3n matrix straight from the
per-tet 12x12 element Hessians, the lumped inertia diagonal and the barrier
stencils written as kappa b''(d) grad_d grad_d^T (not from the packed upper
blocks the oracle reads), and the aggregation operator U is a dense 0/1
matrix.  None of this calls the oracle, so agreement is evidence, not an
echo.
"""
import numpy as np

from paper_2605_04773_gb300 import scenes


def dense_fine_hessian(sc) -> np.ndarray:
    m = sc.meta
    n = sc.n
    H = np.zeros((3 * n, 3 * n))
    tets = m["tets"]
    Hel = m["elem_hess"]
    for e in range(tets.shape[0]):
        dof = (3 * tets[e][:, None] + np.arange(3)).ravel()
        H[np.ix_(dof, dof)] += Hel[e]
    H[np.arange(3 * n), np.arange(3 * n)] += np.repeat(m["mass"] / m["h"] ** 2, 3)
    if sc.n_pairs:
        _, _, b2 = scenes.barrier_derivs(m["pair_d"], m["dhat"])
        kappa = np.broadcast_to(np.asarray(m["pair_kappa"], dtype=float), b2.shape)
        gd = m["pair_grad_d"]
        for p in range(sc.n_pairs):
            dof = (3 * sc.pair_idx[p].astype(np.int64)[:, None] + np.arange(3)).ravel()
            H[np.ix_(dof, dof)] += kappa[p] * b2[p] * np.outer(gd[p], gd[p])
    return H


def dense_from_bsr(row_ptr, col, val, n_rows=None) -> np.ndarray:
    n = (len(row_ptr) - 1) if n_rows is None else n_rows
    A = np.zeros((3 * n, 3 * n))
    for i in range(n):
        for k in range(row_ptr[i], row_ptr[i + 1]):
            j = col[k]
            A[3 * i:3 * i + 3, 3 * j:3 * j + 3] += val[k]
    return A


def aggregation_operator(labels, n_c) -> np.ndarray:
    """U^T as a dense (3 n) x (3 n_c) matrix: identity block at (f, labels[f])."""
    n = len(labels)
    P = np.zeros((3 * n, 3 * n_c))
    for f, c in enumerate(labels):
        P[3 * f:3 * f + 3, 3 * c:3 * c + 3] = np.eye(3)
    return P


def bfs_labels(n, edges, tags):
    """Connected components by breadth-first search, numbered in order of
    each component's smallest vertex (pure Python, small graphs only)."""
    adj = [[] for _ in range(n)]
    for (u, v), t in zip(edges, tags):
        if t:
            adj[u].append(v)
            adj[v].append(u)
    lab = [-1] * n
    nxt = 0
    for s in range(n):
        if lab[s] >= 0:
            continue
        lab[s] = nxt
        queue = [s]
        while queue:
            u = queue.pop()
            for v in adj[u]:
                if lab[v] < 0:
                    lab[v] = nxt
                    queue.append(v)
        nxt += 1
    return np.array(lab, dtype=np.int32), nxt
