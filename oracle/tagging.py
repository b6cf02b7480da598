"""CPU oracle of the Green-strain-increment tagging (Sec. 4.2, Eq. 3).

TEST INFRASTRUCTURE: only the test suite, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference leg of ``bench.py`` may import this module.

Per tet, F = Ds Dm^-1 and the Green strain G = (F^T F - I)/2 at the previous
and the current Newton iterate; a tet whose strain increment has
||G_i - G_{i-1}||_F above the threshold protects (tags 0) every edge it
touches; all other edges are collapsible (tag 1).
"""
from __future__ import annotations

import numpy as np


def green_strain(X_rest, x, tets):
    """G = (F^T F - I)/2 per tet, F = Ds Dm^-1, written out per tet."""
    nt = tets.shape[0]
    G = np.empty((nt, 3, 3))
    for e in range(nt):
        a, b, c, d = tets[e]
        Dm = np.column_stack([X_rest[b] - X_rest[a], X_rest[c] - X_rest[a], X_rest[d] - X_rest[a]])
        Ds = np.column_stack([x[b] - x[a], x[c] - x[a], x[d] - x[a]])
        F = Ds @ np.linalg.inv(Dm)
        G[e] = 0.5 * (F.T @ F - np.eye(3))
    return G


def strain_tags(X_rest, x_prev, x_cur, tets, edges, threshold: float):
    """Tags (uint8 per edge, edges u < v sorted) from the strain increment."""
    dG = green_strain(X_rest, x_cur, tets) - green_strain(X_rest, x_prev, tets)
    norm2 = np.einsum("eij,eij->e", dG, dG)
    hot = norm2 > threshold * threshold
    index = {(int(u), int(v)): k for k, (u, v) in enumerate(edges)}
    tags = np.ones(edges.shape[0], np.uint8)
    for e in np.nonzero(hot)[0]:
        t = tets[e]
        for i in range(4):
            for j in range(i + 1, 4):
                u, v = int(min(t[i], t[j])), int(max(t[i], t[j]))
                tags[index[(u, v)]] = 0
    return tags, np.sqrt(norm2)
