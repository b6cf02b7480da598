"""Pins of the affine-embedding oracle (CPU only)."""
import numpy as np
import scipy.sparse as sp

import oracle
from oracle import affine
from paper_2605_04773_gb300 import scenes


def test_reorder_and_row_bases_by_hand():
    # aggregates of 40, 3, 50, 2 fine nodes, threshold 32: nodes 0 and 2 are
    # affine; rows: node 1 -> 0, node 3 -> 1, node 0 -> 2..5, node 2 -> 6..9
    labels = np.repeat(np.arange(4), [40, 3, 50, 2])
    X = np.random.default_rng(0).standard_normal((labels.size, 3))
    pl = affine.plan(labels, 4, X, 32)
    assert list(pl["dof"]) == [12, 3, 12, 3]
    assert list(pl["base"]) == [2, 0, 6, 1]
    assert pl["n3"] == 2 and pl["n_rows"] == 10
    f = 45  # in aggregate 2 (affine): weights are (X_f, 1)
    assert np.array_equal(pl["fine_w"][f], np.append(X[f], 1.0)) and pl["fine_k"][f] == 4
    assert pl["fine_base"][41] == 0 and pl["fine_k"][41] == 1 and pl["fine_w"][41, 0] == 1.0


def test_without_affine_nodes_it_is_the_plain_galerkin_system():
    sc = scenes.unit_cube(seed=1001)
    lab, nc = oracle.labels(sc.n, sc.edges, sc.tags)
    pl, P, Hc, gc = affine.coarse_system(sc, lab, nc, threshold=10 ** 6)
    assert pl["n_rows"] == nc
    crp, cci, cval = oracle.galerkin(lab, nc, sc.row_ptr, sc.col, sc.val, sc.pair_idx, sc.pair_blk)
    ref = sp.bsr_matrix((cval, cci, crp), shape=(3 * nc, 3 * nc)).toarray()
    assert np.abs(Hc.toarray() - ref).max() <= 1e-12 * np.abs(ref).max()
    assert np.allclose(gc, oracle.coarse_gradient(lab, nc, sc.g).reshape(-1), rtol=1e-13, atol=0)


def test_affine_fields_are_reproduced_exactly():
    # one all-collapsible body, one affine coarse node: when the exact fine
    # step is an affine field of the rest positions, the coarse step finds it
    sc = scenes.tiny_box(seed=41, nx=3, ny=2, nz=2, n_pairs=2, frac=1.0)
    tags = np.ones_like(sc.tags)
    lab, nc = oracle.labels(sc.n, sc.edges, tags)
    assert nc == 1
    H = oracle.fine_system_csr_blocks(sc)
    X = sc.meta["X_rest"]
    rng = np.random.default_rng(5)
    Aff, b = rng.standard_normal((3, 3)), rng.standard_normal(3)
    dx_star = X @ Aff.T + b
    sc.g = -(H @ dx_star.reshape(-1)).reshape(-1, 3)
    out = affine.solve(sc, lab, nc, threshold=4)
    assert out["plan"]["n_rows"] == 4
    assert np.abs(out["dx"] - dx_star).max() <= 1e-9 * np.abs(dx_star).max()
    # the 3-DoF coarsening cannot: it only moves the body rigidly
    plain = affine.solve(sc, lab, nc, threshold=10 ** 6)
    assert np.abs(plain["dx"] - dx_star).max() > 1e-3 * np.abs(dx_star).max()


def test_galerkin_orthogonality_and_symmetry():
    sc = scenes.unit_cube(seed=1001)
    lab, nc = oracle.labels(sc.n, sc.edges, sc.tags)
    out = affine.solve(sc, lab, nc, threshold=32)
    pl = out["plan"]
    assert pl["affine"].any() and (~pl["affine"]).any()
    Hc = out["Hc"].toarray()
    assert np.abs(Hc - Hc.T).max() <= 1e-12 * np.abs(Hc).max()
    assert np.linalg.eigvalsh(Hc).min() > 0
    H = oracle.fine_system_csr_blocks(sc)
    res = out["P"].T @ (H @ out["dx"].reshape(-1) + sc.g.reshape(-1))
    assert np.abs(res).max() <= 1e-9 * np.abs(out["P"].T @ sc.g.reshape(-1)).max()
