"""Pins of the CPU oracle against what the paper and the mathematics fix.

Each test ties one oracle function to something other than itself: the
supplement's worked hashing examples (tests/golden), closed forms, invariants,
dense linear algebra on element stencils, brute force on tiny graphs and
library routines (scipy) for textbook special cases.
"""
import itertools
import json
import os

import numpy as np
import pytest
import scipy.sparse
import scipy.sparse.csgraph
import scipy.sparse.linalg

import oracle
from paper_2605_04773_gb300 import scenes
from tests.dense_reference import aggregation_operator, bfs_labels, dense_fine_hessian, dense_from_bsr

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "supplement_hash_examples.json")


# ---------------------------------------------------------------- labels


def _hash_string(bits, group_size):
    return "".join("1" if (bits >> k) & 1 else "0" for k in reversed(range(group_size)))


@pytest.mark.parametrize("case", json.load(open(GOLDEN))["cases"], ids=lambda c: c["name"])
def test_supplement_worked_examples(case):
    """Supplement Sec. 1.2-1.3: the printed hashes, coarse counts and indices."""
    gs = case["group_size"]
    # the fixture's edge list reproduces the printed direct-neighbour hashes
    init = []
    for v in range(case["n"]):
        h = 1 << (v % gs)
        for (a, b), t in zip(case["edges"], case["tags"]):
            if t and v in (a, b):
                o = b if a == v else a
                if o // gs == v // gs:
                    h |= 1 << (o % gs)
        init.append(_hash_string(h, gs))
    assert init == case["initial_hashes"]
    lab, nc = oracle.labels(case["n"], np.array(case["edges"]), np.array(case["tags"]))
    assert lab.tolist() == case["labels"]
    assert nc == case["n_coarse"]
    # final hash of a node = its component's members inside the group
    for g0 in range(0, case["n"], gs):
        members = list(range(g0, min(g0 + gs, case["n"])))
        final = []
        for v in members:
            h = sum(1 << (u % gs) for u in members if lab[u] == lab[v])
            final.append(_hash_string(h, gs))
        assert final == case["final_hashes"][g0:g0 + gs]
        # footnote of Sec. 1.3: coarse nodes per group = distinct hash values
        assert len(set(final)) == len(set(lab[members].tolist()))


def test_all_collapsible_connected_body_is_one_supernode(unit_cube_scene):
    """Supplement Sec. 1.3: with every tag 1, Map(i) = 0 for all i."""
    sc = unit_cube_scene
    lab, nc = oracle.labels(sc.n, sc.edges, np.ones(sc.n_edges, np.uint8))
    assert nc == 1 and not lab.any()


def test_all_protected_is_identity(unit_cube_scene):
    """Tags all 0: no edge may be collapsed, every fine node is its own super-node."""
    sc = unit_cube_scene
    lab, nc = oracle.labels(sc.n, sc.edges, np.zeros(sc.n_edges, np.uint8))
    assert nc == sc.n and np.array_equal(lab, np.arange(sc.n))


def test_bruteforce_every_tag_pattern():
    """Every tag pattern of random graphs with <= 10 edges against BFS."""
    rng = np.random.default_rng(7)
    for trial in range(12):
        n = int(rng.integers(2, 9))
        allpairs = [(u, v) for u in range(n) for v in range(u + 1, n)]
        ne = int(rng.integers(1, min(10, len(allpairs)) + 1))
        sel = rng.choice(len(allpairs), size=ne, replace=False)
        edges = np.array([allpairs[k] for k in sel], dtype=np.int32)
        for tags in itertools.product([0, 1], repeat=ne):
            tags = np.array(tags, np.uint8)
            lab, nc = oracle.labels(n, edges, tags)
            ref, rnc = bfs_labels(n, edges, tags)
            assert nc == rnc and np.array_equal(lab, ref), (trial, edges.tolist(), tags.tolist())


def test_labels_match_scipy_components(unit_cube_scene):
    """Same partition as scipy's connected_components; labels ranked by the
    smallest member of each component."""
    sc = unit_cube_scene
    rng = np.random.default_rng(3)
    for frac in (0.2, 0.5, 0.7, 0.95):
        tags = (rng.random(sc.n_edges) < frac).astype(np.uint8)
        lab, nc = oracle.labels(sc.n, sc.edges, tags)
        e = sc.edges[tags == 1]
        A = scipy.sparse.coo_matrix((np.ones(len(e)), (e[:, 0], e[:, 1])), shape=(sc.n, sc.n))
        snc, slab = scipy.sparse.csgraph.connected_components(A, directed=False)
        assert nc == snc
        # same partition
        pairs = set(zip(lab.tolist(), slab.tolist()))
        assert len(pairs) == nc
        # canonical ranking: first occurrences appear in increasing label order
        _, first = np.unique(lab, return_index=True)
        assert np.all(np.diff(first) > 0) and first[0] == 0


def test_labels_permutation_invariant_partition(unit_cube_scene):
    sc = unit_cube_scene
    rng = np.random.default_rng(4)
    perm = rng.permutation(sc.n)
    inv = np.argsort(perm)
    lab, nc = oracle.labels(sc.n, sc.edges, sc.tags)
    lab2, nc2 = oracle.labels(sc.n, inv[sc.edges].astype(np.int32), sc.tags)
    assert nc == nc2
    # node v became inv[v]; partitions must agree
    assert len(set(zip(lab.tolist(), lab2[inv].tolist()))) == nc


def test_labels_reject_out_of_range_edge():
    with pytest.raises(oracle.OracleError):
        oracle.labels(3, np.array([[0, 3]]), np.array([1]))


# ---------------------------------------------------------------- coarse system


def test_fine_system_matches_dense_element_assembly(unit_cube_scene):
    """Identity labels: H_c is the full fine Hessian, rebuilt densely from
    the element stencils, inertia and barrier terms kappa b'' gd gd^T."""
    sc = unit_cube_scene
    crp, cci, cval = oracle.fine_system(sc)
    A = dense_from_bsr(crp, cci, cval)
    H = dense_fine_hessian(sc)
    assert np.abs(A - H).max() <= 1e-12 * np.abs(H).max()
    assert all(np.all(np.diff(cci[crp[i]:crp[i + 1]]) > 0) for i in range(sc.n))


def test_all_protected_reproduces_fine_blocks_exactly(unit_cube_scene):
    """All-protected tags: every fine block not touched by a stencil comes
    through bit for bit (single-term sums), and g_c == g exactly."""
    sc = unit_cube_scene
    lab, nc = oracle.labels(sc.n, sc.edges, np.zeros(sc.n_edges, np.uint8))
    crp, cci, cval = oracle.galerkin(lab, nc, sc.row_ptr, sc.col, sc.val, sc.pair_idx[:0], sc.pair_blk[:0])
    for i in range(sc.n):
        for k in range(sc.row_ptr[i], sc.row_ptr[i + 1]):
            j = sc.col[k]
            q = crp[i] + np.searchsorted(cci[crp[i]:crp[i + 1]], j)
            assert np.array_equal(cval[q], sc.val[k])
            q2 = crp[j] + np.searchsorted(cci[crp[j]:crp[j + 1]], i)
            assert np.array_equal(cval[q2], sc.val[k].T)
    assert np.array_equal(oracle.coarse_gradient(lab, nc, sc.g), sc.g)


def test_galerkin_projection_identity(unit_cube_scene):
    """Sec. 4.1: H_c = U H U^T.  Dense check with random u, v: u^T H_c v =
    (U^T u)^T H (U^T v), and the whole matrix to 1e-12 relative."""
    sc = unit_cube_scene
    H = dense_fine_hessian(sc)
    lab, nc = oracle.labels(sc.n, sc.edges, sc.tags)
    crp, cci, cval = oracle.galerkin(lab, nc, sc.row_ptr, sc.col, sc.val, sc.pair_idx, sc.pair_blk)
    Hc = dense_from_bsr(crp, cci, cval)
    P = aggregation_operator(lab, nc)
    ref = P.T @ H @ P
    assert np.abs(Hc - ref).max() <= 1e-12 * np.abs(ref).max()
    rng = np.random.default_rng(5)
    u, v = rng.standard_normal((2, 3 * nc))
    assert abs(u @ Hc @ v - (P @ u) @ H @ (P @ v)) <= 1e-12 * np.abs(ref).max() * np.abs(u).sum() * np.abs(v).sum()


def test_coarse_matrix_symmetric_spd(unit_cube_scene):
    """Supplement Sec. 5: the projected operator inherits SPD-ness."""
    sc = unit_cube_scene
    for frac in (0.0, 0.3, 0.7, 0.9):
        tags = scenes.tags_from_field(sc.edges, scenes.activity_field(sc.meta["X_rest"], np.random.default_rng(11)),
                                      frac) if frac > 0 else np.zeros(sc.n_edges, np.uint8)
        lab, nc = oracle.labels(sc.n, sc.edges, tags)
        crp, cci, cval = oracle.galerkin(lab, nc, sc.row_ptr, sc.col, sc.val, sc.pair_idx, sc.pair_blk)
        Hc = dense_from_bsr(crp, cci, cval)
        # rows (a, b) and (b, a) are summed in different orders: symmetric to rounding
        assert np.abs(Hc - Hc.T).max() <= 1e-14 * np.abs(Hc).max()
        assert np.linalg.eigvalsh(0.5 * (Hc + Hc.T)).min() > 0


def test_force_conservation(unit_cube_scene):
    """Coarsening conserves the total force: sum_c g_c = sum_f g_f."""
    sc = unit_cube_scene
    lab, nc = oracle.labels(sc.n, sc.edges, sc.tags)
    gc = oracle.coarse_gradient(lab, nc, sc.g)
    assert np.allclose(gc.sum(0), sc.g.sum(0), rtol=0, atol=1e-10 * np.abs(sc.g).sum())
    P = aggregation_operator(lab, nc)
    assert np.allclose(gc.ravel(), P.T @ sc.g.ravel(), rtol=0, atol=1e-12 * np.abs(sc.g).max())


def test_single_supernode_closed_form(unit_cube_scene):
    """One super-node: elastic and barrier terms are translation invariant
    (their distance gradients sum to zero), so H_c = (sum m / h^2) I_3 and
    g_c = sum m/h^2 (x - x_hat); the step is the mass-weighted mean offset."""
    sc = unit_cube_scene
    m = sc.meta
    lab, nc = oracle.labels(sc.n, sc.edges, np.ones(sc.n_edges, np.uint8))
    crp, cci, cval = oracle.galerkin(lab, nc, sc.row_ptr, sc.col, sc.val, sc.pair_idx, sc.pair_blk)
    M = m["mass"].sum() / m["h"] ** 2
    assert cci.tolist() == [0]
    assert np.abs(cval[0] - M * np.eye(3)).max() <= 1e-9 * M
    gc = oracle.coarse_gradient(lab, nc, sc.g)
    gexp = ((m["mass"] / m["h"] ** 2)[:, None] * (m["x"] - m["x_hat"])).sum(0)
    assert np.abs(gc[0] - gexp).max() <= 1e-9 * np.abs(sc.g).sum()
    dinv = oracle.block_jacobi(crp, cci, cval)
    y, it, rr, conv = oracle.pcg(crp, cci, cval, dinv, -gc, 1e-12, 10)
    assert conv and it <= 1
    assert np.allclose(y[0], -np.linalg.solve(cval[0], gc[0]), rtol=1e-12, atol=0)


# ---------------------------------------------------------------- solve


@pytest.mark.parametrize("dims", [(1, 1, 1), (2, 2, 2), (3, 2, 1)])
def test_pcg_matches_dense_direct_solve(dims):
    """Tiny meshes: coarse PCG against numpy's dense solve to 1e-10."""
    sc = scenes.tiny_box(seed=100 + sum(dims), nx=dims[0], ny=dims[1], nz=dims[2], n_pairs=3, frac=0.5)
    lab, nc = oracle.labels(sc.n, sc.edges, sc.tags)
    gc = oracle.coarse_gradient(lab, nc, sc.g)
    crp, cci, cval = oracle.galerkin(lab, nc, sc.row_ptr, sc.col, sc.val, sc.pair_idx, sc.pair_blk)
    dinv = oracle.block_jacobi(crp, cci, cval)
    y, it, rr, conv = oracle.pcg(crp, cci, cval, dinv, -gc, 1e-14, 1000)
    ref = np.linalg.solve(dense_from_bsr(crp, cci, cval), -gc.ravel())
    assert conv
    assert np.linalg.norm(y.ravel() - ref) <= 1e-10 * np.linalg.norm(ref)


def test_galerkin_orthogonality_with_fine_hessian(unit_cube_scene):
    """The prolongated step satisfies U (H U^T y + g) = 0 to the PCG
    tolerance, measured with the dense fine Hessian (ties assembly to solve)."""
    sc = unit_cube_scene
    r = oracle.coarsened_step(sc, tol=1e-10)
    H = dense_fine_hessian(sc)
    P = aggregation_operator(r["labels"], r["n_c"])
    res = P.T @ (H @ r["dx"].ravel() + sc.g.ravel())
    assert np.linalg.norm(res) <= 2e-10 * np.linalg.norm(P.T @ sc.g.ravel())
    assert np.array_equal(r["dx"], r["y"][r["labels"]])


def test_fine_pcg_matches_scipy_cg(unit_cube_scene):
    """Identity labels: block-Jacobi PCG against scipy's CG with the same
    preconditioner, both to tight tolerance."""
    sc = unit_cube_scene
    crp, cci, cval = oracle.fine_system(sc)
    dinv = oracle.block_jacobi(crp, cci, cval)
    x, it, rr, conv = oracle.pcg(crp, cci, cval, dinv, -sc.g, 1e-12, 10000)
    A = scipy.sparse.csr_matrix(dense_from_bsr(crp, cci, cval))
    Mb = scipy.sparse.block_diag([scipy.sparse.csr_array(d) for d in dinv], format="csr")
    xs, info = scipy.sparse.linalg.cg(A, -sc.g.ravel(), M=Mb, rtol=1e-12, maxiter=10000)
    assert conv and info == 0
    assert np.linalg.norm(x.ravel() - xs) <= 1e-9 * np.linalg.norm(xs)
    assert np.linalg.norm(A @ x.ravel() + sc.g.ravel()) <= 1.01e-12 * np.linalg.norm(sc.g)


def test_pcg_edge_cases(unit_cube_scene):
    sc = unit_cube_scene
    crp, cci, cval = oracle.fine_system(sc)
    dinv = oracle.block_jacobi(crp, cci, cval)
    x, it, rr, conv = oracle.pcg(crp, cci, cval, dinv, np.zeros((sc.n, 3)), 1e-8, 100)
    assert conv and it == 0 and not x.any()
    x, it, rr, conv = oracle.pcg(crp, cci, cval, dinv, -sc.g, 1e-8, 1)
    assert not conv and it == 1 and rr > 1e-8
    # restart from a converged answer: no further iterations
    x1, _, _, _ = oracle.pcg(crp, cci, cval, dinv, -sc.g, 1e-10, 10000)
    x2, it2, _, conv2 = oracle.pcg(crp, cci, cval, dinv, -sc.g, 1e-6, 100, x0=x1)
    assert conv2 and it2 == 0


def test_block_jacobi_inverts_diagonal(unit_cube_scene):
    sc = unit_cube_scene
    crp, cci, cval = oracle.fine_system(sc)
    dinv = oracle.block_jacobi(crp, cci, cval)
    for i in range(0, sc.n, 37):
        q = crp[i] + np.searchsorted(cci[crp[i]:crp[i + 1]], i)
        assert np.allclose(dinv[i] @ cval[q], np.eye(3), atol=1e-12)


def test_prolongation_is_transpose_of_restriction(unit_cube_scene):
    """Sec. 4.3: d_f = U^T d_c, and <U g, y> = <g, U^T y> (adjointness)."""
    sc = unit_cube_scene
    lab, nc = oracle.labels(sc.n, sc.edges, sc.tags)
    rng = np.random.default_rng(9)
    y = rng.standard_normal((nc, 3))
    dx = oracle.prolongate(lab, y)
    P = aggregation_operator(lab, nc)
    assert np.array_equal(dx.ravel(), P @ y.ravel())
    gc = oracle.coarse_gradient(lab, nc, sc.g)
    assert abs((gc * y).sum() - (sc.g * dx).sum()) <= 1e-10 * np.abs(sc.g).sum() * np.abs(y).max()
