"""Pins of the Green-strain-increment tagging oracle (CPU only)."""
import numpy as np

from oracle import tagging
from paper_2605_04773_gb300 import scenes

THR = 5e-5


def _tet():
    X = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1]], dtype=float)
    return X, np.array([[0, 1, 2, 3]]), scenes.mesh_edges(np.array([[0, 1, 2, 3]]))


def test_green_strain_of_a_stretch():
    # F = diag(s1, s2, s3)  =>  G = diag((s_i^2 - 1) / 2)
    X, tets, _ = _tet()
    s = np.array([1.1, 0.9, 1.3])
    G = tagging.green_strain(X, X * s, tets)[0]
    assert np.allclose(G, np.diag(0.5 * (s * s - 1)), atol=1e-15)


def test_threshold_on_a_single_tet():
    X, tets, edges = _tet()
    # uniaxial stretch s: ||dG||_F = (s^2 - 1) / 2
    for factor, expect in ((2.0, 0), (0.5, 1)):
        s = np.sqrt(1 + 2 * factor * THR)
        x1 = X * np.array([s, 1.0, 1.0])
        tags, norm = tagging.strain_tags(X, X, x1, tets, edges, THR)
        assert abs(norm[0] - factor * THR) <= 1e-12
        assert np.all(tags == expect)


def test_rigid_motion_keeps_every_edge_collapsible():
    sc = scenes.tiny_box(seed=31, nx=2, ny=2, nz=2)
    X, x, tets = sc.meta["X_rest"], sc.meta["x"], sc.meta["tets"]
    rng = np.random.default_rng(3)
    Q, _ = np.linalg.qr(rng.standard_normal((3, 3)))
    Q *= np.sign(np.linalg.det(Q))
    x1 = x @ Q.T + rng.standard_normal(3)
    tags, norm = tagging.strain_tags(X, x, x1, tets, sc.edges, THR)
    assert norm.max() < 1e-12
    assert np.all(tags == 1)


def test_moving_one_vertex_protects_exactly_its_tets_edges():
    sc = scenes.tiny_box(seed=32, nx=3, ny=3, nz=3)
    X, x, tets = sc.meta["X_rest"], sc.meta["x"], sc.meta["tets"]
    v = 21
    x1 = x.copy()
    x1[v] += np.array([0.02, -0.01, 0.015])   # large against THR for every tet around v
    tags, _ = tagging.strain_tags(X, x, x1, tets, sc.edges, THR)
    around = tets[np.any(tets == v, axis=1)]
    expect = set()
    for t in around:
        for i in range(4):
            for j in range(i + 1, 4):
                expect.add((min(t[i], t[j]), max(t[i], t[j])))
    got = {tuple(e) for e, tg in zip(sc.edges.tolist(), tags) if tg == 0}
    assert got == expect
