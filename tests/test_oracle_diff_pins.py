"""Pins of the differentiation-form oracle (CPU only).

The StVK element routine is pinned to its energy by finite differences and
to a hand-computed uniaxial stretch; the projection to eigenvalue facts; the
adjoint gradients to central differences of the whole oracle step (with the
coarse solve converged to machine precision on a small mesh)."""
import numpy as np
import pytest

import oracle
from oracle import adjoint as A
from paper_2605_04773_gb300 import scenes

NU = 0.4


def _random_tet(rng, scale=1.0, strain=0.2):
    X = scale * rng.standard_normal((4, 3))
    while abs(np.linalg.det(X[1:] - X[0])) < 0.05 * scale ** 3:
        X = scale * rng.standard_normal((4, 3))
    return X, X + strain * scale * rng.standard_normal((4, 3))


def test_uniaxial_stretch_energy():
    # Unit right tet, x = diag(s, 1, 1) X: F = diag(s, 1, 1),
    # G = diag((s^2 - 1)/2, 0, 0), Psi = V (mu G00^2 + lam/2 G00^2), V = 1/6.
    X = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1]], dtype=float)
    s, E = 1.3, 2e5
    x = X * np.array([s, 1.0, 1.0])
    mu = E / (2 * (1 + NU))
    lam = E * NU / ((1 + NU) * (1 - 2 * NU))
    G00 = 0.5 * (s * s - 1)
    psi, g, _ = A.stvk_element(X, x, E, NU)
    assert psi == pytest.approx((mu + 0.5 * lam) * G00 ** 2 / 6.0, rel=1e-14)
    # P = F S, S00 = (2 mu + lam) G00: the force on vertex 1 along x is V P00 w_1[0] = V s S00.
    assert g[3] == pytest.approx(s * (2 * mu + lam) * G00 / 6.0, rel=1e-13)
    assert g.reshape(4, 3).sum(0) == pytest.approx(np.zeros(3), abs=1e-9)


def test_gradient_and_hessian_match_finite_differences():
    rng = np.random.default_rng(11)
    for _ in range(3):
        X, x = _random_tet(rng)
        E = 1e5
        _, g, H = A.stvk_element(X, x, E, NU)
        h = 1e-6
        fg = np.zeros(12)
        fH = np.zeros((12, 12))
        for k in range(12):
            xp = x.reshape(-1).copy()
            xm = xp.copy()
            xp[k] += h
            xm[k] -= h
            ep, gp, _ = A.stvk_element(X, xp.reshape(4, 3), E, NU)
            em, gm, _ = A.stvk_element(X, xm.reshape(4, 3), E, NU)
            fg[k] = (ep - em) / (2 * h)
            fH[:, k] = (gp - gm) / (2 * h)
        assert np.abs(fg - g).max() <= 1e-8 * np.abs(g).max()
        assert np.abs(fH - H).max() <= 1e-8 * np.abs(H).max()
        assert np.abs(H - H.T).max() <= 1e-14 * np.abs(H).max()


def test_element_invariances():
    rng = np.random.default_rng(12)
    X, x = _random_tet(rng)
    # rest state: no energy, no force
    psi0, g0, _ = A.stvk_element(X, X, 1e5, NU)
    assert abs(psi0) < 1e-20 and np.abs(g0).max() < 1e-9
    psi, g, H = A.stvk_element(X, x, 1e5, NU)
    # translations are in the Hessian's null space and carry no net force
    for c in range(3):
        t = np.zeros((4, 3))
        t[:, c] = 1.0
        assert np.abs(H @ t.reshape(-1)).max() <= 1e-12 * np.abs(H).max()
        assert abs(g.reshape(4, 3)[:, c].sum()) <= 1e-12 * np.abs(g).max()
    # a rigid rotation of x leaves the energy unchanged
    q, _ = np.linalg.qr(rng.standard_normal((3, 3)))
    q *= np.sign(np.linalg.det(q))
    psi_r, _, _ = A.stvk_element(X, x @ q.T, 1e5, NU)
    assert psi_r == pytest.approx(psi, rel=1e-12)
    # linear in E at fixed nu
    psi2, g2, H2 = A.stvk_element(X, x, 3e5, NU)
    assert psi2 == pytest.approx(3 * psi, rel=1e-14)
    assert np.allclose(H2, 3 * H, rtol=1e-14, atol=0)


def test_psd_projection():
    rng = np.random.default_rng(13)
    Q, _ = np.linalg.qr(rng.standard_normal((12, 12)))
    lam = np.linspace(-3, 8, 12)
    H = Q @ np.diag(lam) @ Q.T
    Hp = A.psd_project(H)
    assert np.allclose(Hp, Q @ np.diag(np.maximum(lam, 0)) @ Q.T, atol=1e-13)
    assert np.linalg.eigvalsh(Hp).min() > -1e-13
    assert np.allclose(A.psd_project(Hp), Hp, atol=1e-13)
    P = Q @ np.diag(np.abs(lam) + 0.1) @ Q.T
    assert np.allclose(A.psd_project(P), P, atol=1e-13)


def test_fine_assembly_matches_generator_and_slow_path():
    sc = scenes.tiny_box(seed=7, nx=3, ny=2, nz=2, n_pairs=3, frac=0.3)
    pr = scenes.diff_problem(sc)
    f = A.forward(pr, pr["E"], pr["X_rest"], tol=1e-12, with_terms=True)
    # the generator sums the same physics with its own code
    assert np.abs(f["fine_val"] - sc.val).max() <= 1e-12 * np.abs(sc.val).max()
    assert np.abs(f["g"] - sc.g).max() <= 1e-12 * np.abs(sc.g).max()
    slow = A.fine_upper(pr["n"], pr["tets"], pr["row_ptr"], pr["col"], f["elem_hess"], pr["mass_h2"])
    assert np.abs(slow - f["fine_val"]).max() <= 1e-13 * np.abs(slow).max()


def _loss(pr, E, X):
    f = A.forward(pr, E, X, tol=1e-14, max_iter=10000)
    assert f["converged"]
    return float(np.sum((f["x_next"] - pr["x_target"]) ** 2)), f


@pytest.fixture(scope="module")
def tiny_adjoint():
    sc = scenes.tiny_box(seed=7, nx=3, ny=3, nz=2, n_pairs=3, frac=0.3)
    pr = scenes.diff_problem(sc)
    L0, f = _loss(pr, pr["E"], pr["X_rest"])
    assert 1 < f["n_c"] < pr["n"]
    ad = A.adjoint(pr, pr["E"], pr["X_rest"], f, 2 * (f["x_next"] - pr["x_target"]), tol=1e-14)
    assert ad["converged"]
    return pr, f, ad


def test_dL_dE_matches_global_central_differences(tiny_adjoint):
    pr, f, ad = tiny_adjoint
    E0 = pr["E"]
    # tets inside one super-node are invisible to the coarse step: zero gradient
    inside = np.all(f["labels"][pr["tets"]] == f["labels"][pr["tets"][:, :1]], axis=1)
    assert inside.any() and (~inside).any()
    scale = np.abs(ad["dL_dE"]).max()
    assert np.abs(ad["dL_dE"][inside]).max() <= 1e-10 * scale
    rng = np.random.default_rng(3)
    for e in rng.choice(np.nonzero(~inside)[0], 6, replace=False):
        d = 1e-5 * E0[e]
        Ep, Em = E0.copy(), E0.copy()
        Ep[e] += d
        Em[e] -= d
        fd = (_loss(pr, Ep, pr["X_rest"])[0] - _loss(pr, Em, pr["X_rest"])[0]) / (2 * d)
        assert abs(fd - ad["dL_dE"][e]) <= 1e-6 * scale


def test_dL_dX_rest_matches_global_central_differences(tiny_adjoint):
    pr, f, ad = tiny_adjoint
    X0 = pr["X_rest"]
    scale = np.abs(ad["dL_dX"]).max()
    rng = np.random.default_rng(4)
    for v in rng.choice(pr["n"], 4, replace=False):
        for c in range(3):
            d = 1e-7
            Xp, Xm = X0.copy(), X0.copy()
            Xp[v, c] += d
            Xm[v, c] -= d
            fd = (_loss(pr, pr["E"], Xp)[0] - _loss(pr, pr["E"], Xm)[0]) / (2 * d)
            assert abs(fd - ad["dL_dX"][v, c]) <= 1e-6 * scale


def test_all_protected_adjoint_is_the_fine_adjoint():
    # with every edge protected U = I: lambda solves the fine system H lambda = v
    sc = scenes.tiny_box(seed=8, nx=2, ny=2, nz=1, n_pairs=2, frac=0.0)
    pr = scenes.diff_problem(sc)
    f = A.forward(pr, pr["E"], pr["X_rest"], tol=1e-14, max_iter=10000)
    assert f["n_c"] == pr["n"]
    v = 2 * (f["x_next"] - pr["x_target"])
    ad = A.adjoint(pr, pr["E"], pr["X_rest"], f, v, tol=1e-14)
    rp, ci, val = oracle.fine_system(sc)
    H = np.zeros((3 * pr["n"], 3 * pr["n"]))
    for i in range(pr["n"]):
        for k in range(rp[i], rp[i + 1]):
            H[3 * i:3 * i + 3, 3 * ci[k]:3 * ci[k] + 3] = val[k]
    lam = np.linalg.solve(H, v.reshape(-1))
    assert np.abs(lam - ad["lam"].reshape(-1)).max() <= 1e-9 * np.abs(lam).max()
