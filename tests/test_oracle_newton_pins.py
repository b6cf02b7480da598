"""Pins of the Newton-loop oracle (Algorithm 1's inner loop, Eq. 1-3) against
closed forms, invariances and finite differences of its own assembled
gradient, not against itself."""
import numpy as np
import pytest

from oracle import newton as N
from oracle.adjoint import GRAVITY
from paper_2605_04773_gb300 import scenes


def _small(n_cells=3, seed=1005):
    sc = scenes.diff_grid(seed=seed, n_cells=n_cells)
    return scenes.newton_problem(sc)


def test_energy_is_inertia_only_under_rigid_motion():
    pr = _small()
    X = pr["X_rest"]
    th = 0.7
    R = np.array([[np.cos(th), -np.sin(th), 0.0], [np.sin(th), np.cos(th), 0.0], [0.0, 0.0, 1.0]])
    x = X @ R.T + np.array([0.3, -0.1, 0.2])
    x_hat = X + pr["h"] ** 2 * GRAVITY
    want = 0.5 * np.sum(pr["mass_h2"] * np.sum((x - x_hat) ** 2, axis=1)) + np.sum(pr["g_extra"] * x)
    got = N.energy(pr, pr["E"], X, x)
    assert abs(got - want) <= 1e-12 * abs(want)


def test_energy_of_uniform_stretch_closed_form():
    pr = _small()
    X = pr["X_rest"]
    pr = dict(pr, g_extra=None)
    s = 1.03
    x = s * X
    E0, nu = 2.5e5, pr["nu"]
    mu, lam = E0 / (2 * (1 + nu)), E0 * nu / ((1 + nu) * (1 - 2 * nu))
    gs = 0.5 * (s * s - 1.0)
    vol = np.prod(X.max(0) - X.min(0))
    psi = vol * (mu * 3 * gs * gs + 0.5 * lam * (3 * gs) ** 2)
    x_hat = X + pr["h"] ** 2 * GRAVITY
    inertia = 0.5 * np.sum(pr["mass_h2"] * np.sum((x - x_hat) ** 2, axis=1))
    got = N.energy(pr, np.full(pr["tets"].shape[0], E0), X, x)
    assert abs(got - (inertia + psi)) <= 1e-11 * (inertia + psi)


def test_energy_central_differences_match_assembled_gradient():
    pr = _small()
    rng = np.random.default_rng(3)
    X = pr["X_rest"]
    x = X + 0.02 * rng.standard_normal(X.shape) / 3
    pr = dict(pr, x=x)
    g, _ = N.gradient_and_hessian(pr, pr["E"], X, x)
    eps = 1e-6
    for v in rng.choice(pr["n"], 6, replace=False):
        for c in range(3):
            xp, xm = x.copy(), x.copy()
            xp[v, c] += eps
            xm[v, c] -= eps
            fd = (N.energy(pr, pr["E"], X, xp) - N.energy(pr, pr["E"], X, xm)) / (2 * eps)
            assert abs(fd - g[v, c]) <= 1e-6 * np.abs(g).max(), (v, c, fd, g[v, c])


def test_backtracking_halves_until_decrease():
    # E(x) = (x - 1)^2 from x = 0 along d = 4: alpha 1 -> 9, 1/2 -> 1 (not < 1), 1/4 -> 0
    f = lambda a: (0.0 + a * 4.0 - 1.0) ** 2  # noqa: E731
    assert N.backtrack(f, 1.0, 30) == (0.25, 0.0, 3)
    # never below: gives up after max_halvings + 1 trials
    assert N.backtrack(lambda a: 2.0, 1.0, 5) == (None, None, 6)


def test_pure_inertia_newton_lands_on_x_hat():
    # E = 0: no elasticity, H = M/h^2; threshold 0 protects every edge, so
    # one iteration solves exactly for x_hat and the next step is zero
    pr = _small()
    X = pr["X_rest"]
    E0 = np.zeros(pr["tets"].shape[0])
    # a noisy previous step: every tet's strain increment is nonzero
    x_last = pr["x"] + 1e-3 * np.random.default_rng(5).standard_normal(pr["x"].shape)
    out = N.newton(pr, E0, X, x_last, threshold=0.0, tol=1e-14, post_iters=0)
    x_hat = X + pr["h"] * pr["v"] + pr["h"] ** 2 * GRAVITY
    assert out["converged"]
    assert len(out["history"]) == 2
    assert out["history"][0]["n_c"] == pr["n"] and out["history"][0]["alpha"] == 1.0
    assert np.abs(out["x"] - x_hat).max() <= 1e-13 * np.abs(x_hat).max()
    assert out["history"][1]["dnorm"] <= 1e-15


def test_newton_decreases_energy_and_converges():
    pr = _small(n_cells=5)
    out = N.newton(pr, pr["E"], pr["X_rest"], pr["x_last"], tol=1e-10)
    hist = out["history"]
    assert out["converged"] and not out["stalled"]
    e = [h_["e_prev"] for h_ in hist] + [hist[-1]["e_new"]]
    assert all(b < a for a, b in zip(e, e[1:]))
    assert hist[-1]["dnorm"] / pr["h"] <= out["eps_d"]
    # the first iteration protects only the impacted corner
    assert 1 < hist[0]["n_c"] < pr["n"]
    # the descent direction is one: g^T d < 0 at every iterate
    x = np.array(pr["x"])
    for h_ in hist:
        g, _ = N.gradient_and_hessian(pr, pr["E"], pr["X_rest"], x)
        assert np.sum(g * h_["d"]) < 0
        x = x + h_["alpha"] * h_["d"]


@pytest.mark.parametrize("post", [0, 10])
def test_full_resolution_newton_is_plain_newton(post):
    # threshold 0: every edge protected -> labels are the identity, the coarse
    # system is the fine one and the loop is plain Newton with PCG; the step
    # then solves H d = -g to the PCG tolerance
    pr = _small()
    x_last = pr["x"] + 1e-3 * np.random.default_rng(6).standard_normal(pr["x"].shape)
    out = N.newton(pr, pr["E"], pr["X_rest"], x_last, threshold=0.0, tol=1e-12, post_iters=post, max_newton=1)
    h0 = out["history"][0]
    assert h0["n_c"] == pr["n"]
    assert np.array_equal(h0["labels"], np.arange(pr["n"]))
    g, val = N.gradient_and_hessian(pr, pr["E"], pr["X_rest"], np.array(pr["x"]))
    import oracle
    rp, ci, cv = oracle.galerkin(np.arange(pr["n"], dtype=np.int32), pr["n"], pr["row_ptr"], pr["col"], val,
                                 np.zeros((0, 4), np.int32), np.zeros((0, 10, 3, 3)))
    res = oracle.spmv(rp, ci, cv, h0["d"]) + g
    assert np.linalg.norm(res) <= 1.05e-12 * np.linalg.norm(g)
