"""GPU parity of the Newton loop (Algorithm 1's inner loop): the energy
kernel, |d|_inf and the whole coarsened Newton loop with backtracking against
the oracle, through the C ABI."""
import numpy as np
import pytest

import oracle
from oracle import newton as N
from oracle.adjoint import GRAVITY
from oracle.tagging import strain_tags
from paper_2605_04773_gb300 import scenes

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _agipc():
    from paper_2605_04773_gb300 import agipc
    return agipc


def _setup(pr):
    agipc = _agipc()
    dp = agipc.DiffDeviceProblem(pr)
    ctx = dp.context()
    dev = dp.x.device
    E = torch.tensor(np.asarray(pr["E"], dtype=np.float64), device=dev)
    X = torch.tensor(pr["X_rest"], dtype=torch.float64, device=dev)
    return agipc, dp, ctx, E, X


@pytest.mark.parametrize("n_cells", [5, 46])
def test_energy_matches_oracle(n_cells):
    sc = scenes.diff_grid(n_cells=n_cells)
    pr = scenes.newton_problem(sc)
    pr["x"] = sc.meta["x"]          # a strained configuration (the scene's displaced positions)
    agipc, dp, ctx, E, X = _setup(pr)
    e = torch.zeros(1, dtype=torch.float64, device=dp.x.device)
    agipc.agipc_stvk_energy(ctx, dp.n, dp.tets, X, dp.x, None, 0.0, dp.xhat_shift, E, dp.nu, dp.mass_h2, dp.g_extra,
                            None, e)
    assert ctx.status() == 0
    want = N.energy(pr, pr["E"], pr["X_rest"], pr["x"])
    assert abs(e.item() - want) <= 1e-12 * abs(want)
    # a trial point x0 + alpha d, written out
    rng = np.random.default_rng(11)
    d = 1e-3 * rng.standard_normal((dp.n, 3))
    alpha = 0.375
    dd = torch.tensor(d, device=dp.x.device)
    xo = torch.empty_like(dp.x)
    agipc.agipc_stvk_energy(ctx, dp.n, dp.tets, X, dp.x, dd, alpha, dp.xhat_shift, E, dp.nu, dp.mass_h2, dp.g_extra,
                            xo, e)
    assert ctx.status() == 0
    xt = pr["x"] + alpha * d
    assert np.array_equal(xo.cpu().numpy(), xt)
    want = N.energy(pr, pr["E"], pr["X_rest"], xt)
    assert abs(e.item() - want) <= 1e-12 * abs(want)
    # deterministic: same bits again
    e2 = torch.zeros_like(e)
    agipc.agipc_stvk_energy(ctx, dp.n, dp.tets, X, dp.x, dd, alpha, dp.xhat_shift, E, dp.nu, dp.mass_h2, dp.g_extra,
                            None, e2)
    assert e2.item() == e.item()
    ctx.close()


def test_energy_rejects_bad_tets_and_aliasing():
    sc = scenes.diff_grid(n_cells=3)
    pr = scenes.newton_problem(sc)
    agipc, dp, ctx, E, X = _setup(pr)
    e = torch.zeros(1, dtype=torch.float64, device=dp.x.device)
    bad = dp.tets.clone()
    bad[5, 2] = dp.n
    agipc.agipc_stvk_energy(ctx, dp.n, bad, X, dp.x, None, 0.0, dp.xhat_shift, E, dp.nu, dp.mass_h2, None, None, e)
    assert ctx.status() == agipc.ERR_BAD_INDEX
    with pytest.raises(agipc.AgipcError):
        agipc.agipc_stvk_energy(ctx, dp.n, dp.tets, X, dp.x, None, 0.0, dp.xhat_shift, E, dp.nu, dp.mass_h2, None,
                                dp.x, e)
    ctx.close()


@pytest.mark.parametrize("m", [0, 1, 31, 1000, 3 * 103823])
def test_max_abs_is_exact(m):
    agipc = _agipc()
    ctx = agipc.Context(max(m, 1), 1, max(m, 1), 1)
    rng = np.random.default_rng(m)
    v = rng.standard_normal(m) * np.exp(rng.uniform(-30, 30, m))
    if m > 2:
        v[m // 2] = -np.abs(v).max() * 1.5     # the largest magnitude is negative
    t = torch.tensor(v, device="cuda")
    out = torch.full((1,), -1.0, dtype=torch.float64, device="cuda")
    agipc.agipc_max_abs(ctx, t, out)
    assert ctx.status() == 0
    assert out.item() == (np.abs(v).max() if m else 0.0)
    ctx.close()


def test_newton_loop_matches_oracle():
    sc = scenes.diff_grid(n_cells=6)
    pr = scenes.newton_problem(sc)
    agipc, dp, ctx, E, X = _setup(pr)
    x_last = torch.tensor(pr["x_last"], device=dp.x.device)
    tol = 1e-10
    sol = agipc.NewtonSolver(ctx, dp, E, X, x_last, tol=tol)
    got = sol.run(keep_labels=True)
    want = N.newton(pr, pr["E"], pr["X_rest"], pr["x_last"], tol=tol)
    assert got["converged"] and want["converged"]
    assert len(got["history"]) == len(want["history"])
    for a, b in zip(got["history"], want["history"]):
        assert a["n_c"] == b["n_c"]
        assert np.array_equal(a["labels"], b["labels"])
        assert a["alpha"] == b["alpha"] and a["trials"] == b["trials"]
        assert abs(a["e_prev"] - b["e_prev"]) <= 1e-11 * abs(b["e_prev"])
        assert a["post_iters"] == b["post_iters"]
        assert np.abs(a["d"] - b["d"]).max() <= 1e-7 * np.abs(b["d"]).max()
        assert abs(a["dnorm"] - b["dnorm"]) <= 1e-7 * b["dnorm"]
    xg = got["x"].cpu().numpy()
    assert np.abs(xg - want["x"]).max() <= 1e-9 * np.abs(want["x"]).max()
    ctx.close()


def test_pure_inertia_newton_lands_on_x_hat():
    sc = scenes.diff_grid(n_cells=4)
    pr = scenes.newton_problem(sc)
    pr["E"] = np.zeros(pr["tets"].shape[0])
    agipc, dp, ctx, E, X = _setup(pr)
    # a noisy previous step: every tet's strain increment is nonzero, so
    # threshold 0 protects every edge
    noise = 1e-3 * np.random.default_rng(5).standard_normal(pr["x"].shape)
    x_last = torch.tensor(pr["x"] + noise, device=dp.x.device)
    got = agipc.NewtonSolver(ctx, dp, E, X, x_last, threshold=0.0, tol=1e-14, post_iters=0).run()
    x_hat = pr["X_rest"] + pr["h"] * pr["v"] + pr["h"] ** 2 * GRAVITY
    assert got["converged"] and got["iterations"] == 2
    assert got["history"][0]["n_c"] == pr["n"] and got["history"][0]["alpha"] == 1.0
    assert np.abs(got["x"].cpu().numpy() - x_hat).max() <= 1e-13 * np.abs(x_hat).max()
    ctx.close()


def test_newton_full_size():
    # the 46^3 workload at the paper's tolerances (PCG 1e-3, eps_d = 1e-3 l)
    sc = scenes.diff_grid()
    pr = scenes.newton_problem(sc)
    agipc, dp, ctx, E, X = _setup(pr)
    x_last = torch.tensor(pr["x_last"], device=dp.x.device)
    sol = agipc.NewtonSolver(ctx, dp, E, X, x_last)
    got = sol.run(keep_labels=True)
    hist = got["history"]
    assert got["converged"] and not got["stalled"]
    e = [h_["e_prev"] for h_ in hist] + [hist[-1]["e_new"]]
    assert all(b < a for a, b in zip(e, e[1:]))
    assert hist[-1]["dnorm"] / pr["h"] <= sol.eps_d
    # first iteration: labels from the oracle's tags against the last step
    tags, _ = strain_tags(pr["X_rest"], pr["x_last"], pr["x"], pr["tets"], pr["edges"], 5e-5)
    lab, nc = oracle.labels(pr["n"], pr["edges"], tags)
    assert hist[0]["n_c"] == nc and np.array_equal(hist[0]["labels"], lab)
    assert 1 < nc < pr["n"]
    # the energies the loop compared, re-evaluated by the oracle along the path
    x = np.array(pr["x"])
    for h_ in hist:
        want = N.energy(pr, pr["E"], pr["X_rest"], x)
        assert abs(h_["e_prev"] - want) <= 1e-12 * abs(want)
        x = x + h_["alpha"] * h_["d"]
    assert np.abs(got["x"].cpu().numpy() - x).max() <= 1e-12 * np.abs(x).max()
    ctx.close()
