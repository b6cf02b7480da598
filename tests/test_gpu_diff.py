"""GPU parity of the differentiation form (fine StVK assembly, adjoint
re-solve and per-element VJP) against the CPU oracle, through the C ABI."""
import numpy as np
import pytest

import oracle
from oracle import adjoint as A
from paper_2605_04773_gb300 import scenes

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _agipc():
    from paper_2605_04773_gb300 import agipc
    return agipc


def _run_gpu(pr, tol, adjoint_tol=None, E=None, X=None):
    agipc = _agipc()
    dp = agipc.DiffDeviceProblem(pr)
    ctx = dp.context()
    step = agipc.DiffStep(ctx, dp, tol=tol, adjoint_tol=adjoint_tol)
    dev = dp.x.device
    E = torch.tensor(pr["E"] if E is None else E, dtype=torch.float64, device=dev, requires_grad=True)
    X = torch.tensor(pr["X_rest"] if X is None else X, dtype=torch.float64, device=dev, requires_grad=True)
    xt = torch.tensor(pr["x_target"], dtype=torch.float64, device=dev)
    x_next = agipc.coarsened_step(E, X, step)
    L = ((x_next - xt) ** 2).sum()
    dE, dX = torch.autograd.grad(L, [E, X])
    rc = ctx.status()
    out = dict(rc=rc, L=float(L.item()), x_next=x_next.detach().cpu().numpy(), dE=dE.cpu().numpy(),
               dX=dX.cpu().numpy(), fine_val=step.fine_val.cpu().numpy().reshape(-1, 3, 3),
               g=step.g.cpu().numpy(), lam=step.lam.cpu().numpy(), dx=step.dx.cpu().numpy(),
               labels=step.labels.cpu().numpy(), iters=int(step.iters.item()), relres=float(step.relres.item()),
               adj_iters=int(step.adj_iters.item()), adj_relres=float(step.adj_relres.item()))
    ctx.close()
    return out


def _rel(a, b, floor=1e-300):
    return float(np.abs(a - b).max() / max(np.abs(b).max(), floor))


@pytest.mark.parametrize("case", ["unit_cube", "tiny_all_protected", "tiny_one_node"])
def test_diff_step_matches_oracle(case):
    if case == "unit_cube":
        sc = scenes.unit_cube(seed=1001)
    elif case == "tiny_all_protected":
        sc = scenes.tiny_box(seed=8, nx=2, ny=2, nz=1, n_pairs=2, frac=0.0)
    else:
        sc = scenes.tiny_box(seed=9, nx=2, ny=2, nz=2, n_pairs=2, frac=1.0)
    pr = scenes.diff_problem(sc)
    got = _run_gpu(pr, tol=1e-12)
    assert got["rc"] == 0, got["rc"]
    f = A.forward(pr, pr["E"], pr["X_rest"], tol=1e-12, with_terms=True)
    assert np.array_equal(got["labels"], f["labels"])
    # fine assembly from elements: same blocks, same gradient
    assert _rel(got["fine_val"], f["fine_val"]) <= 1e-12
    assert _rel(got["g"], f["g"]) <= 1e-12
    assert _rel(got["x_next"] - pr["x"], f["dx"]) <= 1e-8
    ad = A.adjoint(pr, pr["E"], pr["X_rest"], f, 2 * (f["x_next"] - pr["x_target"]), tol=1e-12)
    assert _rel(got["lam"], ad["lam"]) <= 1e-8
    # gradient scales: L spread evenly over the parameters (a tet lying inside
    # one super-node has an exactly zero E-gradient, so the one-node case is
    # all zeros)
    nt = pr["tets"].shape[0]
    floor_E = got["L"] / (pr["E"].mean() * nt)
    floor_X = got["L"] / pr["n"]
    assert _rel(got["dE"], ad["dL_dE"], floor_E) <= 1e-7
    assert _rel(got["dX"], ad["dL_dX"], floor_X) <= 1e-7


@pytest.fixture(scope="module")
def diff_grid_run():
    sc = scenes.diff_grid()
    pr = scenes.diff_problem(sc)
    return pr, _run_gpu(pr, tol=1e-10)


def test_full_size_vjp_matches_element_central_differences(diff_grid_run):
    # 46^3 grid: at the GPU's own adjoint lambda and step dx, the VJP must
    # equal central differences (eps 1e-6) of the oracle's element routine
    # on 32 random tets that straddle super-nodes and on 32 random vertices,
    # to 1e-5 of the sample's largest entry.  The rest-position derivative
    # goes through the eigenvalue clamp, whose divided differences vary fast
    # when a positive and a negative eigenvalue are both near zero; there the
    # difference quotient's own truncation error, estimated by
    # |FD(eps) - FD(eps/10)|, is added to the tolerance.
    pr, got = diff_grid_run
    assert got["rc"] == 0, got["rc"]
    rng = np.random.default_rng(2024)
    tets = pr["tets"]
    straddle = np.nonzero(~np.all(got["labels"][tets] == got["labels"][tets[:, :1]], axis=1))[0]
    elems = rng.choice(straddle, 32, replace=False)
    verts = rng.choice(pr["n"], 32, replace=False)
    dE_ref, dX_ref = A.vjp(pr, pr["E"], pr["X_rest"], got["lam"], got["dx"], eps=1e-6, vertices=verts,
                           elements=elems)
    _, dX_fine = A.vjp(pr, pr["E"], pr["X_rest"], got["lam"], got["dx"], eps=1e-7, vertices=verts,
                       elements=elems[:1])
    sE = np.abs(dE_ref[elems]).max()
    sX = np.abs(dX_ref[verts]).max()
    assert np.abs(got["dE"][elems] - dE_ref[elems]).max() <= 1e-5 * sE
    trunc = np.abs(dX_ref[verts] - dX_fine[verts])
    assert np.all(np.abs(got["dX"][verts] - dX_ref[verts]) <= 1e-5 * sX + trunc)


def test_full_size_gradient_matches_oracle(diff_grid_run):
    pr, got = diff_grid_run
    assert got["rc"] == 0, got["rc"]
    assert got["relres"] <= 1.01e-10 and got["adj_relres"] <= 1.01e-10
    f = A.forward(pr, pr["E"], pr["X_rest"], tol=1e-10, with_terms=True)
    assert np.array_equal(got["labels"], f["labels"])
    assert _rel(got["fine_val"], f["fine_val"]) <= 1e-12
    rng = np.random.default_rng(7)
    verts = rng.choice(pr["n"], 32, replace=False)
    v = 2 * (f["x_next"] - pr["x_target"])
    ad = A.adjoint(pr, pr["E"], pr["X_rest"], f, v, tol=1e-10, vertices=verts, eps=1e-6)
    ad7 = A.adjoint(pr, pr["E"], pr["X_rest"], f, v, tol=1e-10, vertices=verts, eps=1e-7, elements=[0])
    # both solves stop at 1e-10 relative residual: the gradients agree to the
    # solves' accuracy times the conditioning, far below the 1e-5 target; the
    # oracle's rest-position gradient is a central difference, whose own
    # truncation error |FD(1e-6) - FD(1e-7)| is added to the tolerance
    assert _rel(got["x_next"] - pr["x"], f["dx"]) <= 1e-6
    assert _rel(got["dE"], ad["dL_dE"]) <= 1e-5
    sX = np.abs(ad["dL_dX"][verts]).max()
    trunc = np.abs(ad["dL_dX"][verts] - ad7["dL_dX"][verts])
    assert np.all(np.abs(got["dX"][verts] - ad["dL_dX"][verts]) <= 1e-5 * sX + trunc)


def test_full_size_adjoint_matches_central_differences_of_L(diff_grid_run):
    # dL/dE and dL/dX_rest from the adjoint re-solve against central
    # differences of L = |x_next - x_target|^2 itself, each L evaluated by the
    # GPU forward step (fine StVK assembly, the same labels, coarse assembly,
    # PCG to 1e-12, prolongation) on the 46^3 grid.  A single tet moves L by
    # about 3.5e-13 of its value when its E changes by 1e-6, below the FP64
    # rounding noise of the solve, so the differences are taken along
    # directions over many parameters at once: d = E o sign(dL/dE) on all
    # tets and on three random halves of them (eps = 1e-6 relative), and
    # d = cell o sign(dL/dX) on all rest coordinates and a random half (eps =
    # 1e-7).  Scaling E leaves the PSD clamp's eigenvectors unchanged, so L is
    # smooth along the E directions.
    agipc = _agipc()
    pr, _ = diff_grid_run
    dp = agipc.DiffDeviceProblem(pr)
    ctx = dp.context()
    dev = dp.x.device
    step = agipc.DiffStep(ctx, dp, tol=1e-12)
    xt = torch.tensor(pr["x_target"], dtype=torch.float64, device=dev)
    X0 = torch.tensor(pr["X_rest"], dtype=torch.float64, device=dev)
    E0 = torch.tensor(pr["E"], dtype=torch.float64, device=dev)

    def L_of(E, X):
        d = (step.forward(E, X) - xt).reshape(-1)
        assert ctx.status() == agipc.OK
        return float(torch.dot(d, d).item())

    v = 2 * (step.forward(E0, X0) - xt)
    step.backward(v)
    assert ctx.status() == agipc.OK
    dE, dX = step.dL_dE.clone(), step.dL_dX.clone()
    rng = np.random.default_rng(31)
    cell = 1.0 / 46
    dirs_E = [torch.sign(dE) * E0]
    for _ in range(3):
        mask = torch.tensor(rng.random(dE.numel()) < 0.5, device=dev)
        dirs_E.append(torch.sign(dE) * E0 * mask)
    for d in dirs_E:
        eps = 1e-6
        fd = (L_of(E0 + eps * d, X0) - L_of(E0 - eps * d, X0)) / (2 * eps)
        adj = float(torch.dot(dE, d).item())
        assert abs(fd - adj) <= 1e-5 * abs(adj), (fd, adj)
    dirs_X = [torch.sign(dX) * cell,
              torch.sign(dX) * cell * torch.tensor(rng.random(dX.shape) < 0.5, device=dev)]
    for d in dirs_X:
        eps = 1e-7
        fd = (L_of(E0, X0 + eps * d) - L_of(E0, X0 - eps * d)) / (2 * eps)
        adj = float(torch.dot(dX.reshape(-1), d.reshape(-1)).item())
        assert abs(fd - adj) <= 1e-5 * abs(adj), (fd, adj)
    ctx.close()


def test_bad_tet_index_sets_status():
    agipc = _agipc()
    sc = scenes.tiny_box(seed=10, nx=1, ny=1, nz=1, n_pairs=0)
    pr = scenes.diff_problem(sc)
    pr["tets"] = pr["tets"].copy()
    pr["tets"][0, 2] = pr["n"] + 5
    dp = agipc.DiffDeviceProblem(pr)
    ctx = dp.context()
    step = agipc.DiffStep(ctx, dp, tol=1e-8)
    E = torch.tensor(pr["E"], dtype=torch.float64, device=dp.x.device)
    X = torch.tensor(pr["X_rest"], dtype=torch.float64, device=dp.x.device)
    agipc.agipc_fine_assemble_stvk(ctx, dp.n, dp.tets, X, dp.x, dp.xhat_shift, E, dp.nu, dp.mass_h2, None,
                                   dp.row_ptr, dp.col, step.fine_val, step.g, step.workspace)
    assert ctx.status() == agipc.ERR_BAD_INDEX
    ctx.close()
