"""CUDA path vs the CPU oracle, element by element, through the C ABI.

Labels and the coarse sparsity structure are integer work and must match
bit for bit.  Coarse blocks and the coarse gradient are FP64 sums whose
order differs from the oracle's: each entry must agree within 1e-12 times the
sum of the magnitudes of its contributions (the oracle applied to |H|), and
the whole matrix within 1e-12 in the Frobenius norm.  A PCG solution is
judged by its true FP64 residual with the oracle's H_c and g_c, which must be
within the requested tolerance (5 % slack for the recurrence-vs-true
residual gap).
"""
import copy

import numpy as np
import pytest
import torch

import oracle
from paper_2605_04773_gb300 import agipc, scenes

pytestmark = pytest.mark.gpu

VAL_RTOL = 1e-12


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2605_04773_gb300 import build
    build.build()
    agipc.load()


@pytest.fixture(scope="module")
def domino_full():
    return scenes.domino_grid(seed=1002)


def _run(sc, tags=None, tol=1e-8, max_iter=100000, assembly_run=None, streamed=False):
    ds = agipc.DeviceScene(sc)
    ctx = ds.context()
    if assembly_run is not None:
        ctx.set_assembly_run(assembly_run)
    step = agipc.CoarsenedStep(ctx, ds, tol=tol, max_iter=max_iter, streamed=streamed)
    if tags is not None:
        step.aggregate(torch.from_numpy(np.ascontiguousarray(tags, np.uint8)).cuda())
        step.assemble()
        step.solve()
        step.prolongate()
    else:
        step.run()
    rc = ctx.status()
    out = step.host()
    ctx.close()
    return rc, out


def _check_coarse(sc, got, tags):
    lab, nc = oracle.labels(sc.n, sc.edges, tags)
    assert got["n_c"] == nc
    assert np.array_equal(got["labels"], lab)
    crp, cci, cval = oracle.galerkin(lab, nc, sc.row_ptr, sc.col, sc.val, sc.pair_idx, sc.pair_blk)
    assert np.array_equal(got["row_ptr"], crp)
    assert np.array_equal(got["col"], cci)
    _, _, mag = oracle.galerkin(lab, nc, sc.row_ptr, sc.col, np.abs(sc.val), sc.pair_idx, np.abs(sc.pair_blk))
    err = np.abs(got["val"] - cval)
    assert np.all(err <= VAL_RTOL * mag + 1e-300), err.max()
    assert np.linalg.norm(got["val"] - cval) <= VAL_RTOL * np.linalg.norm(cval)
    # the GPU output mirrors its upper triangle: exactly symmetric
    for a in range(0, nc, max(1, nc // 64)):
        for k in range(crp[a], crp[a + 1]):
            b = cci[k]
            q = crp[b] + np.searchsorted(cci[crp[b]:crp[b + 1]], a)
            assert np.array_equal(got["val"][k], got["val"][q].T)
    gc = oracle.coarse_gradient(lab, nc, sc.g)
    gmag = oracle.coarse_gradient(lab, nc, np.abs(sc.g))
    assert np.all(np.abs(got["g_c"] - gc) <= VAL_RTOL * gmag + 1e-300)
    dinv = oracle.block_jacobi(crp, cci, cval)
    assert np.abs(got["dinv"] - dinv).max() <= 1e-10 * np.abs(dinv).max()
    return crp, cci, cval, gc


def _check_solve(got, crp, cci, cval, gc, tol):
    res = oracle.spmv(crp, cci, cval, got["y"]) + gc
    rel = np.linalg.norm(res) / np.linalg.norm(gc)
    assert rel <= 1.05 * tol, rel
    assert got["relres"] <= tol
    assert np.array_equal(got["dx"], got["y"][got["labels"]])
    return rel


# ------------------------------------------------------------------ labels


@pytest.mark.parametrize("pattern", ["scene", "none", "all", "random30", "random95"])
def test_labels_bit_exact_unit_cube(pattern):
    sc = scenes.unit_cube(seed=1001)
    rng = np.random.default_rng(21)
    tags = {"scene": sc.tags, "none": np.zeros(sc.n_edges, np.uint8), "all": np.ones(sc.n_edges, np.uint8),
            "random30": (rng.random(sc.n_edges) < 0.3).astype(np.uint8),
            "random95": (rng.random(sc.n_edges) < 0.95).astype(np.uint8)}[pattern]
    rc, got = _run(sc, tags)
    assert rc == agipc.OK
    _check_coarse(sc, got, tags)


@pytest.mark.parametrize("dims", [(1, 1, 1), (2, 3, 1), (3, 3, 3), (5, 1, 2), (7, 6, 5)])
def test_ragged_boxes_full_path(dims):
    """Node counts that are not multiples of the 32-node group, tiny systems."""
    sc = scenes.tiny_box(seed=300 + sum(dims), nx=dims[0], ny=dims[1], nz=dims[2], n_pairs=3, frac=0.6)
    rc, got = _run(sc, tol=1e-10)
    assert rc == agipc.OK
    crp, cci, cval, gc = _check_coarse(sc, got, sc.tags)
    _check_solve(got, crp, cci, cval, gc, 1e-10)


def test_labels_random_graph_any_edge_order():
    """Edges in random order and orientation, self-loops and duplicates."""
    rng = np.random.default_rng(5)
    n = 5000
    e = rng.integers(0, n, size=(12000, 2)).astype(np.int32)
    e = np.concatenate([e, e[:100], np.stack([np.arange(50), np.arange(50)], 1).astype(np.int32)])
    tags = (rng.random(e.shape[0]) < 0.5).astype(np.uint8)
    ctx = agipc.Context(n, e.shape[0], 1, 0)
    labels = torch.empty(n, dtype=torch.int32, device="cuda")
    nc = torch.zeros(1, dtype=torch.int32, device="cuda")
    agipc.agipc_aggregate(ctx, n, torch.from_numpy(e).cuda(), torch.from_numpy(tags).cuda(), labels, nc)
    assert ctx.status() == agipc.OK
    ref, rnc = oracle.labels(n, e, tags)
    assert int(nc.item()) == rnc and np.array_equal(labels.cpu().numpy(), ref)
    # repeat: bitwise identical whatever the scheduling
    labels2 = torch.empty_like(labels)
    agipc.agipc_aggregate(ctx, n, torch.from_numpy(e).cuda(), torch.from_numpy(tags).cuda(), labels2, nc)
    assert torch.equal(labels, labels2)
    ctx.close()


def test_labels_no_edges():
    ctx = agipc.Context(100, 1, 1, 0)
    labels = torch.empty(100, dtype=torch.int32, device="cuda")
    nc = torch.zeros(1, dtype=torch.int32, device="cuda")
    e = torch.zeros(0, 2, dtype=torch.int32, device="cuda")
    t = torch.zeros(0, dtype=torch.uint8, device="cuda")
    agipc.agipc_aggregate(ctx, 100, e, t, labels, nc)
    assert ctx.status() == agipc.OK
    assert int(nc.item()) == 100 and torch.equal(labels.cpu(), torch.arange(100, dtype=torch.int32))
    ctx.close()


# ------------------------------------------------------------------ full path


@pytest.mark.parametrize("streamed", [False, True])
def test_unit_cube_full_path_parity(streamed):
    # streamed: the 16-warp kernel on a 60-block coarse system, one ragged
    # slice for the whole GPU (every other warp idle)
    sc = scenes.unit_cube(seed=1001)
    rc, got = _run(sc, tol=1e-8, streamed=streamed)
    assert rc == agipc.OK
    crp, cci, cval, gc = _check_coarse(sc, got, sc.tags)
    _check_solve(got, crp, cci, cval, gc, 1e-8)
    ref = oracle.coarsened_step(sc, tol=1e-8)
    assert abs(got["iters"] - ref["iters"]) <= 2
    assert np.linalg.norm(got["dx"] - ref["dx"]) <= 1e-6 * np.linalg.norm(ref["dx"])


@pytest.mark.parametrize("cells", [8, 14])
def test_long_coarse_rows(cells):
    """One large interior aggregate wrapped in protected boundary vertices:
    its coarse row holds hundreds of blocks (spanning many warp lanes and
    several slices), next to many short rows, so the SpMV joins rows both
    ways (shuffle scan for long chains, the walk for short ones)."""
    sc = scenes.tiny_box(seed=77 + cells, nx=cells, ny=cells, nz=cells, n_pairs=4, frac=0.5)
    X = sc.meta["X_rest"]
    lo, hi = X.min(0), X.max(0)
    cell = (hi[0] - lo[0]) / cells
    interior = np.all((X > lo + 0.5 * cell) & (X < hi - 0.5 * cell), axis=1)
    tags = (interior[sc.edges[:, 0]] & interior[sc.edges[:, 1]]).astype(np.uint8)
    rc, got = _run(sc, tags, tol=1e-10)
    assert rc == agipc.OK
    crp, cci, cval, gc = _check_coarse(sc, got, tags)
    assert np.diff(crp).max() > 256   # longer than two 128-block slices
    _check_solve(got, crp, cci, cval, gc, 1e-10)


def test_single_supernode_and_all_protected():
    sc = scenes.unit_cube(seed=1003)
    rc, got = _run(sc, np.ones(sc.n_edges, np.uint8), tol=1e-12)
    assert rc == agipc.OK and got["n_c"] == 1
    crp, cci, cval, gc = _check_coarse(sc, got, np.ones(sc.n_edges, np.uint8))
    assert np.allclose(got["y"][0], -np.linalg.solve(cval[0], gc[0]), rtol=1e-10, atol=0)
    rc, got = _run(sc, np.zeros(sc.n_edges, np.uint8), tol=1e-8)
    assert rc == agipc.OK and got["n_c"] == sc.n
    crp, cci, cval, gc = _check_coarse(sc, got, np.zeros(sc.n_edges, np.uint8))
    _check_solve(got, crp, cci, cval, gc, 1e-8)


@pytest.mark.parametrize("assembly_run", [4, 8, 16, 32])
def test_domino_small_multibody(assembly_run):
    # every launch shape of the coarse reduction (terms per lane) meets the
    # same per-entry bar: only the order of the atomics changes
    sc = scenes.domino_grid(seed=77, gx=2, gy=2, dims=(3, 5, 8), n_pairs=2000)
    rc, got = _run(sc, tol=1e-8, assembly_run=assembly_run)
    assert rc == agipc.OK
    crp, cci, cval, gc = _check_coarse(sc, got, sc.tags)
    _check_solve(got, crp, cci, cval, gc, 1e-8)


def test_domino_full_size_parity(domino_full):
    """The 64-box, 145,600-vertex, 200k-stencil workload in the bench's launch
    configuration: labels and structure bit-exact, blocks to 1e-12, solve to
    1e-6 (true residual)."""
    sc = domino_full
    rc, got = _run(sc, tol=1e-6)
    assert rc == agipc.OK
    crp, cci, cval, gc = _check_coarse(sc, got, sc.tags)
    _check_solve(got, crp, cci, cval, gc, 1e-6)


@pytest.mark.parametrize("streamed", [False, True])
def test_fine_arm_full_size(domino_full, streamed):
    """Identity labels: the fine system in full storage and fine PCG to 1e-6,
    in both kernel layouts (2.28 M blocks: both stream it from HBM)."""
    sc = domino_full
    ds = agipc.DeviceScene(sc)
    ctx = ds.context()
    fs = agipc.FineStep(ctx, ds, tol=1e-6, streamed=streamed)
    fs.run()
    assert ctx.status() == agipc.OK
    got = fs.host()
    frp, fci, fval = oracle.fine_system(sc)
    assert np.array_equal(got["row_ptr"], frp) and np.array_equal(got["col"], fci)
    assert np.linalg.norm(got["val"] - fval) <= VAL_RTOL * np.linalg.norm(fval)
    res = oracle.spmv(frp, fci, fval, got["y"]) + sc.g
    assert np.linalg.norm(res) <= 1.05e-6 * np.linalg.norm(sc.g)
    ctx.close()


# ------------------------------------------------------------------ status / edge cases


def test_host_pipeline_matches_single_steps():
    """Steps fed from pinned host buffers through the two-buffer pipeline give
    the dx of plain steps on the same inputs (and every step's own inputs:
    the right-hand sides differ from step to step)."""
    sc = scenes.unit_cube(seed=1001)
    a, b = agipc.DeviceScene(sc), agipc.DeviceScene(sc)
    ctx = a.context()
    base = {f: getattr(a, f).cpu() for f in agipc.SCENE_INPUTS}
    host, outs = [], []
    for s in (1.0, 2.0, -0.5, 3.0):
        d = {f: t.clone().pin_memory() for f, t in base.items()}
        d["g"] = (base["g"] * s).pin_memory()
        host.append(d)
        outs.append(torch.empty(sc.n, 3, dtype=torch.float64).pin_memory())
    pipe = agipc.HostPipeline(ctx, (a, b), tol=1e-12)
    pipe.run(host, outs)
    torch.cuda.synchronize()
    assert ctx.status() == agipc.OK
    ref = agipc.DeviceScene(sc)
    step = agipc.CoarsenedStep(ctx, ref, tol=1e-12)
    for k, d in enumerate(host):
        ref.g.copy_(d["g"])
        step.run()
        want = step.dx.cpu()
        assert ctx.status() == agipc.OK
        assert torch.abs(outs[k] - want).max() <= 1e-10 * torch.abs(want).max()
    ctx.close()


@pytest.mark.parametrize("streamed", [False, True])
def test_status_not_converged_and_zero_rhs(streamed):
    sc = scenes.unit_cube(seed=1001)
    ds = agipc.DeviceScene(sc)
    ctx = ds.context()
    step = agipc.CoarsenedStep(ctx, ds, tol=1e-12, max_iter=1, streamed=streamed)
    step.run()
    assert ctx.status() == agipc.ERR_NOT_CONVERGED
    assert int(step.iters.item()) == 1
    step.g_c.zero_()
    step.solve()
    assert ctx.status() == agipc.OK
    assert int(step.iters.item()) == 0 and not step.y[: int(step.n_c.item())].any()
    ctx.close()


def test_assembly_run_accepts_only_its_lengths():
    sc = scenes.unit_cube(seed=1001)
    ds = agipc.DeviceScene(sc)
    ctx = ds.context()
    for bad in (0, 2, 7, 64, -8):
        with pytest.raises(agipc.AgipcError):
            ctx.set_assembly_run(bad)
    for good in (4, 8, 16, 32):
        ctx.set_assembly_run(good)
    ctx.close()


def test_status_bad_index_and_capacity():
    sc = scenes.unit_cube(seed=1001)
    ds = agipc.DeviceScene(sc)
    ctx = ds.context()
    bad = ds.edges.clone()
    bad[7, 1] = sc.n + 5
    labels = torch.empty(sc.n, dtype=torch.int32, device="cuda")
    nc = torch.zeros(1, dtype=torch.int32, device="cuda")
    agipc.agipc_aggregate(ctx, sc.n, bad, ds.tags, labels, nc)
    assert ctx.status() == agipc.ERR_BAD_INDEX
    step = agipc.CoarsenedStep(ctx, ds, tol=1e-8)
    step.aggregate()
    small_col = torch.empty(10, dtype=torch.int32, device="cuda")
    small_val = torch.empty(10, 9, dtype=torch.float64, device="cuda")
    agipc.agipc_assemble_coarse(ctx, ds.n, step.labels, step.n_c, ds.row_ptr, ds.col, ds.val, ds.pair_idx,
                                ds.pair_blk, ds.g, step.row_ptr, small_col, small_val, step.nnz, step.g_c, step.dinv)
    assert ctx.status() == agipc.ERR_CAPACITY
    with pytest.raises(agipc.AgipcError):
        agipc.agipc_aggregate(ctx, sc.n + 1, ds.edges, ds.tags, labels, nc)
    ctx.close()


def test_pcg_deterministic():
    sc = scenes.unit_cube(seed=1001)
    ds = agipc.DeviceScene(sc)
    ctx = ds.context()
    step = agipc.CoarsenedStep(ctx, ds, tol=1e-8)
    step.run()
    y1 = step.y.clone()
    step.solve()
    assert ctx.status() == agipc.OK
    assert torch.equal(y1, step.y)
    ctx.close()


@pytest.mark.parametrize("streamed", [False, True])
@pytest.mark.parametrize("seed", [1001, 1011, "domino_4x4"])
def test_post_coarsening_matches_oracle_cg_from_dx(seed, streamed):
    # Sec. 4.3: at most 10 fine PCG iterations started from the prolongated
    # coarse step.  Both sides start from the oracle's dx (an input here),
    # run exactly 10 iterations, and must agree; CG never raises the energy.
    # The 330,332-block domino streams its fine matrix in both layouts (the
    # 8-warp one by bulk copies after the initial guess's A x0 pass).
    if seed == "domino_4x4":
        sc = scenes.domino_grid(seed=1003, gx=4, gy=4, dims=(8, 8, 16), n_pairs=20000, small_gap_frac=0.02)
    else:
        sc = scenes.unit_cube(seed=seed)
    ref = oracle.coarsened_step(sc, tol=1e-8)
    rp, ci, val = oracle.fine_system(sc)
    dinv = oracle.block_jacobi(rp, ci, val)
    x_or, it_or, rr_or, _ = oracle.pcg(rp, ci, val, dinv, -sc.g, 1e-14, 10, x0=ref["dx"])
    assert it_or == 10
    ds = agipc.DeviceScene(sc)
    ctx = ds.context()
    post = agipc.PostCoarsening(ctx, ds, tol=1e-14, max_iter=10)
    post.fine.inner.streamed = streamed
    post.assemble()
    x = post.refine(torch.tensor(ref["dx"], dtype=torch.float64, device=ds.g.device))
    rc = ctx.status()
    assert rc == agipc.ERR_NOT_CONVERGED  # capped at 10, as asked
    got = x.cpu().numpy()
    it = int(post.fine.inner.iters.item())
    rr = float(post.fine.inner.relres.item())
    ctx.close()
    assert it == 10
    assert np.abs(got - x_or).max() <= 1e-9 * np.abs(x_or).max()
    assert abs(rr - rr_or) <= 1e-6 * rr_or
    g = sc.g.reshape(-1)

    def energy(v):
        return g @ v.reshape(-1) + 0.5 * v.reshape(-1) @ oracle.spmv(rp, ci, val, v).reshape(-1)

    assert energy(got) <= energy(ref["dx"]) + 1e-12 * abs(energy(ref["dx"]))


@pytest.mark.parametrize("streamed", [False, True])
@pytest.mark.parametrize("case", ["unit_cube", "domino_4x4"])
def test_fine_pcg_both_layouts(case, streamed):
    # FP64 PCG on a fine system (identity labels) in both kernel layouts: 8
    # warps per SM (the unit cube stays in shared memory; the 4x4 domino's
    # 330,332 blocks = 2,581 slices exceed the 1,216 it holds and stream) and
    # 16 warps per SM (always streamed, one slice buffer per warp: the unit
    # cube leaves most warps idle, the domino gives some warps two slices and
    # ends in a ragged 92-block slice).  Structure bit-exact, true residual.
    if case == "unit_cube":
        sc = scenes.unit_cube(seed=1001)
    else:
        sc = scenes.domino_grid(seed=1003, gx=4, gy=4, dims=(8, 8, 16), n_pairs=20000, small_gap_frac=0.02)
    tol = 1e-8
    ds = agipc.DeviceScene(sc)
    ctx = ds.context()
    fs = agipc.FineStep(ctx, ds, tol=tol, streamed=streamed)
    fs.run()
    assert ctx.status() == agipc.OK
    got = fs.host()
    ctx.close()
    frp, fci, fval = oracle.fine_system(sc)
    assert np.array_equal(got["row_ptr"], frp) and np.array_equal(got["col"], fci)
    if case == "domino_4x4":
        assert frp[-1] > 1216 * 128 and frp[-1] % 128 != 0
    res = oracle.spmv(frp, fci, fval, got["y"]) + sc.g
    assert np.linalg.norm(res) <= 1.05 * tol * np.linalg.norm(sc.g)


def test_pcg_initial_guess_zero_rhs_returns_zero():
    sc = scenes.tiny_box(seed=21, nx=2, ny=2, nz=2)
    sc.g = np.zeros_like(sc.g)
    ds = agipc.DeviceScene(sc)
    ctx = ds.context()
    post = agipc.PostCoarsening(ctx, ds, tol=1e-10, max_iter=10)
    post.assemble()
    x = post.refine(torch.ones(sc.n, 3, dtype=torch.float64, device=ds.g.device))
    assert ctx.status() == 0
    assert float(x.abs().max()) == 0.0
    assert int(post.fine.inner.iters.item()) == 0
    ctx.close()


@pytest.mark.parametrize("amp", [0.0, 8e-6, 2e-3])
def test_strain_tags_match_oracle(amp):
    # Sec. 4.2, Eq. 3: tags from the Green-strain increment between two
    # iterates; bit-exact against the oracle (FP64 decision on both sides)
    from oracle import tagging
    sc = scenes.unit_cube(seed=1001)
    X, x, tets = sc.meta["X_rest"], sc.meta["x"], sc.meta["tets"]
    rng = np.random.default_rng(11)
    # a smooth random displacement plus a localized bump
    x1 = x + amp * np.sin(3.0 * X @ rng.standard_normal((3, 3)))
    x1[rng.choice(sc.n, 5, replace=False)] += 0.01
    ref, _ = tagging.strain_tags(X, x, x1, tets, sc.edges, 5e-5)
    t = lambda a, dt: torch.tensor(np.ascontiguousarray(a), dtype=dt, device="cuda")  # noqa: E731
    ds = agipc.DeviceScene(sc)
    ctx = ds.context()
    tags = torch.empty(sc.n_edges, dtype=torch.uint8, device="cuda")
    agipc.agipc_strain_tags(ctx, sc.n, t(tets, torch.int32), t(X, torch.float64), t(x, torch.float64),
                            t(x1, torch.float64), 5e-5, ds.row_ptr, ds.col, tags)
    assert ctx.status() == 0
    ctx.close()
    got = tags.cpu().numpy()
    assert np.array_equal(got, ref)
    if amp == 8e-6:  # a mix of protected and collapsible edges
        assert 0 < (ref == 0).sum() < ref.size


@pytest.mark.parametrize("case", ["unit_cube", "domino_2x2"])
def test_affine_embedding_matches_oracle(case):
    # Sec. 4.2, Eq. 4: aggregates of more than 32 fine nodes get 12 DoF; the
    # expanded Galerkin system, its gradient, solve and prolongation against
    # the oracle's explicit P^T H P
    from oracle import affine
    import scipy.sparse as sps
    if case == "unit_cube":
        sc = scenes.unit_cube(seed=1001)
    else:
        sc = scenes.domino_grid(seed=1002, gx=2, gy=2, n_pairs=2000)
    lab, nc = oracle.labels(sc.n, sc.edges, sc.tags)
    pl, P, Hc, gc = affine.coarse_system(sc, lab, nc, threshold=32)
    assert pl["affine"].any() and (~pl["affine"]).any()
    ds = agipc.DeviceScene(sc)
    ctx = ds.context()
    st = agipc.AffineStep(ctx, ds, sc.meta["X_rest"], tol=1e-10, threshold=32)
    st.run()
    rc = ctx.status()
    got = st.host()
    ctx.close()
    assert rc == 0, rc
    assert np.array_equal(got["labels"], lab)
    assert got["n_rows"] == pl["n_rows"]
    assert np.array_equal(got["coarse_base"], pl["base"])
    assert np.array_equal(got["coarse_k"], np.where(pl["affine"], 4, 1))
    nr = pl["n_rows"]
    H_gpu = sps.bsr_matrix((got["a_val"], got["a_col"], got["a_row_ptr"]), shape=(3 * nr, 3 * nr)).toarray()
    H_ref = Hc.toarray()
    # each entry within 1e-12 of the sum of the magnitudes of its terms:
    # |P|^T |H| |P| with |H| assembled from the absolute block values
    absc = copy.copy(sc)
    absc.val = np.abs(sc.val)
    absc.pair_blk = np.abs(sc.pair_blk)
    Pa = abs(P)
    H_mag = (Pa.T @ oracle.fine_system_csr_blocks(absc) @ Pa).toarray()
    assert np.all(np.abs(H_gpu - H_ref) <= VAL_RTOL * H_mag + 1e-300)
    g_mag = Pa.T @ np.abs(sc.g.reshape(-1))
    assert np.all(np.abs(got["a_gc"].reshape(-1) - gc) <= VAL_RTOL * g_mag + 1e-300)
    y = got["y"].reshape(-1)
    assert np.linalg.norm(H_ref @ y + gc) <= 1.05e-10 * np.linalg.norm(gc)
    assert np.abs(got["dx"].reshape(-1) - P @ y).max() <= 1e-13 * np.abs(P @ y).max()
