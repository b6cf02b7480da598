"""GPU parity of the batched form: many uneven instances in one block-diagonal
problem, per-instance PCG in one persistent launch, against the oracle run on
each instance alone (through the C ABI)."""
import numpy as np
import pytest

import oracle
from paper_2605_04773_gb300 import scenes

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-6


def _agipc():
    from paper_2605_04773_gb300 import agipc
    return agipc


def _rounded(sc):
    """The instance with its FP32 inputs widened back to FP64 (the values the
    batched form actually sums)."""
    sc.val = sc.val.astype(np.float32).astype(np.float64)
    sc.pair_blk = sc.pair_blk.astype(np.float32).astype(np.float64)
    return sc


def _check_instance(batch, got, i, tol=TOL):
    sc = _rounded(batch.instance(i))
    v0, v1 = int(batch.vert_ptr[i]), int(batch.vert_ptr[i + 1])
    c0, c1 = int(got["inst_row"][i]), int(got["inst_row"][i + 1])
    lab, nc = oracle.labels(sc.n, sc.edges, sc.tags)
    assert np.array_equal(got["labels"][v0:v1] - c0, lab), i
    assert c1 - c0 == nc
    crp, cci, cval = oracle.galerkin(lab, nc, sc.row_ptr, sc.col, sc.val, sc.pair_idx, sc.pair_blk)
    grp = got["row_ptr"][c0:c1 + 1]
    b0, b1 = int(grp[0]), int(grp[-1])
    assert np.array_equal(grp - b0, crp)
    assert np.array_equal(got["col"][b0:b1] - c0, cci)
    # the FP64 master sums the widened FP32 inputs exactly as the FP64 path
    # sums its inputs: each entry within 1e-12 of the sum of the magnitudes
    # of its contributions (the oracle applied to |H|)
    _, _, mag = oracle.galerkin(lab, nc, sc.row_ptr, sc.col, np.abs(sc.val), sc.pair_idx, np.abs(sc.pair_blk))
    assert np.all(np.abs(got["val"][b0:b1] - cval) <= 1e-12 * mag + 1e-300), i
    gc = oracle.coarse_gradient(lab, nc, sc.g)
    gmag = oracle.coarse_gradient(lab, nc, np.abs(sc.g))
    assert np.all(np.abs(got["g_c"][c0:c1] - gc) <= 1e-12 * gmag + 1e-300), i
    # the solution's true FP64 residual with the oracle's coarse matrix
    y = got["y"][c0:c1]
    res = oracle.spmv(crp, cci, cval, y) + gc
    nb = np.linalg.norm(gc)
    if nb > 0:
        assert np.linalg.norm(res) <= 1.05 * tol * nb, (i, np.linalg.norm(res) / nb, got["relres"][i])
    assert got["relres"][i] <= tol
    assert np.array_equal(got["dx"][v0:v1], y[lab])


def _run(batch, tile=5, tol=TOL):
    agipc = _agipc()
    bd = agipc.BatchDevice(batch)
    ctx = bd.context()
    st = agipc.BatchedStep(ctx, bd, tol=tol, tile=tile)
    st.run()
    rc = ctx.status()
    got = st.host()
    ctx.close()
    return rc, got


@pytest.mark.parametrize("tile", [4, 5, 6, 8])
def test_small_batch_matches_oracle_per_instance(tile):
    batch = scenes.batch_instances(seed=2001, n_inst=9, v_range=(150, 3000), with_values=True)
    rc, got = _run(batch, tile=tile)
    assert rc == 0, rc
    assert len(set(got["iters"].tolist())) > 1  # instances stop independently
    for i in range(batch.n_inst):
        _check_instance(batch, got, i)


def test_degenerate_instances():
    # all-protected (n_c = n) next to nearly all-collapsible instances, and a
    # single-instance batch
    a = scenes.batch_instances(seed=2002, n_inst=3, v_range=(100, 600), frac_range=(0.0, 0.0), with_values=True)
    rc, got = _run(a)
    assert rc == 0
    assert got["n_c"] == a.n
    for i in range(a.n_inst):
        _check_instance(a, got, i)
    b = scenes.batch_instances(seed=2003, n_inst=4, v_range=(100, 600), frac_range=(0.999, 1.0), with_values=True)
    rc, got = _run(b)
    assert rc == 0
    for i in range(b.n_inst):
        _check_instance(b, got, i)
    c = scenes.batch_instances(seed=2004, n_inst=1, v_range=(2000, 2500), with_values=True)
    rc, got = _run(c)
    assert rc == 0
    _check_instance(c, got, 0)


def test_graph_replay_matches_eager():
    agipc = _agipc()
    batch = scenes.batch_instances(seed=2005, n_inst=12, v_range=(150, 2000), with_values=True)
    bd = agipc.BatchDevice(batch)
    ctx = bd.context()
    st = agipc.BatchedStep(ctx, bd, tol=TOL)
    st.run()
    assert ctx.status() == 0
    eager = st.host()
    st.capture()
    st.y.zero_()
    st.dx.zero_()
    st.replay()
    assert ctx.status() == 0
    rep = st.host()
    ctx.close()
    assert np.array_equal(rep["labels"], eager["labels"])
    assert np.array_equal(rep["col"], eager["col"])
    for i in range(batch.n_inst):
        _check_instance(batch, rep, i)


def test_autotuner_picks_both_launch_shapes(tmp_path):
    agipc = _agipc()
    batch = scenes.batch_instances(seed=2006, n_inst=16, v_range=(500, 4000), with_values=True)
    bd = agipc.BatchDevice(batch)
    ctx = bd.context()
    st = agipc.BatchedStep(ctx, bd, tol=TOL)
    tile, ms = agipc.autotune_batched(st, cache=str(tmp_path / "tune.json"))
    assert tile in agipc.BATCH_TILES and set(ms) == {str(t) for t in agipc.BATCH_TILES}
    run = st.assembly_run
    assert run in agipc.ASSEMBLY_RUNS and set(st.assembly_ms) == {str(r) for r in agipc.ASSEMBLY_RUNS}
    assert ctx.assembly_run == run
    # the cache holds both launch shapes and a second call reuses them
    import json
    ent = next(iter(json.load(open(tmp_path / "tune.json")).values()))
    assert ent["tile"] == tile and ent["assembly_run"] == run
    tile2, _ = agipc.autotune_batched(st, cache=str(tmp_path / "tune.json"))
    assert tile2 == tile and st.assembly_run == run
    st.run()
    assert ctx.status() == 0
    got = st.host()
    ctx.close()
    for i in range(0, batch.n_inst, 3):
        _check_instance(batch, got, i)


def test_full_batch_sampled_instances():
    # the 256-instance workload in the bench's configuration; the sampled
    # instances carry numpy-built values, the rest GPU-built ones
    rng = np.random.default_rng(7)
    sample = sorted(int(i) for i in rng.choice(256, 5, replace=False))
    batch = scenes.batch_instances(with_values=set(sample))
    rc, got = _run(batch)
    assert rc == 0, rc
    assert np.all(got["relres"] <= TOL)
    for i in sample:
        _check_instance(batch, got, i)
    # labels of every instance, bit-exact against the oracle (cheap)
    for i in range(0, 256, 16):
        v0, v1 = int(batch.vert_ptr[i]), int(batch.vert_ptr[i + 1])
        e_sel = (batch.edges[:, 0] >= v0) & (batch.edges[:, 0] < v1)
        lab, nc = oracle.labels(v1 - v0, batch.edges[e_sel] - v0, batch.tags[e_sel])
        assert np.array_equal(got["labels"][v0:v1] - got["inst_row"][i], lab)


def test_bad_cross_instance_block_sets_status():
    agipc = _agipc()
    batch = scenes.batch_instances(seed=2007, n_inst=2, v_range=(200, 300), with_values=True)
    bd = agipc.BatchDevice(batch)
    ctx = bd.context()
    st = agipc.BatchedStep(ctx, bd, tol=TOL)
    st.run()
    assert ctx.status() == 0
    # claim one instance: the coarse columns of the second leave it
    one = torch.tensor([0, int(st.n_c.item())], dtype=torch.int32, device=bd.g.device)
    half = torch.tensor([0, int(st.inst_row[1].item()), int(st.n_c.item())], dtype=torch.int32, device=bd.g.device)
    half[1] = max(1, int(half[1].item()) - 1)  # cut inside the first instance
    agipc.agipc_pcg_batched(ctx, 2, half, bd.n, st.row_ptr, st.col, st.val, st.val32, st.dinv32, st.g_c, st.y, TOL,
                            1000, -1, 20, 5, st.iters[:2], st.relres[:2])
    assert ctx.status() == agipc.ERR_BAD_INDEX
    agipc.agipc_pcg_batched(ctx, 1, one, bd.n, st.row_ptr, st.col, st.val, st.val32, st.dinv32, st.g_c, st.y, TOL,
                            1000, -1, 20, 5, st.iters[:1], st.relres[:1])
    assert ctx.status() == 0
    ctx.close()
