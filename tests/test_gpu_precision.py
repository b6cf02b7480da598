"""Precision form (FP32 blocks, SpMV and preconditioner, FP64 dots and FP64
residual replacement) against the oracle.

The FP64 master coarse matrix must equal the oracle's U H U^T of the same
rounded inputs (FP32 blocks widened to FP64, small-gap stencils in FP64) to
the 1e-12 bar of the FP64 path, and the FP32 copy must be its exact rounding.
The solve is judged by its true FP64 residual with that master matrix.  The
difference to the all-FP64 step (unrounded inputs) is the precision form's
error; the paper fixes no bound for it (all its runs are FP64), so it is
reported and only checked for sanity.
"""
import numpy as np
import pytest
import torch

import oracle
from oracle import precision
from paper_2605_04773_gb300 import agipc, scenes

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2605_04773_gb300 import build
    build.build()
    agipc.load()


def _mixed(sc, tol, streamed=False):
    ds = agipc.MixedDeviceScene(sc)
    ctx = ds.context()
    st = agipc.MixedStep(ctx, ds, tol=tol, streamed=streamed)
    stages = {}
    for name, f in (("aggregate", st.aggregate), ("assemble", st.assemble), ("solve", st.solve),
                    ("prolongate", st.prolongate)):
        f()
        stages[name] = ctx.status()
    out = st.host()
    ctx.close()
    rc = next((v for v in stages.values() if v != agipc.OK), agipc.OK)
    assert rc == agipc.OK, (stages, out["iters"], out["relres"])
    return rc, out


def _check(sc, got, tol):
    pi = precision.scene_split(sc)
    lab, nc = oracle.labels(sc.n, sc.edges, sc.tags)
    assert got["n_c"] == nc and np.array_equal(got["labels"], lab)
    pidx = np.concatenate([pi["pair_idx32"], pi["pair_idx64"]])
    pblk = np.concatenate([pi["pair_blk32"].astype(np.float64), pi["pair_blk64"]])
    val = pi["val32"].astype(np.float64)
    crp, cci, cval = oracle.galerkin(lab, nc, sc.row_ptr, sc.col, val, pidx, pblk)
    _, _, mag = oracle.galerkin(lab, nc, sc.row_ptr, sc.col, np.abs(val), pidx, np.abs(pblk))
    assert np.array_equal(got["row_ptr"], crp) and np.array_equal(got["col"], cci)
    assert np.all(np.abs(got["val"] - cval) <= 1e-12 * mag + 1e-300)
    assert np.array_equal(got["val32"], got["val"].astype(np.float32))
    gc = oracle.coarse_gradient(lab, nc, sc.g)
    res = oracle.spmv(crp, cci, cval, got["y"]) + gc
    rel = np.linalg.norm(res) / np.linalg.norm(gc)
    assert rel <= 1.05 * tol, rel
    assert np.array_equal(got["dx"], got["y"][got["labels"]])
    return rel


@pytest.mark.parametrize("streamed", [False, True])
def test_precision_form_unit_cube(streamed):
    # streamed: the 16-warp kernel on the tiny coarse system (one ragged
    # slice, every other warp idle; residual replacements included)
    sc = scenes.unit_cube(seed=1001)
    rc, got = _mixed(sc, 1e-8, streamed=streamed)
    assert rc == agipc.OK
    _check(sc, got, 1e-8)
    ref = oracle.coarsened_step(sc, tol=1e-12)
    err = np.linalg.norm(got["dx"] - ref["dx"]) / np.linalg.norm(ref["dx"])
    assert err < 1e-3, err


def test_precision_form_domino_with_small_gaps():
    sc = scenes.domino_grid(seed=1003, gx=3, gy=3, dims=(4, 8, 12), n_pairs=6000, small_gap_frac=0.02)
    pi = precision.scene_split(sc)
    assert pi["pair_idx64"].shape[0] > 0
    rc, got = _mixed(sc, 1e-6)
    assert rc == agipc.OK
    _check(sc, got, 1e-6)


def test_precision_form_refinement_off_and_not_converged_status():
    sc = scenes.unit_cube(seed=1001)
    ds = agipc.MixedDeviceScene(sc)
    ctx = ds.context()
    st = agipc.MixedStep(ctx, ds, tol=1e-12, max_iter=3)
    st.run()
    assert ctx.status() == agipc.ERR_NOT_CONVERGED
    st2 = agipc.MixedStep(ctx, ds, tol=1e-5, refine_every=0)
    st2.run()
    assert ctx.status() == agipc.OK
    ctx.close()


@pytest.mark.parametrize("case", ["small_gaps", "no_small_gaps", "all_small", "no_pairs"])
def test_precision_split_matches_oracle(case):
    # agipc_precision_split against the oracle's rule, bit for bit: the same
    # FP64 comparison gap < limit, round-to-nearest FP32 values, input order
    # kept in both lists
    if case == "no_pairs":
        sc = scenes.tiny_box(seed=4, nx=2, ny=2, nz=2, n_pairs=0)
    else:
        sc = scenes.domino_grid(seed=1003, gx=2, gy=2, dims=(3, 6, 8), n_pairs=3000,
                                small_gap_frac={"small_gaps": 0.05, "no_small_gaps": 0.0, "all_small": 1.0}[case])
    want = precision.scene_split(sc)
    ds = agipc.MixedDeviceScene(sc)
    assert np.array_equal(ds.val32.cpu().numpy(), want["val32"].reshape(-1, 9))
    for k, w in (("pair_idx32", want["pair_idx32"]), ("pair_blk32", want["pair_blk32"]),
                 ("pair_idx64", want["pair_idx64"]), ("pair_blk64", want["pair_blk64"])):
        got = getattr(ds, k).cpu().numpy()
        assert got.shape[0] == w.shape[0], k
        assert np.array_equal(got.reshape(w.shape), w), k
    if case == "no_small_gaps":
        assert want["pair_idx64"].shape[0] == 0
    if case == "all_small":
        assert want["pair_idx32"].shape[0] == 0


def test_precision_form_c3_errors_vs_fp64_oracle():
    # The precision form on the full C3 scene (the 64-box domino with 1 % of
    # the gaps below 0.05 dhat) against the FP64 oracle on the unrounded
    # inputs.  The paper fixes no bound (it is all FP64), so the bounds come
    # from the FP32 storage: the true coarse residual with the unrounded H_c
    # is at most the solve's residual with its FP64 master (1.05 tol) plus
    # u |H_c|_abs |y| with u = 2^-24 (every FP32 input entry is within u of
    # its FP64 value); dx and the energy decrease are printed for the record.
    sc = scenes.domino_grid(seed=1003, small_gap_frac=0.01)
    tol = 1e-6
    rc, got = _mixed(sc, tol)
    assert rc == agipc.OK
    ref = oracle.coarsened_step(sc, tol=1e-12)
    lab, nc = oracle.labels(sc.n, sc.edges, sc.tags)
    crp, cci, cval = oracle.galerkin(lab, nc, sc.row_ptr, sc.col, sc.val, sc.pair_idx, sc.pair_blk)
    _, _, mag = oracle.galerkin(lab, nc, sc.row_ptr, sc.col, np.abs(sc.val), sc.pair_idx, np.abs(sc.pair_blk))
    gc = oracle.coarse_gradient(lab, nc, sc.g)
    y = got["y"]
    nb = np.linalg.norm(gc)
    res = np.linalg.norm(oracle.spmv(crp, cci, cval, y) + gc) / nb
    bound = 1.05 * tol + 2.0 ** -24 * np.linalg.norm(oracle.spmv(crp, cci, mag, np.abs(y))) / nb
    assert res <= bound, (res, bound)
    dx_err = np.linalg.norm(got["dx"] - ref["dx"]) / np.linalg.norm(ref["dx"])
    rp, ci, fv = oracle.fine_system(sc)
    g = sc.g.reshape(-1)

    def decrease(dx):
        return float(g @ dx.reshape(-1) + 0.5 * dx.reshape(-1) @ oracle.spmv(rp, ci, fv, dx).reshape(-1))

    e_ref, e_got = decrease(ref["dx"]), decrease(got["dx"])
    e_err = abs(e_got - e_ref) / abs(e_ref)
    print("C3 vs FP64 oracle: coarse residual %.3e (bound %.3e), dx rel err %.3e, energy decrease rel err %.3e"
          % (res, bound, dx_err, e_err))
    assert dx_err < 1e-3 and e_err < 1e-6


def _fine_mixed(sc, tol, streamed):
    ds = agipc.MixedDeviceScene(sc)
    ctx = ds.context()
    st = agipc.MixedFineStep(ctx, ds, tol=tol, streamed=streamed)
    st.assemble()
    ctx.check()
    st.solve()
    rc = ctx.status()
    out = st.host()
    ctx.close()
    assert rc == agipc.OK, (rc, out["iters"], out["relres"])
    return out


@pytest.mark.parametrize("streamed", [False, True])
@pytest.mark.parametrize("case", ["unit_cube", "domino_4x4"])
def test_precision_form_fine_system_both_layouts(case, streamed):
    # The precision-form PCG on a fine system (identity labels, contacts
    # merged) in both kernel layouts: 8 warps per SM (the unit cube's matrix
    # stays in shared memory; the 4x4 domino's 330,332 blocks = 2,581 slices
    # exceed the 1,216 it holds and stream) and 16 warps per SM (always
    # streamed: the unit cube leaves most warps without a slice, the domino
    # gives some warps two, and its last slice is ragged, 92 blocks, so it
    # takes the zero-filling copy path while full slices go by bulk copy).
    # Judged by the true FP64 residual with the oracle's fine matrix of the
    # same rounded inputs.
    if case == "unit_cube":
        sc = scenes.unit_cube(seed=1001)
    else:
        sc = scenes.domino_grid(seed=1003, gx=4, gy=4, dims=(8, 8, 16), n_pairs=20000, small_gap_frac=0.02)
    tol = 1e-8
    got = _fine_mixed(sc, tol, streamed)
    pi = precision.scene_split(sc)
    ident = np.arange(sc.n, dtype=np.int32)
    pidx = np.concatenate([pi["pair_idx32"], pi["pair_idx64"]])
    pblk = np.concatenate([pi["pair_blk32"].astype(np.float64), pi["pair_blk64"]])
    crp, cci, cval = oracle.galerkin(ident, sc.n, sc.row_ptr, sc.col, pi["val32"].astype(np.float64), pidx, pblk)
    assert np.array_equal(got["row_ptr"], crp) and np.array_equal(got["col"], cci)
    if case == "domino_4x4":
        assert crp[-1] > 1216 * 128 and crp[-1] % 128 != 0
    g = sc.g.reshape(-1, 3)
    rel = np.linalg.norm(oracle.spmv(crp, cci, cval, got["y"]) + g) / np.linalg.norm(g)
    assert rel <= 1.05 * tol, rel
