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
from paper_2605_04773_gb300 import agipc, scenes

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2605_04773_gb300 import build
    build.build()
    agipc.load()


def _mixed(sc, tol):
    ds = agipc.MixedDeviceScene(sc)
    ctx = ds.context()
    st = agipc.MixedStep(ctx, ds, tol=tol)
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
    pi = scenes.precision_inputs(sc)
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


def test_precision_form_unit_cube():
    sc = scenes.unit_cube(seed=1001)
    rc, got = _mixed(sc, 1e-8)
    assert rc == agipc.OK
    _check(sc, got, 1e-8)
    ref = oracle.coarsened_step(sc, tol=1e-12)
    err = np.linalg.norm(got["dx"] - ref["dx"]) / np.linalg.norm(ref["dx"])
    assert err < 1e-3, err


def test_precision_form_domino_with_small_gaps():
    sc = scenes.domino_grid(seed=1003, gx=3, gy=3, dims=(4, 8, 12), n_pairs=6000, small_gap_frac=0.02)
    pi = scenes.precision_inputs(sc)
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
